// Compiled packed H·v kernels: one entry per (shape, elements per lane, label width).
#pragma once

#include <vector>

#include "hvp_lane.cuh"

namespace ftlm {

// Shape ids: one block of dimension 1..12 (Section 3's limit on d_Gamma; real
// forms of complex and quaternionic irreps count their real dimension), and the
// full real irrep sets of I_h, O_h and T_d in canonical irrep order (dimensions
// ascending).
enum {
    kShapeD1 = 0, kShapeD2, kShapeD3, kShapeD4, kShapeD5, kShapeD6, kShapeD7, kShapeD8, kShapeD9, kShapeD10,
    kShapeD11, kShapeD12, kShapeIh, kShapeOh, kShapeTd, kNumShapes
};
constexpr bool shape_is_single(int shape) { return shape >= kShapeD1 && shape <= kShapeD12; }
constexpr bool shape_is_wide(int shape) { return shape >= kShapeD6 && shape <= kShapeD12; }
using ShapeIh = Shape<1, 1, 3, 3, 3, 3, 4, 4, 5, 5>;
using ShapeOh = Shape<1, 1, 1, 1, 2, 2, 3, 3, 3, 3>;
using ShapeTd = Shape<1, 1, 2, 3, 3>;

template <typename VT>
struct HvpOps {
    int (*occupancy)(const HvpArgs<VT> &, int warps, int nbuf);
    ftlm_status (*launch)(HvpArgs<VT>, const HvpGeom &, cudaStream_t);
    int max_threads;
    int tile_fixed;  // representatives per tile fixed by the kernel (0: chosen with the geometry)
};

#define FTLM_HVP_OPS_M(VT, ST, SH, GPL, HALF, MODE)                                              \
    HvpOps<VT> {                                                                                   \
        &hvp_occupancy_t<VT, ST, SH, GPL, HALF, MODE>, &hvp_launch_t<VT, ST, SH, GPL, HALF, MODE>, \
            hvp_max_threads<VT, SH>(), 0                                                           \
    }
// one thread per representative (table mode, one block, B = 1; hvp_lane.cuh)
#define FTLM_HVP_LANE_OPS(VT, ST, D) \
    HvpOps<VT> { &hvp_lane_occupancy_t<VT, ST, D>, &hvp_lane_launch_t<VT, ST, D>, kLaneThreads, kLaneThreads }
#define FTLM_HVP_OPS(VT, ST, SH, GPL, HALF) FTLM_HVP_OPS_M(VT, ST, SH, GPL, HALF, 0)

template <typename VT>
struct HvpPlan {
    HvpArgs<VT> a;
    HvpGeom geo;
    const HvpOps<VT> *ops = nullptr;
    int mode = 0;                     // 0: on-the-fly search; 1: entry table; 2: entry-table build
    uint64_t rows_total = 0;          // packed rows over all parts (profiling)
    std::vector<uint64_t> tile0, ntile;  // per part: first tile and tile count
};

// packed.cu
template <typename VT>
void hvp_part_of(const ftlm_sector *s, const PackedSet *ps, const ftlm_basis *const *blocks, const void *x, void *y,
                 HvpPart<VT> &p);
// esize: bytes of a stored vector element (sizeof(VT), or 2 for FP16 storage with VT = float)
template <typename VT>
ftlm_status hvp_plan(const ftlm_sector *s, const PackedSet *ps, std::vector<HvpPart<VT>> &parts, int B, int esize,
                     HvpPlan<VT> &plan, cudaStream_t tune_stream);
template <typename VT>
ftlm_status hvp_launch_plan(const HvpPlan<VT> &plan, double *dot_part, cudaStream_t stream, bool timed);
// pieces of a plan (packed.cu): sector-wide arguments, geometry, tile order
template <typename VT>
void hvp_fill_common(const ftlm_sector *s, const PackedSet *ps, int B, int esize, HvpArgs<VT> &a);
template <typename VT>
ftlm_status hvp_choose_geom(const HvpOps<VT> *ops, HvpArgs<VT> a, bool tma, HvpGeom &geo);
template <typename VT>
void hvp_retile(HvpPlan<VT> &plan, std::vector<HvpPart<VT>> &parts);
// entries.cu: the sector's optional entry table
ftlm_status entry_table_build(ftlm_sector *s, cudaStream_t stream);
void entry_table_free(ftlm_sector *s);

// null if the combination is not compiled (gpl: 2 for |G| <= 64, 4 for |G| <= 128)
const HvpOps<float> *hvp_ops_single_f32(int shape, int gpl, bool half);
const HvpOps<float> *hvp_ops_multi_f32(int shape, int gpl, bool half);
const HvpOps<double> *hvp_ops_single_f64(int shape, int gpl, bool half);
const HvpOps<double> *hvp_ops_multi_f64(int shape, int gpl, bool half);
const HvpOps<float> *hvp_ops_single_f16(int shape, int gpl, bool half);  // FP16 storage, FP32 arithmetic
const HvpOps<float> *hvp_ops_multi_f16(int shape, int gpl, bool half);
// one block of dimension 6..12 (label search with 4 elements per lane, any |G| <= 128):
// kind 0 search, 1 table, 2 table with one thread per representative (B = 1)
const HvpOps<float> *hvp_ops_wide_f32(int shape, bool half, int kind);
const HvpOps<double> *hvp_ops_wide_f64(int shape, bool half, int kind);
const HvpOps<float> *hvp_ops_wide_f16(int shape, bool half, int kind);
// table mode (flips from the sector's entry table), shapes D1..D5, I_h, O_h, T_d; esize 8, 4 or 2
const HvpOps<double> *hvp_ops_table_f64(int shape);
const HvpOps<float> *hvp_ops_table_f32(int shape);
const HvpOps<float> *hvp_ops_table_f16(int shape);
// table mode, one thread per representative: single blocks (shapes D1..D5) at B = 1
const HvpOps<double> *hvp_ops_lane_f64(int shape);
const HvpOps<float> *hvp_ops_lane_f32(int shape);
const HvpOps<float> *hvp_ops_lane_f16(int shape);
// build mode (writes the entry table; no gathers or outputs)
const HvpOps<float> *hvp_ops_build(int gpl, bool half);

}  // namespace ftlm
