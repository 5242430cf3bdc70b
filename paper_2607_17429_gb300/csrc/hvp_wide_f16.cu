// Packed H·v kernels for one block of dimension 6..12 (FP16 vector storage with FP32 arithmetic): the
// label search with four group elements per lane (any |G| <= 128), the entry-table
// kernel and the one-thread-per-representative entry-table kernel (B = 1).
#include "hvp_ops.h"

namespace ftlm {

const HvpOps<float> *hvp_ops_wide_f16(int shape, bool half, int kind) {
    static const HvpOps<float> tab[7][4] = {
#define ROW(D)                                                                                              \
    {FTLM_HVP_OPS(float, __half, Shape<D>, 4, false), FTLM_HVP_OPS(float, __half, Shape<D>, 4, true),              \
     FTLM_HVP_OPS_M(float, __half, Shape<D>, 2, false, 1), FTLM_HVP_LANE_OPS(float, __half, D)}
        ROW(6), ROW(7), ROW(8), ROW(9), ROW(10), ROW(11), ROW(12)
#undef ROW
    };
    if (!shape_is_wide(shape) || kind < 0 || kind > 2) return nullptr;
    const int col = kind == 0 ? (half ? 1 : 0) : kind + 1;
    return &tab[shape - kShapeD6][col];
}

}  // namespace ftlm
