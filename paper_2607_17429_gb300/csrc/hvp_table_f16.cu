// Packed H·v kernels in table mode (flips read from the sector's entry table), every compiled
// block shape, FP16 vector storage with FP32 arithmetic.
#include "hvp_ops.h"

namespace ftlm {

const HvpOps<float> *hvp_ops_table_f16(int shape) {
    static const HvpOps<float> tab[8] = {
        FTLM_HVP_OPS_M(float, __half, Shape<1>, 2, false, 1), FTLM_HVP_OPS_M(float, __half, Shape<2>, 2, false, 1),
        FTLM_HVP_OPS_M(float, __half, Shape<3>, 2, false, 1), FTLM_HVP_OPS_M(float, __half, Shape<4>, 2, false, 1),
        FTLM_HVP_OPS_M(float, __half, Shape<5>, 2, false, 1), FTLM_HVP_OPS_M(float, __half, ShapeIh, 2, false, 1),
        FTLM_HVP_OPS_M(float, __half, ShapeOh, 2, false, 1), FTLM_HVP_OPS_M(float, __half, ShapeTd, 2, false, 1)};
    if (shape >= kShapeD1 && shape <= kShapeD5) return &tab[shape - kShapeD1];
    if (shape >= kShapeIh && shape <= kShapeTd) return &tab[5 + shape - kShapeIh];
    return nullptr;
}

const HvpOps<float> *hvp_ops_lane_f16(int shape) {
    static const HvpOps<float> tab[5] = {FTLM_HVP_LANE_OPS(float, __half, 1), FTLM_HVP_LANE_OPS(float, __half, 2),
                                       FTLM_HVP_LANE_OPS(float, __half, 3), FTLM_HVP_LANE_OPS(float, __half, 4),
                                       FTLM_HVP_LANE_OPS(float, __half, 5)};
    if (shape < kShapeD1 || shape > kShapeD5) return nullptr;
    return &tab[shape - kShapeD1];
}

}  // namespace ftlm
