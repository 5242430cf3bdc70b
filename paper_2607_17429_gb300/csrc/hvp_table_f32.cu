// Packed H·v kernels in table mode (flips read from the sector's entry table), every compiled
// block shape, float vectors.
#include "hvp_ops.h"

namespace ftlm {

const HvpOps<float> *hvp_ops_table_f32(int shape) {
    static const HvpOps<float> tab[8] = {
        FTLM_HVP_OPS_M(float, float, Shape<1>, 2, false, 1), FTLM_HVP_OPS_M(float, float, Shape<2>, 2, false, 1),
        FTLM_HVP_OPS_M(float, float, Shape<3>, 2, false, 1), FTLM_HVP_OPS_M(float, float, Shape<4>, 2, false, 1),
        FTLM_HVP_OPS_M(float, float, Shape<5>, 2, false, 1), FTLM_HVP_OPS_M(float, float, ShapeIh, 2, false, 1),
        FTLM_HVP_OPS_M(float, float, ShapeOh, 2, false, 1), FTLM_HVP_OPS_M(float, float, ShapeTd, 2, false, 1)};
    if (shape >= kShapeD1 && shape <= kShapeD5) return &tab[shape - kShapeD1];
    if (shape >= kShapeIh && shape <= kShapeTd) return &tab[5 + shape - kShapeIh];
    return nullptr;
}

const HvpOps<float> *hvp_ops_lane_f32(int shape) {
    static const HvpOps<float> tab[5] = {FTLM_HVP_LANE_OPS(float, float, 1), FTLM_HVP_LANE_OPS(float, float, 2),
                                       FTLM_HVP_LANE_OPS(float, float, 3), FTLM_HVP_LANE_OPS(float, float, 4),
                                       FTLM_HVP_LANE_OPS(float, float, 5)};
    if (shape < kShapeD1 || shape > kShapeD5) return nullptr;
    return &tab[shape - kShapeD1];
}

}  // namespace ftlm
