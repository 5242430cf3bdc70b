// Packed H·v kernels in table mode (flips read from the sector's entry table), every compiled
// block shape, double vectors.
#include "hvp_ops.h"

namespace ftlm {

const HvpOps<double> *hvp_ops_table_f64(int shape) {
    static const HvpOps<double> tab[8] = {
        FTLM_HVP_OPS_M(double, double, Shape<1>, 2, false, 1), FTLM_HVP_OPS_M(double, double, Shape<2>, 2, false, 1),
        FTLM_HVP_OPS_M(double, double, Shape<3>, 2, false, 1), FTLM_HVP_OPS_M(double, double, Shape<4>, 2, false, 1),
        FTLM_HVP_OPS_M(double, double, Shape<5>, 2, false, 1), FTLM_HVP_OPS_M(double, double, ShapeIh, 2, false, 1),
        FTLM_HVP_OPS_M(double, double, ShapeOh, 2, false, 1), FTLM_HVP_OPS_M(double, double, ShapeTd, 2, false, 1)};
    if (shape >= kShapeD1 && shape <= kShapeD5) return &tab[shape - kShapeD1];
    if (shape >= kShapeIh && shape <= kShapeTd) return &tab[5 + shape - kShapeIh];
    return nullptr;
}

const HvpOps<double> *hvp_ops_lane_f64(int shape) {
    static const HvpOps<double> tab[5] = {FTLM_HVP_LANE_OPS(double, double, 1), FTLM_HVP_LANE_OPS(double, double, 2),
                                       FTLM_HVP_LANE_OPS(double, double, 3), FTLM_HVP_LANE_OPS(double, double, 4),
                                       FTLM_HVP_LANE_OPS(double, double, 5)};
    if (shape < kShapeD1 || shape > kShapeD5) return nullptr;
    return &tab[shape - kShapeD1];
}

}  // namespace ftlm
