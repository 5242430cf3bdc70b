// Packed H·v kernels for the full irrep sets of I_h (|G| = 120), O_h (48) and T_d (24),
// FP16 vector storage with FP32 arithmetic.
#include "hvp_ops.h"

namespace ftlm {

const HvpOps<float> *hvp_ops_multi_f16(int shape, int gpl, bool half) {
    static const HvpOps<float> ih[2] = {FTLM_HVP_OPS(float, __half, ShapeIh, 4, false), FTLM_HVP_OPS(float, __half, ShapeIh, 4, true)};
    static const HvpOps<float> oh[2] = {FTLM_HVP_OPS(float, __half, ShapeOh, 2, false), FTLM_HVP_OPS(float, __half, ShapeOh, 2, true)};
    static const HvpOps<float> td[2] = {FTLM_HVP_OPS(float, __half, ShapeTd, 2, false), FTLM_HVP_OPS(float, __half, ShapeTd, 2, true)};
    const int h = half ? 1 : 0;
    if (shape == kShapeIh && gpl == 4) return &ih[h];
    if (shape == kShapeOh && gpl == 2) return &oh[h];
    if (shape == kShapeTd && gpl == 2) return &td[h];
    return nullptr;
}

}  // namespace ftlm
