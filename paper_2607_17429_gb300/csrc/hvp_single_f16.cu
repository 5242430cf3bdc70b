// Packed H·v kernels, one block of dimension 1..5, FP16 vector storage with FP32 arithmetic.
#include "hvp_ops.h"

namespace ftlm {

const HvpOps<float> *hvp_ops_single_f16(int shape, int gpl, bool half) {
    static const HvpOps<float> tab[5][2][2] = {
#define ROW(D) \
    {{FTLM_HVP_OPS(float, __half, Shape<D>, 2, false), FTLM_HVP_OPS(float, __half, Shape<D>, 2, true)}, \
     {FTLM_HVP_OPS(float, __half, Shape<D>, 4, false), FTLM_HVP_OPS(float, __half, Shape<D>, 4, true)}}
        ROW(1), ROW(2), ROW(3), ROW(4), ROW(5)
#undef ROW
    };
    if (shape < kShapeD1 || shape > kShapeD5 || (gpl != 2 && gpl != 4)) return nullptr;
    return &tab[shape - kShapeD1][gpl == 4][half ? 1 : 0];
}

}  // namespace ftlm
