// Build mode of the packed H·v kernel: the representative search and lookup of every
// ladder flip, written to the sector's entry table (no gathers, no outputs).
#include "hvp_ops.h"

namespace ftlm {

const HvpOps<float> *hvp_ops_build(int gpl, bool half) {
    static const HvpOps<float> tab[2][2] = {
        {FTLM_HVP_OPS_M(float, float, Shape<1>, 2, false, 2), FTLM_HVP_OPS_M(float, float, Shape<1>, 2, true, 2)},
        {FTLM_HVP_OPS_M(float, float, Shape<1>, 4, false, 2), FTLM_HVP_OPS_M(float, float, Shape<1>, 4, true, 2)}};
    if (gpl != 2 && gpl != 4) return nullptr;
    return &tab[gpl == 4][half ? 1 : 0];
}

}  // namespace ftlm
