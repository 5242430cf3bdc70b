// Packed H·v kernels for one block of dimension 6..12 (double vectors): the
// label search with four group elements per lane (any |G| <= 128), the entry-table
// kernel and the one-thread-per-representative entry-table kernel (B = 1).
#include "hvp_ops.h"

namespace ftlm {

const HvpOps<double> *hvp_ops_wide_f64(int shape, bool half, int kind) {
    static const HvpOps<double> tab[7][4] = {
#define ROW(D)                                                                                              \
    {FTLM_HVP_OPS(double, double, Shape<D>, 4, false), FTLM_HVP_OPS(double, double, Shape<D>, 4, true),              \
     FTLM_HVP_OPS_M(double, double, Shape<D>, 2, false, 1), FTLM_HVP_LANE_OPS(double, double, D)}
        ROW(6), ROW(7), ROW(8), ROW(9), ROW(10), ROW(11), ROW(12)
#undef ROW
    };
    if (!shape_is_wide(shape) || kind < 0 || kind > 2) return nullptr;
    const int col = kind == 0 ? (half ? 1 : 0) : kind + 1;
    return &tab[shape - kShapeD6][col];
}

}  // namespace ftlm
