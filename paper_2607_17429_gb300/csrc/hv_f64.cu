// FP64 instantiations of the H·v kernel.
#include "hv_impl.cuh"

namespace ftlm {
ftlm_status hv_launch_f64(const ftlm_basis *bs, int B, const double *x, double *y, cudaStream_t stream) {
    HvArgs<double> a;
    fill_hv_args<double>(bs, B, a, bs->d_sqrtS, bs->d_V, bs->d_rhoT);
    a.bonds = bs->sec->d_bonds;
    return launch_hv<double>(a, bs->sec->half, x, y, stream);
}
}  // namespace ftlm
