// F64 instantiations of the H·v kernel: one block (ftlm_hv) or a multi-block set (ftlm_hv_multi).
#include "hv_kernel.cuh"

namespace ftlm {

ftlm_status hv_launch_f64(const ftlm_basis *bs, int B, const double *x, double *y, cudaStream_t stream) {
    HvArgs<double> a;
    const ftlm_basis *blocks[1] = {bs};
    const int rho_off[1] = {0};
    const double *V[1] = {bs->d_V};
    const double *xs[1] = {x};
    double *ys[1] = {y};
    fill_hv_args<double>(bs->sec, B, 1, blocks, bs->d_off, bs->d_ntab, bs->d_sqrtS, bs->d_rhoT,
                      bs->rho_elems, rho_off, V, xs, ys, a);
    return launch_hv<double>(a, bs->sec->half, stream);
}

ftlm_status hv_multi_launch_f64(const ftlm_multiblock *mb, int B, const double *const *x, double *const *y,
                               cudaStream_t stream) {
    HvArgs<double> a;
    const double *V[kMaxK];
    for (int k = 0; k < mb->K; ++k) V[k] = mb->blocks[k]->d_V;
    fill_hv_args<double>(mb->sec, B, mb->K, mb->blocks.data(), mb->d_offm, mb->d_ntab, mb->blocks[0]->d_sqrtS,
                      mb->d_rhoT, mb->rho_total, mb->rho_off.data(), V, x, y, a);
    return launch_hv<double>(a, mb->sec->half, stream);
}

}  // namespace ftlm
