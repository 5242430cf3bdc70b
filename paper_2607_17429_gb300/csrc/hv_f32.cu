// F32 instantiations of the H·v kernel: one block (ftlm_hv) or a multi-block set (ftlm_hv_multi).
#include "hv_kernel.cuh"

namespace ftlm {

ftlm_status hv_launch_f32(const ftlm_basis *bs, int B, const float *x, float *y, cudaStream_t stream) {
    HvArgs<float> a;
    const ftlm_basis *blocks[1] = {bs};
    const int rho_off[1] = {0};
    const float *V[1] = {bs->d_Vf};
    const float *xs[1] = {x};
    float *ys[1] = {y};
    fill_hv_args<float>(bs->sec, B, 1, blocks, bs->d_off, bs->d_ntab, bs->d_sqrtSf, bs->d_rhoTf,
                      bs->rho_elemsf, rho_off, V, xs, ys, a);
    return launch_hv<float>(a, bs->sec->half, stream);
}

ftlm_status hv_multi_launch_f32(const ftlm_multiblock *mb, int B, const float *const *x, float *const *y,
                               cudaStream_t stream) {
    HvArgs<float> a;
    const float *V[kMaxK];
    for (int k = 0; k < mb->K; ++k) V[k] = mb->blocks[k]->d_Vf;
    fill_hv_args<float>(mb->sec, B, mb->K, mb->blocks.data(), mb->d_offm, mb->d_ntab, mb->blocks[0]->d_sqrtSf,
                      mb->d_rhoTf, mb->rho_totalf, mb->rho_offf.data(), V, x, y, a);
    return launch_hv<float>(a, mb->sec->half, stream);
}

}  // namespace ftlm
