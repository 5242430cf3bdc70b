// F32 instantiation of the per-block-layout multi-block H·v kernel (ftlm_hv_multi).
#include "hv_kernel.cuh"

namespace ftlm {

ftlm_status hv_multi_launch_f32(const ftlm_multiblock *mb, int B, const float *const *x, float *const *y,
                               cudaStream_t stream) {
    for (int k = 0; k < mb->K; ++k)  // this per-block layout kernel is specialised for d_Gamma <= 5
        if (mb->blocks[k]->d > 5)
            return fail(FTLM_EUNSUPPORTED, "d_Gamma = %d needs the packed layout (ftlm_hv_packed)", mb->blocks[k]->d);
    HvArgs<float> a;
    const float *V[kMaxK];
    for (int k = 0; k < mb->K; ++k) V[k] = mb->blocks[k]->d_Vf;
    fill_hv_args<float>(mb->sec, B, mb->K, mb->blocks.data(), mb->d_offm, mb->d_ntab, mb->blocks[0]->d_sqrtSf,
                      mb->d_rhoTf, mb->rho_totalf, mb->rho_offf.data(), V, x, y, a);
    return launch_hv<float>(a, mb->sec->half, stream);
}

}  // namespace ftlm
