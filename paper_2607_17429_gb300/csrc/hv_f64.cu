// F64 instantiation of the per-block-layout multi-block H·v kernel (ftlm_hv_multi).
#include "hv_kernel.cuh"

namespace ftlm {

ftlm_status hv_multi_launch_f64(const ftlm_multiblock *mb, int B, const double *const *x, double *const *y,
                               cudaStream_t stream) {
    for (int k = 0; k < mb->K; ++k)  // this per-block layout kernel is specialised for d_Gamma <= 5
        if (mb->blocks[k]->d > 5)
            return fail(FTLM_EUNSUPPORTED, "d_Gamma = %d needs the packed layout (ftlm_hv_packed)", mb->blocks[k]->d);
    HvArgs<double> a;
    const double *V[kMaxK];
    for (int k = 0; k < mb->K; ++k) V[k] = mb->blocks[k]->d_V;
    fill_hv_args<double>(mb->sec, B, mb->K, mb->blocks.data(), mb->d_offm, mb->d_ntab, mb->blocks[0]->d_sqrtS,
                      mb->d_rhoT, mb->rho_total, mb->rho_off.data(), V, x, y, a);
    return launch_hv<double>(a, mb->sec->half, stream);
}

}  // namespace ftlm
