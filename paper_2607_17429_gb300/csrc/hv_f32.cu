// FP32 instantiations of the H·v kernel (mixed-precision path: FP32 vectors and arithmetic).
#include "hv_impl.cuh"

namespace ftlm {
ftlm_status hv_launch_f32(const ftlm_basis *bs, int B, const float *x, float *y, cudaStream_t stream) {
    HvArgs<float> a;
    fill_hv_args<float>(bs, B, a, bs->d_sqrtSf, bs->d_Vf, bs->d_rhoTf);
    a.bonds = bs->sec->d_bonds;
    return launch_hv<float>(a, bs->sec->half, x, y, stream);
}
}  // namespace ftlm
