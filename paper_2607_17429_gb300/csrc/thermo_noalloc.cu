// ftlm_thermo_noalloc: the thermal-sum pipeline (Ritz pairs -> E0 -> Z, E, C, chi)
// for callers that cannot allocate device memory.  Its only scratch, the
// intermediate Ritz values and weights plus an error word, lives in one
// file-scope device array of fixed size instead of cudaMalloc'd buffers.
#include "ritz_thermo.cuh"

namespace ftlm {
namespace {

constexpr size_t kNoAllocEntries = size_t(1) << 19;  // chains x steps held in the fixed scratch (2 x 4 MiB)

// [0, N): Ritz values, [N, 2N): weights, [2N]: error word.  Every GPU that
// loads the library holds this array until the process exits.
static __device__ __align__(256) double g_thermo_scratch[2 * kNoAllocEntries + 32];

// Device address of the scratch in the current context.  Looked up on every
// call, not cached: after a context reset (cudaDeviceReset) the module is
// loaded again and the array may sit at another address.  Under lazy module
// loading the first look-up on a device is what loads the module, and with it
// reserves the array.
ftlm_status scratch_on_current_device(double **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_thermo_scratch);
    if (e != cudaSuccess || !p)
        return fail(FTLM_ECUDA, "cudaGetSymbolAddress of the thermal scratch failed: %s", cudaGetErrorString(e));
    *out = static_cast<double *>(p);
    return FTLM_OK;
}

}  // namespace
}  // namespace ftlm

using namespace ftlm;

extern "C" ftlm_status ftlm_thermo_noalloc(int n_chains, int ld, const int *m, const double *alpha,
                                           const double *beta, const double *weight, const double *msq, int n_T,
                                           const double *T, double g, double *out, double *E0, void *cuda_stream) {
    if (n_chains == 0) {  // warm-up: make the scratch and the three kernels resident on the current device
        double *scr = nullptr;
        ftlm_status st = scratch_on_current_device(&scr);
        if (st != FTLM_OK) return st;
        cudaFuncAttributes fa;  // under lazy loading, querying a kernel loads it
        FTLM_CUDA(cudaFuncGetAttributes(&fa, ritz_kernel));
        FTLM_CUDA(cudaFuncGetAttributes(&fa, ground_energy));
        FTLM_CUDA(cudaFuncGetAttributes(&fa, thermo_kernel));
        return FTLM_OK;
    }
    if (n_chains < 1 || ld < 1 || n_T < 1 || !m || !alpha || !beta || !weight || !msq || !T || !out || !E0)
        return fail(FTLM_EINVAL, "bad arguments");
    if (ld > kMaxSteps) return fail(FTLM_EINVAL, "ld = %d exceeds %d steps", ld, kMaxSteps);
    if ((size_t)n_chains * (size_t)ld > kNoAllocEntries)
        return fail(FTLM_EINVAL, "n_chains * ld = %zu exceeds the fixed scratch of %zu Ritz entries",
                    (size_t)n_chains * (size_t)ld, kNoAllocEntries);
    double *scr = nullptr;
    ftlm_status st = scratch_on_current_device(&scr);
    if (st != FTLM_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double *theta = scr, *w = scr + kNoAllocEntries;
    int *err = reinterpret_cast<int *>(scr + 2 * kNoAllocEntries);
    FTLM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));  // the array keeps the previous call's contents
    count_launch(3);
    ritz_kernel<<<(n_chains + 63) / 64, 64, 0, s>>>(n_chains, ld, m, alpha, beta, theta, w, err);
    ThermoIn in{n_chains, ld, m, theta, w, weight, msq};
    ground_energy<<<1, kThermoThreads, 0, s>>>(in, E0);
    thermo_kernel<<<n_T, kThermoThreads, 0, s>>>(in, T, E0, g, out, n_T);
    FTLM_CUDA(cudaGetLastError());
    int h_err = 0;
    FTLM_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    FTLM_CUDA(cudaStreamSynchronize(s));
    if (h_err) return fail(FTLM_EINTERNAL, "tridiagonal eigensolve failed or steps exceed ld (code %d)", h_err);
    return FTLM_OK;
}
