// Launch counting and H·v timing (CUDA events on the launching stream).
#include <mutex>
#include <vector>

#include "common.cuh"

namespace ftlm {

namespace {
std::mutex g_mu;
std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_on{0};
struct Pending {
    cudaEvent_t a, b;
    uint64_t rows;
};
std::vector<Pending> g_pending;
uint64_t g_hv_launches = 0, g_hv_rows = 0;
double g_hv_ms = 0.0;
unsigned long long *g_flips[256] = {};  // per device: flip counter of the packed H·v
}  // namespace

// Device counter of ladder flips processed by the packed H·v while profiling
// (allocated once per device on first use; null if that fails).
unsigned long long *profile_flip_counter() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_flips[dev]) {
        void *p = nullptr;
        if (cudaMalloc(&p, sizeof(unsigned long long)) != cudaSuccess) return nullptr;
        cudaMemset(p, 0, sizeof(unsigned long long));
        g_flips[dev] = static_cast<unsigned long long *>(p);
    }
    return g_flips[dev];
}

void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
bool profiling_on() { return g_on.load(std::memory_order_relaxed) != 0; }

void hv_timer_begin(cudaStream_t st, cudaEvent_t *a, cudaEvent_t *b) {
    *a = *b = nullptr;
    if (!profiling_on()) return;
    if (cudaEventCreate(a) != cudaSuccess || cudaEventCreate(b) != cudaSuccess) {
        *a = *b = nullptr;
        return;
    }
    cudaEventRecord(*a, st);
}

void hv_timer_end(cudaStream_t st, cudaEvent_t a, cudaEvent_t b, uint64_t rows) {
    if (!a) return;
    cudaEventRecord(b, st);
    std::lock_guard<std::mutex> lk(g_mu);
    g_pending.push_back({a, b, rows});
}

// H·v time measured elsewhere (events recorded inside a captured graph).
void hv_profile_add(double ms, uint64_t rows) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_hv_ms += ms;
    g_hv_rows += rows;
    ++g_hv_launches;
}

}  // namespace ftlm

using namespace ftlm;

extern "C" {

ftlm_status ftlm_profile_enable(int on) {
    g_on.store(on ? 1 : 0);
    return FTLM_OK;
}

ftlm_status ftlm_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &p : g_pending) {
        cudaEventSynchronize(p.b);
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    g_pending.clear();
    g_hv_launches = g_hv_rows = 0;
    g_hv_ms = 0.0;
    g_launches.store(0);
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 256 && g_flips[dev]) {
        cudaDeviceSynchronize();
        cudaMemset(g_flips[dev], 0, sizeof(unsigned long long));
    }
    return FTLM_OK;
}

ftlm_status ftlm_profile_get(ftlm_profile *out) {
    if (!out) return fail(FTLM_EINVAL, "out is NULL");
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &p : g_pending) {
        float ms = 0.f;
        FTLM_CUDA(cudaEventSynchronize(p.b));
        FTLM_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
        g_hv_ms += ms;
        g_hv_rows += p.rows;
        ++g_hv_launches;
    }
    g_pending.clear();
    out->kernel_launches = g_launches.load();
    out->hv_launches = g_hv_launches;
    out->hv_ms = g_hv_ms;
    out->hv_rows = g_hv_rows;
    out->hv_flips = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 256 && g_flips[dev]) {
        unsigned long long f = 0;
        FTLM_CUDA(cudaDeviceSynchronize());
        FTLM_CUDA(cudaMemcpy(&f, g_flips[dev], sizeof(f), cudaMemcpyDeviceToHost));
        out->hv_flips = f;
    }
    return FTLM_OK;
}

}  // extern "C"
