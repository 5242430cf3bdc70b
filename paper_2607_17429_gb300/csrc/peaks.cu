// Roofline denominators measured on the device the library runs on.
//
// The H·v kernel mixes integer work (the representative search: XOR or add of a
// precomputed image with a per-bond delta, then an unsigned min), shared-memory
// table loads, FP32/FP64 FMAs (the Eq. 15 contraction) and random gathers of
// block-vector rows.  Which of these binds depends on the configuration, so each
// one gets a probe that measures its sustained rate with the clocks and the
// power state of the moment:
//   FTLM_PEAK_LOP3, _MIN_U32, _ADD_U64 : integer lane-operations per second
//   FTLM_PEAK_FFMA32, _DFMA64          : fused multiply-adds per second (lanes)
//   FTLM_PEAK_LDS32                    : conflict-free 32-bit shared loads per second (lanes)
//   FTLM_PEAK_GATHER                   : bytes per second of random, aligned
//                                        segments of `seg` bytes read from a
//                                        buffer of `span` bytes (LDG.128 per lane)
//   FTLM_PEAK_STREAM                   : bytes per second of a read+write copy
//                                        of `span` bytes (the STREAM copy kernel)
// Every probe runs a fixed grid of 4 CTAs per SM, warms up once and is timed with
// CUDA events on the caller's stream.
#include <stdint.h>

#include <algorithm>

#include "common.cuh"

namespace ftlm {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

template <int OP>
__global__ void alu_probe(uint32_t seed, int iters, uint32_t *sink) {
    uint32_t a[kChains], b[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        a[c] = seed * (threadIdx.x + 7 * c + 1) + blockIdx.x;
        b[c] = seed ^ (0x9E3779B9u * (c + 1));
    }
    uint64_t q[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) q[c] = ((uint64_t)a[c] << 32) | b[c];
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (OP == 0) {
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[c]) : "r"(b[c]), "r"(seed));
            } else if (OP == 1) {
                asm volatile("min.u32 %0, %0, %1;" : "+r"(a[c]) : "r"(b[c]));
            } else {
                asm volatile("add.u64 %0, %0, %1;" : "+l"(q[c]) : "l"((uint64_t)b[c] | 1ull));
            }
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc ^= a[c] ^ b[c] ^ (uint32_t)q[c] ^ (uint32_t)(q[c] >> 32);
    if (acc == 0x12345678u) sink[0] = acc;  // practically never: defeats dead-code elimination
}

template <typename T>
__global__ void fma_probe(T seed, int iters, T *sink) {
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (T)(threadIdx.x * 0.001 + c);
    const T m = (T)0.999999, s = (T)1e-7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = a[c] * m + s;
    }
    T acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += a[c];
    if (acc == (T)-1.2345) sink[0] = acc;
}

__global__ void lds_probe(int iters, uint32_t *sink) {
    __shared__ uint32_t tab[4096];
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) tab[i] = (uint32_t)(i * 2654435761u) & 0xfe0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(tab);
    uint32_t idx[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) idx[c] = (uint32_t)(c * 512);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            // row base from the previous load (a multiple of 32 words), lane-consecutive words
            uint32_t v;
            const uint32_t addr = base + 4u * ((idx[c] + (uint32_t)lane) & 4095u);
            asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
            idx[c] = (v + 32u * (uint32_t)c) & 4064u;
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc ^= idx[c];
    if (acc == 0x7fffffffu) sink[0] = acc;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// One warp per segment at a time; 16-byte loads, seg/16 per segment spread over the lanes.
// Segment indices are hashed and masked to a power-of-two count (no integer division).
__global__ void gather_probe(const uint4 *buf, uint64_t seg_mask, int seg_u4, int per_warp, uint32_t *sink) {
    const int lane = threadIdx.x & 31;
    const uint64_t wg = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t acc = 0;
    for (int it = 0; it < per_warp; it += 4) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {  // four independent segments in flight per warp
            const uint64_t s = mix64(wg * 0x100000001ull + (uint64_t)(it + u)) & seg_mask;
            const uint4 *p = buf + s * (uint64_t)seg_u4;
            v[u] = make_uint4(0, 0, 0, 0);
            for (int q = lane; q < seg_u4; q += 32) {
                const uint4 t = __ldcg(p + q);
                v[u].x ^= t.x;
                v[u].y ^= t.y;
                v[u].z ^= t.z;
                v[u].w ^= t.w;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
    if (acc == 0x13572468u) sink[0] = acc;
}

// Segments of at most 64 bytes: every lane gathers its own segments (four in flight), as the
// one-thread-per-representative H·v does with its 8..60-byte rows.
__global__ void gather_lane_probe(const uint4 *buf, uint64_t seg_mask, int seg_u4, int per_lane, uint32_t *sink) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (int it = 0; it < per_lane; it += 4) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t s = mix64(t * 0x100000001ull + (uint64_t)(it + u)) & seg_mask;
            const uint4 *p = buf + s * (uint64_t)seg_u4;
            v[u] = __ldcg(p);
            for (int q = 1; q < seg_u4; ++q) {
                const uint4 w = __ldcg(p + q);
                v[u].x ^= w.x;
                v[u].y ^= w.y;
                v[u].z ^= w.z;
                v[u].w ^= w.w;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
    if (acc == 0x13572468u) sink[0] = acc;
}

__global__ void copy_probe(const uint4 *src, uint4 *dst, uint64_t n) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = __ldcs(src + i);
}

template <typename F>
ftlm_status time_it(F launch, cudaStream_t st, double *ms) {
    cudaEvent_t a, b;
    FTLM_CUDA(cudaEventCreate(&a));
    FTLM_CUDA(cudaEventCreate(&b));
    launch();  // warm-up
    FTLM_CUDA(cudaGetLastError());
    FTLM_CUDA(cudaEventRecord(a, st));
    launch();
    FTLM_CUDA(cudaEventRecord(b, st));
    FTLM_CUDA(cudaEventSynchronize(b));
    float f = 0.f;
    FTLM_CUDA(cudaEventElapsedTime(&f, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms = f;
    return FTLM_OK;
}

}  // namespace
}  // namespace ftlm

using namespace ftlm;

extern "C" ftlm_status ftlm_peak_probe(int kind, uint64_t span, int seg, void *cuda_stream, double *rate) {
    if (!rate) return fail(FTLM_EINVAL, "rate is NULL");
    *rate = 0.0;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = kNumSMs;
    FTLM_CUDA(cudaGetDevice(&dev));
    FTLM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * 4;
    const double lanes = (double)grid * kProbeThreads;
    DevBuf<uint32_t> sink;
    FTLM_CUDA(sink.alloc(4));
    double ms = 0.0;
    ftlm_status s = FTLM_OK;
    switch (kind) {
        case FTLM_PEAK_LOP3:
        case FTLM_PEAK_MIN_U32:
        case FTLM_PEAK_ADD_U64: {
            const int iters = 1 << 16;
            auto go = [&] {
                if (kind == FTLM_PEAK_LOP3) alu_probe<0><<<grid, kProbeThreads, 0, st>>>(12345u, iters, sink.p);
                if (kind == FTLM_PEAK_MIN_U32) alu_probe<1><<<grid, kProbeThreads, 0, st>>>(12345u, iters, sink.p);
                if (kind == FTLM_PEAK_ADD_U64) alu_probe<2><<<grid, kProbeThreads, 0, st>>>(12345u, iters, sink.p);
            };
            if ((s = time_it(go, st, &ms)) != FTLM_OK) return s;
            *rate = lanes * iters * kChains / (ms * 1e-3);
            break;
        }
        case FTLM_PEAK_FFMA32: {
            const int iters = 1 << 16;
            DevBuf<float> fs;
            FTLM_CUDA(fs.alloc(1));
            auto go = [&] { fma_probe<float><<<grid, kProbeThreads, 0, st>>>(1.0f, iters, fs.p); };
            if ((s = time_it(go, st, &ms)) != FTLM_OK) return s;
            *rate = lanes * iters * kChains / (ms * 1e-3);
            break;
        }
        case FTLM_PEAK_DFMA64: {
            const int iters = 1 << 12;
            DevBuf<double> ds;
            FTLM_CUDA(ds.alloc(1));
            auto go = [&] { fma_probe<double><<<grid, kProbeThreads, 0, st>>>(1.0, iters, ds.p); };
            if ((s = time_it(go, st, &ms)) != FTLM_OK) return s;
            *rate = lanes * iters * kChains / (ms * 1e-3);
            break;
        }
        case FTLM_PEAK_LDS32: {
            const int iters = 1 << 14;
            auto go = [&] { lds_probe<<<grid, kProbeThreads, 0, st>>>(iters, sink.p); };
            if ((s = time_it(go, st, &ms)) != FTLM_OK) return s;
            *rate = lanes * iters * kChains / (ms * 1e-3);
            break;
        }
        case FTLM_PEAK_GATHER: {
            if (seg < 16 || seg % 16 || span < (uint64_t)seg || span > (64ull << 30))
                return fail(FTLM_EINVAL, "gather probe: seg a multiple of 16, seg <= span <= 64 GiB");
            DevBuf<uint4> buf;
            FTLM_CUDA(buf.alloc(span / 16));
            FTLM_CUDA(cudaMemsetAsync(buf.p, 0x5a, span / 16 * 16, st));
            uint64_t n_seg = 1;
            while (2 * n_seg <= span / (uint64_t)seg) n_seg *= 2;
            if (seg <= 64) {  // one segment per lane: about 1 GB of segments per timed launch
                const uint64_t lanes_all = (uint64_t)grid * kProbeThreads;
                int per_lane = (int)std::min<uint64_t>(1 << 12, ((1ull << 30) / (uint64_t)seg + lanes_all - 1) / lanes_all);
                per_lane = (per_lane + 3) & ~3;
                auto go = [&] {
                    gather_lane_probe<<<grid, kProbeThreads, 0, st>>>(buf.p, n_seg - 1, seg / 16, per_lane, sink.p);
                };
                if ((s = time_it(go, st, &ms)) != FTLM_OK) return s;
                *rate = (double)lanes_all * per_lane * seg / (ms * 1e-3);
                break;
            }
            const int warps = grid * kProbeThreads / 32;
            // about 4 GB of segments per timed launch
            int per_warp = (int)std::min<uint64_t>(1 << 16, ((4ull << 30) / (uint64_t)seg + warps - 1) / warps);
            per_warp = (per_warp + 3) & ~3;
            auto go = [&] { gather_probe<<<grid, kProbeThreads, 0, st>>>(buf.p, n_seg - 1, seg / 16, per_warp, sink.p); };
            if ((s = time_it(go, st, &ms)) != FTLM_OK) return s;
            *rate = (double)warps * per_warp * seg / (ms * 1e-3);
            break;
        }
        case FTLM_PEAK_STREAM: {
            if (span < 16 || span > (64ull << 30)) return fail(FTLM_EINVAL, "stream probe: 16 B <= span <= 64 GiB");
            DevBuf<uint4> a, b;
            FTLM_CUDA(a.alloc(span / 16));
            FTLM_CUDA(b.alloc(span / 16));
            FTLM_CUDA(cudaMemsetAsync(a.p, 1, span / 16 * 16, st));
            auto go = [&] { copy_probe<<<grid, kProbeThreads * 4, 0, st>>>(a.p, b.p, span / 16); };
            if ((s = time_it(go, st, &ms)) != FTLM_OK) return s;
            *rate = 2.0 * (double)(span / 16 * 16) / (ms * 1e-3);
            break;
        }
        default:
            return fail(FTLM_EINVAL, "unknown probe kind %d", kind);
    }
    count_launch(2);
    FTLM_CUDA(cudaStreamSynchronize(st));
    return FTLM_OK;
}
