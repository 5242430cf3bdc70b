// Device helpers shared by the CUDA translation units of libftlm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

#define FTLM_CUDA(call)                                                                                   \
    do {                                                                                                  \
        cudaError_t _e = (call);                                                                          \
        if (_e != cudaSuccess)                                                                            \
            return ::ftlm::fail(_e == cudaErrorMemoryAllocation ? FTLM_ENOMEM : FTLM_ECUDA, "%s: %s (%s:%d)", \
                                #call, cudaGetErrorString(_e), __FILE__, __LINE__);                       \
    } while (0)

namespace ftlm {

void hv_timer_begin(cudaStream_t st, cudaEvent_t *a, cudaEvent_t *b);
void hv_timer_end(cudaStream_t st, cudaEvent_t a, cudaEvent_t b, uint64_t rows);

constexpr int kNumSMs = 152;  // GB300; grids are multiples of this
constexpr unsigned kFull = 0xffffffffu;

// Device buffer that frees itself unless released.
template <typename T>
struct DevBuf {
    T *p = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t n) {
        if (p) cudaFree(p);
        p = nullptr;
        return cudaMalloc((void **)&p, (n ? n : 1) * sizeof(T));
    }
    T *release() {
        T *q = p;
        p = nullptr;
        return q;
    }
};

// Exclusive prefix sum (uint64) of n values given by a functor v(i); out[0..n], out[n] = total.
// Three passes: tile sums, scan of tile sums in one block, tile-local scan with carry-in.
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename F>
__global__ void scan_tile_sums(F v, uint64_t n, uint64_t *tile_sums) {
    __shared__ uint64_t warp_sums[kScanThreads / 32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    uint64_t s = 0;
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        uint64_t i = base + (uint64_t)t * kScanThreads + threadIdx.x;
        if (i < n) s += v(i);
    }
    for (int o = 16; o; o >>= 1) s += __shfl_down_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t tot = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) tot += warp_sums[w];
        tile_sums[blockIdx.x] = tot;
    }
}

// In-place exclusive scan of the tile sums by one block (1024 threads), chunk by chunk.
static __global__ void scan_serial_tiles(uint64_t *tile_sums, uint64_t n_tiles) {
    __shared__ uint64_t warp_sums[32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint64_t c0 = 0; c0 < n_tiles; c0 += 1024) {
        const uint64_t i = c0 + threadIdx.x;
        const uint64_t x = i < n_tiles ? tile_sums[i] : 0;
        uint64_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(kFull, incl, o);
            if ((threadIdx.x & 31) >= o) incl += y;
        }
        if ((threadIdx.x & 31) == 31) warp_sums[threadIdx.x >> 5] = incl;
        __syncthreads();
        uint64_t wbase = carry;
        for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) wbase += warp_sums[w];
        if (i < n_tiles) tile_sums[i] = wbase + incl - x;
        __syncthreads();
        if (threadIdx.x == 1023) carry = wbase + incl;
        __syncthreads();
    }
}

template <typename F>
__global__ void scan_tiles(F v, uint64_t n, const uint64_t *tile_offsets, uint64_t *out) {
    __shared__ uint64_t warp_sums[kScanThreads / 32];
    __shared__ uint64_t carry;
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    if (threadIdx.x == 0) carry = tile_offsets[blockIdx.x];
    __syncthreads();
    for (int t = 0; t < kScanItems; ++t) {
        uint64_t i = base + (uint64_t)t * kScanThreads + threadIdx.x;
        uint64_t x = i < n ? v(i) : 0;
        uint64_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(kFull, incl, o);
            if ((threadIdx.x & 31) >= o) incl += y;
        }
        if ((threadIdx.x & 31) == 31) warp_sums[threadIdx.x >> 5] = incl;
        __syncthreads();
        uint64_t wbase = carry;
        for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) wbase += warp_sums[w];
        if (i < n) out[i] = wbase + incl - x;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry = wbase + incl;
        __syncthreads();
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = carry;
}

// Host driver: out must hold n + 1 entries.  Synchronous on stream; returns the total.
template <typename F>
ftlm_status exclusive_scan(F v, uint64_t n, uint64_t *out, cudaStream_t stream, uint64_t *total) {
    const uint64_t n_tiles = (n + kScanTile - 1) / kScanTile;
    if (n_tiles == 0) {
        FTLM_CUDA(cudaMemsetAsync(out, 0, sizeof(uint64_t), stream));
        *total = 0;
        return FTLM_OK;
    }
    DevBuf<uint64_t> tiles;
    FTLM_CUDA(tiles.alloc(n_tiles + 1));
    count_launch(3);
    scan_tile_sums<<<(unsigned)n_tiles, kScanThreads, 0, stream>>>(v, n, tiles.p);
    FTLM_CUDA(cudaGetLastError());
    scan_serial_tiles<<<1, 1024, 0, stream>>>(tiles.p, n_tiles);
    FTLM_CUDA(cudaGetLastError());
    scan_tiles<<<(unsigned)n_tiles, kScanThreads, 0, stream>>>(v, n, tiles.p, out);
    FTLM_CUDA(cudaGetLastError());
    FTLM_CUDA(cudaMemcpyAsync(total, out + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, stream));
    FTLM_CUDA(cudaStreamSynchronize(stream));
    return FTLM_OK;
}

}  // namespace ftlm
