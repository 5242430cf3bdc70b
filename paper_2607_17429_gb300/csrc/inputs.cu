// Seeded test inputs at any block size, and representative lookup by label.
//
// ftlm_fill_label_keyed writes the label-keyed block vector: the entry (r, k, b)
// depends only on the base-(2s+1) label of representative r (Eq. 2), the row k
// within r and the right-hand side b, through SplitMix64 (Steele, Lea and
// Flood, OOPSLA'14):
//   z = label * 4096 + k * 64 + b + seed * 0x632BE59BD9B4E019   (mod 2^64)
//   value = (splitmix64(z) >> 11) * 2^-52 - 1                    in [-1, 1)
// A checker can regenerate any row from the label alone, without the sector
// table, so rows of a block too large for a host copy can be verified.
// ftlm_basis_rows finds representatives of a block by packed label.
#include <vector>

#include "common.cuh"

namespace ftlm {
namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <typename VT>
__global__ void fill_label_keyed(const uint64_t *labels, const uint16_t *stab_id, const uint8_t *ntab,
                                 const uint64_t *off, uint64_t n_reps, int N, int bits, int d, int B, uint64_t seed,
                                 VT *x) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_reps) return;
    const uint64_t p = labels[i];
    uint64_t lab = 0;  // base-d label of Eq. 2: site N-1 is the most significant digit
    for (int k = N - 1; k >= 0; --k) lab = lab * (uint64_t)d + ((p >> (bits * k)) & ((1ull << bits) - 1));
    const int n = ntab[stab_id[i]];
    const uint64_t o = off[i];
    const uint64_t base = lab * 4096ull + seed * 0x632BE59BD9B4E019ull;
    for (int k = 0; k < n; ++k)
        for (int b = 0; b < B; ++b) {
            const uint64_t h = splitmix64(base + (uint64_t)k * 64ull + (uint64_t)b);
            x[(o + k) * B + b] = (VT)((double)(h >> 11) * 0x1p-52 - 1.0);
        }
}

__global__ void rows_of_labels(const uint64_t *labels, uint64_t n_reps, const uint32_t *bucket, uint64_t n_buckets,
                               int shift, const uint16_t *stab_id, const uint8_t *ntab, const uint64_t *off,
                               const uint64_t *query, int n, int64_t *first, int *nrows) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint64_t key = query[q];
    const uint64_t bk = key >> shift;
    int64_t f = -1;
    int c = 0;
    if (bk < n_buckets) {
        uint32_t lo = bucket[bk], hi = bucket[bk + 1];
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (labels[mid] < key)
                lo = mid + 1;
            else
                hi = mid;
        }
        if (lo < n_reps && labels[lo] == key) {
            f = (int64_t)off[lo];
            c = ntab[stab_id[lo]];
        }
    }
    first[q] = f;
    nrows[q] = c;
}

}  // namespace
}  // namespace ftlm

using namespace ftlm;

extern "C" {

ftlm_status ftlm_fill_label_keyed(const ftlm_basis *b, ftlm_dtype dtype, int B, uint64_t seed, void *x,
                                  void *cuda_stream) {
    if (!b || !x) return fail(FTLM_EINVAL, "NULL argument");
    if (B < 1 || B > 64) return fail(FTLM_EINVAL, "B must be in 1..64 (4096 / 64 rows per label)");
    const ftlm_sector *s = b->sec;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const uint64_t n = s->n_reps;
    if (n == 0) return FTLM_OK;
    count_launch();
    if (dtype == FTLM_F64)
        fill_label_keyed<double><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            s->d_labels, s->d_stab_id, b->d_ntab, b->d_off, n, s->N, s->bits, s->two_s + 1, B, seed, (double *)x);
    else if (dtype == FTLM_F32)
        fill_label_keyed<float><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            s->d_labels, s->d_stab_id, b->d_ntab, b->d_off, n, s->N, s->bits, s->two_s + 1, B, seed, (float *)x);
    else
        return fail(FTLM_EINVAL, "unknown dtype");
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

ftlm_status ftlm_basis_rows(const ftlm_basis *b, int n, const uint64_t *labels, int64_t *first_row, int *n_rows,
                            void *cuda_stream) {
    if (!b || n < 0 || (n && (!labels || !first_row || !n_rows))) return fail(FTLM_EINVAL, "bad arguments");
    if (n == 0) return FTLM_OK;
    const ftlm_sector *s = b->sec;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    DevBuf<uint64_t> dq;
    DevBuf<int64_t> df;
    DevBuf<int> dn;
    FTLM_CUDA(dq.alloc(n));
    FTLM_CUDA(df.alloc(n));
    FTLM_CUDA(dn.alloc(n));
    FTLM_CUDA(cudaMemcpyAsync(dq.p, labels, (size_t)n * 8, cudaMemcpyHostToDevice, st));
    count_launch();
    rows_of_labels<<<(n + 255) / 256, 256, 0, st>>>(s->d_labels, s->n_reps, s->d_bucket, s->n_buckets,
                                                    s->bucket_shift, s->d_stab_id, b->d_ntab, b->d_off, dq.p, n,
                                                    df.p, dn.p);
    FTLM_CUDA(cudaGetLastError());
    FTLM_CUDA(cudaMemcpyAsync(first_row, df.p, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
    FTLM_CUDA(cudaMemcpyAsync(n_rows, dn.p, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
    FTLM_CUDA(cudaStreamSynchronize(st));
    return FTLM_OK;
}

}  // extern "C"
