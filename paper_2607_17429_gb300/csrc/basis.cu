// Sector and block preparation on the GPU (Sections 2.3 and 3 of arXiv 2607.17429).
//
// Sector (irrep independent, Section 3's first phase):
//   enumerate the S^z sector (digit sum A = N s + M, Section 2.1) in ascending
//   label order by unranking chunk starts and stepping to the next label with
//   the same digit sum; keep a label when no group element maps it to a smaller
//   one (orbit minimum, Section 2.3); its stabilizer (Eq. 8) is the set of
//   elements that fix it.  Two passes (count, then write at prefix-sum offsets)
//   keep the table sorted without a sort.  Stabilizer subgroups get small ids
//   (0 = trivial).  A bucket index on the high label bits serves the lookup.
// Block (irrep dependent, second phase): per stabilizer id n_Gamma (character
//   count), V_r (Eq. 11) and sqrt|Stab|; per representative the row offset
//   (Eq. 13 prefix sum).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "common.cuh"
#include "contract.cuh"

namespace ftlm {

namespace {

constexpr int kEnumThreads = 256;

struct EnumArgs {
    int N, bits, dmax, A, G;  // G: elements acting on the sector (2|G| with the spin flip)
    uint64_t dim;          // sector dimension
    uint64_t chunk;        // labels per thread
    uint64_t n_threads;    // total threads
    const uint64_t *cnt;   // [(N+1)][(A+1)] ways for k low digits to sum to a
    const uint8_t *src;    // [G][N] src[g][t] = pi_g^{-1}(t), + N when g also flips the spin
};

__device__ __forceinline__ unsigned digit(uint64_t n, int k, int bits, unsigned dmask) {
    return (unsigned)(n >> (bits * k)) & dmask;
}

// label of the given rank (ascending order) among digit strings with sum A
__device__ uint64_t unrank(const EnumArgs &a, uint64_t rank) {
    uint64_t n = 0;
    int rem = a.A;
    for (int t = a.N - 1; t >= 0; --t) {
        int v = 0;
        for (; v <= a.dmax && v <= rem; ++v) {
            uint64_t c = a.cnt[t * (a.A + 1) + (rem - v)];
            if (rank < c) break;
            rank -= c;
        }
        n |= (uint64_t)v << (a.bits * t);
        rem -= v;
    }
    return n;
}

// next larger label with the same digit sum
__device__ uint64_t next_label(const EnumArgs &a, uint64_t n) {
    const unsigned dmask = (1u << a.bits) - 1;
    int below = 0, p = 0;
    for (; p < a.N; ++p) {
        unsigned v = digit(n, p, a.bits, dmask);
        if (v < (unsigned)a.dmax && below > 0) break;
        below += v;
    }
    if (p >= a.N) return ~0ull;
    const int sh = a.bits * (p + 1);
    const uint64_t hi = sh < 64 ? (n >> sh) << sh : 0;  // digits above position p are kept
    unsigned vp = digit(n, p, a.bits, dmask) + 1;
    uint64_t m = hi | ((uint64_t)vp << (a.bits * p));
    int rest = below - 1;
    for (int t = 0; t < p && rest > 0; ++t) {
        int v = rest < a.dmax ? rest : a.dmax;
        m |= (uint64_t)v << (a.bits * t);
        rest -= v;
    }
    return m;
}

// 0: not a representative; 1: representative with trivial stabilizer; 2: with nontrivial one.
// mask (if non-null) receives the stabilizer bitmask.
__device__ int rep_test(const EnumArgs &a, const uint8_t *src, uint64_t n, uint64_t *mask) {
    const unsigned dmask = (1u << a.bits) - 1;
    int nontrivial = 0;
    if (mask) {
        mask[0] = 1;
        mask[1] = mask[2] = mask[3] = 0;
    }
    for (int g = 1; g < a.G; ++g) {
        const uint8_t *s = src + g * a.N;
        int t = a.N - 1;
        unsigned u = 0, v = 0;
        for (; t >= 0; --t) {
            const int sk = s[t];
            u = sk < a.N ? digit(n, sk, a.bits, dmask) : (unsigned)a.dmax - digit(n, sk - a.N, a.bits, dmask);
            v = digit(n, t, a.bits, dmask);
            if (u != v) break;
        }
        if (t < 0) {
            nontrivial = 1;
            if (mask) mask[g >> 6] |= 1ull << (g & 63);
        } else if (u < v) {
            return 0;
        }
    }
    return 1 + nontrivial;
}

__global__ void enum_count(EnumArgs a, uint32_t *counts, unsigned long long *n_nontrivial) {
    extern __shared__ uint8_t s_src[];
    for (int i = threadIdx.x; i < a.G * a.N; i += blockDim.x) s_src[i] = a.src[i];
    __syncthreads();
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned c = 0, nt = 0;
    if (t < a.n_threads) {
        uint64_t r0 = t * a.chunk, r1 = min(r0 + a.chunk, a.dim);
        uint64_t n = unrank(a, r0);
        for (uint64_t r = r0; r < r1; ++r) {
            int k = rep_test(a, s_src, n, nullptr);
            c += k > 0;
            nt += k == 2;
            if (r + 1 < r1) n = next_label(a, n);
        }
        counts[t] = c;
    }
    for (int o = 16; o; o >>= 1) nt += __shfl_down_sync(kFull, nt, o);
    if ((threadIdx.x & 31) == 0 && nt) atomicAdd(n_nontrivial, (unsigned long long)nt);
}

__global__ void enum_write(EnumArgs a, const uint64_t *offsets, uint64_t *labels, unsigned long long *side_count,
                           uint64_t *side, unsigned long long side_cap) {
    extern __shared__ uint8_t s_src[];
    for (int i = threadIdx.x; i < a.G * a.N; i += blockDim.x) s_src[i] = a.src[i];
    __syncthreads();
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_threads) return;
    uint64_t pos = offsets[t];
    uint64_t r0 = t * a.chunk, r1 = min(r0 + a.chunk, a.dim);
    uint64_t n = unrank(a, r0);
    uint64_t mask[4];
    for (uint64_t r = r0; r < r1; ++r) {
        int k = rep_test(a, s_src, n, mask);
        if (k) {
            labels[pos] = n;
            if (k == 2) {
                unsigned long long q = atomicAdd(side_count, 1ull);
                if (q < side_cap) {
                    side[5 * q] = pos;
                    for (int w = 0; w < 4; ++w) side[5 * q + 1 + w] = mask[w];
                }
            }
            ++pos;
        }
        if (r + 1 < r1) n = next_label(a, n);
    }
}

// masks as 4-word keys compared from the highest word down (the host sorts them the same way)
__device__ __forceinline__ bool mask_less(const uint64_t *a, const uint64_t *b) {
    for (int w = 3; w >= 0; --w)
        if (a[w] != b[w]) return a[w] < b[w];
    return false;
}

__global__ void assign_stab_ids(const uint64_t *side, uint64_t n_side, const uint64_t *masks, int n_masks,
                                uint16_t *stab_id) {
    const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_side) return;
    const uint64_t *m = side + 5 * q + 1;
    int lo = 0, hi = n_masks;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (mask_less(masks + 4 * mid, m))
            lo = mid + 1;
        else
            hi = mid;
    }
    stab_id[side[5 * q]] = (uint16_t)(lo + 1);
}

__global__ void build_buckets(const uint64_t *labels, uint64_t n_reps, int shift, uint64_t n_buckets,
                              uint32_t *bucket) {
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b > n_buckets) return;
    if (b == n_buckets) {
        bucket[b] = (uint32_t)n_reps;
        return;
    }
    const uint64_t key = shift >= 64 ? 0 : (b << shift);
    uint64_t lo = 0, hi = n_reps;
    while (lo < hi) {
        uint64_t mid = (lo + hi) >> 1;
        if (labels[mid] < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    bucket[b] = (uint32_t)lo;
}

struct NGammaOf {
    const uint16_t *stab_id;
    const uint8_t *ntab;
    __device__ uint64_t operator()(uint64_t i) const { return ntab[stab_id[i]]; }
};

struct CountsOf {
    const uint32_t *counts;
    __device__ uint64_t operator()(uint64_t i) const { return counts[i]; }
};

int bits_for(int two_s) {
    int b = 1;
    while ((1 << b) < two_s + 1) ++b;
    return b;
}

void free_sector(ftlm_sector *s) {
    if (!s) return;
    cudaFree(s->d_labels);
    cudaFree(s->d_stab_id);
    cudaFree(s->d_bucket);
    cudaFree(s->d_lut);
    cudaFree(s->d_lut2);
    cudaFree(s->d_pos);
    cudaFree(s->d_dtab);
    cudaFree(s->d_bonds);
    cudaFree(s->d_err);
    cudaFree(s->d_eoff);
    cudaFree(s->d_ent);
    delete s;
}

ftlm_status build_search_tables(ftlm_sector *s) {
    const int N = s->N, G = s->G, nb = s->grp.n_bonds();
    const int32_t *P = s->grp.perms.data();
    std::vector<uint8_t> bnd(2 * nb);
    for (int t = 0; t < 2 * nb; ++t) bnd[t] = (uint8_t)s->grp.bonds[t];
    FTLM_CUDA(cudaMalloc((void **)&s->d_bonds, bnd.size() + 1));
    FTLM_CUDA(cudaMemcpy(s->d_bonds, bnd.data(), bnd.size(), cudaMemcpyHostToDevice));
    auto pi = [&](int g, int k) { return P[(size_t)(g < G ? g : 0) * N + k]; };  // padded with the identity
    if (s->half) {
        s->n_chunks = (N + 3) / 4;
        std::vector<uint32_t> lut((size_t)s->n_chunks * 16 * kMaxG, 0);
        for (int c = 0; c < s->n_chunks; ++c)
            for (int v = 0; v < 16; ++v)
                for (int g = 0; g < kMaxG; ++g) {
                    uint32_t img = 0;
                    for (int t = 0; t < 4; ++t)
                        if (((v >> t) & 1) && 4 * c + t < N) img |= 1u << pi(g, 4 * c + t);
                    lut[((size_t)c * 16 + v) * kMaxG + g] = img;
                }
        std::vector<uint32_t> dt((size_t)nb * kMaxG);
        for (int e = 0; e < nb; ++e)
            for (int g = 0; g < kMaxG; ++g)
                dt[(size_t)e * kMaxG + g] = (1u << pi(g, s->grp.bonds[2 * e])) | (1u << pi(g, s->grp.bonds[2 * e + 1]));
        FTLM_CUDA(cudaMalloc((void **)&s->d_lut, lut.size() * 4));
        s->n_chunks2 = (N + 1) / 2;  // 2-site chunks for the packed kernel
        std::vector<uint32_t> lut2((size_t)s->n_chunks2 * 4 * kMaxG, 0);
        for (int c = 0; c < s->n_chunks2; ++c)
            for (int v = 0; v < 4; ++v)
                for (int g = 0; g < kMaxG; ++g) {
                    uint32_t img = 0;
                    for (int t = 0; t < 2; ++t)
                        if (((v >> t) & 1) && 2 * c + t < N) img |= 1u << pi(g, 2 * c + t);
                    lut2[((size_t)c * 4 + v) * kMaxG + g] = img;
                }
        FTLM_CUDA(cudaMalloc((void **)&s->d_lut2, lut2.size() * 4));
        FTLM_CUDA(cudaMemcpy(s->d_lut2, lut2.data(), lut2.size() * 4, cudaMemcpyHostToDevice));
        s->device_bytes += lut2.size() * 4;
        FTLM_CUDA(cudaMemcpy(s->d_lut, lut.data(), lut.size() * 4, cudaMemcpyHostToDevice));
        FTLM_CUDA(cudaMalloc(&s->d_dtab, dt.size() * 4));
        FTLM_CUDA(cudaMemcpy(s->d_dtab, dt.data(), dt.size() * 4, cudaMemcpyHostToDevice));
        s->device_bytes += lut.size() * 4 + dt.size() * 4;
    } else {
        std::vector<uint8_t> pos((size_t)kMaxG * 64, 0);
        for (int g = 0; g < kMaxG; ++g)
            for (int k = 0; k < N; ++k) pos[(size_t)g * 64 + k] = (uint8_t)(s->bits * pi(g, k));
        std::vector<int64_t> dt((size_t)nb * kMaxG);
        for (int e = 0; e < nb; ++e)
            for (int g = 0; g < kMaxG; ++g) {
                uint64_t ui = 1ull << (s->bits * pi(g, s->grp.bonds[2 * e]));
                uint64_t uj = 1ull << (s->bits * pi(g, s->grp.bonds[2 * e + 1]));
                dt[(size_t)e * kMaxG + g] = (int64_t)(ui - uj);
            }
        FTLM_CUDA(cudaMalloc((void **)&s->d_pos, pos.size()));
        FTLM_CUDA(cudaMemcpy(s->d_pos, pos.data(), pos.size(), cudaMemcpyHostToDevice));
        FTLM_CUDA(cudaMalloc(&s->d_dtab, dt.size() * 8));
        FTLM_CUDA(cudaMemcpy(s->d_dtab, dt.data(), dt.size() * 8, cudaMemcpyHostToDevice));
        s->device_bytes += pos.size() + dt.size() * 8;
    }
    return FTLM_OK;
}

// G x Z_2 (the spin flip at M = 0, Section 2.2) as a group acting on labels: element g + z|G| is
// the signed permutation pi_g(k) + z N; irreps Gamma_i+ (2i: rho(g, z) = rho(g)) and Gamma_i-
// (2i + 1: rho(g, z) = (-1)^z rho(g)), interleaved as the canonical irrep order puts them.
GroupData spin_flip_extension(const GroupData &g) {
    GroupData x = g;
    const int G = g.G, N = g.N;
    x.G = 2 * G;
    x.perms.resize((size_t)2 * G * N);
    for (size_t i = 0; i < (size_t)G * N; ++i) x.perms[(size_t)G * N + i] = g.perms[i] + N;
    x.inv.resize(2 * G);
    for (int i = 0; i < G; ++i) x.inv[G + i] = g.inv[i] + G;
    x.mult.assign((size_t)4 * G * G, 0);
    for (int z = 0; z < 2; ++z)
        for (int w = 0; w < 2; ++w)
            for (int i = 0; i < G; ++i)
                for (int j = 0; j < G; ++j)
                    x.mult[(size_t)(i + z * G) * 2 * G + (j + w * G)] = g.mult[(size_t)i * G + j] + (z ^ w) * G;
    x.irreps.clear();
    for (const Irrep &ir : g.irreps)
        for (int sgn = 1; sgn >= -1; sgn -= 2) {
            Irrep e;
            e.dim = ir.dim;
            e.fs = ir.fs;
            e.chars.resize(2 * G);
            for (int i = 0; i < G; ++i) e.chars[i] = ir.chars[i], e.chars[G + i] = sgn * ir.chars[i];
            if (!ir.rho.empty()) {
                const size_t dd = (size_t)ir.dim * ir.dim;
                e.rho.resize(2 * G * dd);
                for (size_t t = 0; t < G * dd; ++t) e.rho[t] = ir.rho[t], e.rho[G * dd + t] = sgn * ir.rho[t];
            }
            x.irreps.push_back(std::move(e));
        }
    return x;
}

ftlm_status build_sector_impl(const GroupData &grp_in, int two_s, int two_M, int flip, cudaStream_t stream,
                              ftlm_sector *s) {
    const int N = grp_in.N, G = grp_in.G;
    if (two_s < 1) return fail(FTLM_EINVAL, "two_s must be >= 1");
    if (flip && two_M != 0) return fail(FTLM_EINVAL, "the spin flip is a symmetry of the M = 0 sector only");
    const GroupData grp = flip ? spin_flip_extension(grp_in) : grp_in;
    const int GX = grp.G;  // elements acting on labels
    if ((N * two_s + two_M) % 2) return fail(FTLM_EINVAL, "N s + M is not an integer");
    const int A = (N * two_s + two_M) / 2;
    if (A < 0 || A > N * two_s) return fail(FTLM_EINVAL, "M out of range");
    const int bits = bits_for(two_s);
    if (N * bits > 64) return fail(FTLM_EUNSUPPORTED, "N * bits = %d exceeds 64", N * bits);
    if (G > kMaxG) return fail(FTLM_EUNSUPPORTED, "|G| = %d exceeds %d on the GPU path", G, kMaxG);
    if (grp.n_bonds() > kMaxBonds) return fail(FTLM_EUNSUPPORTED, "more than %d bonds", kMaxBonds);
    s->grp = grp;
    s->two_s = two_s;
    s->two_M = two_M;
    s->bits = bits;
    s->N = N;
    s->G = G;
    s->A = A;
    s->flip = flip;
    s->half = (two_s == 1 && N <= 32);
    s->flipc = 0;
    for (int k = 0; k < N; ++k) s->flipc |= (uint64_t)two_s << (bits * k);
    // counting table: cnt[k][a] = #strings of k digits (0..2s) with sum a
    std::vector<uint64_t> cnt((size_t)(N + 1) * (A + 1), 0);
    cnt[0] = 1;
    for (int k = 1; k <= N; ++k)
        for (int a = 0; a <= A; ++a) {
            uint64_t v = 0;
            for (int t = 0; t <= two_s && t <= a; ++t) v += cnt[(size_t)(k - 1) * (A + 1) + (a - t)];
            cnt[(size_t)k * (A + 1) + a] = v;
        }
    s->sector_dim = cnt[(size_t)N * (A + 1) + A];
    std::vector<uint8_t> src((size_t)GX * N);
    for (int g = 0; g < GX; ++g)
        for (int k = 0; k < N; ++k) {
            const int p = grp.perms[(size_t)g * N + k];  // >= N: the digit is also flipped
            src[(size_t)g * N + (p % N)] = (uint8_t)(k + (p >= N ? N : 0));
        }
    FTLM_CUDA(cudaMalloc((void **)&s->d_err, sizeof(int)));
    FTLM_CUDA(cudaMemset(s->d_err, 0, sizeof(int)));
    s->device_bytes += sizeof(int);
    {
        ftlm_status st = build_search_tables(s);
        if (st != FTLM_OK) return st;
    }
    if (s->sector_dim == 0) return fail(FTLM_EINVAL, "empty sector");
    DevBuf<uint64_t> d_cnt;
    DevBuf<uint8_t> d_src;
    FTLM_CUDA(d_cnt.alloc(cnt.size()));
    FTLM_CUDA(d_src.alloc(src.size()));
    FTLM_CUDA(cudaMemcpyAsync(d_cnt.p, cnt.data(), cnt.size() * 8, cudaMemcpyHostToDevice, stream));
    FTLM_CUDA(cudaMemcpyAsync(d_src.p, src.data(), src.size(), cudaMemcpyHostToDevice, stream));
    EnumArgs ea;
    ea.N = N;
    ea.bits = bits;
    ea.dmax = two_s;
    ea.A = A;
    ea.G = GX;
    ea.dim = s->sector_dim;
    ea.chunk = s->sector_dim > (1ull << 32) ? 256 : 32;
    ea.n_threads = (s->sector_dim + ea.chunk - 1) / ea.chunk;
    ea.cnt = d_cnt.p;
    ea.src = d_src.p;
    const uint64_t n_blocks = (ea.n_threads + kEnumThreads - 1) / kEnumThreads;
    const size_t smem = (size_t)GX * N;
    DevBuf<uint32_t> counts;
    DevBuf<uint64_t> offsets;
    DevBuf<unsigned long long> nontriv;
    FTLM_CUDA(counts.alloc(ea.n_threads));
    FTLM_CUDA(offsets.alloc(ea.n_threads + 1));
    FTLM_CUDA(nontriv.alloc(2));
    FTLM_CUDA(cudaMemsetAsync(nontriv.p, 0, 2 * sizeof(unsigned long long), stream));
    count_launch();
    enum_count<<<(unsigned)n_blocks, kEnumThreads, smem, stream>>>(ea, counts.p, nontriv.p);
    FTLM_CUDA(cudaGetLastError());
    uint64_t n_reps = 0;
    {
        ftlm_status st = exclusive_scan(CountsOf{counts.p}, ea.n_threads, offsets.p, stream, &n_reps);
        if (st != FTLM_OK) return st;
    }
    if (n_reps >= 0xffffffffull) return fail(FTLM_EUNSUPPORTED, "more than 2^32-1 representatives");
    unsigned long long n_side = 0;
    FTLM_CUDA(cudaMemcpyAsync(&n_side, nontriv.p, sizeof(n_side), cudaMemcpyDeviceToHost, stream));
    FTLM_CUDA(cudaStreamSynchronize(stream));
    s->n_reps = n_reps;
    FTLM_CUDA(cudaMalloc((void **)&s->d_labels, n_reps * 8));
    FTLM_CUDA(cudaMalloc((void **)&s->d_stab_id, n_reps * 2));
    s->device_bytes += n_reps * 10;
    FTLM_CUDA(cudaMemsetAsync(s->d_stab_id, 0, n_reps * 2, stream));
    DevBuf<uint64_t> side;
    FTLM_CUDA(side.alloc(5 * n_side + 5));
    FTLM_CUDA(cudaMemsetAsync(nontriv.p, 0, sizeof(unsigned long long), stream));
    count_launch();
    enum_write<<<(unsigned)n_blocks, kEnumThreads, smem, stream>>>(ea, offsets.p, s->d_labels, nontriv.p, side.p,
                                                                   n_side);
    FTLM_CUDA(cudaGetLastError());
    // stabilizer subgroups: dedupe masks on the host, ids ordered by mask
    std::vector<uint64_t> h_side(5 * n_side);
    if (n_side)
        FTLM_CUDA(cudaMemcpyAsync(h_side.data(), side.p, h_side.size() * 8, cudaMemcpyDeviceToHost, stream));
    FTLM_CUDA(cudaStreamSynchronize(stream));
    std::vector<std::array<uint64_t, 4>> uniq;  // (m3, m2, m1, m0): the device's comparison order
    for (unsigned long long q = 0; q < n_side; ++q)
        uniq.push_back({h_side[5 * q + 4], h_side[5 * q + 3], h_side[5 * q + 2], h_side[5 * q + 1]});
    std::sort(uniq.begin(), uniq.end());
    uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
    if (uniq.size() + 1 > 65535) return fail(FTLM_EUNSUPPORTED, "too many stabilizer subgroups");
    s->stab_masks.clear();
    s->stab_elems.clear();
    s->stab_masks.push_back({1ull, 0ull, 0ull, 0ull});
    s->stab_elems.push_back({0});
    std::vector<uint64_t> masks_flat;
    for (auto &u : uniq) {
        const std::array<uint64_t, 4> m = {u[3], u[2], u[1], u[0]};  // word w holds elements 64w..64w+63
        s->stab_masks.push_back(m);
        std::vector<int> el;
        for (int g = 0; g < GX; ++g)
            if ((m[g >> 6] >> (g & 63)) & 1) el.push_back(g);
        s->stab_elems.push_back(el);
        for (int w = 0; w < 4; ++w) masks_flat.push_back(m[w]);
    }
    if (n_side) {
        DevBuf<uint64_t> d_masks;
        FTLM_CUDA(d_masks.alloc(masks_flat.size()));
        FTLM_CUDA(cudaMemcpyAsync(d_masks.p, masks_flat.data(), masks_flat.size() * 8, cudaMemcpyHostToDevice,
                                  stream));
        count_launch();
        assign_stab_ids<<<(unsigned)((n_side + 255) / 256), 256, 0, stream>>>(side.p, n_side, d_masks.p,
                                                                               (int)uniq.size(), s->d_stab_id);
        FTLM_CUDA(cudaGetLastError());
        FTLM_CUDA(cudaStreamSynchronize(stream));
    }
    // bucket index on the high bits of the label
    uint64_t max_label = 0;
    FTLM_CUDA(cudaMemcpyAsync(&max_label, s->d_labels + (n_reps - 1), 8, cudaMemcpyDeviceToHost, stream));
    FTLM_CUDA(cudaStreamSynchronize(stream));
    int lb = 1;
    while (lb < 31 && (1ull << lb) < n_reps) ++lb;  // about one bucket per representative
    int width = 1;
    while (width < 64 && (max_label >> width)) ++width;
    s->bucket_shift = width > lb ? width - lb : 0;
    s->n_buckets = (max_label >> s->bucket_shift) + 1;
    FTLM_CUDA(cudaMalloc((void **)&s->d_bucket, (s->n_buckets + 1) * 4));
    s->device_bytes += (s->n_buckets + 1) * 4;
    count_launch();
    build_buckets<<<(unsigned)((s->n_buckets + 256) / 256), 256, 0, stream>>>(s->d_labels, n_reps, s->bucket_shift,
                                                                                s->n_buckets, s->d_bucket);
    FTLM_CUDA(cudaGetLastError());
    FTLM_CUDA(cudaStreamSynchronize(stream));
    return FTLM_OK;
}

// Eq. 11 basis of the projector range: MGS over the columns of (1/|S|) sum_h rho(h).
ftlm_status stabilizer_tables(const GroupData &grp, const Irrep &ir, const std::vector<int> &S, int &nG, double *V,
                              double &sqrtS) {
    const int d = ir.dim;
    double chi = 0.0;
    for (int h : S) chi += ir.chars[h];
    const double val = chi / (double)S.size();
    nG = (int)lround(val);
    if (fabs(val - nG) > 1e-6) return fail(FTLM_EIRREP, "n_Gamma is not an integer");
    std::vector<double> P((size_t)d * d, 0.0);
    for (int h : S)
        for (int t = 0; t < d * d; ++t) P[t] += ir.rho[(size_t)h * d * d + t];
    for (double &p : P) p /= (double)S.size();
    std::vector<std::vector<double>> Q;
    for (int j = 0; j < d; ++j) {
        std::vector<double> v(d);
        for (int i = 0; i < d; ++i) v[i] = P[(size_t)i * d + j];
        for (auto &q : Q) {
            double dot = 0.0;
            for (int i = 0; i < d; ++i) dot += q[i] * v[i];
            for (int i = 0; i < d; ++i) v[i] -= dot * q[i];
        }
        double nrm = 0.0;
        for (int i = 0; i < d; ++i) nrm += v[i] * v[i];
        nrm = sqrt(nrm);
        if (nrm > 1e-8) {
            for (double &x : v) x /= nrm;
            Q.push_back(v);
        }
    }
    if ((int)Q.size() != nG) return fail(FTLM_EIRREP, "projector rank %d differs from n_Gamma %d", (int)Q.size(), nG);
    for (int i = 0; i < d * d; ++i) V[i] = 0.0;
    for (int k = 0; k < nG; ++k)
        for (int i = 0; i < d; ++i) V[i * d + k] = Q[k][i];
    sqrtS = sqrt((double)S.size());
    return FTLM_OK;
}

void free_block(ftlm_basis *b) {
    if (!b) return;
    cudaFree(b->d_off);
    cudaFree(b->d_ntab);
    cudaFree(b->d_sqrtS);
    cudaFree(b->d_sqrtSf);
    cudaFree(b->d_V);
    cudaFree(b->d_Vf);
    cudaFree(b->d_rhoT);
    cudaFree(b->d_rhoTf);
    packed_set_free(b->ps);
    if (b->sec) sector_release(b->sec);
    delete b;
}

ftlm_status build_block_impl(ftlm_sector *s, int irrep, cudaStream_t stream, ftlm_basis *b) {
    const GroupData &grp = s->grp;
    if (irrep < 0 || irrep >= (int)grp.irreps.size()) return fail(FTLM_EINVAL, "irrep index out of range");
    const Irrep &ir = grp.irreps[irrep];
    if (ir.dim > kMaxD) return fail(FTLM_EUNSUPPORTED, "d_Gamma = %d exceeds %d", ir.dim, kMaxD);
    const int d = ir.dim, G = grp.G;
    b->irrep = irrep;
    b->d = d;
    const size_t ns = s->stab_elems.size();
    std::vector<uint8_t> ntab(ns);
    std::vector<double> V(ns * d * d), sq(ns);
    for (size_t t = 0; t < ns; ++t) {
        int nG;
        ftlm_status st = stabilizer_tables(grp, ir, s->stab_elems[t], nG, &V[t * d * d], sq[t]);
        if (st != FTLM_OK) return st;
        ntab[t] = (uint8_t)nG;
    }
    b->h_ntab = ntab;
    std::vector<float> Vf(V.begin(), V.end()), sqf(sq.begin(), sq.end());
    b->rho_elems = rho_table_elems<double>(G, d);
    b->rho_elemsf = rho_table_elems<float>(G, d);
    std::vector<double> rhoT(b->rho_elems, 0.0);
    std::vector<float> rhoTf(b->rho_elemsf, 0.0f);
    const int RP = rho_row(d);
    for (int g = 0; g < G; ++g)
        for (int r = 0; r < d; ++r)
            for (int c = 0; c < d; ++c) {
                const double v = ir.rho[((size_t)g * d + c) * d + r];
                rhoT[((size_t)g * d + r) * RP + c] = v;
                rhoTf[((size_t)g * d + r) * RP + c] = (float)v;
            }
    FTLM_CUDA(cudaMalloc((void **)&b->d_ntab, ns));
    FTLM_CUDA(cudaMalloc((void **)&b->d_sqrtS, ns * 8));
    FTLM_CUDA(cudaMalloc((void **)&b->d_sqrtSf, ns * 4));
    FTLM_CUDA(cudaMalloc((void **)&b->d_V, V.size() * 8));
    FTLM_CUDA(cudaMalloc((void **)&b->d_Vf, V.size() * 4));
    FTLM_CUDA(cudaMalloc((void **)&b->d_rhoT, rhoT.size() * 8));
    FTLM_CUDA(cudaMalloc((void **)&b->d_rhoTf, rhoTf.size() * 4));
    FTLM_CUDA(cudaMalloc((void **)&b->d_off, (s->n_reps + 1) * 8));
    b->device_bytes = ns * 13 + V.size() * 12 + rhoT.size() * 8 + rhoTf.size() * 4 + (s->n_reps + 1) * 8;
    FTLM_CUDA(cudaMemcpyAsync(b->d_ntab, ntab.data(), ns, cudaMemcpyHostToDevice, stream));
    FTLM_CUDA(cudaMemcpyAsync(b->d_sqrtS, sq.data(), ns * 8, cudaMemcpyHostToDevice, stream));
    FTLM_CUDA(cudaMemcpyAsync(b->d_sqrtSf, sqf.data(), ns * 4, cudaMemcpyHostToDevice, stream));
    FTLM_CUDA(cudaMemcpyAsync(b->d_V, V.data(), V.size() * 8, cudaMemcpyHostToDevice, stream));
    FTLM_CUDA(cudaMemcpyAsync(b->d_Vf, Vf.data(), Vf.size() * 4, cudaMemcpyHostToDevice, stream));
    FTLM_CUDA(cudaMemcpyAsync(b->d_rhoT, rhoT.data(), rhoT.size() * 8, cudaMemcpyHostToDevice, stream));
    FTLM_CUDA(cudaMemcpyAsync(b->d_rhoTf, rhoTf.data(), rhoTf.size() * 4, cudaMemcpyHostToDevice, stream));
    FTLM_CUDA(cudaStreamSynchronize(stream));  // host staging vectors go out of scope
    uint64_t dim = 0;
    ftlm_status st = exclusive_scan(NGammaOf{s->d_stab_id, b->d_ntab}, s->n_reps, b->d_off, stream, &dim);
    if (st != FTLM_OK) return st;
    b->dim = dim;
    const ftlm_basis *one[1] = {b};
    return packed_set_build(s, 1, one, stream, &b->ps);
}

__global__ void interleave_offsets(const uint64_t *const *offs, int K, uint64_t n_reps, uint64_t *offm) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_reps) return;
    for (int k = 0; k < K; ++k) offm[i * K + k] = offs[k][i];
}

void free_multiblock(ftlm_multiblock *mb) {
    if (!mb) return;
    for (auto *b : mb->blocks) free_block(b);
    cudaFree(mb->d_offm);
    cudaFree(mb->d_ntab);
    cudaFree(mb->d_rhoT);
    cudaFree(mb->d_rhoTf);
    packed_set_free(mb->ps);
    if (mb->sec) sector_release(mb->sec);
    delete mb;
}

ftlm_status build_multiblock_impl(ftlm_sector *s, int n, const int *irreps, cudaStream_t stream,
                                  ftlm_multiblock *mb) {
    mb->K = n;
    const size_t ns = s->stab_elems.size();
    std::vector<uint8_t> ntab((size_t)n * ns);
    std::vector<double> rho;
    std::vector<float> rhof;
    for (int k = 0; k < n; ++k) {
        ftlm_basis *b = new (std::nothrow) ftlm_basis();
        if (!b) return fail(FTLM_ENOMEM, "host allocation failed");
        s->refs.fetch_add(1);
        b->sec = s;
        mb->blocks.push_back(b);
        ftlm_status st = build_block_impl(s, irreps[k], stream, b);
        if (st != FTLM_OK) return st;
        std::copy(b->h_ntab.begin(), b->h_ntab.end(), ntab.begin() + (size_t)k * ns);
        const Irrep &ir = s->grp.irreps[irreps[k]];
        const int d = ir.dim, G = s->G, RP = rho_row(d);
        mb->d.push_back(d);
        mb->rho_off.push_back((int)rho.size());
        mb->rho_offf.push_back((int)rhof.size());
        rho.resize(rho.size() + rho_table_elems<double>(G, d), 0.0);
        rhof.resize(rhof.size() + rho_table_elems<float>(G, d), 0.0f);
        for (int g = 0; g < G; ++g)
            for (int r = 0; r < d; ++r)
                for (int c = 0; c < d; ++c) {
                    const double v = ir.rho[((size_t)g * d + c) * d + r];
                    rho[mb->rho_off.back() + ((size_t)g * d + r) * RP + c] = v;
                    rhof[mb->rho_offf.back() + ((size_t)g * d + r) * RP + c] = (float)v;
                }
        mb->device_bytes += b->device_bytes;
    }
    mb->rho_total = (int)rho.size();
    mb->rho_totalf = (int)rhof.size();
    std::vector<const uint64_t *> offs(n);
    for (int k = 0; k < n; ++k) offs[k] = mb->blocks[k]->d_off;
    DevBuf<const uint64_t *> d_offs;
    FTLM_CUDA(d_offs.alloc(n));
    FTLM_CUDA(cudaMemcpyAsync(d_offs.p, offs.data(), n * sizeof(void *), cudaMemcpyHostToDevice, stream));
    FTLM_CUDA(cudaMalloc((void **)&mb->d_offm, s->n_reps * n * 8 + 8));
    FTLM_CUDA(cudaMalloc((void **)&mb->d_ntab, ntab.size()));
    FTLM_CUDA(cudaMalloc((void **)&mb->d_rhoT, rho.size() * 8));
    FTLM_CUDA(cudaMalloc((void **)&mb->d_rhoTf, rhof.size() * 4));
    mb->device_bytes += s->n_reps * n * 8 + ntab.size() + rho.size() * 8 + rhof.size() * 4;
    FTLM_CUDA(cudaMemcpyAsync(mb->d_ntab, ntab.data(), ntab.size(), cudaMemcpyHostToDevice, stream));
    FTLM_CUDA(cudaMemcpyAsync(mb->d_rhoT, rho.data(), rho.size() * 8, cudaMemcpyHostToDevice, stream));
    FTLM_CUDA(cudaMemcpyAsync(mb->d_rhoTf, rhof.data(), rhof.size() * 4, cudaMemcpyHostToDevice, stream));
    count_launch();
    interleave_offsets<<<(unsigned)((s->n_reps + 255) / 256), 256, 0, stream>>>(d_offs.p, n, s->n_reps, mb->d_offm);
    FTLM_CUDA(cudaGetLastError());
    FTLM_CUDA(cudaStreamSynchronize(stream));
    if (n <= kPMaxK && packed_shape_id(n, mb->d.data()) >= 0) {
        ftlm_status st = packed_set_build(s, n, mb->blocks.data(), stream, &mb->ps);
        if (st != FTLM_OK) return st;
        mb->device_bytes += mb->ps->device_bytes;
    }
    return FTLM_OK;
}

}  // namespace

void sector_release(ftlm_sector *s) {
    if (s && s->refs.fetch_sub(1) == 1) free_sector(s);
}

}  // namespace ftlm

using namespace ftlm;

extern "C" {

ftlm_status ftlm_build_sector(const ftlm_group *g, int two_s, int two_M, void *cuda_stream, ftlm_sector **out) {
    if (!g || !out) return fail(FTLM_EINVAL, "NULL argument");
    *out = nullptr;
    ftlm_sector *s = new (std::nothrow) ftlm_sector();
    if (!s) return fail(FTLM_ENOMEM, "host allocation failed");
    ftlm_status st = build_sector_impl(g->d, two_s, two_M, 0, (cudaStream_t)cuda_stream, s);
    if (st != FTLM_OK) {
        cudaStreamSynchronize((cudaStream_t)cuda_stream);
        free_sector(s);
        return st;
    }
    *out = s;
    return FTLM_OK;
}

ftlm_status ftlm_build_sector_flip(const ftlm_group *g, int two_s, void *cuda_stream, ftlm_sector **out) {
    if (!g || !out) return fail(FTLM_EINVAL, "NULL argument");
    *out = nullptr;
    if ((g->d.N * two_s) % 2) return fail(FTLM_EINVAL, "N s is not an integer: no M = 0 sector");
    ftlm_sector *s = new (std::nothrow) ftlm_sector();
    if (!s) return fail(FTLM_ENOMEM, "host allocation failed");
    ftlm_status st = build_sector_impl(g->d, two_s, 0, 1, (cudaStream_t)cuda_stream, s);
    if (st != FTLM_OK) {
        cudaStreamSynchronize((cudaStream_t)cuda_stream);
        free_sector(s);
        return st;
    }
    *out = s;
    return FTLM_OK;
}

ftlm_status ftlm_sector_symmetry(const ftlm_sector *s, int *order, int *n_irreps, int *flip) {
    if (!s) return fail(FTLM_EINVAL, "sector is NULL");
    if (order) *order = s->grp.G;
    if (n_irreps) *n_irreps = (int)s->grp.irreps.size();
    if (flip) *flip = s->flip;
    return FTLM_OK;
}

ftlm_status ftlm_sector_info(const ftlm_sector *s, uint64_t *n_reps, uint64_t *sector_dim, size_t *device_bytes) {
    if (!s) return fail(FTLM_EINVAL, "sector is NULL");
    if (n_reps) *n_reps = s->n_reps;
    if (sector_dim) *sector_dim = s->sector_dim;
    if (device_bytes) *device_bytes = s->device_bytes;
    return FTLM_OK;
}

ftlm_status ftlm_sector_export(const ftlm_sector *s, uint64_t *labels, uint64_t *stab_mask) {
    if (!s) return fail(FTLM_EINVAL, "sector is NULL");
    if (labels) FTLM_CUDA(cudaMemcpy(labels, s->d_labels, s->n_reps * 8, cudaMemcpyDeviceToHost));
    if (stab_mask) {
        const int W = s->flip ? 4 : 2;
        std::vector<uint16_t> ids(s->n_reps);
        FTLM_CUDA(cudaMemcpy(ids.data(), s->d_stab_id, s->n_reps * 2, cudaMemcpyDeviceToHost));
        for (uint64_t i = 0; i < s->n_reps; ++i)
            for (int w = 0; w < W; ++w) stab_mask[W * i + w] = s->stab_masks[ids[i]][w];
    }
    return FTLM_OK;
}

void ftlm_sector_free(ftlm_sector *s) { sector_release(s); }

ftlm_status ftlm_build_block(const ftlm_sector *s_const, int irrep, void *cuda_stream, ftlm_basis **out) {
    if (!s_const || !out) return fail(FTLM_EINVAL, "NULL argument");
    *out = nullptr;
    ftlm_sector *s = const_cast<ftlm_sector *>(s_const);
    ftlm_basis *b = new (std::nothrow) ftlm_basis();
    if (!b) return fail(FTLM_ENOMEM, "host allocation failed");
    s->refs.fetch_add(1);
    b->sec = s;
    ftlm_status st = build_block_impl(s, irrep, (cudaStream_t)cuda_stream, b);
    if (st != FTLM_OK) {
        cudaStreamSynchronize((cudaStream_t)cuda_stream);
        free_block(b);
        return st;
    }
    *out = b;
    return FTLM_OK;
}

ftlm_status ftlm_build_basis(const ftlm_group *g, int two_s, int two_M, int irrep, void *cuda_stream,
                             ftlm_basis **out) {
    ftlm_sector *s = nullptr;
    ftlm_status st = ftlm_build_sector(g, two_s, two_M, cuda_stream, &s);
    if (st != FTLM_OK) return st;
    st = ftlm_build_block(s, irrep, cuda_stream, out);
    sector_release(s);  // the block holds its own reference
    return st;
}

ftlm_status ftlm_basis_info(const ftlm_basis *b, uint64_t *n_reps, uint64_t *dim, size_t *device_bytes) {
    if (!b) return fail(FTLM_EINVAL, "basis is NULL");
    if (n_reps) *n_reps = b->sec->n_reps;
    if (dim) *dim = b->dim;
    if (device_bytes) *device_bytes = b->device_bytes + b->sec->device_bytes;
    return FTLM_OK;
}

ftlm_status ftlm_basis_export(const ftlm_basis *b, uint64_t *labels, uint64_t *stab_mask, uint8_t *n_gamma,
                              uint64_t *offsets) {
    if (!b) return fail(FTLM_EINVAL, "basis is NULL");
    ftlm_status st = ftlm_sector_export(b->sec, labels, stab_mask);
    if (st != FTLM_OK) return st;
    const uint64_t n = b->sec->n_reps;
    if (n_gamma) {
        std::vector<uint16_t> ids(n);
        FTLM_CUDA(cudaMemcpy(ids.data(), b->sec->d_stab_id, n * 2, cudaMemcpyDeviceToHost));
        for (uint64_t i = 0; i < n; ++i) n_gamma[i] = b->h_ntab[ids[i]];
    }
    if (offsets) FTLM_CUDA(cudaMemcpy(offsets, b->d_off, (n + 1) * 8, cudaMemcpyDeviceToHost));
    return FTLM_OK;
}

void ftlm_basis_free(ftlm_basis *b) { free_block(b); }

ftlm_status ftlm_build_multiblock(const ftlm_sector *s_const, int n_blocks, const int *irreps, void *cuda_stream,
                                  ftlm_multiblock **out) {
    if (!s_const || !irreps || !out) return fail(FTLM_EINVAL, "NULL argument");
    if (n_blocks < 1 || n_blocks > 16) return fail(FTLM_EINVAL, "n_blocks must be in 1..16");
    *out = nullptr;
    ftlm_sector *s = const_cast<ftlm_sector *>(s_const);
    ftlm_multiblock *mb = new (std::nothrow) ftlm_multiblock();
    if (!mb) return fail(FTLM_ENOMEM, "host allocation failed");
    s->refs.fetch_add(1);
    mb->sec = s;
    ftlm_status st = build_multiblock_impl(s, n_blocks, irreps, (cudaStream_t)cuda_stream, mb);
    if (st != FTLM_OK) {
        cudaStreamSynchronize((cudaStream_t)cuda_stream);
        free_multiblock(mb);
        return st;
    }
    *out = mb;
    return FTLM_OK;
}

ftlm_status ftlm_multiblock_info(const ftlm_multiblock *mb, int *n_blocks, uint64_t *dims, size_t *device_bytes) {
    if (!mb) return fail(FTLM_EINVAL, "multiblock is NULL");
    if (n_blocks) *n_blocks = mb->K;
    if (dims)
        for (int k = 0; k < mb->K; ++k) dims[k] = mb->blocks[k]->dim;
    if (device_bytes) *device_bytes = mb->device_bytes + mb->sec->device_bytes;
    return FTLM_OK;
}

ftlm_status ftlm_multiblock_block(const ftlm_multiblock *mb, int k, const ftlm_basis **out) {
    if (!mb || !out || k < 0 || k >= mb->K) return fail(FTLM_EINVAL, "bad arguments");
    *out = mb->blocks[k];
    return FTLM_OK;
}

void ftlm_multiblock_free(ftlm_multiblock *mb) { free_multiblock(mb); }

ftlm_status ftlm_basis_check(const ftlm_basis *b, void *cuda_stream) {
    if (!b) return fail(FTLM_EINVAL, "basis is NULL");
    FTLM_CUDA(cudaStreamSynchronize((cudaStream_t)cuda_stream));
    int err = 0;
    FTLM_CUDA(cudaMemcpy(&err, b->sec->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        FTLM_CUDA(cudaMemset(b->sec->d_err, 0, sizeof(int)));
        if (err & 8) return fail(FTLM_ETIMEOUT, "a bounded device wait gave up (code %d)", err);
        return fail(FTLM_EINTERNAL, "device bounds check tripped (code %d)", err);
    }
    return FTLM_OK;
}

}  // extern "C"
