// Symmetry-adapted H·v kernel (Eqs. 15-16 of arXiv 2607.17429, pull form) for
// K >= 1 irrep blocks of one S^z sector in one launch.
//
// One warp per output representative r (persistent grid-stride walk over the
// sorted table):
//  1. images I_g = U(g) r for the lane's group elements g = lane + 32c, from a
//     shared table (s = 1/2: image of every 4-site nibble; general s: the bit
//     position of every site after g);
//  2. lanes over bonds: diagonal term J sum m_i m_j (Eq. 16) and the admissible
//     ladder flips (Eq. 3), compacted with ballots;
//  3. representative search per flip: U(g) a = I_g XOR mask_g(bond) (s = 1/2)
//     or I_g +- delta_g(bond), one table load and one integer op per candidate;
//     redux.sync min over the warp gives r' = min O(a) and the smallest
//     minimising element g*, with a = U(g_e) r', g_e = g*^{-1};
//  4. lookup of r' (one lane per flip): bucket on the high label bits, binary
//     search in the sorted table; the flip record (index, stabilizer id, g*,
//     c_a) goes to the warp's shared-memory slot;
//  5. per block k with n_k(r) > 0 (steps 1-4 are irrep independent and run
//     once): lanes = (flip group, right-hand side) accumulate
//       z += c_a sqrt|Stab r'| rho_k(g*)^T V_k(r') x_k(r')   (rho(g_e) = rho(g*)^T)
//     with the contraction specialised on d_k, then
//       y_k(r) = V_k(r)^T z / sqrt|Stab r| + diag x_k(r).
// Row offsets are [n_reps][K] (one record per lookup).  FP32 keeps the rho
// tables in shared memory; FP64 reads them through the read-only cache.
#pragma once

#include <type_traits>

#include "contract.cuh"

namespace ftlm {

constexpr int kMaxK = 16;

template <typename VT>
__host__ __device__ constexpr int hv_threads() {
    return sizeof(VT) == 8 ? 512 : 1024;
}
template <bool HALF>
__host__ __device__ constexpr int hv_max_flips() {
    return HALF ? 64 : 128;  // one flip per bond (s = 1/2) or two
}

template <typename VT>
struct HvArgs {
    int N, G, n_bonds, bits, two_s, n_chunks, bucket_shift, B, K, n_sid;
    uint64_t n_reps, n_buckets, n_rows_total;
    VT J;
    VT up[8], dn[8];  // sqrt(s(s+1) - m(m+1)), sqrt(s(s+1) - m(m-1)) per digit a = m + s
    const uint64_t *labels;
    const uint16_t *stab_id;
    const uint32_t *bucket;
    const uint32_t *lut;
    const uint8_t *pos;
    const void *dtab;
    const uint8_t *bonds;  // [n_bonds][2]
    const uint64_t *off;   // [n_reps][K] row offsets
    const uint8_t *ntab;   // [K][n_sid]
    const VT *sqrtS;       // [n_sid]
    const VT *rhoT;        // padded tables concatenated, block k at rho_off[k]
    int rho_total;
    int d[kMaxK], rho_off[kMaxK];
    const VT *V[kMaxK];    // [n_sid][d_k][d_k]
    const VT *x[kMaxK];
    VT *y[kMaxK];
    int *err;
};

__device__ __forceinline__ unsigned hv_digit(uint64_t n, int k, int bits) {
    return (unsigned)(n >> (bits * k)) & ((1u << bits) - 1);
}

// position of the n-th (0-based) set bit of m
__device__ __forceinline__ int nth_set_bit(uint32_t m, int n) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const uint32_t lo = m & ((1u << w) - 1u);
        const int c = __popc(lo);
        if (n >= c) {
            n -= c;
            m >>= w;
            pos += w;
        } else {
            m = lo;
        }
    }
    return pos;
}

template <typename VT>
struct HvLayout {
    size_t o_dtab, o_rho, o_bond, o_flip, total;
};

template <typename VT, bool HALF>
__host__ __device__ inline HvLayout<VT> hv_layout(int n_chunks, int n_bonds, int rho_total, int warps) {
    HvLayout<VT> L;
    size_t o = HALF ? (size_t)n_chunks * 16 * kMaxG * 4 : (size_t)kMaxG * 64;
    o = (o + 15) & ~(size_t)15;
    L.o_dtab = o;
    o += (size_t)n_bonds * kMaxG * (HALF ? 4 : 8);
    o = (o + 15) & ~(size_t)15;
    L.o_rho = o;
    if (sizeof(VT) == 4) o += (size_t)rho_total * sizeof(VT);
    o = (o + 15) & ~(size_t)15;
    L.o_bond = o;
    o += (size_t)n_bonds * 2;
    o = (o + 15) & ~(size_t)15;
    L.o_flip = o;
    o += (size_t)warps * hv_max_flips<HALF>() * (8 + sizeof(VT));
    L.total = o;
    return L;
}

// Block k's pass over the flips of one representative (steps 5 and 6).
template <typename VT, int BT, int D>
__device__ __forceinline__ void block_pass(const HvArgs<VT> &a, int k, uint64_t rep, int sid, int n_rk, int nf,
                                           VT diag, const uint32_t *f_idx, const uint32_t *f_sg, const VT *f_c,
                                           const VT *rk, int lane) {
    constexpr int P = 32 / BT;
    constexpr int RP = rho_row(D);
    const int b = lane % BT, fg = lane / BT;
    const int B = a.B, K = a.K;
    const VT *xk = a.x[k];
    const VT *Vk = a.V[k];
    VT z[D];
#pragma unroll
    for (int i = 0; i < D; ++i) z[i] = (VT)0;
    for (int t = 0; t < nf; t += P) {
        const int f = t + fg;
        if (f < nf && b < B) {
            const uint32_t sg = f_sg[f];
            const int sid_j = (int)(sg >> 8), g_j = (int)(sg & 255u);
            const int n_j = __ldg(a.ntab + k * a.n_sid + sid_j);
            if (n_j > 0) {
                const uint64_t off_j = __ldg(a.off + (uint64_t)f_idx[f] * K + k);
                const VT cf = f_c[f] * __ldg(a.sqrtS + sid_j);
                contract_flip<VT, D>(rk + g_j * D * RP, xk + off_j * B + b, B, sid_j, n_j, Vk + (size_t)sid_j * D * D,
                                     cf, z);
            }
        }
    }
#pragma unroll
    for (int w = BT; w < 32; w <<= 1)
#pragma unroll
        for (int i = 0; i < D; ++i) z[i] += __shfl_xor_sync(kFull, z[i], w);
    if (b < B) {
        const VT inv_sq = (VT)1 / __ldg(a.sqrtS + sid);
        const VT *Vr = Vk + (size_t)sid * D * D;
        const uint64_t off_r = __ldg(a.off + rep * K + k);
        VT *yk = a.y[k];
        for (int kk = fg; kk < n_rk; kk += P) {
            VT val = (VT)0;
#pragma unroll
            for (int be = 0; be < D; ++be) val += __ldg(Vr + be * D + kk) * z[be];
            const size_t row = (off_r + kk) * B + b;
            yk[row] = val * inv_sq + diag * __ldg(xk + row);
        }
    }
}

template <typename VT, int BT, int GPL, bool HALF>
__global__ void __launch_bounds__(hv_threads<VT>(), 1) hv_kernel(HvArgs<VT> a) {
    using LT = typename std::conditional<HALF, uint32_t, uint64_t>::type;
    constexpr int MAXF = hv_max_flips<HALF>();
    extern __shared__ __align__(16) uint8_t smem[];
    const int warps = blockDim.x >> 5;
    const HvLayout<VT> L = hv_layout<VT, HALF>(a.n_chunks, a.n_bonds, a.rho_total, warps);
    {
        const size_t n_tab = HALF ? (size_t)a.n_chunks * 16 * kMaxG * 4 : (size_t)kMaxG * 64;
        const uint4 *src0 = reinterpret_cast<const uint4 *>(HALF ? (const void *)a.lut : (const void *)a.pos);
        for (size_t i = threadIdx.x; i < n_tab / 16; i += blockDim.x) reinterpret_cast<uint4 *>(smem)[i] = src0[i];
        const size_t n_dt = (size_t)a.n_bonds * kMaxG * (HALF ? 4 : 8);
        const uint4 *src1 = reinterpret_cast<const uint4 *>(a.dtab);
        for (size_t i = threadIdx.x; i < n_dt / 16; i += blockDim.x)
            reinterpret_cast<uint4 *>(smem + L.o_dtab)[i] = src1[i];
        if (sizeof(VT) == 4) {
            const uint4 *src2 = reinterpret_cast<const uint4 *>(a.rhoT);
            for (int i = threadIdx.x; i < a.rho_total * (int)sizeof(VT) / 16; i += blockDim.x)
                reinterpret_cast<uint4 *>(smem + L.o_rho)[i] = src2[i];
        }
        for (int i = threadIdx.x; i < 2 * a.n_bonds; i += blockDim.x) smem[L.o_bond + i] = a.bonds[i];
    }
    __syncthreads();
    const uint32_t *s_lut = reinterpret_cast<const uint32_t *>(smem);
    const uint8_t *s_pos = smem;
    const LT *s_dtab = reinterpret_cast<const LT *>(smem + L.o_dtab);
    const VT *rho_base = sizeof(VT) == 4 ? reinterpret_cast<const VT *>(smem + L.o_rho) : a.rhoT;
    const uint8_t *s_bond = smem + L.o_bond;
    const int wid = threadIdx.x >> 5;
    uint32_t *f_idx = reinterpret_cast<uint32_t *>(smem + L.o_flip) + (size_t)wid * MAXF * 2;
    uint32_t *f_sg = f_idx + MAXF;
    VT *f_c = reinterpret_cast<VT *>(smem + L.o_flip + (size_t)warps * MAXF * 8) + (size_t)wid * MAXF;

    const int lane = threadIdx.x & 31;
    const int K = a.K;
    const uint64_t nw = (uint64_t)gridDim.x * warps;
    const VT halfJ = a.J * (VT)0.5;

    for (uint64_t rep = (uint64_t)blockIdx.x * warps + wid; rep < a.n_reps; rep += nw) {
        const int sid = a.stab_id[rep];
        const bool act = lane < K && __ldg(a.ntab + lane * a.n_sid + sid) > 0;
        if (__ballot_sync(kFull, act) == 0u) continue;  // no block has rows for this orbit
        const LT lab = (LT)a.labels[rep];

        // 1. images of r under the lane's elements
        LT I[GPL];
#pragma unroll
        for (int c = 0; c < GPL; ++c) {
            const int g = lane + 32 * c;
            LT v = 0;
            if (HALF) {
                for (int q = 0; q < a.n_chunks; ++q) v |= s_lut[(q * 16 + (int)((lab >> (4 * q)) & 15)) * kMaxG + g];
            } else {
                for (int k = 0; k < a.N; ++k) v += (LT)hv_digit(lab, k, a.bits) << s_pos[g * 64 + k];
            }
            I[c] = v;
        }
        // 2. diagonal term and admissible flips
        uint32_t m[4] = {0u, 0u, 0u, 0u};
        int diag4 = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = lane + 32 * h;
            const bool has = e < a.n_bonds;
            int ai = 0, aj = 0;
            if (has) {
                ai = (int)hv_digit(lab, s_bond[2 * e], a.bits);
                aj = (int)hv_digit(lab, s_bond[2 * e + 1], a.bits);
                diag4 += (2 * ai - a.two_s) * (2 * aj - a.two_s);
            }
            if (HALF) {
                m[h] = __ballot_sync(kFull, has && ai != aj);
            } else {
                m[2 * h] = __ballot_sync(kFull, has && ai < a.two_s && aj > 0);      // s_i^+ s_j^-
                m[2 * h + 1] = __ballot_sync(kFull, has && ai > 0 && aj < a.two_s);  // s_i^- s_j^+
            }
        }
        diag4 = __reduce_add_sync(kFull, diag4);
        const VT diag = a.J * (VT)diag4 * (VT)0.25;
        const int nf = __popc(m[0]) + __popc(m[1]) + __popc(m[2]) + __popc(m[3]);

        // 3-4. search and lookup, 32 flips per round; records to shared memory
        for (int base = 0; base < nf; base += 32) {
            const int nround = min(32, nf - base);
            int my_e = 0, my_sg = 1;
            VT my_c = (VT)0;
            if (lane < nround) {
                int f = base + lane, w = 0;
                while (f >= __popc(m[w])) {
                    f -= __popc(m[w]);
                    ++w;
                }
                const int bit = nth_set_bit(m[w], f);
                if (HALF) {
                    my_e = bit + 32 * w;
                    my_c = halfJ;
                } else {
                    my_e = bit + 32 * (w >> 1);
                    my_sg = (w & 1) ? -1 : 1;
                    const int ai = (int)hv_digit(lab, s_bond[2 * my_e], a.bits);
                    const int aj = (int)hv_digit(lab, s_bond[2 * my_e + 1], a.bits);
                    my_c = halfJ * (my_sg > 0 ? a.up[ai] * a.dn[aj] : a.dn[ai] * a.up[aj]);
                }
            }
            LT my_rp = 0;
            int my_g = 0;
            for (int j = 0; j < nround; ++j) {
                const int e = __shfl_sync(kFull, my_e, j);
                const int sg = HALF ? 1 : __shfl_sync(kFull, my_sg, j);
                LT best = 0;
                int bg = 0;
#pragma unroll
                for (int c = 0; c < GPL; ++c) {
                    const int g = lane + 32 * c;
                    LT cand;
                    if (HALF) {
                        cand = I[c] ^ s_dtab[e * kMaxG + g];
                    } else {
                        const LT dlt = s_dtab[e * kMaxG + g];
                        cand = sg > 0 ? I[c] + dlt : I[c] - dlt;
                    }
                    if (c == 0 || cand < best) {
                        best = cand;
                        bg = g;
                    }
                }
                LT mn;
                if (HALF) {
                    mn = (LT)__reduce_min_sync(kFull, (unsigned)best);
                } else {
                    const unsigned hi = __reduce_min_sync(kFull, (unsigned)(best >> 32));
                    const unsigned lo = __reduce_min_sync(kFull, (unsigned)(best >> 32) == hi ? (unsigned)best : ~0u);
                    mn = ((LT)hi << 32) | (LT)lo;
                }
                const int gs = (int)__reduce_min_sync(kFull, best == mn ? (unsigned)bg : 0xffffu);
                if (lane == j) {
                    my_rp = mn;
                    my_g = gs;
                }
            }
            if (lane < nround) {
                const uint64_t key = (uint64_t)my_rp;
                const uint64_t bk = key >> a.bucket_shift;
                uint32_t idx = 0;
                int sid_f = 0;
                bool found = false;
                if (bk < a.n_buckets) {
                    uint32_t lo = __ldg(a.bucket + bk), hi = __ldg(a.bucket + bk + 1);
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (__ldg(a.labels + mid) < key)
                            lo = mid + 1;
                        else
                            hi = mid;
                    }
                    if (lo < a.n_reps && __ldg(a.labels + lo) == key) {
                        found = true;
                        idx = lo;
                        sid_f = __ldg(a.stab_id + lo);
                    }
                }
                if (!found) {
                    atomicOr(a.err, 1);
                    my_c = (VT)0;
                }
                f_idx[base + lane] = idx;
                f_sg[base + lane] = ((uint32_t)sid_f << 8) | (uint32_t)my_g;
                f_c[base + lane] = my_c;
            }
        }
        __syncwarp();

        // 5-6. contraction and output, block by block
        for (int k = 0; k < K; ++k) {
            const int n_rk = __ldg(a.ntab + k * a.n_sid + sid);
            if (n_rk == 0) continue;
            const VT *rk = rho_base + a.rho_off[k];
            switch (a.d[k]) {
                case 1: block_pass<VT, BT, 1>(a, k, rep, sid, n_rk, nf, diag, f_idx, f_sg, f_c, rk, lane); break;
                case 2: block_pass<VT, BT, 2>(a, k, rep, sid, n_rk, nf, diag, f_idx, f_sg, f_c, rk, lane); break;
                case 3: block_pass<VT, BT, 3>(a, k, rep, sid, n_rk, nf, diag, f_idx, f_sg, f_c, rk, lane); break;
                case 4: block_pass<VT, BT, 4>(a, k, rep, sid, n_rk, nf, diag, f_idx, f_sg, f_c, rk, lane); break;
                default: block_pass<VT, BT, 5>(a, k, rep, sid, n_rk, nf, diag, f_idx, f_sg, f_c, rk, lane); break;
            }
        }
        __syncwarp();
    }
}

template <typename VT, int BT, int GPL, bool HALF>
ftlm_status launch_hv_t(const HvArgs<VT> &a, cudaStream_t stream) {
    auto kern = hv_kernel<VT, BT, GPL, HALF>;
    constexpr int threads = hv_threads<VT>();
    const size_t smem = hv_layout<VT, HALF>(a.n_chunks, a.n_bonds, a.rho_total, threads / 32).total;
    FTLM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    FTLM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return fail(FTLM_EUNSUPPORTED, "H·v kernel does not fit on an SM (shared memory %zu B)", smem);
    int dev = 0, sms = kNumSMs;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t need = (a.n_reps + threads / 32 - 1) / (threads / 32);
    uint64_t grid = (uint64_t)sms * per_sm;
    if (need < grid) grid = need ? need : 1;
    cudaEvent_t e0, e1;
    hv_timer_begin(stream, &e0, &e1);
    kern<<<(unsigned)grid, threads, smem, stream>>>(a);
    count_launch();
    FTLM_CUDA(cudaGetLastError());
    hv_timer_end(stream, e0, e1, a.n_rows_total);
    return FTLM_OK;
}

template <typename VT, int GPL, bool HALF>
ftlm_status launch_hv_b(const HvArgs<VT> &a, cudaStream_t stream) {
    if (a.B <= 1) return launch_hv_t<VT, 1, GPL, HALF>(a, stream);
    if (a.B <= 2) return launch_hv_t<VT, 2, GPL, HALF>(a, stream);
    if (a.B <= 4) return launch_hv_t<VT, 4, GPL, HALF>(a, stream);
    if (a.B <= 8) return launch_hv_t<VT, 8, GPL, HALF>(a, stream);
    if (a.B <= 16) return launch_hv_t<VT, 16, GPL, HALF>(a, stream);
    return launch_hv_t<VT, 32, GPL, HALF>(a, stream);
}

template <typename VT>
ftlm_status launch_hv(const HvArgs<VT> &a, bool half, cudaStream_t stream) {
    if (a.G <= 64) return half ? launch_hv_b<VT, 2, true>(a, stream) : launch_hv_b<VT, 2, false>(a, stream);
    return half ? launch_hv_b<VT, 4, true>(a, stream) : launch_hv_b<VT, 4, false>(a, stream);
}

// Argument block from the sector and K blocks (rho tables and offsets given by the caller).
template <typename VT>
void fill_hv_args(const ftlm_sector *s, int B, int K, const ftlm_basis *const *blocks, const uint64_t *off,
                  const uint8_t *ntab, const VT *sqrtS, const VT *rhoT, int rho_total, const int *rho_off,
                  const VT *const *V, const VT *const *x, VT *const *y, HvArgs<VT> &a) {
    a.N = s->N;
    a.G = s->G;
    a.n_bonds = s->grp.n_bonds();
    a.bits = s->bits;
    a.two_s = s->two_s;
    a.n_chunks = s->n_chunks;
    a.bucket_shift = s->bucket_shift;
    a.B = B;
    a.K = K;
    a.n_sid = (int)s->stab_elems.size();
    a.n_reps = s->n_reps;
    a.n_buckets = s->n_buckets;
    a.J = (VT)s->grp.J;
    const double sp = 0.5 * s->two_s, ss1 = sp * (sp + 1.0);
    for (int i = 0; i < 8; ++i) {
        const double mm = i - sp;
        const double u = ss1 - mm * (mm + 1.0), dn = ss1 - mm * (mm - 1.0);
        a.up[i] = (VT)(u > 0 ? sqrt(u) : 0.0);
        a.dn[i] = (VT)(dn > 0 ? sqrt(dn) : 0.0);
    }
    a.labels = s->d_labels;
    a.stab_id = s->d_stab_id;
    a.bucket = s->d_bucket;
    a.lut = s->d_lut;
    a.pos = s->d_pos;
    a.dtab = s->d_dtab;
    a.bonds = s->d_bonds;
    a.off = off;
    a.ntab = ntab;
    a.sqrtS = sqrtS;
    a.rhoT = rhoT;
    a.rho_total = rho_total;
    a.err = s->d_err;
    a.n_rows_total = 0;
    for (int k = 0; k < kMaxK; ++k) {
        const bool in = k < K;
        a.d[k] = in ? blocks[k]->d : 0;
        a.rho_off[k] = in ? rho_off[k] : 0;
        a.V[k] = in ? V[k] : nullptr;
        a.x[k] = in ? x[k] : nullptr;
        a.y[k] = in ? y[k] : nullptr;
        if (in) a.n_rows_total += blocks[k]->dim * (uint64_t)B;
    }
}

}  // namespace ftlm
