// Symmetry-adapted H·v kernel (Eqs. 15-16 of arXiv 2607.17429, pull form).
//
// One warp per output representative r (grid-stride over the sorted table):
//  1. images I_g = U(g) r for the lane's group elements g = lane + 32c, from a
//     shared-memory table (s = 1/2: image of every 4-site nibble; general s:
//     target bit position of every site);
//  2. lanes over bonds: diagonal term J sum m_i m_j (Eq. 16) and the admissible
//     ladder flips (Eq. 3), compacted with ballots;
//  3. representative search per flip: U(g) a = I_g XOR mask_g(bond) (s = 1/2) or
//     I_g +- delta_g(bond) (general s), so each candidate is one table load and
//     one integer op; warp min-reduction (redux.sync) gives r' = min O(a) and the
//     smallest minimising element g*, a = U(g_e) r' with g_e = g*^{-1};
//  4. lookup of r' (one lane per flip): bucket on the high label bits, then a
//     binary search in the sorted table; n_Gamma(r') = 0 skips the flip;
//  5. contraction (lanes = flip group x right-hand side): u = V_r' x_r',
//     z += c_a sqrt|Stab r'| rho(g*)^T u   (rho(g_e) = rho(g*)^T for real irreps);
//  6. y_r = V_r^T z / sqrt|Stab r| + diag x_r.
// All tables are staged in shared memory once per block; the grid is a
// multiple of the SM count and every block walks representatives persistently.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace ftlm {

constexpr int kHvThreads = 512;

template <typename VT>
struct HvArgs {
    int N, G, n_bonds, bits, two_s, d, n_chunks, bucket_shift, B;
    uint64_t n_reps, n_buckets;
    uint64_t n_rows_total;  // dim * B (for profiling)
    VT J;
    VT up[8], dn[8];  // sqrt(s(s+1) - m(m+1)), sqrt(s(s+1) - m(m-1)) per digit a = m + s
    const uint64_t *labels;
    const uint16_t *stab_id;
    const uint64_t *off;
    const uint32_t *bucket;
    const uint32_t *lut;
    const uint8_t *pos;
    const void *dtab;
    const uint8_t *bonds;  // [n_bonds][2]
    const uint8_t *ntab;
    const VT *sqrtS;
    const VT *V;
    const VT *rhoT;
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
size_t hv_smem_bytes(bool half, int n_chunks, int n_bonds, int G, int d) {
    size_t s = half ? (size_t)n_chunks * 16 * kMaxG * 4 : (size_t)kMaxG * 64;
    s = (s + 15) & ~(size_t)15;
    s += (size_t)n_bonds * kMaxG * (half ? 4 : 8);
    s = (s + 15) & ~(size_t)15;
    s += (size_t)G * d * d * sizeof(VT);
    s = (s + 15) & ~(size_t)15;
    s += (size_t)n_bonds * 2;
    return s;
}

template <typename VT, int BT, int GPL, bool HALF>
__global__ void __launch_bounds__(kHvThreads) hv_kernel(HvArgs<VT> a, const VT *__restrict__ x, VT *__restrict__ y) {
    using LT = typename std::conditional<HALF, uint32_t, uint64_t>::type;
    extern __shared__ __align__(16) uint8_t smem[];
    size_t o = 0;
    const uint32_t *s_lut = reinterpret_cast<const uint32_t *>(smem);
    const uint8_t *s_pos = smem;
    o = HALF ? (size_t)a.n_chunks * 16 * kMaxG * 4 : (size_t)kMaxG * 64;
    o = (o + 15) & ~(size_t)15;
    const size_t o_dtab = o;
    o += (size_t)a.n_bonds * kMaxG * (HALF ? 4 : 8);
    o = (o + 15) & ~(size_t)15;
    const size_t o_rho = o;
    o += (size_t)a.G * a.d * a.d * sizeof(VT);
    o = (o + 15) & ~(size_t)15;
    const size_t o_bond = o;
    {
        // stage the tables (16-byte vector copies; every region is a multiple of 16 bytes but the last)
        const size_t n_tab = HALF ? (size_t)a.n_chunks * 16 * kMaxG * 4 : (size_t)kMaxG * 64;
        const uint4 *src0 = reinterpret_cast<const uint4 *>(HALF ? (const void *)a.lut : (const void *)a.pos);
        for (size_t i = threadIdx.x; i < n_tab / 16; i += blockDim.x) reinterpret_cast<uint4 *>(smem)[i] = src0[i];
        const size_t n_dt = (size_t)a.n_bonds * kMaxG * (HALF ? 4 : 8);
        const uint4 *src1 = reinterpret_cast<const uint4 *>(a.dtab);
        for (size_t i = threadIdx.x; i < n_dt / 16; i += blockDim.x)
            reinterpret_cast<uint4 *>(smem + o_dtab)[i] = src1[i];
        VT *s_rho_w = reinterpret_cast<VT *>(smem + o_rho);
        for (int i = threadIdx.x; i < a.G * a.d * a.d; i += blockDim.x) s_rho_w[i] = a.rhoT[i];
        for (int i = threadIdx.x; i < 2 * a.n_bonds; i += blockDim.x) smem[o_bond + i] = a.bonds[i];
    }
    __syncthreads();
    const LT *s_dtab = reinterpret_cast<const LT *>(smem + o_dtab);
    const VT *s_rho = reinterpret_cast<const VT *>(smem + o_rho);
    const uint8_t *s_bond = smem + o_bond;

    constexpr int P = 32 / BT;  // flip groups in the contraction
    const int lane = threadIdx.x & 31;
    const int b = lane % BT, fg = lane / BT;
    const int d = a.d;
    const int B = a.B;
    const uint64_t warps_per_block = blockDim.x >> 5;
    const uint64_t nw = (uint64_t)gridDim.x * warps_per_block;
    const VT halfJ = a.J * (VT)0.5;

    for (uint64_t rep = (uint64_t)blockIdx.x * warps_per_block + (threadIdx.x >> 5); rep < a.n_reps; rep += nw) {
        const int sid = a.stab_id[rep];
        const int n_r = a.ntab[sid];
        if (n_r == 0) continue;  // warp-uniform
        const LT lab = (LT)a.labels[rep];
        const uint64_t off_r = a.off[rep];

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

        // 2. diagonal term and admissible flips (lanes over bonds)
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

        VT z[kMaxD];
#pragma unroll
        for (int i = 0; i < kMaxD; ++i) z[i] = (VT)0;

        for (int base = 0; base < nf; base += 32) {
            const int nround = min(32, nf - base);
            // the lane's flip (base + lane): bond, sign, coefficient (Eq. 3)
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
            // 3. representative search, one flip at a time across the warp
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
            // 4. lookup of r' in the sorted table (one lane per flip)
            int my_n = 0, my_sid = 0;
            uint64_t my_off = 0;
            if (lane < nround) {
                const uint64_t key = (uint64_t)my_rp;
                const uint64_t bk = key >> a.bucket_shift;
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
                        my_sid = __ldg(a.stab_id + lo);
                        my_n = __ldg(a.ntab + my_sid);
                        my_off = __ldg(a.off + lo);
                    }
                }
                if (!found) atomicOr(a.err, 1);
            }
            // 5. contraction: lane = (flip group fg, right-hand side b)
            for (int t = 0; t < nround; t += P) {
                const int j = t + fg;
                const int srcl = j < nround ? j : 0;
                const int n_j = __shfl_sync(kFull, my_n, srcl);
                const uint64_t off_j = __shfl_sync(kFull, my_off, srcl);
                const int sid_j = __shfl_sync(kFull, my_sid, srcl);
                const int g_j = __shfl_sync(kFull, my_g, srcl);
                const VT c_j = __shfl_sync(kFull, my_c, srcl);
                if (j < nround && n_j > 0 && b < B) {
                    const VT *xr = x + off_j * B + b;
                    VT u[kMaxD];
                    if (sid_j == 0) {
#pragma unroll
                        for (int g2 = 0; g2 < kMaxD; ++g2) u[g2] = g2 < d ? __ldg(xr + (size_t)g2 * B) : (VT)0;
                    } else {
                        const VT *Vt = a.V + (size_t)sid_j * d * d;
#pragma unroll
                        for (int g2 = 0; g2 < kMaxD; ++g2) u[g2] = (VT)0;
                        for (int kp = 0; kp < n_j; ++kp) {
                            const VT xv = __ldg(xr + (size_t)kp * B);
#pragma unroll
                            for (int g2 = 0; g2 < kMaxD; ++g2)
                                if (g2 < d) u[g2] += __ldg(Vt + g2 * d + kp) * xv;
                        }
                    }
                    const VT cf = c_j * __ldg(a.sqrtS + sid_j);
                    const VT *R = s_rho + g_j * d * d;
#pragma unroll
                    for (int be = 0; be < kMaxD; ++be) {
                        if (be < d) {
                            VT acc = (VT)0;
#pragma unroll
                            for (int ga = 0; ga < kMaxD; ++ga)
                                if (ga < d) acc += R[be * d + ga] * u[ga];
                            z[be] += cf * acc;
                        }
                    }
                }
            }
        }
        // reduce over flip groups
#pragma unroll
        for (int w = BT; w < 32; w <<= 1)
#pragma unroll
            for (int i = 0; i < kMaxD; ++i) z[i] += __shfl_xor_sync(kFull, z[i], w);
        // 6. y_r = V_r^T z / sqrt|Stab r| + diag x_r
        if (b < B) {
            const VT inv_sq = (VT)1 / __ldg(a.sqrtS + sid);
            const VT *Vr = a.V + (size_t)sid * d * d;
            for (int k = fg; k < n_r; k += P) {
                VT val = (VT)0;
#pragma unroll
                for (int be = 0; be < kMaxD; ++be)
                    if (be < d) val += __ldg(Vr + be * d + k) * z[be];
                const size_t row = (off_r + k) * B + b;
                y[row] = val * inv_sq + diag * __ldg(x + row);
            }
        }
    }
}

template <typename VT, int BT, int GPL, bool HALF>
ftlm_status launch_hv_t(const HvArgs<VT> &a, const VT *x, VT *y, cudaStream_t stream) {
    auto kern = hv_kernel<VT, BT, GPL, HALF>;
    const size_t smem = hv_smem_bytes<VT>(HALF, a.n_chunks, a.n_bonds, a.G, a.d);
    FTLM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    FTLM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kHvThreads, smem));
    if (per_sm < 1) return fail(FTLM_EUNSUPPORTED, "H·v kernel does not fit on an SM (smem %zu)", smem);
    int dev = 0, sms = kNumSMs;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t need = (a.n_reps + kHvThreads / 32 - 1) / (kHvThreads / 32);
    uint64_t grid = (uint64_t)sms * per_sm;
    if (need < grid) grid = need ? need : 1;
    cudaEvent_t e0, e1;
    hv_timer_begin(stream, &e0, &e1);
    kern<<<(unsigned)grid, kHvThreads, smem, stream>>>(a, x, y);
    count_launch();
    FTLM_CUDA(cudaGetLastError());
    hv_timer_end(stream, e0, e1, a.n_rows_total);
    return FTLM_OK;
}

template <typename VT, int GPL, bool HALF>
ftlm_status launch_hv_b(const HvArgs<VT> &a, const VT *x, VT *y, cudaStream_t stream) {
    if (a.B <= 1) return launch_hv_t<VT, 1, GPL, HALF>(a, x, y, stream);
    if (a.B <= 2) return launch_hv_t<VT, 2, GPL, HALF>(a, x, y, stream);
    if (a.B <= 4) return launch_hv_t<VT, 4, GPL, HALF>(a, x, y, stream);
    if (a.B <= 8) return launch_hv_t<VT, 8, GPL, HALF>(a, x, y, stream);
    if (a.B <= 16) return launch_hv_t<VT, 16, GPL, HALF>(a, x, y, stream);
    return launch_hv_t<VT, 32, GPL, HALF>(a, x, y, stream);
}

template <typename VT>
ftlm_status launch_hv(const HvArgs<VT> &a, bool half, const VT *x, VT *y, cudaStream_t stream) {
    if (a.G <= 64) {
        return half ? launch_hv_b<VT, 2, true>(a, x, y, stream) : launch_hv_b<VT, 2, false>(a, x, y, stream);
    }
    return half ? launch_hv_b<VT, 4, true>(a, x, y, stream) : launch_hv_b<VT, 4, false>(a, x, y, stream);
}

// fill the argument block shared by both precisions
template <typename VT>
void fill_hv_args(const ftlm_basis *bs, int B, HvArgs<VT> &a, const VT *sqrtS, const VT *V, const VT *rhoT) {
    const ftlm_sector *s = bs->sec;
    a.N = s->N;
    a.G = s->G;
    a.n_bonds = s->grp.n_bonds();
    a.bits = s->bits;
    a.two_s = s->two_s;
    a.d = bs->d;
    a.n_chunks = s->n_chunks;
    a.bucket_shift = s->bucket_shift;
    a.B = B;
    a.n_rows_total = bs->dim * (uint64_t)B;
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
    a.off = bs->d_off;
    a.bucket = s->d_bucket;
    a.lut = s->d_lut;
    a.pos = s->d_pos;
    a.dtab = s->d_dtab;
    a.ntab = bs->d_ntab;
    a.sqrtS = sqrtS;
    a.V = V;
    a.rhoT = rhoT;
    a.err = s->d_err;
}

}  // namespace ftlm
