// Packed symmetry-adapted H·v (Eqs. 15-16 of arXiv 2607.17429, pull form).
//
// A "packed set" holds K irrep blocks of one S^z sector with their rows
// interleaved by representative, in lifted coordinates: representative r owns
// the W = sum_k d_k rows (k, gamma), gamma < d_k, holding x~_k(r) = V_k(r)
// x_k(r), the block-k coefficients of r mapped into the d_k-dimensional irrep
// space by V_r of Eq. 11 ([rows][B], B right-hand sides per row).  V_r has
// orthonormal columns, so the lift is an isometry: inner products and norms
// (the Lanczos alpha, beta) are those of the block vectors, and H acts as
//   y~_k(r) = P_k(r) z_k(r) / sqrt|Stab r| + diag x~_k(r),
//   z_k(r)  = sum_flips c_a sqrt|Stab r'| rho_k(g*)^T x~_k(r'),
// with the projector P_k(r) = V_k(r) V_k(r)^T (the identity for a trivial
// stabilizer).  Every segment has the same W rows, r' owns rows r' W .. r' W +
// W - 1, and the flip contraction never touches V.  The block dimensions form a
// compile-time Shape, so the contraction unrolls over the blocks with register
// accumulators; K = 1 is a single block.
//
// One warp per output representative r; representatives are walked in tiles
// (a tile never crosses a part; several sectors may form one launch as parts):
//  1. the record of r (label, stabilizer id); its own rows are prefetched by
//     a bulk copy (bulk-copy path);
//  2. images I_g = U(g) r for the lane's elements g = lane + 32c (2-site LUT for
//     s = 1/2, bit-field positions otherwise), the diagonal term J sum m_i m_j
//     (Eq. 16) and the admissible ladder flips (Eq. 3) by ballots;
//  3. per flip, the orbit minimum r' = min_g U(g) a over the warp (redux.sync)
//     with the smallest minimising element g*, so a = U(g_e) r', g_e = g*^{-1};
//  4. lookup of r' (lane per flip): bucket on the high label bits, then binary
//     search over the 16-byte records (label, segment offset, stabilizer id);
//  5. gathers: the segments of Q = 32/BT flips at a time go to the warp's
//     staging buffer, by bulk copies completing on an mbarrier (bulk-copy path,
//     nbuf groups in flight) or by lane copies (direct path);
//  6. lanes = (flip group, right-hand side) accumulate z for every block;
//  7. z is summed over flip groups and y~(r) written; optionally <x~_k, y~_k>
//     per right-hand side is accumulated (products exact, double-float per
//     representative, FP64 per CTA) for the fused Lanczos step.
// Every mbarrier wait is bounded by a caller-set cycle budget; when it runs out
// the warp records the timeout, drains its copies in flight and stops working,
// while still taking part in the CTA barriers of the reductions.
#pragma once

#include <cuda_fp16.h>

#include <mutex>
#include <type_traits>
#include <utility>

#include "contract.cuh"
#include "ptx.cuh"

namespace ftlm {

constexpr int kPMaxParts = 4096;  // parts (sectors) per launch
constexpr int kErrMissingRep = 1, kErrWaitTimeout = 8;
constexpr int kMaxBuf = 4;  // staging buffers in flight per warp

// ---------------------------------------------------------------- compile-time block shapes

template <int k, int... Ds>
struct NthDim;
template <int D0, int... Ds>
struct NthDim<0, D0, Ds...> {
    static constexpr int value = D0;
};
template <int k, int D0, int... Ds>
struct NthDim<k, D0, Ds...> {
    static constexpr int value = NthDim<k - 1, Ds...>::value;
};
template <int k, int... Ds>
struct ZOff {
    static constexpr int value = ZOff<k - 1, Ds...>::value + NthDim<k - 1, Ds...>::value;
};
template <int... Ds>
struct ZOff<0, Ds...> {
    static constexpr int value = 0;
};

template <int... Ds>
struct Shape {
    static constexpr int K = sizeof...(Ds);
    static constexpr int W = (0 + ... + Ds);  // z rows = sum of d_k
    template <int k>
    static constexpr int D = NthDim<k, Ds...>::value;
    template <int k>
    static constexpr int Z = ZOff<k, Ds...>::value;
};

template <class F, int... I>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F &&f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// ---------------------------------------------------------------- arguments

template <typename VT>
struct HvpPart {
    uint64_t n_reps;
    uint64_t tile0;          // first tile of this part in the launch's tile order
    const HvRec *rec;        // [n_reps], ascending labels; rec.off = index * W
    const uint32_t *bucket;  // [n_buckets + 1]
    uint64_t n_buckets;
    int bucket_shift;
    int n_sid;
    const uint8_t *wtab;     // [n_sid] sum over k of n_k(sid) (0: the orbit has no rows in the set)
    const VT *sqrtS;         // [n_sid]
    const VT *Pj[kPMaxK];    // block k: [n_sid][d_k][d_k] projector V V^T
    const void *x;           // lifted [n_reps * W][B] of the storage type (VT, or FP16 with VT = float)
    void *y;
    const uint64_t *eoff;    // entry table of the sector ([n_reps + 1]; table and build modes)
    HvEntry *ent;            // [n_entries] (read in table mode, written in build mode)
};

template <typename VT>
struct HvpArgs {
    int N, G, n_bonds, bits, two_s, n_chunks;
    int flip;                // G x Z_2 at M = 0: candidates U(g) a and their spin flips
    unsigned long long flipc;  // flip(n) = n ^ flipc (s = 1/2) or flipc - n
    unsigned neg;            // bit k: block k is a Gamma- block (rho(g, 1) = -rho(g))
    VT J;
    VT up[8], dn[8];         // sqrt(s(s+1) - m(m+1)), sqrt(s(s+1) - m(m-1)) per digit a = m + s
    const uint32_t *lut2;    // s = 1/2: [n_chunks][4][kMaxG] image of a 2-site chunk
    const uint8_t *pos;      // general s: [kMaxG][64] bit position of site k after g
    const void *dtab;        // [n_bonds][kMaxG] XOR masks (s = 1/2) or signed deltas
    const uint8_t *bonds;    // [n_bonds][2]
    const VT *rhoT;          // rho(g) of the K blocks, row-major with padded rows, block k at rho_off[k]
    int rho_total;
    int rho_off[kPMaxK];
    int n_parts;
    HvpPart<VT> part0;           // the part when n_parts == 1
    const HvpPart<VT> *parts;    // device array when n_parts > 1
    uint64_t n_tiles;
    int tile_reps;
    int B, BT, lgBT, nbuf, tma;
    int esize;               // bytes of one stored vector element (sizeof(VT), or 2 for FP16 storage)
    int stage_elems;         // stored elements of one staging buffer
    int slot_elems;          // stored elements of one flip's slot (W * B rounded up to 16 bytes, then padded)
    int rho_smem;            // FP32: rho tables staged in shared memory (else read through L1)
    int own;                 // bulk-copy path: prefetch the representative's own rows into shared memory
    unsigned long long wait_limit;
    int *err;
    double *dot_part;        // [n_parts][gridDim.x][K][B] partial <x_k, y_k>, or null
    unsigned long long *flips;  // profiling: ladder flips processed (one atomic per representative), or null
};

// ---------------------------------------------------------------- shared-memory layout

struct HvpLayout {
    size_t o_dtab, o_rho, o_bond, o_red, o_flip, o_fc, o_bar, o_stage, per_warp_stage, own_elems, total;
};

template <typename VT, bool HALF>
__host__ __device__ inline HvpLayout hvp_layout(int n_chunks, int n_bonds, int rho_total, int warps, int K, int W,
                                                int B, int nbuf, int stage_elems, int own, int esize,
                                                bool search_tables = true) {
    constexpr int MAXF = HALF ? 64 : 128;
    HvpLayout L;
    size_t o = !search_tables ? 0 : HALF ? (size_t)n_chunks * 4 * kMaxG * 4 : (size_t)kMaxG * 64;
    o = (o + 15) & ~(size_t)15;
    L.o_dtab = o;
    if (search_tables) o += (size_t)n_bonds * kMaxG * (HALF ? 4 : 8);
    o = (o + 15) & ~(size_t)15;
    L.o_rho = o;
    if (sizeof(VT) == 4) o += (size_t)rho_total * sizeof(VT);
    o = (o + 15) & ~(size_t)15;
    L.o_bond = o;
    o += (size_t)n_bonds * 2;
    o = (o + 15) & ~(size_t)15;
    L.o_red = o;  // [K][B] doubles: CTA reduction of <x, y>
    o += (size_t)K * B * 8;
    o = (o + 15) & ~(size_t)15;
    L.o_flip = o;  // per warp: off[MAXF], sg[MAXF] (u32)
    o += (size_t)warps * MAXF * 8;
    L.o_fc = o;    // per warp: c[MAXF] (VT)
    o += (size_t)warps * MAXF * sizeof(VT);
    o = (o + 15) & ~(size_t)15;
    L.o_bar = o;   // per warp: kMaxBuf ring barriers and one for the representative's own rows
    o += (size_t)warps * 8 * (kMaxBuf + 1);
    o = (o + 127) & ~(size_t)127;
    L.o_stage = o;  // per warp: nbuf staging buffers, then the representative's own rows
    L.own_elems = own ? ((size_t)W * B * esize + 15) / 16 * 16 / esize : 0;
    L.per_warp_stage = ((size_t)nbuf * stage_elems * esize + L.own_elems * esize + 127) & ~(size_t)127;
    o += (size_t)warps * L.per_warp_stage;
    L.total = o;
    return L;
}

__device__ __forceinline__ unsigned hvp_digit(uint64_t n, int k, int bits) {
    return (unsigned)(n >> (bits * k)) & ((1u << bits) - 1);
}

// position of the n-th (0-based) set bit of m
__device__ __forceinline__ int hvp_nth_set_bit(uint32_t m, int n) {
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

// ---------------------------------------------------------------- exact-product dot accumulation

// FP32 vectors: x*y exactly as (p, e) with p = fl(xy), e = fma(x, y, -p); the
// pair is added to a double-float accumulator (hi, lo) by TwoSum.
struct DotAcc32 {
    float hi, lo;
    __device__ __forceinline__ void zero() { hi = lo = 0.f; }
    __device__ __forceinline__ void add(float x, float y) {
        const float p = x * y;
        const float e = fmaf(x, y, -p);
        const float s = hi + p;
        const float bp = s - hi;
        const float err = (hi - (s - bp)) + (p - bp);
        hi = s;
        lo += err + e;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
struct DotAcc64 {
    double v;
    __device__ __forceinline__ void zero() { v = 0.0; }
    __device__ __forceinline__ void add(double x, double y) { v = fma(x, y, v); }
    __device__ __forceinline__ double value() const { return v; }
};
template <typename VT>
using DotAcc = typename std::conditional<sizeof(VT) == 4, DotAcc32, DotAcc64>::type;

// ---------------------------------------------------------------- contraction of one flip, one block

template <typename VT, int D, int Z, int W>
__device__ __forceinline__ void hvp_contract_block(const VT *__restrict__ R, const VT *__restrict__ xs, int B, int b,
                                                   int sid, int nk, int ko, const VT *__restrict__ Vk, VT cf,
                                                   VT (&z)[W]) {
    constexpr int RP = rho_row(D);
    VT u[D];
    if (sid == 0) {
#pragma unroll
        for (int g2 = 0; g2 < D; ++g2) u[g2] = xs[(Z + g2) * B + b];
    } else {
#pragma unroll
        for (int g2 = 0; g2 < D; ++g2) u[g2] = (VT)0;
        const VT *Vs = Vk + (size_t)sid * D * D;
        for (int kp = 0; kp < nk; ++kp) {
            const VT xv = xs[(ko + kp) * B + b];
#pragma unroll
            for (int g2 = 0; g2 < D; ++g2) u[g2] += __ldg(Vs + g2 * D + kp) * xv;
        }
    }
#pragma unroll
    for (int be = 0; be < D; ++be) {
        VT row[RP];
        load_row<VT, RP>(R + be * RP, row);
        VT acc = row[0] * u[0];
#pragma unroll
        for (int ga = 1; ga < D; ++ga) acc += row[ga] * u[ga];
        z[Z + be] += cf * acc;
    }
}

// ---------------------------------------------------------------- contraction of one flip, one block

__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// two FP32 FMAs in one instruction (sm_100 and later): d = a * b + c, element-wise
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// z[beta] += cf * sum_gamma R[gamma * RP + beta] u[gamma] for beta < D.  FP32 with
// D >= 2 runs pairs of output rows through fma.f32x2 (rows of R padded to RP,
// an even count); otherwise scalar FMAs.  Same products and summation order
// over gamma either way (the first product is a multiply, as a fused
// multiply-add onto zero would round it).
template <typename VT, int D, int RP>
__device__ __forceinline__ void hvp_rows(const VT *__restrict__ R, const VT (&u)[D], VT cf, VT *z) {
    if constexpr (sizeof(VT) == 4 && D >= 2) {
        constexpr int NP = (D + 1) / 2;
        unsigned long long acc[NP];
#pragma unroll
        for (int ga = 0; ga < D; ++ga) {
            VT row[RP];
            load_row<VT, RP>(R + ga * RP, row);
            const unsigned long long uu = f2_pack(u[ga], u[ga]);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const unsigned long long rr = f2_pack(row[2 * q], row[2 * q + 1]);
                acc[q] = ga == 0 ? f2_mul(rr, uu) : f2_fma(rr, uu, acc[q]);
            }
        }
        const unsigned long long cc = f2_pack(cf, cf);
#pragma unroll
        for (int q = 0; q < D / 2; ++q) {  // z pairs += cf * acc, the same FMA per element
            float lo, hi;
            f2_unpack(f2_fma(acc[q], cc, f2_pack(z[2 * q], z[2 * q + 1])), lo, hi);
            z[2 * q] = lo;
            z[2 * q + 1] = hi;
        }
        if constexpr (D % 2) {
            float lo, hi;
            f2_unpack(acc[NP - 1], lo, hi);
            z[D - 1] += cf * lo;
        }
    } else {
        VT acc[D];
#pragma unroll
        for (int be = 0; be < D; ++be) acc[be] = (VT)0;
#pragma unroll
        for (int ga = 0; ga < D; ++ga) {
            VT row[RP];
            load_row<VT, RP>(R + ga * RP, row);
#pragma unroll
            for (int be = 0; be < D; ++be) acc[be] += row[be] * u[ga];
        }
#pragma unroll
        for (int be = 0; be < D; ++be) z[be] += cf * acc[be];
    }
}

// ---------------------------------------------------------------- storage conversions

// Stored vector elements are VT, or FP16 for FP32 arithmetic (read widened to
// FP32, written rounded to nearest).
template <typename VT, typename ST>
__device__ __forceinline__ VT st_get(ST v) {
    if constexpr (std::is_same<ST, __half>::value)
        return __half2float(v);
    else
        return (VT)v;
}
template <typename VT, typename ST>
__device__ __forceinline__ ST st_put(VT v) {
    if constexpr (std::is_same<ST, __half>::value)
        return __float2half_rn(v);
    else
        return (ST)v;
}

// ---------------------------------------------------------------- the kernel

// threads per CTA at most: 1024 for FP32 one-block shapes, fewer when registers are scarcer
template <typename VT, class SH>
__host__ __device__ constexpr int hvp_max_threads() {
    return (sizeof(VT) == 8 || SH::W > 8) ? 512 : 768;
}

// MODE 0: search (steps 1-4 on the fly); 1: table (flips read from the
// sector's entry table, no images, search or lookup); 2: build (steps 1-4,
// then the flips are written to the entry table; no gathers or outputs).
template <typename VT, typename ST, class SH, int GPL, bool HALF, int MODE>
__global__ void __launch_bounds__(hvp_max_threads<VT, SH>(), 1) hvp_kernel(const __grid_constant__ HvpArgs<VT> a) {
    using LT = typename std::conditional<HALF, uint32_t, uint64_t>::type;
    constexpr int K = SH::K;
    constexpr int W = SH::W;
    constexpr int MAXF = HALF ? 64 : 128;
    extern __shared__ __align__(128) uint8_t smem[];
    const int warps = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const HvpLayout L = hvp_layout<VT, HALF>(a.n_chunks, a.n_bonds, a.rho_smem ? a.rho_total : 0, warps, K, W, a.B,
                                             a.nbuf, a.stage_elems, MODE != 2 && a.tma && a.own, (int)sizeof(ST),
                                             MODE != 1);
    const bool own_on = MODE != 2 && a.tma && a.own;
    if (MODE != 1) {
        const size_t n_tab = HALF ? (size_t)a.n_chunks * 4 * kMaxG * 4 : (size_t)kMaxG * 64;
        const uint4 *src0 = reinterpret_cast<const uint4 *>(HALF ? (const void *)a.lut2 : (const void *)a.pos);
        for (size_t i = threadIdx.x; i < n_tab / 16; i += blockDim.x) reinterpret_cast<uint4 *>(smem)[i] = src0[i];
        const size_t n_dt = (size_t)a.n_bonds * kMaxG * (HALF ? 4 : 8);
        const uint4 *src1 = reinterpret_cast<const uint4 *>(a.dtab);
        for (size_t i = threadIdx.x; i < n_dt / 16; i += blockDim.x)
            reinterpret_cast<uint4 *>(smem + L.o_dtab)[i] = src1[i];
    }
    {
        if (a.rho_smem) {
            const uint4 *src2 = reinterpret_cast<const uint4 *>(a.rhoT);
            for (int i = threadIdx.x; i < a.rho_total * (int)sizeof(VT) / 16; i += blockDim.x)
                reinterpret_cast<uint4 *>(smem + L.o_rho)[i] = src2[i];
        }
        for (int i = threadIdx.x; i < 2 * a.n_bonds; i += blockDim.x) smem[L.o_bond + i] = a.bonds[i];
        double *red = reinterpret_cast<double *>(smem + L.o_red);
        for (int i = threadIdx.x; i < K * a.B; i += blockDim.x) red[i] = 0.0;
        if (lane <= kMaxBuf) mbar_init(smem_u32(smem + L.o_bar + 8 * ((kMaxBuf + 1) * wid + lane)), 1);
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncthreads();
    const uint32_t *s_lut = reinterpret_cast<const uint32_t *>(smem);
    const uint8_t *s_pos = smem;
    const LT *s_dtab = reinterpret_cast<const LT *>(smem + L.o_dtab);
    const VT *rho_base = a.rho_smem ? reinterpret_cast<const VT *>(smem + L.o_rho) : a.rhoT;
    const uint8_t *s_bond = smem + L.o_bond;
    double *red = reinterpret_cast<double *>(smem + L.o_red);
    uint32_t *f_off = reinterpret_cast<uint32_t *>(smem + L.o_flip) + (size_t)wid * MAXF * 2;
    uint32_t *f_sg = f_off + MAXF;
    VT *f_c = reinterpret_cast<VT *>(smem + L.o_fc) + (size_t)wid * MAXF;
    const uint32_t bar0 = smem_u32(smem + L.o_bar + 8 * (kMaxBuf + 1) * wid);
    const uint32_t bar_own = bar0 + 8 * kMaxBuf;
    ST *stage = reinterpret_cast<ST *>(smem + L.o_stage + (size_t)wid * L.per_warp_stage);
    const uint32_t stage_s = smem_u32(stage);
    ST *own = stage + (size_t)a.nbuf * a.stage_elems;  // the representative's own rows (bulk-copy path)
    const uint32_t own_s = smem_u32(own);

    const int B = a.B, BT = a.BT;
    const int Q = 32 >> a.lgBT;        // flip groups per warp
    const int b = lane & (BT - 1);
    const int fg = lane >> a.lgBT;
    const VT halfJ = a.J * (VT)0.5;
    uint32_t parity = 0;               // bit i: phase parity of buffer i (bit kMaxBuf: own rows)
    uint32_t pending = 0;              // bit i: copies in flight into buffer i
    bool dead = false;                 // a wait ran out: no more work for this warp
    DotAcc<VT> dacc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) dacc[k].zero();
    const bool want_dot = a.dot_part != nullptr;
    int cur_part = -1;
    unsigned long long n_flips = 0;  // profiling: flips of this warp, one atomic at the end

    // CTA-wide flush of the per-lane dot accumulators into the partials of part p
    auto flush = [&](int p) {
        double v[K];
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = dacc[k].value();
#pragma unroll
        for (int k = 0; k < K; ++k)
            for (int w = BT; w < 32; w <<= 1) v[k] += __shfl_xor_sync(kFullMask, v[k], w);
        for (int w = 0; w < warps; ++w) {  // fixed order over warps: deterministic sums
            __syncthreads();
            if (wid == w && lane < B) {
#pragma unroll
                for (int k = 0; k < K; ++k) red[k * B + lane] += v[k];
            }
        }
        __syncthreads();
        double *dst = a.dot_part + ((size_t)p * gridDim.x + blockIdx.x) * K * B;
        for (int i = threadIdx.x; i < K * B; i += blockDim.x) {
            dst[i] = red[i];
            red[i] = 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; ++k) dacc[k].zero();
    };

    for (uint64_t t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        int p = 0;
        if (a.n_parts > 1) {  // last part whose first tile is <= t
            int lo = 0, hi = a.n_parts - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(&a.parts[mid].tile0) <= t)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            p = lo;
        }
        if (want_dot && p != cur_part) {
            if (cur_part >= 0) flush(cur_part);
            cur_part = p;
        }
        const HvpPart<VT> &P = a.n_parts == 1 ? a.part0 : a.parts[p];
        const uint64_t n_reps = P.n_reps;
        const uint64_t r0 = (t - P.tile0) * (uint64_t)a.tile_reps;
        const uint64_t r1 = min(r0 + (uint64_t)a.tile_reps, n_reps);
        const HvRec *rec = P.rec;
        const VT *sqrtS = P.sqrtS;
        const ST *__restrict__ x = static_cast<const ST *>(P.x);
        ST *__restrict__ y = static_cast<ST *>(P.y);
        for (uint64_t rep = r0 + wid; rep < r1 && !dead; rep += warps) {
            const HvRec rr = rec[rep];
            const int sid = (int)rr.sid;
            const size_t seg = (size_t)rr.off * B;  // first element of r's W rows
            if (MODE != 2 && sid != 0 && __ldg(P.wtab + sid) == 0) {  // no block has rows for this orbit: y~(r) = 0
                for (int e = lane; e < W * B; e += 32) y[seg + e] = st_put<VT, ST>((VT)0);
                continue;
            }
            const LT lab = (LT)rr.label;
            if (MODE != 2 && !own_on) {  // the own rows are read in the epilogue: start bringing them into L2 now
                const uint32_t bytes = (uint32_t)(W * B * (int)sizeof(ST));
                const char *src = reinterpret_cast<const char *>(x + seg);
                for (uint32_t o = (uint32_t)lane * 128u; o < bytes; o += 32u * 128u) prefetch_l2(src + o);
                if (lane == 31) prefetch_l2(src + bytes - 1);  // the last line when the segment is not aligned
            }
            if (own_on) {  // the representative's own rows (diagonal term, <x~, y~>) land during the search
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    const uint32_t bytes = (uint32_t)(W * B * (int)sizeof(ST));
                    mbar_arrive_expect_tx(bar_own, bytes);
                    bulk_copy_g2s(own_s, x + seg, bytes, bar_own);
                }
                pending |= 1u << kMaxBuf;
            }

            int nf = 0;
            VT diag = (VT)0;
            if constexpr (MODE == 1) {  // diagonal term, and the flips from the entry table
                int diag4 = 0;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int e = lane + 32 * h;
                    if (e < a.n_bonds)
                        diag4 += (2 * (int)hvp_digit(lab, s_bond[2 * e], a.bits) - a.two_s) *
                                 (2 * (int)hvp_digit(lab, s_bond[2 * e + 1], a.bits) - a.two_s);
                }
                diag4 = __reduce_add_sync(kFullMask, diag4);
                diag = a.J * (VT)diag4 * (VT)0.25;
                const uint64_t e0 = __ldg(P.eoff + rep);
                nf = (int)(__ldg(P.eoff + rep + 1) - e0);
                n_flips += (unsigned long long)nf;
                for (int base = lane; base < nf; base += 32) {
                    const uint2 raw = __ldg(reinterpret_cast<const uint2 *>(P.ent + e0 + base));
                    const uint32_t tgt = raw.x, g8 = raw.y & 255u, es = (raw.y >> 8) & 255u, sidf = raw.y >> 16;
                    VT c = halfJ;
                    if (a.two_s != 1) {
                        const int e = (int)(es & 127u);
                        const int ai = (int)hvp_digit(lab, s_bond[2 * e], a.bits);
                        const int aj = (int)hvp_digit(lab, s_bond[2 * e + 1], a.bits);
                        c = halfJ * ((es & 128u) == 0 ? a.up[ai] * a.dn[aj] : a.dn[ai] * a.up[aj]);
                    }
                    f_off[base] = tgt * (uint32_t)W;
                    f_sg[base] = (sidf << 8) | g8;
                    f_c[base] = c * __ldg(sqrtS + sidf);
                }
            } else {
            // 1. images of r under the lane's elements
            LT I[GPL];
#pragma unroll
            for (int c = 0; c < GPL; ++c) {
                const int g = lane + 32 * c;
                LT v = 0;
                if (HALF) {
                    for (int q = 0; q < a.n_chunks; ++q)
                        v |= s_lut[(q * 4 + (int)((lab >> (2 * q)) & 3)) * kMaxG + g];
                } else {
                    for (int k = 0; k < a.N; ++k) v += (LT)hvp_digit(lab, k, a.bits) << s_pos[g * 64 + k];
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
                    ai = (int)hvp_digit(lab, s_bond[2 * e], a.bits);
                    aj = (int)hvp_digit(lab, s_bond[2 * e + 1], a.bits);
                    diag4 += (2 * ai - a.two_s) * (2 * aj - a.two_s);
                }
                if (HALF) {
                    m[h] = __ballot_sync(kFullMask, has && ai != aj);
                } else {
                    m[2 * h] = __ballot_sync(kFullMask, has && ai < a.two_s && aj > 0);      // s_i^+ s_j^-
                    m[2 * h + 1] = __ballot_sync(kFullMask, has && ai > 0 && aj < a.two_s);  // s_i^- s_j^+
                }
            }
            diag4 = __reduce_add_sync(kFullMask, diag4);
            diag = a.J * (VT)diag4 * (VT)0.25;
            nf = __popc(m[0]) + __popc(m[1]) + __popc(m[2]) + __popc(m[3]);
            n_flips += (unsigned long long)nf;
            if (MODE == 2 && lane == 0 && (uint64_t)nf != P.eoff[rep + 1] - P.eoff[rep])
                atomicOr(a.err, kErrMissingRep);  // the count pass and the kernel disagree

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
                    const int bit = hvp_nth_set_bit(m[w], f);
                    if (HALF) {
                        my_e = bit + 32 * w;
                        my_c = halfJ;
                    } else {
                        my_e = bit + 32 * (w >> 1);
                        my_sg = (w & 1) ? -1 : 1;
                        const int ai = (int)hvp_digit(lab, s_bond[2 * my_e], a.bits);
                        const int aj = (int)hvp_digit(lab, s_bond[2 * my_e + 1], a.bits);
                        my_c = halfJ * (my_sg > 0 ? a.up[ai] * a.dn[aj] : a.dn[ai] * a.up[aj]);
                    }
                }
                LT my_rp = 0;
                int my_g = 0;
                // one flip's orbit minimum over the warp; FL: also the spin-flipped candidates
                // (G x Z_2, elements (g, 1) after all of G: index 128 + g)
                auto search = [&](int j, auto FL) {
                    const int e = __shfl_sync(kFullMask, my_e, j);
                    const int sg = HALF ? 1 : __shfl_sync(kFullMask, my_sg, j);
                    LT best = 0;
                    int bg = 0;
                    LT cands[GPL];
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
                        cands[c] = cand;
                        if (c == 0 || cand < best) {
                            best = cand;
                            bg = g;
                        }
                    }
                    if constexpr (decltype(FL)::value) {  // after all of G, in index order: strict <
#pragma unroll
                        for (int c = 0; c < GPL; ++c) {
                            const LT cf = HALF ? (cands[c] ^ (LT)a.flipc) : ((LT)a.flipc - cands[c]);
                            if (cf < best) {
                                best = cf;
                                bg = (lane + 32 * c) | 128;
                            }
                        }
                    }
                    LT mn;
                    if (HALF) {
                        mn = (LT)__reduce_min_sync(kFullMask, (unsigned)best);
                    } else {
                        const unsigned hi = __reduce_min_sync(kFullMask, (unsigned)((uint64_t)best >> 32));
                        const unsigned lo = __reduce_min_sync(
                            kFullMask, (unsigned)((uint64_t)best >> 32) == hi ? (unsigned)best : ~0u);
                        mn = (LT)(((uint64_t)hi << 32) | (uint64_t)lo);
                    }
                    const int gs = (int)__reduce_min_sync(kFullMask, best == mn ? (unsigned)bg : 0xffffu);
                    if (lane == j) {
                        my_rp = mn;
                        my_g = gs;
                    }
                };
                if (!a.flip) {
#pragma unroll 2
                    for (int j = 0; j < nround; ++j) search(j, std::false_type{});
                } else {
                    for (int j = 0; j < nround; ++j) search(j, std::true_type{});
                }
                if (lane < nround) {
                    const uint64_t key = (uint64_t)my_rp;
                    const uint64_t bk = key >> P.bucket_shift;
                    uint32_t off_f = 0, sid_f = 0, idx_f = 0;
                    bool found = false;
                    if (bk < P.n_buckets) {
                        uint32_t lo = __ldg(P.bucket + bk), hi = __ldg(P.bucket + bk + 1);
                        const uint32_t hi0 = hi;
                        uint4 hrec = make_uint4(0, 0, 0, 0);
                        while (lo < hi) {
                            const uint32_t mid = (lo + hi) >> 1;
                            const uint4 rm = __ldg(reinterpret_cast<const uint4 *>(rec + mid));
                            const uint64_t lm = ((uint64_t)rm.y << 32) | rm.x;
                            if (lm < key) {
                                lo = mid + 1;
                            } else {
                                hi = mid;
                                hrec = rm;
                            }
                        }
                        if (lo < hi0 && ((((uint64_t)hrec.y << 32) | hrec.x) == key)) {
                            found = true;
                            off_f = hrec.z;
                            sid_f = hrec.w;
                            idx_f = lo;
                        }
                    }
                    if (!found) {
                        atomicOr(a.err, kErrMissingRep);
                        my_c = (VT)0;
                    }
                    if constexpr (MODE == 2) {
                        const uint64_t slot = P.eoff[rep] + (uint64_t)(base + lane);
                        if (slot < P.eoff[rep + 1]) {
                            HvEntry en;
                            en.tgt = idx_f;
                            en.g = (uint8_t)my_g;
                            en.esign = (uint8_t)(my_e | (my_sg < 0 ? 128 : 0));
                            en.sid = (uint16_t)sid_f;
                            P.ent[slot] = en;
                        }
                    } else {
                        f_off[base + lane] = off_f;
                        f_sg[base + lane] = (sid_f << 8) | (uint32_t)my_g;  // g* < |G| <= 128, bit 7: spin flip
                        f_c[base + lane] = my_c * __ldg(sqrtS + sid_f);      // c_a sqrt|Stab r'|
                    }
                }
            }
            }  // search and lookup
            if constexpr (MODE == 2) continue;  // build mode: the flips are in the table
            __syncwarp();

            // 5-6. gathers and contraction, Q flips per group
            VT z[W];
#pragma unroll
            for (int i = 0; i < W; ++i) z[i] = (VT)0;
            const int n_groups = (nf + Q - 1) / Q;
            const int nbuf = a.nbuf;
            auto fill = [&](int grp) {
                const int buf = grp % nbuf;
                const int j = grp * Q + (a.tma ? lane : fg);
                if (a.tma) {
                    const uint32_t bytes = (lane < Q && j < nf) ? (uint32_t)(W * B * (int)sizeof(ST)) : 0u;
                    const uint32_t total = (uint32_t)min(Q, nf - grp * Q) * (uint32_t)(W * B * (int)sizeof(ST));
                    const uint32_t bar = bar0 + 8 * buf;
                    fence_proxy_async_smem();  // earlier generic reads of the buffer before the async writes
                    __syncwarp();
                    if (lane == 0) mbar_arrive_expect_tx(bar, total);
                    __syncwarp();
                    if (bytes)
                        bulk_copy_g2s(stage_s + (uint32_t)(((size_t)buf * a.stage_elems + (size_t)lane * a.slot_elems) *
                                                           sizeof(ST)),
                                      x + (size_t)f_off[j] * B, bytes, bar);
                    pending |= 1u << buf;
                } else {
                    if (j < nf && b < B) {
                        const ST *src = x + (size_t)f_off[j] * B + b;
                        ST *dst = stage + (size_t)buf * a.stage_elems + (size_t)fg * a.slot_elems + b;
                        ST v[W];
#pragma unroll
                        for (int r = 0; r < W; ++r) v[r] = __ldg(src + r * B);
#pragma unroll
                        for (int r = 0; r < W; ++r) dst[r * B] = v[r];
                    }
                    __syncwarp();
                }
            };
            const int npro = min(nbuf, n_groups);
            for (int grp = 0; grp < npro; ++grp) fill(grp);
            for (int grp = 0; grp < n_groups; ++grp) {
                const int buf = grp % nbuf;
                if (a.tma) {
                    if (!mbar_wait_bounded(bar0 + 8 * buf, (parity >> buf) & 1u, a.wait_limit)) {
                        dead = true;
                        break;
                    }
                    parity ^= 1u << buf;
                    pending &= ~(1u << buf);
                }
                const int j = grp * Q + fg;
                if (j < nf && b < B) {
                    const int g_j = (int)(f_sg[j] & 127u);
                    const unsigned negj = (f_sg[j] & 128u) ? a.neg : 0u;  // (g*, 1) in a Gamma- block: -rho(g*)
                    const VT cf = f_c[j];
                    const ST *xs = stage + (size_t)buf * a.stage_elems + (size_t)fg * a.slot_elems + b;
                    static_for<K>([&](auto kc) {
                        constexpr int k = decltype(kc)::value;
                        constexpr int D = SH::template D<k>;
                        constexpr int Zk = SH::template Z<k>;
                        constexpr int RP = rho_row(D);
                        // R[gamma][beta] = rho_k(g*)[gamma][beta]; z_beta += cf sum_gamma R[gamma][beta] u_gamma
                        const VT *R = rho_base + a.rho_off[k] + (size_t)g_j * D * RP;
                        VT u[D];
#pragma unroll
                        for (int g2 = 0; g2 < D; ++g2) u[g2] = st_get<VT, ST>(xs[(Zk + g2) * B]);
                        hvp_rows<VT, D, RP>(R, u, ((negj >> k) & 1u) ? -cf : cf, z + Zk);
                    });
                }
                __syncwarp();
                if (grp + nbuf < n_groups) fill(grp + nbuf);
            }
            if (dead) {  // a wait ran out: record it, let the copies in flight land, stop
                if (lane == 0) atomicOr(a.err, kErrWaitTimeout);
                for (int bi = 0; bi <= kMaxBuf; ++bi)
                    if ((pending >> bi) & 1u) mbar_wait_bounded(bar0 + 8 * bi, (parity >> bi) & 1u, kDrainCycles);
                pending = 0;
                break;
            }

            // 7. sum over flip groups, output rows, <x~, y~>
            VT *zs = reinterpret_cast<VT *>(stage);  // the staging buffers are idle here
            // Four flip groups whose partial rows fit in the staging buffers: every lane stores its
            // rows ([fg][row][b], a group stride of W BT + BT elements keeps the stores conflict-free),
            // then each lane adds the four partials of W BT / 32 entries in the order the shuffle
            // butterfly below uses, (z0 + z1) + (z2 + z3), into group 0's slice: the same sums.
            const int zstride = W * BT + BT;
            const bool zq = Q == 4 && (size_t)4 * zstride * sizeof(VT) <= (size_t)nbuf * a.stage_elems * sizeof(ST);
            if (zq) {
#pragma unroll
                for (int i = 0; i < W; ++i) zs[fg * zstride + i * BT + b] = z[i];
                __syncwarp();
                for (int e = lane; e < W * BT; e += 32)
                    zs[e] = (zs[e] + zs[zstride + e]) + (zs[2 * zstride + e] + zs[3 * zstride + e]);
            } else {
#pragma unroll
                for (int i = 0; i < W; ++i)
                    for (int w = BT; w < 32; w <<= 1) z[i] += __shfl_xor_sync(kFullMask, z[i], w);
            }
            if (own_on) {
                if (!mbar_wait_bounded(bar_own, (parity >> kMaxBuf) & 1u, a.wait_limit)) {
                    if (lane == 0) atomicOr(a.err, kErrWaitTimeout);
                    mbar_wait_bounded(bar_own, (parity >> kMaxBuf) & 1u, kDrainCycles);
                    pending = 0;
                    dead = true;
                    break;
                }
                parity ^= 1u << kMaxBuf;
                pending &= ~(1u << kMaxBuf);
            }
            if (!zq && fg == 0) {
#pragma unroll
                for (int i = 0; i < W; ++i) zs[i * BT + b] = z[i];
            }
            __syncwarp();
            if (b < B) {
                const VT inv_sq = sid == 0 ? (VT)1 : (VT)1 / __ldg(sqrtS + sid);
                static_for<K>([&](auto kc) {
                    constexpr int k = decltype(kc)::value;
                    constexpr int D = SH::template D<k>;
                    constexpr int Zk = SH::template Z<k>;
                    for (int gam = fg; gam < D; gam += Q) {
                        VT val;
                        if (sid == 0) {
                            val = zs[(Zk + gam) * BT + b];
                        } else {  // projector onto the range of V_k(r)
                            const VT *Pr = P.Pj[k] + ((size_t)sid * D + gam) * D;
                            val = (VT)0;
#pragma unroll
                            for (int be = 0; be < D; ++be) val += __ldg(Pr + be) * zs[(Zk + be) * BT + b];
                            val *= inv_sq;
                        }
                        const size_t e = seg + (size_t)(Zk + gam) * B + b;
                        const VT xv = st_get<VT, ST>(own_on ? own[(Zk + gam) * B + b] : __ldg(x + e));
                        const ST ys = st_put<VT, ST>(val + diag * xv);
                        y[e] = ys;
                        if (want_dot) dacc[k].add(xv, st_get<VT, ST>(ys));  // the values as stored
                    }
                });
            }
            __syncwarp();
        }
    }
    if (want_dot && cur_part >= 0) flush(cur_part);
    if (a.flips && lane == 0 && n_flips) atomicAdd(a.flips, n_flips);
}

// ---------------------------------------------------------------- host side

struct HvpGeom {
    int warps, nbuf, tma, tile_reps, grid, rho_smem, own;
};

template <typename VT, typename ST, class SH, int GPL, bool HALF, int MODE>
size_t hvp_smem_t(const HvpArgs<VT> &a, int warps, int nbuf) {
    return hvp_layout<VT, HALF>(a.n_chunks, a.n_bonds, a.rho_smem ? a.rho_total : 0, warps, SH::K, SH::W, a.B, nbuf,
                                a.stage_elems, MODE != 2 && a.tma && a.own, (int)sizeof(ST), MODE != 1)
        .total;
}

// CTAs per SM for the given geometry (0 if it does not fit); sets the shared-memory attribute.
template <typename VT, typename ST, class SH, int GPL, bool HALF, int MODE>
int hvp_occupancy_t(const HvpArgs<VT> &a, int warps, int nbuf) {
    auto kern = hvp_kernel<VT, ST, SH, GPL, HALF, MODE>;
    if (warps * 32 > hvp_max_threads<VT, SH>()) return 0;
    const size_t smem = hvp_smem_t<VT, ST, SH, GPL, HALF, MODE>(a, warps, nbuf);
    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem > (size_t)max_smem) return 0;
    {  // the attribute is only ever raised: a plan made on another thread never invalidates a launch
        static std::mutex mu;
        static int raised[64] = {};
        std::lock_guard<std::mutex> lk(mu);
        const int d = dev & 63;
        if ((int)smem > raised[d]) {
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                return 0;
            raised[d] = (int)smem;
        }
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem) != cudaSuccess) return 0;
    return per_sm;
}

template <typename VT, typename ST, class SH, int GPL, bool HALF, int MODE>
ftlm_status hvp_launch_t(HvpArgs<VT> a, const HvpGeom &geo, cudaStream_t stream) {
    auto kern = hvp_kernel<VT, ST, SH, GPL, HALF, MODE>;
    a.nbuf = geo.nbuf;
    a.tma = geo.tma;
    a.tile_reps = geo.tile_reps;
    a.rho_smem = geo.rho_smem;
    a.own = geo.own;
    const size_t smem = hvp_smem_t<VT, ST, SH, GPL, HALF, MODE>(a, geo.warps, geo.nbuf);
    kern<<<(unsigned)geo.grid, geo.warps * 32, smem, stream>>>(a);
    count_launch();
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

}  // namespace ftlm
