// Table-mode H·v with one thread per output representative, for one block
// (K = 1) and one right-hand side (B = 1): Eqs. 15-16 in the pull form with the
// flips read from the sector's entry table (Section 3).  A warp of the search
// or table kernel works on one representative at a time; with B = 1 most of its
// lanes idle and each representative is a chain of dependent memory round trips
// (record, entry offsets, entries, gathers).  Here every thread walks its own
// representative's entries, so a warp keeps 32 such chains in flight.  The
// contributions are summed in entry order (the warp kernels sum them per flip
// group and then across groups), so results agree with theirs to rounding.
#pragma once

#include "hvp.cuh"

namespace ftlm {

constexpr int kLaneThreads = 256;
constexpr int kLaneFlips = 2;  // flips whose entries and rows are loaded before the first is summed

__host__ __device__ constexpr int lane_gcd(int a, int b) { return b == 0 ? a : lane_gcd(b, a % b); }

// Element j of a span of 32-bit words (j a compile-time constant after unrolling).
template <typename ST>
__device__ __forceinline__ ST span_elem(const uint32_t *w, int j) {
    if constexpr (sizeof(ST) == 2) {
        return __ushort_as_half((unsigned short)(w[j >> 1] >> (16 * (j & 1))));
    } else if constexpr (sizeof(ST) == 4) {
        return __uint_as_float(w[j]);
    } else {
        return __hiloint2double((int)w[2 * j + 1], (int)w[2 * j]);
    }
}

// The D stored elements of row r of x (D * sizeof(ST) bytes from byte r * D * sizeof(ST)).  A row
// starts at a multiple of gcd(D * sizeof(ST), 16) bytes past a 16-byte boundary, so the L aligned
// 16-byte words from that boundary cover it: L vector loads per lane instead of D scalar ones, a
// warp's gather then takes about 32 L sector lookups in L1 instead of 32 D.  The row is picked
// out of the words by its offset (selects over the possible offsets, no local memory).  Rows
// whose covering words would pass the end of x (n_elems elements), or an x that is not 16-byte
// aligned, take scalar loads.
template <typename VT, typename ST, int D>
__device__ __forceinline__ void lane_row(const ST *__restrict__ x, uint64_t r, uint64_t n_elems, bool vec,
                                         VT (&u)[D]) {
    constexpr int E = (int)sizeof(ST), RB = D * E, PER = 16 / E;
    constexpr int G = lane_gcd(RB, 16);
    constexpr int L = (16 - G + RB + 15) / 16;  // words covering a row at the largest offset
    constexpr int STEP = G / E, NOFF = 16 / G;  // offsets 0, STEP, ..., (NOFF - 1) STEP elements
    const uint64_t e0 = r * D, w0 = e0 / PER;
    if (vec && (w0 + L) * PER <= n_elems) {
        uint32_t w[4 * L];
#pragma unroll
        for (int l = 0; l < L; ++l) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(x) + w0 + l);
            w[4 * l] = v.x;
            w[4 * l + 1] = v.y;
            w[4 * l + 2] = v.z;
            w[4 * l + 3] = v.w;
        }
        const int off = (int)(e0 - w0 * PER);
#pragma unroll
        for (int g = 0; g < D; ++g) u[g] = st_get<VT, ST>(span_elem<ST>(w, g));
#pragma unroll
        for (int k = 1; k < NOFF; ++k) {
            const bool hit = off == k * STEP;
#pragma unroll
            for (int g = 0; g < D; ++g) {
                const VT v = st_get<VT, ST>(span_elem<ST>(w, k * STEP + g));
                u[g] = hit ? v : u[g];
            }
        }
    } else {
#pragma unroll
        for (int g = 0; g < D; ++g) u[g] = st_get<VT, ST>(__ldg(x + e0 + g));
    }
}

template <typename VT, typename ST, int D>
__global__ void __launch_bounds__(kLaneThreads) hvp_lane_kernel(const __grid_constant__ HvpArgs<VT> a) {
    constexpr int RP = rho_row(D);
    extern __shared__ __align__(128) uint8_t smem[];
    VT *s_rho = reinterpret_cast<VT *>(smem);  // rho(g) of the block, [G][D][RP]
    uint8_t *s_bond = smem + (((size_t)a.rho_total * sizeof(VT) + 15) & ~(size_t)15);
    __shared__ double red[kLaneThreads / 32];
    for (int i = threadIdx.x; i < a.rho_total; i += blockDim.x) s_rho[i] = a.rhoT[i];
    for (int i = threadIdx.x; i < 2 * a.n_bonds; i += blockDim.x) s_bond[i] = a.bonds[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const VT halfJ = a.J * (VT)0.5;
    const bool want_dot = a.dot_part != nullptr;
    DotAcc<VT> dacc;
    dacc.zero();
    int cur_part = -1;
    unsigned long long n_flips = 0;  // profiling: one atomic per warp at the end
    auto flush = [&](int p) {  // CTA sum of the per-thread <x, y> in a fixed order
        double v = dacc.value();
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
        __syncthreads();
        if (lane == 0) red[wid] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            a.dot_part[(size_t)p * gridDim.x + blockIdx.x] = t;
        }
        dacc.zero();
    };
    for (uint64_t t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        int p = 0;
        if (a.n_parts > 1) {
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
        const uint64_t rep = (t - P.tile0) * (uint64_t)a.tile_reps + threadIdx.x;
        if (rep >= P.n_reps) continue;
        const ST *__restrict__ x = static_cast<const ST *>(P.x);
        ST *__restrict__ y = static_cast<ST *>(P.y);
        const uint64_t n_elems = P.n_reps * (uint64_t)D;
        const bool vec = (reinterpret_cast<uintptr_t>(x) & 15) == 0;
        const HvRec rr = P.rec[rep];
        const int sid = (int)rr.sid;
        const size_t seg = rr.off;  // W = D rows, B = 1
        if (sid != 0 && __ldg(P.wtab + sid) == 0) {
#pragma unroll
            for (int g = 0; g < D; ++g) y[seg + g] = st_put<VT, ST>((VT)0);
            continue;
        }
        const uint64_t lab = rr.label;
        int diag4 = 0;
        for (int e = 0; e < a.n_bonds; ++e)
            diag4 += (2 * (int)hvp_digit(lab, s_bond[2 * e], a.bits) - a.two_s) *
                     (2 * (int)hvp_digit(lab, s_bond[2 * e + 1], a.bits) - a.two_s);
        const VT diag = a.J * (VT)diag4 * (VT)0.25;
        const uint64_t e0 = __ldg(P.eoff + rep), e1 = __ldg(P.eoff + rep + 1);
        n_flips += e1 - e0;
        VT z[D];
#pragma unroll
        for (int g = 0; g < D; ++g) z[g] = (VT)0;
        // one flip: coefficient of Eq. 3 times sqrt|Stab r'| (the 1/sqrt|Stab r| comes last), gather of
        // the target's row, z += cf rho(g*)^T u; flips are summed in entry order
        auto coef = [&](uint2 raw) {
            const uint32_t g8 = raw.y & 255u, es = (raw.y >> 8) & 255u, sidf = raw.y >> 16;
            VT c = halfJ;
            if (a.two_s != 1) {
                const int b = (int)(es & 127u);
                const int ai = (int)hvp_digit(lab, s_bond[2 * b], a.bits);
                const int aj = (int)hvp_digit(lab, s_bond[2 * b + 1], a.bits);
                c = halfJ * ((es & 128u) == 0 ? a.up[ai] * a.dn[aj] : a.dn[ai] * a.up[aj]);
            }
            VT cf = c * __ldg(P.sqrtS + sidf);
            if ((g8 & 128u) && (a.neg & 1u)) cf = -cf;  // (g*, 1) in a Gamma- block
            return cf;
        };
        auto accumulate = [&](uint2 raw, VT cf, const VT(&u)[D]) {
            const VT *R = s_rho + (size_t)(raw.y & 127u) * D * RP;
#pragma unroll
            for (int be = 0; be < D; ++be) {
                VT acc = R[be] * u[0];
#pragma unroll
                for (int ga = 1; ga < D; ++ga) acc += R[ga * RP + be] * u[ga];
                z[be] += cf * acc;
            }
        };
        uint64_t e = e0;
        for (; e + kLaneFlips <= e1; e += kLaneFlips) {  // kLaneFlips gathers in flight per thread
            uint2 r[kLaneFlips];
            VT u[kLaneFlips][D];
#pragma unroll
            for (int q = 0; q < kLaneFlips; ++q) r[q] = __ldg(reinterpret_cast<const uint2 *>(P.ent + e + q));
#pragma unroll
            for (int q = 0; q < kLaneFlips; ++q) lane_row<VT, ST, D>(x, r[q].x, n_elems, vec, u[q]);
#pragma unroll
            for (int q = 0; q < kLaneFlips; ++q) accumulate(r[q], coef(r[q]), u[q]);
        }
        for (; e < e1; ++e) {
            const uint2 r0 = __ldg(reinterpret_cast<const uint2 *>(P.ent + e));
            VT u0[D];
            lane_row<VT, ST, D>(x, r0.x, n_elems, vec, u0);
            accumulate(r0, coef(r0), u0);
        }
        VT val[D];
        if (sid == 0) {
#pragma unroll
            for (int g = 0; g < D; ++g) val[g] = z[g];
        } else {  // projector onto the range of V(r), and 1/sqrt|Stab r|
            const VT inv_sq = (VT)1 / __ldg(P.sqrtS + sid);
            const VT *Pr = P.Pj[0] + (size_t)sid * D * D;
#pragma unroll
            for (int g = 0; g < D; ++g) {
                VT v = (VT)0;
#pragma unroll
                for (int be = 0; be < D; ++be) v += __ldg(Pr + g * D + be) * z[be];
                val[g] = v * inv_sq;
            }
        }
        VT xo[D];
        lane_row<VT, ST, D>(x, rep, n_elems, vec, xo);
#pragma unroll
        for (int g = 0; g < D; ++g) {
            const VT xv = xo[g];
            const ST ys = st_put<VT, ST>(val[g] + diag * xv);
            y[seg + g] = ys;
            if (want_dot) dacc.add(xv, st_get<VT, ST>(ys));
        }
    }
    if (want_dot && cur_part >= 0) flush(cur_part);
    if (a.flips) {
        for (int o = 16; o; o >>= 1) n_flips += __shfl_xor_sync(kFullMask, n_flips, o);
        if (lane == 0 && n_flips) atomicAdd(a.flips, n_flips);
    }
}

template <typename VT, typename ST, int D>
size_t hvp_lane_smem(const HvpArgs<VT> &a) {
    return (((size_t)a.rho_total * sizeof(VT) + 15) & ~(size_t)15) + (size_t)2 * a.n_bonds + 16;
}

template <typename VT, typename ST, int D>
int hvp_lane_occupancy_t(const HvpArgs<VT> &a, int warps, int) {
    if (warps * 32 != kLaneThreads) return 0;
    auto kern = hvp_lane_kernel<VT, ST, D>;
    const size_t smem = hvp_lane_smem<VT, ST, D>(a);
    {  // raised only, as for the warp kernels
        static std::mutex mu;
        static int raised[64] = {};
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> lk(mu);
        if ((int)smem > raised[dev & 63]) {
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                return 0;
            raised[dev & 63] = (int)smem;
        }
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLaneThreads, smem) != cudaSuccess) return 0;
    return per_sm;
}

template <typename VT, typename ST, int D>
ftlm_status hvp_lane_launch_t(HvpArgs<VT> a, const HvpGeom &geo, cudaStream_t stream) {
    a.tile_reps = geo.tile_reps;
    hvp_lane_kernel<VT, ST, D><<<(unsigned)geo.grid, kLaneThreads, hvp_lane_smem<VT, ST, D>(a), stream>>>(a);
    count_launch();
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}

}  // namespace ftlm
