// FTLM Lanczos chains on packed sets (Section 2.2 of arXiv 2607.17429), batched
// through one packed H·v launch per step, with the step loop captured in a
// CUDA graph.
//
// The vectors are kept unnormalised: u_j with v_j = s_j u_j.  One step j is
//   A  y = H u_j (packed H·v) with <u_j, y> per (block, chain) fused into
//      the H·v epilogue;
//   fA alpha_j = s_j^2 <u_j, y>; coefficients (s_j, alpha_j s_j, beta_j s_{j-1});
//   U  w = s_j y - alpha_j s_j u_j - beta_j s_{j-1} u_{j-1}  (= H v_j - alpha_j v_j
//      - beta_j v_{j-1}), written over y, with |w|^2 per (block, chain);
//   fB beta_{j+1} = |w|, stop test, s_{j+1} = 1 / beta_{j+1}, u_{j+1} = w.
// Dot products and norms: exact products, double-float sums per representative
// and lane (FP32 vectors) or FP64 (FP64 vectors), FP64 across lanes and CTAs in a
// fixed order, so repeated runs give identical coefficients.  A chain stops
// after step j when beta_{j+1} <= tol (|alpha_j| + beta_j) (tol 1e-12 for FP64,
// 1e-6 for FP32 vectors) or when j + 1 = min(n_steps, dim).
//
// Several packed sets of the same group and shape (for instance every S^z
// sector of a cluster) run as the parts of one launch per kernel.
#include <string.h>

#include <algorithm>
#include <vector>

#include "hvp_ops.h"
#include "lanczos_packed.h"
#include "philox.cuh"
#include "ritz_thermo.cuh"

namespace ftlm {

void hv_profile_add(double ms, uint64_t rows);
unsigned long long wait_limit_cycles();

namespace {

constexpr int kLzThreads = 256;

template <typename VT>
struct LzPart {
    uint64_t n_reps;
    uint64_t tile0;
    const HvRec *rec;
    const uint8_t *ntab;           // [n_sid][K] n_k(sid)
    const VT *V[kPMaxK];           // block k: [n_sid][d_k][d_k] (Eq. 11), lifts the start vectors
    const uint64_t *boff[kPMaxK];  // block k's row offsets [n_reps] (start-vector counters)
    uint32_t key1[kPMaxK];         // Philox key word 1 of block k (block id)
    int entry0;                    // index of (part, block 0, chain 0) in the state arrays: p * K * B
    void *y;                       // start vectors: output, of the storage type
};

template <typename VT>
struct LzArgs {
    int n_parts;
    LzPart<VT> part0;
    const LzPart<VT> *parts;
    uint64_t n_tiles;
    int tile_reps;
    int B, BT, lgBT;
    int dims[kPMaxK], zoff[kPMaxK];
    int rng;
    uint32_t chain0, key0;
    double *norm_part;     // [n_parts][gridDim.x][K][B]
};

// Start vectors u_0 (Philox per block row index and chain, lifted by V_k(r)),
// with |u_0|^2 per (block, chain) as per-CTA partials.  Rows of representative
// r: r W + Z_k + gamma.
template <typename VT, typename ST, int K>
__global__ void __launch_bounds__(kLzThreads) lzp_start(const __grid_constant__ LzArgs<VT> a) {
    __shared__ double red[kPMaxK * 32];
    const int warps = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int B = a.B, BT = a.BT;
    const int Q = 32 >> a.lgBT;
    const int b = lane & (BT - 1), fg = lane >> a.lgBT;
    for (int i = threadIdx.x; i < K * B; i += blockDim.x) red[i] = 0.0;
    __syncthreads();
    DotAcc<VT> acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k].zero();
    int cur = -1;
    auto flush = [&](int p) {
        double v[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            v[k] = acc[k].value();
            for (int w = BT; w < 32; w <<= 1) v[k] += __shfl_xor_sync(kFullMask, v[k], w);
        }
        for (int w = 0; w < warps; ++w) {
            __syncthreads();
            if (wid == w && lane < B) {
#pragma unroll
                for (int k = 0; k < K; ++k) red[k * B + lane] += v[k];
            }
        }
        __syncthreads();
        double *dst = a.norm_part + ((size_t)p * gridDim.x + blockIdx.x) * K * B;
        for (int i = threadIdx.x; i < K * B; i += blockDim.x) {
            dst[i] = red[i];
            red[i] = 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k].zero();
    };
    for (uint64_t t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        int p = 0;
        if (a.n_parts > 1) {
            int lo = 0, hi = a.n_parts - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.parts[mid].tile0 <= t)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            p = lo;
        }
        const LzPart<VT> &P = a.n_parts == 1 ? a.part0 : a.parts[p];
        if (p != cur) {
            if (cur >= 0) flush(cur);
            cur = p;
        }
        const uint64_t r0 = (t - P.tile0) * (uint64_t)a.tile_reps;
        const uint64_t r1 = min(r0 + (uint64_t)a.tile_reps, P.n_reps);
        for (uint64_t rep = r0 + wid; rep < r1; rep += warps) {
            const HvRec rr = P.rec[rep];
            const int sid = (int)rr.sid;
            if (b >= B) continue;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int D = a.dims[k];
                for (int gam = fg; gam < D; gam += Q) {
                    const size_t e = ((size_t)rr.off + a.zoff[k] + gam) * B + b;
                    const uint64_t row0 = __ldg(P.boff[k] + rep);
                    VT v;
                    if (sid == 0) {
                        v = start_value_t<VT>(row0 + (uint64_t)gam, a.chain0 + (uint32_t)b, a.key0, P.key1[k], a.rng);
                    } else {  // lift the n_k(r) coefficients: V_k(r) x_k(r)
                        const int nk = __ldg(P.ntab + sid * K + k);
                        const VT *Vr = P.V[k] + ((size_t)sid * D + gam) * D;
                        v = (VT)0;
                        for (int q = 0; q < nk; ++q)
                            v += __ldg(Vr + q) * start_value_t<VT>(row0 + (uint64_t)q, a.chain0 + (uint32_t)b,
                                                                   a.key0, P.key1[k], a.rng);
                    }
                    const ST sv = st_put<VT, ST>(v);
                    static_cast<ST *>(P.y)[e] = sv;
                    const VT vs = st_get<VT, ST>(sv);  // norms of the values as stored
                    acc[k].add(vs, vs);
                }
            }
        }
    }
    if (cur >= 0) flush(cur);
}

// The update on the flat packed vector.  Rows of every representative are
// consecutive W-row segments, so element e of a part has row (e / B) mod W and
// chain e mod B; with a thread count that is a multiple of W * B every thread of
// the grid-stride loop sees one fixed (row, chain), hence one block k, one set
// of coefficients and one accumulator.  Parts are processed one after another;
// per part every CTA writes its partial |w|^2 per (block, chain).
template <typename VT>
struct LzUpd {
    int n_parts, W, B, K, has_prev;
    int blk_of_row[32];         // block of each row of a segment
    const uint64_t *elem0;      // [n_parts + 1] first element of each part in the vectors
    const int *entry0;          // [n_parts] p * K * B
    void *y;                    // in: H u_j, out: w (storage type)
    const void *u, *up;
    const VT *coef;             // [entries][3]
    double *norm_part;          // [n_parts][gridDim.x][K][B]
};

template <typename VT, typename ST>
__global__ void __launch_bounds__(kLzThreads) lzp_update(const __grid_constant__ LzUpd<VT> a) {
    __shared__ double red[kLzThreads];
    const int B = a.B, WB = a.W * a.B, K = a.K;
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int tb = (int)(g % (uint64_t)WB);
    const int k = a.blk_of_row[tb / B], b = tb % B;
    for (int p = 0; p < a.n_parts; ++p) {
        const uint64_t e0 = a.elem0[p], n = a.elem0[p + 1] - e0;
        const VT *c = a.coef + ((size_t)a.entry0[p] + k * B + b) * 3;
        const VT cy = c[0], cu = c[1], cp = a.has_prev ? c[2] : (VT)0;
        ST *y = static_cast<ST *>(a.y) + e0;
        const ST *u = static_cast<const ST *>(a.u) + e0;
        const ST *up = static_cast<const ST *>(a.up) + e0;
        DotAcc<VT> acc;
        acc.zero();
        uint64_t e = g;
        for (; e + 3 * T < n; e += 4 * T) {  // four elements in flight per thread
            VT yv[4], uv[4], pv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                yv[q] = st_get<VT, ST>(y[e + q * T]);
                uv[q] = st_get<VT, ST>(__ldg(u + e + q * T));
                pv[q] = a.has_prev ? st_get<VT, ST>(__ldg(up + e + q * T)) : (VT)0;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const ST ws = st_put<VT, ST>(cy * yv[q] - cu * uv[q] - cp * pv[q]);
                y[e + q * T] = ws;
                const VT w = st_get<VT, ST>(ws);
                acc.add(w, w);
            }
        }
        for (; e < n; e += T) {
            const VT wv = cy * st_get<VT, ST>(y[e]) - cu * st_get<VT, ST>(__ldg(u + e)) -
                          (a.has_prev ? cp * st_get<VT, ST>(__ldg(up + e)) : (VT)0);
            const ST ws = st_put<VT, ST>(wv);
            y[e] = ws;
            const VT w = st_get<VT, ST>(ws);
            acc.add(w, w);
        }
        red[threadIdx.x] = acc.value();
        __syncthreads();
        if ((int)threadIdx.x < K * B) {  // fixed order over the CTA's threads
            const int kk = threadIdx.x / B, bb = threadIdx.x % B;
            const uint64_t gb = (uint64_t)blockIdx.x * blockDim.x;
            double sum = 0.0;
            for (int i = 0; i < (int)blockDim.x; ++i) {
                const int tbi = (int)((gb + i) % (uint64_t)WB);
                if (a.blk_of_row[tbi / B] == kk && tbi % B == bb) sum += red[i];
            }
            a.norm_part[((size_t)p * gridDim.x + blockIdx.x) * K * B + threadIdx.x] = sum;
        }
        __syncthreads();
    }
}

struct LzState {
    double *alpha, *beta;       // [n_steps][entries]
    double *s, *s_prev, *bprev; // [entries]
    double *sig;                // [entries] power-of-two scale of the stored u_{j+1} (FP16 storage; else 1)
    const double *rms_rows;     // [n_parts * K] sqrt(packed rows of the block) / (16 Hmax): the scale target
    int *active, *steps;        // [entries]
    const int *m_max;           // [n_parts * K]
    double *coef64;             // [entries][3]
    float *coef32;              // [entries][3]
};

// One CTA per part, one thread per (block, chain).  Sums the per-CTA partials of
// the CTAs that processed tiles of the part (tile order fixed, so the sum is too).
// mode 0: start-vector norms; 1: alpha_j and the update coefficients; 2: beta_{j+1}.
// With `scaled` (FP16 storage) the update writes sigma w instead of w, sigma the
// per-block power of two 2^floor(log2(sqrt(rows) / (16 Hmax))) with Hmax = |J|
// n_bonds s(s+1) >= |H|: since |w| = beta_{j+1} <= |H v_j| <= Hmax, the stored
// components have a root mean square at most 1/16 and no component can exceed
// sqrt(rows) / 16, independently of the block dimension (the subnormal range of
// FP16 that a fixed scale would reach in large blocks is avoided).  sigma
// multiplies the three coefficients, beta_{j+1} = |sigma w| / sigma, and the next
// scale s_{j+1} = 1 / |sigma w| (v_{j+1} = sigma w / (sigma beta_{j+1})).  Without
// it sigma = 1 and the recurrence is unchanged.
// Slices of the partial sums per (block, chain): the CTA of a part has K B x kFinSlices threads.
constexpr int kFinThreads = 1024;
__host__ __device__ inline int fin_slices(int KB) { return KB >= kFinThreads ? 1 : (kFinThreads / KB < 8 ? kFinThreads / KB : 8); }

__global__ void lzp_finalize(int mode, int j, int K, int B, int grid, const uint64_t *tile0, const uint64_t *ntile,
                             const double *part, LzState st, double tol, int scaled) {
    const int p = blockIdx.x, KB = K * B, S = fin_slices(KB);
    const int t = threadIdx.x % KB, sl = threadIdx.x / KB;
    __shared__ double sl_sum[kFinThreads];  // [slice][K B]
    const int k = t / B, b = t % B;
    const size_t e = ((size_t)p * K + k) * B + b;
    const uint64_t nt = ntile[p], t0 = tile0[p];
    // The partials of the CTAs that worked on part p, summed in a fixed order: slice sl takes
    // partials sl, sl + S, ... in four interleaved running sums (loads in flight), the slices are
    // then added in slice order; the association depends on the partial count only.
    const uint64_t n = nt >= (uint64_t)grid ? (uint64_t)grid : nt;
    const uint64_t c0 = nt >= (uint64_t)grid ? 0 : t0 % (uint64_t)grid;
    auto at = [&](uint64_t i) {
        uint64_t c = c0 + i;
        if (c >= (uint64_t)grid) c -= (uint64_t)grid;
        return part[(((size_t)p * grid + c) * K + k) * B + b];
    };
    if (sl < S && t < KB) {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        uint64_t i = (uint64_t)sl;
        for (; i + 3 * (uint64_t)S < n; i += 4 * (uint64_t)S) {
            const double v0 = at(i), v1 = at(i + S), v2 = at(i + 2 * S), v3 = at(i + 3 * S);
            acc[0] += v0;
            acc[1] += v1;
            acc[2] += v2;
            acc[3] += v3;
        }
        if (i < n) acc[0] += at(i);  // at most three left
        if (i + S < n) acc[1] += at(i + S);
        if (i + 2 * (uint64_t)S < n) acc[2] += at(i + 2 * S);
        sl_sum[sl * KB + t] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    }
    __syncthreads();
    if (sl != 0 || t >= KB) return;
    double sum = sl_sum[t];
    for (int q = 1; q < S; ++q) sum += sl_sum[q * KB + t];
    const size_t E = (size_t)gridDim.x * K * B;
    if (mode == 0) {
        const double n = sqrt(sum);
        const bool on = n > 0.0 && st.m_max[p * K + k] > 0;
        st.s[e] = on ? 1.0 / n : 0.0;
        st.s_prev[e] = 0.0;
        st.bprev[e] = 0.0;
        st.sig[e] = 1.0;
        st.active[e] = on ? 1 : 0;
        st.steps[e] = 0;
    } else if (mode == 1) {
        double c0 = 0.0, c1 = 0.0, c2 = 0.0, al = 0.0;
        if (st.active[e]) {
            const double s = st.s[e];
            al = s * s * sum;
            c0 = s;
            c1 = al * s;
            c2 = j > 0 ? st.bprev[e] * st.s_prev[e] : 0.0;
            double sig = 1.0;
            if (scaled) {
                const double ex = floor(log2(st.rms_rows[p * K + k]));
                sig = ldexp(1.0, (int)fmin(fmax(ex, -100.0), 100.0));
            }
            st.sig[e] = sig;
            c0 *= sig;
            c1 *= sig;
            c2 *= sig;
        }
        st.alpha[(size_t)j * E + e] = al;
        st.coef64[3 * e] = c0;
        st.coef64[3 * e + 1] = c1;
        st.coef64[3 * e + 2] = c2;
        st.coef32[3 * e] = (float)c0;
        st.coef32[3 * e + 1] = (float)c1;
        st.coef32[3 * e + 2] = (float)c2;
    } else {
        if (!st.active[e]) {
            st.beta[(size_t)j * E + e] = 0.0;
            return;
        }
        const double bn = sqrt(sum);           // |sigma w| of the stored vector
        const double be = bn / st.sig[e];      // beta_{j+1} = |w|
        const double al = st.alpha[(size_t)j * E + e];
        st.beta[(size_t)j * E + e] = be;
        if (j + 1 >= st.m_max[p * K + k] || be <= tol * (fabs(al) + st.bprev[e])) {
            st.active[e] = 0;
            st.steps[e] = j + 1;
        } else {
            st.s_prev[e] = st.s[e];
            st.s[e] = 1.0 / bn;
            st.bprev[e] = be;
        }
    }
}

template <typename VT, typename ST>
ftlm_status lzp_start_launch(int K, const LzArgs<VT> &a, int grid, cudaStream_t st) {
    count_launch();
    switch (K) {
        case 1: lzp_start<VT, ST, 1><<<grid, kLzThreads, 0, st>>>(a); break;
        case 5: lzp_start<VT, ST, 5><<<grid, kLzThreads, 0, st>>>(a); break;
        case 10: lzp_start<VT, ST, 10><<<grid, kLzThreads, 0, st>>>(a); break;
        default: return fail(FTLM_EUNSUPPORTED, "no recurrence kernel for %d blocks", K);
    }
    FTLM_CUDA(cudaGetLastError());
    return FTLM_OK;
}


}  // namespace

template <typename VT, typename ST>
ftlm_status lanczos_packed_st(const std::vector<LzSetIn> &sets, int R, int n_steps, uint64_t seed, int rng,
                              cudaStream_t stream, double *alpha, double *beta, int *steps_done) {
    constexpr bool kScaled = sizeof(ST) < sizeof(VT);
    const int P = (int)sets.size();
    const PackedSet *ps0 = sets[0].ps;
    const int K = ps0->K;
    const size_t out_n = (size_t)P * K * R;
    for (size_t i = 0; i < out_n; ++i) steps_done[i] = 0;
    for (size_t i = 0; i < out_n * n_steps; ++i) alpha[i] = beta[i] = 0.0;
    const int Bmax = std::min(R, kMaxB);
    std::vector<uint64_t> row0(P + 1, 0);
    std::vector<int> m_max((size_t)P * K);
    int m_all = 0;
    for (int p = 0; p < P; ++p) {
        row0[p + 1] = row0[p] + sets[p].ps->rows;
        for (int k = 0; k < K; ++k) {
            const int lim = sets[p].n_steps > 0 ? std::min(sets[p].n_steps, n_steps) : n_steps;
            m_max[(size_t)p * K + k] = (int)std::min<uint64_t>((uint64_t)lim, sets[p].blocks[k]->dim);
            m_all = std::max(m_all, m_max[(size_t)p * K + k]);
        }
    }
    if (m_all == 0) return FTLM_OK;
    const uint64_t rows = row0[P];
    DevBuf<ST> vb[3];
    for (int q = 0; q < 3; ++q) FTLM_CUDA(vb[q].alloc(std::max<uint64_t>(rows, 1) * Bmax));
    const size_t E = (size_t)P * K * Bmax;
    DevBuf<double> dstate;
    DevBuf<float> fstate;
    DevBuf<int> istate;
    FTLM_CUDA(dstate.alloc(2 * (size_t)n_steps * E + 7 * E + (size_t)P * K));
    FTLM_CUDA(fstate.alloc(3 * E));
    FTLM_CUDA(istate.alloc(2 * E + (size_t)P * K));
    LzState st;
    st.alpha = dstate.p;
    st.beta = dstate.p + (size_t)n_steps * E;
    st.s = st.beta + (size_t)n_steps * E;
    st.s_prev = st.s + E;
    st.bprev = st.s_prev + E;
    st.coef64 = st.bprev + E;
    st.sig = st.coef64 + 3 * E;
    st.rms_rows = st.sig + E;
    {
        std::vector<double> rr((size_t)P * K);
        for (int p = 0; p < P; ++p) {
            const ftlm_sector *sp = sets[p].sec;
            const double sp1 = 0.5 * sp->two_s * (0.5 * sp->two_s + 1.0);
            const double hmax = std::max(1e-300, fabs(sp->grp.J) * sp->grp.n_bonds() * sp1);  // >= |H|
            for (int k = 0; k < K; ++k)
                rr[(size_t)p * K + k] = sqrt((double)sp->n_reps * ps0->dims[k]) / (16.0 * hmax);
        }
        FTLM_CUDA(cudaMemcpyAsync(st.sig + E, rr.data(), rr.size() * 8, cudaMemcpyHostToDevice, stream));
    }
    st.coef32 = fstate.p;
    st.active = istate.p;
    st.steps = istate.p + E;
    st.m_max = istate.p + 2 * E;
    FTLM_CUDA(cudaMemcpyAsync(istate.p + 2 * E, m_max.data(), m_max.size() * sizeof(int), cudaMemcpyHostToDevice,
                              stream));
    DevBuf<int> derr;
    FTLM_CUDA(derr.alloc(1));
    FTLM_CUDA(cudaMemsetAsync(derr.p, 0, sizeof(int), stream));
    int dev = 0, sms = kNumSMs;
    FTLM_CUDA(cudaGetDevice(&dev));
    FTLM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const double tol = sizeof(ST) == 8 ? 1e-12 : (sizeof(ST) == 4 ? 1e-6 : 1e-3);
    const char *ng = getenv("FTLM_NO_GRAPH");
    const bool use_graph = !(ng && strcmp(ng, "1") == 0);
    std::vector<double> ha, hb;
    std::vector<int> hs;

    for (int chain0 = 0; chain0 < R; chain0 += Bmax) {
        const int B = std::min(Bmax, R - chain0);
        const size_t EB = (size_t)P * K * B;  // entries of this batch
        // ---- H·v plans for the three rotations: x = vb[j % 3], y = vb[(j + 1) % 3]
        HvpPlan<VT> plan[3];
        std::vector<HvpPart<VT>> hparts[3];
        DevBuf<HvpPart<VT>> d_hparts[3];
        for (int q = 0; q < 3; ++q) {
            hparts[q].resize(P);
            for (int p = 0; p < P; ++p)
                hvp_part_of<VT>(sets[p].sec, sets[p].ps, sets[p].blocks, vb[q].p + row0[p] * B,
                                vb[(q + 1) % 3].p + row0[p] * B, hparts[q][p]);
            ftlm_status s0 = hvp_plan<VT>(sets[0].sec, ps0, hparts[q], B, (int)sizeof(ST), plan[q], stream);
            if (s0 != FTLM_OK) return s0;
            plan[q].a.err = derr.p;  // this call's own error word (launches on the same sector may run concurrently)
            plan[q].rows_total = rows;
            if (P > 1) {
                FTLM_CUDA(d_hparts[q].alloc(P));
                FTLM_CUDA(cudaMemcpyAsync(d_hparts[q].p, hparts[q].data(), P * sizeof(HvpPart<VT>),
                                          cudaMemcpyHostToDevice, stream));
                plan[q].a.parts = d_hparts[q].p;
            }
        }
        const int hv_grid = plan[0].geo.grid;
        DevBuf<double> hv_part, lz_part;
        FTLM_CUDA(hv_part.alloc((size_t)P * hv_grid * K * B));
        DevBuf<uint64_t> tiles;  // hv tile0, hv ntile, lz tile0, lz ntile
        FTLM_CUDA(tiles.alloc(4 * (size_t)P));
        // ---- recurrence kernels: tiles of 64 representatives, up to 8 CTAs per SM
        const int lz_tile = 64;
        std::vector<uint64_t> tinfo(4 * (size_t)P);
        uint64_t lz_tiles = 0;
        for (int p = 0; p < P; ++p) {
            tinfo[p] = plan[0].tile0[p];
            tinfo[P + p] = plan[0].ntile[p];
            const uint64_t nt = (sets[p].sec->n_reps + lz_tile - 1) / lz_tile;
            tinfo[2 * P + p] = lz_tiles;
            tinfo[3 * P + p] = nt;
            lz_tiles += nt;
        }
        const int lz_grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(lz_tiles, (uint64_t)sms * 8));
        FTLM_CUDA(lz_part.alloc((size_t)P * lz_grid * K * B));
        FTLM_CUDA(cudaMemcpyAsync(tiles.p, tinfo.data(), tinfo.size() * 8, cudaMemcpyHostToDevice, stream));
        std::vector<LzPart<VT>> lparts(P);  // start vectors
        DevBuf<LzPart<VT>> d_lparts;
        LzArgs<VT> la;
        for (int p = 0; p < P; ++p) {
            LzPart<VT> &lp = lparts[p];
            memset(&lp, 0, sizeof(lp));
            lp.n_reps = sets[p].sec->n_reps;
            lp.tile0 = tinfo[2 * P + p];
            lp.rec = sets[p].ps->d_rec;
            lp.ntab = sets[p].ps->d_ntab;
            for (int k = 0; k < K; ++k) {
                lp.V[k] = sizeof(VT) == 8 ? reinterpret_cast<const VT *>(sets[p].blocks[k]->d_V)
                                          : reinterpret_cast<const VT *>(sets[p].blocks[k]->d_Vf);
                lp.boff[k] = sets[p].blocks[k]->d_off;
                lp.key1[k] = (uint32_t)sets[p].block_ids[k];
            }
            lp.entry0 = p * K * B;
            lp.y = vb[0].p + row0[p] * B;
        }
        memset(&la, 0, sizeof(la));
        la.n_parts = P;
        if (P == 1) {
            la.part0 = lparts[0];
        } else {
            FTLM_CUDA(d_lparts.alloc(P));
            FTLM_CUDA(cudaMemcpyAsync(d_lparts.p, lparts.data(), P * sizeof(LzPart<VT>), cudaMemcpyHostToDevice,
                                      stream));
            la.parts = d_lparts.p;
        }
        la.n_tiles = lz_tiles;
        la.tile_reps = lz_tile;
        la.B = B;
        la.BT = plan[0].a.BT;
        la.lgBT = plan[0].a.lgBT;
        {
            int z = 0;
            for (int k = 0; k < K; ++k) {
                la.dims[k] = ps0->dims[k];
                la.zoff[k] = z;
                z += ps0->dims[k];
            }
        }
        la.rng = rng;
        la.chain0 = (uint32_t)chain0;
        la.key0 = (uint32_t)seed;
        la.norm_part = lz_part.p;
        const uint64_t *hv_t0 = tiles.p, *hv_nt = tiles.p + P, *lz_t0 = tiles.p + 2 * P, *lz_nt = tiles.p + 3 * P;
        // flat update: grid a multiple of W*B / gcd(W*B, threads) so every thread keeps one (row, chain)
        const int WB = ps0->W * B;
        int gg = WB, tt = kLzThreads;
        while (tt) {
            const int r = gg % tt;
            gg = tt;
            tt = r;
        }
        const int gstep = WB / gg;
        const int up_grid = std::max(gstep, (sms * 8 + gstep - 1) / gstep * gstep);
        DevBuf<double> up_part;
        FTLM_CUDA(up_part.alloc((size_t)P * up_grid * K * B));
        std::vector<uint64_t> elem0(P + 1), ut(2 * (size_t)P);
        std::vector<int> ent(P);
        for (int p = 0; p <= P; ++p) elem0[p] = row0[p] * (uint64_t)B;
        for (int p = 0; p < P; ++p) {
            ent[p] = p * K * B;
            ut[p] = 0;
            ut[P + p] = (uint64_t)up_grid;  // every CTA writes a partial of every part
        }
        DevBuf<uint64_t> d_elem0, d_ut;
        DevBuf<int> d_ent;
        FTLM_CUDA(d_elem0.alloc(P + 1));
        FTLM_CUDA(d_ut.alloc(2 * (size_t)P));
        FTLM_CUDA(d_ent.alloc(P));
        FTLM_CUDA(cudaMemcpyAsync(d_elem0.p, elem0.data(), (P + 1) * 8, cudaMemcpyHostToDevice, stream));
        FTLM_CUDA(cudaMemcpyAsync(d_ut.p, ut.data(), 2 * (size_t)P * 8, cudaMemcpyHostToDevice, stream));
        FTLM_CUDA(cudaMemcpyAsync(d_ent.p, ent.data(), P * sizeof(int), cudaMemcpyHostToDevice, stream));
        LzUpd<VT> ua[3];
        for (int q = 0; q < 3; ++q) {
            LzUpd<VT> &U = ua[q];
            memset(&U, 0, sizeof(U));
            U.n_parts = P;
            U.W = ps0->W;
            U.B = B;
            U.K = K;
            int r = 0;
            for (int k = 0; k < K; ++k)
                for (int d = 0; d < ps0->dims[k]; ++d) U.blk_of_row[r++] = k;
            U.elem0 = d_elem0.p;
            U.entry0 = d_ent.p;
            U.y = vb[(q + 1) % 3].p;
            U.u = vb[q].p;
            U.up = vb[(q + 2) % 3].p;
            U.coef = sizeof(VT) == 8 ? reinterpret_cast<const VT *>(st.coef64)
                                     : reinterpret_cast<const VT *>(st.coef32);
            U.norm_part = up_part.p;
        }
        // ---- start vectors and their norms
        ftlm_status s1 = lzp_start_launch<VT, ST>(K, la, lz_grid, stream);
        if (s1 != FTLM_OK) return s1;
        count_launch();
        lzp_finalize<<<P, K * B * fin_slices(K * B), 0, stream>>>(0, 0, K, B, lz_grid, lz_t0, lz_nt, lz_part.p, st, tol, kScaled);
        FTLM_CUDA(cudaGetLastError());
        // ---- the step loop (captured once on a private stream, replayed once on the caller's)
        const bool prof = profiling_on();
        std::vector<cudaEvent_t> ev;
        auto steps = [&](cudaStream_t ss, bool capture) -> ftlm_status {
            for (int j = 0; j < m_all; ++j) {
                const int q = j % 3;
                if (prof) {
                    cudaEvent_t e0, e1;
                    FTLM_CUDA(cudaEventCreate(&e0));
                    FTLM_CUDA(cudaEventCreate(&e1));
                    ev.push_back(e0);
                    ev.push_back(e1);
                    FTLM_CUDA(capture ? cudaEventRecordWithFlags(e0, ss, cudaEventRecordExternal)
                                      : cudaEventRecord(e0, ss));
                }
                ftlm_status s2 = hvp_launch_plan<VT>(plan[q], hv_part.p, ss, false);
                if (s2 != FTLM_OK) return s2;
                if (prof)
                    FTLM_CUDA(capture ? cudaEventRecordWithFlags(ev.back(), ss, cudaEventRecordExternal)
                                      : cudaEventRecord(ev.back(), ss));
                count_launch();
                lzp_finalize<<<P, K * B * fin_slices(K * B), 0, ss>>>(1, j, K, B, hv_grid, hv_t0, hv_nt, hv_part.p, st, tol, kScaled);
                FTLM_CUDA(cudaGetLastError());
                LzUpd<VT> U = ua[q];
                U.has_prev = j > 0;
                count_launch();
                lzp_update<VT, ST><<<up_grid, kLzThreads, 0, ss>>>(U);
                FTLM_CUDA(cudaGetLastError());
                count_launch();
                lzp_finalize<<<P, K * B * fin_slices(K * B), 0, ss>>>(2, j, K, B, up_grid, d_ut.p, d_ut.p + P, up_part.p, st, tol,
                                                  kScaled);
                FTLM_CUDA(cudaGetLastError());
            }
            return FTLM_OK;
        };
        if (prof) profile_flip_counter();  // allocated before the capture (no allocation while capturing)
        if (use_graph) {
            cudaStream_t cap = nullptr;
            FTLM_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (ce != cudaSuccess) {
                cudaStreamDestroy(cap);
                return fail(FTLM_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
            }
            ftlm_status s3 = steps(cap, true);
            ce = cudaStreamEndCapture(cap, &graph);  // always end the capture, even after a failed launch
            cudaStreamDestroy(cap);
            if (s3 != FTLM_OK) {
                if (graph) cudaGraphDestroy(graph);
                return s3;
            }
            if (ce != cudaSuccess) return fail(FTLM_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
            ce = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return fail(FTLM_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
            ce = cudaGraphLaunch(exec, stream);
            cudaError_t ce2 = cudaStreamSynchronize(stream);
            cudaGraphExecDestroy(exec);
            if (ce != cudaSuccess || ce2 != cudaSuccess)
                return fail(FTLM_ECUDA, "graph launch: %s", cudaGetErrorString(ce != cudaSuccess ? ce : ce2));
        } else {
            ftlm_status s3 = steps(stream, false);
            if (s3 != FTLM_OK) return s3;
            FTLM_CUDA(cudaStreamSynchronize(stream));
        }
        if (prof) {
            for (size_t i = 0; i + 1 < ev.size(); i += 2) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) hv_profile_add(ms, rows * B);
            }
            for (auto e : ev) cudaEventDestroy(e);
        }
        // ---- results of the batch
        ha.resize((size_t)n_steps * E);
        hb.resize((size_t)n_steps * E);
        hs.resize(E);
        FTLM_CUDA(cudaMemcpyAsync(ha.data(), st.alpha, (size_t)n_steps * E * 8, cudaMemcpyDeviceToHost, stream));
        FTLM_CUDA(cudaMemcpyAsync(hb.data(), st.beta, (size_t)n_steps * E * 8, cudaMemcpyDeviceToHost, stream));
        FTLM_CUDA(cudaMemcpyAsync(hs.data(), st.steps, E * sizeof(int), cudaMemcpyDeviceToHost, stream));
        FTLM_CUDA(cudaStreamSynchronize(stream));
        {
            int err = 0;
            FTLM_CUDA(cudaMemcpyAsync(&err, derr.p, sizeof(int), cudaMemcpyDeviceToHost, stream));
            FTLM_CUDA(cudaStreamSynchronize(stream));
            if (err) {
                if (err & kErrWaitTimeout) return fail(FTLM_ETIMEOUT, "a bounded device wait gave up in H·v");
                return fail(FTLM_EINTERNAL, "device bounds check tripped in H·v (code %d)", err);
            }
        }
        for (int p = 0; p < P; ++p)
            for (int k = 0; k < K; ++k)
                for (int b = 0; b < B; ++b) {
                    const size_t e = ((size_t)p * K + k) * B + b;
                    const size_t o = ((size_t)p * K + k) * R + chain0 + b;
                    const int m = hs[e];
                    steps_done[o] = m;
                    for (int jj = 0; jj < m; ++jj) {
                        alpha[o * n_steps + jj] = ha[(size_t)jj * EB + e];
                        beta[o * n_steps + jj] = hb[(size_t)jj * EB + e];
                    }
                }
    }
    return FTLM_OK;
}

template <typename VT>
ftlm_status lanczos_packed(const std::vector<LzSetIn> &sets, int R, int n_steps, uint64_t seed, int rng,
                           cudaStream_t stream, double *alpha, double *beta, int *steps_done, int esize) {
    if (esize == (int)sizeof(VT))
        return lanczos_packed_st<VT, VT>(sets, R, n_steps, seed, rng, stream, alpha, beta, steps_done);
    if constexpr (sizeof(VT) == 4) {
        if (esize == 2)
            return lanczos_packed_st<float, __half>(sets, R, n_steps, seed, rng, stream, alpha, beta, steps_done);
    }
    return fail(FTLM_EINVAL, "no %d-byte storage for this arithmetic type", esize);
}

template ftlm_status lanczos_packed<float>(const std::vector<LzSetIn> &, int, int, uint64_t, int, cudaStream_t,
                                           double *, double *, int *, int);
template ftlm_status lanczos_packed<double>(const std::vector<LzSetIn> &, int, int, uint64_t, int, cudaStream_t,
                                            double *, double *, int *, int);

}  // namespace ftlm
