// FTLM on the GPU (Section 2.2 of arXiv 2607.17429): start vectors, the
// three-term Lanczos recurrence with FP64 dot products and norms, the FP64
// tridiagonal eigensolve, and the thermal sums of Eqs. 5-7 with Eq. 14 weights.
//
// Reductions are deterministic: a fixed grid, a fixed row partition per block
// and a fixed summation order, so repeated runs give identical coefficients.
#include <float.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "lanczos_packed.h"
#include "philox.cuh"
#include "ritz_thermo.cuh"

namespace ftlm {

ftlm_status hv_multi_launch_f64(const ftlm_multiblock *mb, int B, const double *const *x, double *const *y,
                               cudaStream_t stream);
ftlm_status hv_multi_launch_f32(const ftlm_multiblock *mb, int B, const float *const *x, float *const *y,
                               cudaStream_t stream);

namespace {

constexpr int kRedBlocks = kNumSMs * 4;  // fixed reduction grid (deterministic order)
constexpr int kRedThreads = 256;

// Threads of a reduction block are (row lane r, column b): t = r * B + b.
__device__ __forceinline__ int red_rows(int B) { return kRedThreads / B; }

__device__ void block_partial(double acc, int B, double *partials) {
    __shared__ double s[kRedThreads];
    const int nr = red_rows(B);
    const int t = threadIdx.x;
    s[t] = (t < nr * B) ? acc : 0.0;
    __syncthreads();
    if (t < B) {
        double sum = 0.0;
        for (int r = 0; r < nr; ++r) sum += s[r * B + t];
        partials[(size_t)blockIdx.x * B + t] = sum;
    }
}

template <typename VT>
__global__ void lz_random(VT *v, uint64_t dim, int B, int Bc, uint32_t chain0, uint32_t k0, uint32_t k1, int rng,
                          double *partials) {
    const int nr = red_rows(B);
    const int r = threadIdx.x / B, b = threadIdx.x % B;
    double acc = 0.0;
    if (r < nr) {
        for (uint64_t i = (uint64_t)blockIdx.x * nr + r; i < dim; i += (uint64_t)gridDim.x * nr) {
            double val = b < Bc ? start_value(i, chain0 + b, k0, k1, rng) : 0.0;
            const VT st = (VT)val;
            v[i * B + b] = st;
            acc += (double)st * (double)st;
        }
    }
    block_partial(acc, B, partials);
}

template <typename VT>
__global__ void lz_dot(const VT *v, const VT *w, uint64_t dim, int B, double *partials) {
    const int nr = red_rows(B);
    const int r = threadIdx.x / B, b = threadIdx.x % B;
    double acc = 0.0;
    if (r < nr)
        for (uint64_t i = (uint64_t)blockIdx.x * nr + r; i < dim; i += (uint64_t)gridDim.x * nr)
            acc += (double)v[i * B + b] * (double)w[i * B + b];
    block_partial(acc, B, partials);
}

struct LzState {
    double *alpha;      // [n_steps][B]
    double *beta;       // [n_steps][B]
    double *beta_prev;  // [B]
    double *scale;      // [B] 1/norm of the vector being normalised
    int *active;        // [B]
    int *steps;         // [B]
};

// w -= alpha v + beta_prev v_prev, partial |w|^2
template <typename VT>
__global__ void lz_update(VT *w, const VT *v, const VT *vp, uint64_t dim, int B, int j, LzState st, double *partials) {
    const int nr = red_rows(B);
    const int r = threadIdx.x / B, b = threadIdx.x % B;
    double acc = 0.0;
    if (r < nr) {
        const double al = st.alpha[(size_t)j * B + b], bp = st.beta_prev[b];
        for (uint64_t i = (uint64_t)blockIdx.x * nr + r; i < dim; i += (uint64_t)gridDim.x * nr) {
            const size_t e = i * B + b;
            const VT nw = (VT)((double)w[e] - al * (double)v[e] - bp * (double)vp[e]);
            w[e] = nw;
            acc += (double)nw * (double)nw;
        }
    }
    block_partial(acc, B, partials);
}

template <typename VT>
__global__ void lz_scale(VT *w, uint64_t dim, int B, LzState st) {
    const uint64_t n = dim * (uint64_t)B;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (uint64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e % B);
        w[e] = st.active[b] ? (VT)((double)w[e] * st.scale[b]) : (VT)0;
    }
}

__device__ double sum_partials(const double *p, int B, int b) {
    double s = 0.0;
    for (int k = 0; k < kRedBlocks; ++k) s += p[(size_t)k * B + b];
    return s;
}

__global__ void fin_norm(const double *p, int B, LzState st) {
    const int b = threadIdx.x;
    if (b >= B) return;
    const double n = sqrt(sum_partials(p, B, b));
    st.scale[b] = n > 0 ? 1.0 / n : 0.0;
    st.active[b] = n > 0;
    st.steps[b] = 0;
    st.beta_prev[b] = 0.0;
}

__global__ void fin_alpha(const double *p, int B, int j, LzState st) {
    const int b = threadIdx.x;
    if (b >= B) return;
    st.alpha[(size_t)j * B + b] = st.active[b] ? sum_partials(p, B, b) : 0.0;
}

__global__ void fin_beta(const double *p, int B, int j, int m_max, double tol, LzState st) {
    const int b = threadIdx.x;
    if (b >= B) return;
    if (!st.active[b]) {
        st.beta[(size_t)j * B + b] = 0.0;
        return;
    }
    const double bn = sqrt(sum_partials(p, B, b));
    const double al = st.alpha[(size_t)j * B + b];
    st.beta[(size_t)j * B + b] = bn;
    if (j + 1 >= m_max || bn <= tol * (fabs(al) + st.beta_prev[b])) {
        st.active[b] = 0;
        st.steps[b] = j + 1;
    } else {
        st.beta_prev[b] = bn;
        st.scale[b] = 1.0 / bn;
    }
}

template <typename VT>
ftlm_status hv_multi_any(const ftlm_multiblock *mb, int B, const VT *const *x, VT *const *y, cudaStream_t st);
template <>
ftlm_status hv_multi_any<double>(const ftlm_multiblock *mb, int B, const double *const *x, double *const *y,
                                 cudaStream_t st) {
    return hv_multi_launch_f64(mb, B, x, y, st);
}
template <>
ftlm_status hv_multi_any<float>(const ftlm_multiblock *mb, int B, const float *const *x, float *const *y,
                                cudaStream_t st) {
    return hv_multi_launch_f32(mb, B, x, y, st);
}

// Lanczos on every block of a multi-block set in lockstep: one multi-block H·v
// per step, then the per-block recurrence kernels.
template <typename VT>
ftlm_status lanczos_multi_impl(const ftlm_multiblock *mb, int R, int n_steps, uint64_t seed, const uint64_t *ids,
                               int rng, cudaStream_t stream, double *alpha, double *beta, int *steps_done) {
    const int K = mb->K;
    const int Bmax = std::min(R, kMaxB);
    for (size_t i = 0; i < (size_t)K * R; ++i) steps_done[i] = 0;
    for (size_t i = 0; i < (size_t)K * R * n_steps; ++i) alpha[i] = beta[i] = 0.0;
    std::vector<uint64_t> dim(K);
    std::vector<int> m_max(K);
    int m_all = 0;
    for (int k = 0; k < K; ++k) {
        dim[k] = mb->blocks[k]->dim;
        m_max[k] = (int)std::min<uint64_t>((uint64_t)n_steps, dim[k]);
        m_all = std::max(m_all, m_max[k]);
    }
    std::vector<DevBuf<VT>> vec(3 * K);
    for (int k = 0; k < K; ++k)
        for (int q = 0; q < 3; ++q) FTLM_CUDA(vec[3 * k + q].alloc(std::max<uint64_t>(dim[k], 1) * Bmax));
    const size_t per_state = (size_t)2 * n_steps * Bmax + 2 * Bmax;
    DevBuf<double> partials, dstate;
    DevBuf<int> istate;
    FTLM_CUDA(partials.alloc((size_t)kRedBlocks * Bmax));
    FTLM_CUDA(dstate.alloc(per_state * K));
    FTLM_CUDA(istate.alloc((size_t)2 * Bmax * K));
    std::vector<LzState> st(K);
    for (int k = 0; k < K; ++k) {
        double *base = dstate.p + per_state * k;
        st[k].alpha = base;
        st[k].beta = base + (size_t)n_steps * Bmax;
        st[k].beta_prev = base + (size_t)2 * n_steps * Bmax;
        st[k].scale = st[k].beta_prev + Bmax;
        st[k].active = istate.p + (size_t)2 * Bmax * k;
        st[k].steps = st[k].active + Bmax;
    }
    std::vector<double> ha((size_t)n_steps * Bmax), hb((size_t)n_steps * Bmax);
    std::vector<int> hs(Bmax);
    const int scale_blocks = kNumSMs * 8;
    std::vector<const VT *> xs(K);
    std::vector<VT *> ys(K), vp(K), v(K), w(K);
    for (int chain0 = 0; chain0 < R; chain0 += Bmax) {
        const int B = std::min(Bmax, R - chain0);
        FTLM_CUDA(cudaMemsetAsync(dstate.p, 0, per_state * K * sizeof(double), stream));
        for (int k = 0; k < K; ++k) {
            vp[k] = vec[3 * k].p;
            v[k] = vec[3 * k + 1].p;
            w[k] = vec[3 * k + 2].p;
            if (dim[k] == 0) continue;
            FTLM_CUDA(cudaMemsetAsync(vp[k], 0, dim[k] * B * sizeof(VT), stream));
            count_launch(3);
            lz_random<VT><<<kRedBlocks, kRedThreads, 0, stream>>>(v[k], dim[k], B, B, (uint32_t)chain0, (uint32_t)seed,
                                                                  (uint32_t)ids[k], rng, partials.p);
            fin_norm<<<1, 32, 0, stream>>>(partials.p, B, st[k]);
            lz_scale<VT><<<scale_blocks, 256, 0, stream>>>(v[k], dim[k], B, st[k]);
            FTLM_CUDA(cudaGetLastError());
        }
        for (int j = 0; j < m_all; ++j) {
            for (int k = 0; k < K; ++k) {
                xs[k] = v[k];
                ys[k] = w[k];
            }
            ftlm_status sst = hv_multi_any<VT>(mb, B, xs.data(), ys.data(), stream);
            if (sst != FTLM_OK) return sst;
            for (int k = 0; k < K; ++k) {
                if (j >= m_max[k]) continue;
                count_launch(5);
                lz_dot<VT><<<kRedBlocks, kRedThreads, 0, stream>>>(v[k], w[k], dim[k], B, partials.p);
                fin_alpha<<<1, 32, 0, stream>>>(partials.p, B, j, st[k]);
                lz_update<VT><<<kRedBlocks, kRedThreads, 0, stream>>>(w[k], v[k], vp[k], dim[k], B, j, st[k],
                                                                      partials.p);
                fin_beta<<<1, 32, 0, stream>>>(partials.p, B, j, m_max[k], sizeof(VT) == 8 ? 1e-12 : 1e-6, st[k]);
                lz_scale<VT><<<scale_blocks, 256, 0, stream>>>(w[k], dim[k], B, st[k]);
                FTLM_CUDA(cudaGetLastError());
                VT *t = vp[k];
                vp[k] = v[k];
                v[k] = w[k];
                w[k] = t;
            }
        }
        for (int k = 0; k < K; ++k) {
            if (dim[k] == 0) continue;
            FTLM_CUDA(cudaMemcpyAsync(ha.data(), st[k].alpha, (size_t)n_steps * B * 8, cudaMemcpyDeviceToHost, stream));
            FTLM_CUDA(cudaMemcpyAsync(hb.data(), st[k].beta, (size_t)n_steps * B * 8, cudaMemcpyDeviceToHost, stream));
            FTLM_CUDA(cudaMemcpyAsync(hs.data(), st[k].steps, (size_t)B * 4, cudaMemcpyDeviceToHost, stream));
            FTLM_CUDA(cudaStreamSynchronize(stream));
            for (int b = 0; b < B; ++b) {
                const int r = chain0 + b;
                const size_t kr = (size_t)k * R + r;
                steps_done[kr] = hs[b];
                for (int jj = 0; jj < hs[b]; ++jj) {
                    alpha[kr * n_steps + jj] = ha[(size_t)jj * B + b];
                    beta[kr * n_steps + jj] = hb[(size_t)jj * B + b];
                }
            }
        }
        int err = 0;
        FTLM_CUDA(cudaMemcpy(&err, mb->sec->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (err) return fail(FTLM_EINTERNAL, "device bounds check tripped in H·v (code %d)", err);
    }
    return FTLM_OK;
}

}  // namespace
}  // namespace ftlm

using namespace ftlm;

extern "C" {

ftlm_status ftlm_lanczos(const ftlm_basis *b, ftlm_dtype dtype, int R, int n_steps, uint64_t seed, uint64_t block_id,
                         ftlm_rng rng, void *cuda_stream, double *alpha, double *beta, int *steps_done) {
    if (!b || !alpha || !beta || !steps_done) return fail(FTLM_EINVAL, "NULL argument");
    if (R < 1 || n_steps < 1 || n_steps > kMaxSteps) return fail(FTLM_EINVAL, "R >= 1 and 1 <= n_steps <= 512");
    if (rng != FTLM_GAUSS && rng != FTLM_RADEMACHER) return fail(FTLM_EINVAL, "unknown rng");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const ftlm_basis *one[1] = {b};
    std::vector<LzSetIn> sets{{b->sec, b->ps, one, &block_id}};
    if (dtype == FTLM_F64) return lanczos_packed<double>(sets, R, n_steps, seed, rng, st, alpha, beta, steps_done, 8);
    if (dtype == FTLM_F32) return lanczos_packed<float>(sets, R, n_steps, seed, rng, st, alpha, beta, steps_done, 4);
    if (dtype == FTLM_F16) return lanczos_packed<float>(sets, R, n_steps, seed, rng, st, alpha, beta, steps_done, 2);
    return fail(FTLM_EINVAL, "unknown dtype");
}

ftlm_status ftlm_hv_multi(const ftlm_multiblock *mb, ftlm_dtype dtype, int B, const void *const *x,
                          void *const *y, void *cuda_stream) {
    if (!mb || !x || !y) return fail(FTLM_EINVAL, "NULL argument");
    if (mb->sec->flip) return fail(FTLM_EUNSUPPORTED, "spin-flip sectors run on the packed layout (ftlm_hv_packed)");
    if (B < 1 || B > kMaxB) return fail(FTLM_EINVAL, "B must be in 1..%d", kMaxB);
    for (int k = 0; k < mb->K; ++k)
        if (!x[k] || !y[k]) return fail(FTLM_EINVAL, "NULL vector for block %d", k);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (dtype == FTLM_F64)
        return hv_multi_launch_f64(mb, B, (const double *const *)x, (double *const *)y, st);
    if (dtype == FTLM_F32) return hv_multi_launch_f32(mb, B, (const float *const *)x, (float *const *)y, st);
    return fail(FTLM_EINVAL, "unknown dtype");
}

ftlm_status ftlm_lanczos_multi(const ftlm_multiblock *mb, ftlm_dtype dtype, int R, int n_steps, uint64_t seed,
                               const uint64_t *block_ids, ftlm_rng rng, void *cuda_stream, double *alpha,
                               double *beta, int *steps_done) {
    if (!mb || !block_ids || !alpha || !beta || !steps_done) return fail(FTLM_EINVAL, "NULL argument");
    if (R < 1 || n_steps < 1 || n_steps > kMaxSteps) return fail(FTLM_EINVAL, "R >= 1 and 1 <= n_steps <= 512");
    if (rng != FTLM_GAUSS && rng != FTLM_RADEMACHER) return fail(FTLM_EINVAL, "unknown rng");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (mb->ps) {  // packed layout: one launch per kernel for all blocks
        std::vector<LzSetIn> sets{{mb->sec, mb->ps, mb->blocks.data(), block_ids}};
        if (dtype == FTLM_F64)
            return lanczos_packed<double>(sets, R, n_steps, seed, rng, st, alpha, beta, steps_done, 8);
        if (dtype == FTLM_F32)
            return lanczos_packed<float>(sets, R, n_steps, seed, rng, st, alpha, beta, steps_done, 4);
        if (dtype == FTLM_F16)
            return lanczos_packed<float>(sets, R, n_steps, seed, rng, st, alpha, beta, steps_done, 2);
        return fail(FTLM_EINVAL, "unknown dtype");
    }
    if (mb->sec->flip) return fail(FTLM_EUNSUPPORTED, "spin-flip sectors need a compiled packed block shape");
    if (dtype == FTLM_F64)
        return lanczos_multi_impl<double>(mb, R, n_steps, seed, block_ids, rng, st, alpha, beta, steps_done);
    if (dtype == FTLM_F32)
        return lanczos_multi_impl<float>(mb, R, n_steps, seed, block_ids, rng, st, alpha, beta, steps_done);
    return fail(FTLM_EINVAL, "unknown dtype");
}

ftlm_status ftlm_lanczos_sets(int n_sets, const ftlm_multiblock *const *sets, ftlm_dtype dtype, int R, int n_steps,
                              uint64_t seed, const uint64_t *block_ids, ftlm_rng rng, void *cuda_stream,
                              double *alpha, double *beta, int *steps_done) {
    if (n_sets < 1 || !sets || !block_ids || !alpha || !beta || !steps_done) return fail(FTLM_EINVAL, "bad arguments");
    if (R < 1 || n_steps < 1 || n_steps > kMaxSteps) return fail(FTLM_EINVAL, "R >= 1 and 1 <= n_steps <= 512");
    if (rng != FTLM_GAUSS && rng != FTLM_RADEMACHER) return fail(FTLM_EINVAL, "unknown rng");
    const ftlm_multiblock *m0 = sets[0];
    if (!m0 || !m0->ps) return fail(FTLM_EUNSUPPORTED, "set 0 has no packed layout");
    const int K = m0->K;
    std::vector<LzSetIn> in;
    for (int i = 0; i < n_sets; ++i) {
        const ftlm_multiblock *m = sets[i];
        if (!m || !m->ps) return fail(FTLM_EUNSUPPORTED, "set %d has no packed layout", i);
        const GroupData &g0 = m0->sec->grp, &g = m->sec->grp;
        bool same = m->K == K && m->ps->shape == m0->ps->shape && m->sec->two_s == m0->sec->two_s &&
                    g.perms == g0.perms && g.bonds == g0.bonds && g.J == g0.J && g.irreps.size() == g0.irreps.size();
        for (int k = 0; same && k < K; ++k) {
            same = m->blocks[k]->irrep == m0->blocks[k]->irrep &&
                   g.irreps[m->blocks[k]->irrep].rho == g0.irreps[m0->blocks[k]->irrep].rho;
        }
        if (!same) return fail(FTLM_EINVAL, "set %d differs from set 0 in group, spin, bonds or irreps", i);
        in.push_back({m->sec, m->ps, m->blocks.data(), block_ids + (size_t)i * K});
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (dtype == FTLM_F64) return lanczos_packed<double>(in, R, n_steps, seed, rng, st, alpha, beta, steps_done, 8);
    if (dtype == FTLM_F32) return lanczos_packed<float>(in, R, n_steps, seed, rng, st, alpha, beta, steps_done, 4);
    if (dtype == FTLM_F16) return lanczos_packed<float>(in, R, n_steps, seed, rng, st, alpha, beta, steps_done, 2);
    return fail(FTLM_EINVAL, "unknown dtype");
}

ftlm_status ftlm_ritz(int n_chains, int ld, const int *m, const double *alpha, const double *beta, double *theta,
                      double *w, void *cuda_stream) {
    if (n_chains < 0 || ld < 1 || ld > kMaxSteps || !m || !alpha || !beta || !theta || !w)
        return fail(FTLM_EINVAL, "bad arguments");
    if (n_chains == 0) return FTLM_OK;
    for (int c = 0; c < n_chains; ++c)
        if (m[c] < 0 || m[c] > ld) return fail(FTLM_EINVAL, "steps out of range");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t n = (size_t)n_chains * ld;
    DevBuf<double> da, db, dt, dw;
    DevBuf<int> dm, derr;
    FTLM_CUDA(da.alloc(n));
    FTLM_CUDA(db.alloc(n));
    FTLM_CUDA(dt.alloc(n));
    FTLM_CUDA(dw.alloc(n));
    FTLM_CUDA(dm.alloc(n_chains));
    FTLM_CUDA(derr.alloc(1));
    FTLM_CUDA(cudaMemcpyAsync(da.p, alpha, n * 8, cudaMemcpyHostToDevice, st));
    FTLM_CUDA(cudaMemcpyAsync(db.p, beta, n * 8, cudaMemcpyHostToDevice, st));
    FTLM_CUDA(cudaMemcpyAsync(dm.p, m, n_chains * 4, cudaMemcpyHostToDevice, st));
    FTLM_CUDA(cudaMemsetAsync(derr.p, 0, 4, st));
    count_launch();
    ritz_kernel<<<(n_chains + 63) / 64, 64, 0, st>>>(n_chains, ld, dm.p, da.p, db.p, dt.p, dw.p, derr.p);
    FTLM_CUDA(cudaGetLastError());
    int err = 0;
    FTLM_CUDA(cudaMemcpyAsync(theta, dt.p, n * 8, cudaMemcpyDeviceToHost, st));
    FTLM_CUDA(cudaMemcpyAsync(w, dw.p, n * 8, cudaMemcpyDeviceToHost, st));
    FTLM_CUDA(cudaMemcpyAsync(&err, derr.p, 4, cudaMemcpyDeviceToHost, st));
    FTLM_CUDA(cudaStreamSynchronize(st));
    if (err) return fail(FTLM_EINTERNAL, "tridiagonal eigensolve did not converge");
    return FTLM_OK;
}

ftlm_status ftlm_thermo(int n_blocks, const ftlm_block *blocks, int n_T, const double *T, double g, double *lnZ,
                        double *E, double *C, double *chi, double *E0, void *cuda_stream) {
    if (n_blocks < 1 || !blocks || n_T < 1 || !T) return fail(FTLM_EINVAL, "bad arguments");
    for (int t = 0; t < n_T; ++t)
        if (!(T[t] > 0)) return fail(FTLM_EINVAL, "temperatures must be positive");
    int ld = 1, n_chains = 0;
    for (int k = 0; k < n_blocks; ++k) {
        const ftlm_block &bl = blocks[k];
        if (bl.R < 1 || bl.ld < 1 || !bl.steps_done || !bl.alpha || !bl.beta) return fail(FTLM_EINVAL, "bad block");
        for (int r = 0; r < bl.R; ++r) {
            if (bl.steps_done[r] < 0 || bl.steps_done[r] > bl.ld) return fail(FTLM_EINVAL, "steps out of range");
            ld = std::max(ld, bl.steps_done[r]);
        }
        n_chains += bl.R;
    }
    if (ld > kMaxSteps) return fail(FTLM_EINVAL, "too many steps");
    std::vector<double> a((size_t)n_chains * ld, 0.0), b((size_t)n_chains * ld, 0.0), Wc(n_chains), Msq(n_chains);
    std::vector<int> m(n_chains);
    int c = 0;
    for (int k = 0; k < n_blocks; ++k) {
        const ftlm_block &bl = blocks[k];
        const double mult = bl.two_M > 0 ? 2.0 : 1.0;
        for (int r = 0; r < bl.R; ++r, ++c) {
            m[c] = bl.steps_done[r];
            for (int j = 0; j < m[c]; ++j) {
                a[(size_t)c * ld + j] = bl.alpha[(size_t)r * bl.ld + j];
                b[(size_t)c * ld + j] = bl.beta[(size_t)r * bl.ld + j];
            }
            Wc[c] = mult * bl.d_gamma * (double)bl.dim / bl.R;
            Msq[c] = 0.25 * bl.two_M * bl.two_M;
        }
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t n = (size_t)n_chains * ld;
    DevBuf<double> da, db, dt, dw, dW, dM, dT, dE0, dout;
    DevBuf<int> dm, derr;
    FTLM_CUDA(da.alloc(n));
    FTLM_CUDA(db.alloc(n));
    FTLM_CUDA(dt.alloc(n));
    FTLM_CUDA(dw.alloc(n));
    FTLM_CUDA(dW.alloc(n_chains));
    FTLM_CUDA(dM.alloc(n_chains));
    FTLM_CUDA(dT.alloc(n_T));
    FTLM_CUDA(dE0.alloc(1));
    FTLM_CUDA(dout.alloc((size_t)4 * n_T));
    FTLM_CUDA(dm.alloc(n_chains));
    FTLM_CUDA(derr.alloc(1));
    FTLM_CUDA(cudaMemcpyAsync(da.p, a.data(), n * 8, cudaMemcpyHostToDevice, st));
    FTLM_CUDA(cudaMemcpyAsync(db.p, b.data(), n * 8, cudaMemcpyHostToDevice, st));
    FTLM_CUDA(cudaMemcpyAsync(dW.p, Wc.data(), n_chains * 8, cudaMemcpyHostToDevice, st));
    FTLM_CUDA(cudaMemcpyAsync(dM.p, Msq.data(), n_chains * 8, cudaMemcpyHostToDevice, st));
    FTLM_CUDA(cudaMemcpyAsync(dm.p, m.data(), n_chains * 4, cudaMemcpyHostToDevice, st));
    FTLM_CUDA(cudaMemcpyAsync(dT.p, T, n_T * 8, cudaMemcpyHostToDevice, st));
    FTLM_CUDA(cudaMemsetAsync(derr.p, 0, 4, st));
    count_launch();
    ritz_kernel<<<(n_chains + 63) / 64, 64, 0, st>>>(n_chains, ld, dm.p, da.p, db.p, dt.p, dw.p, derr.p);
    ThermoIn in{n_chains, ld, dm.p, dt.p, dw.p, dW.p, dM.p};
    count_launch();
    ground_energy<<<1, kRedThreads, 0, st>>>(in, dE0.p);
    count_launch();
    thermo_kernel<<<n_T, kRedThreads, 0, st>>>(in, dT.p, dE0.p, g, dout.p, n_T);
    FTLM_CUDA(cudaGetLastError());
    std::vector<double> out((size_t)4 * n_T);
    double e0 = 0.0;
    int err = 0;
    FTLM_CUDA(cudaMemcpyAsync(out.data(), dout.p, out.size() * 8, cudaMemcpyDeviceToHost, st));
    FTLM_CUDA(cudaMemcpyAsync(&e0, dE0.p, 8, cudaMemcpyDeviceToHost, st));
    FTLM_CUDA(cudaMemcpyAsync(&err, derr.p, 4, cudaMemcpyDeviceToHost, st));
    FTLM_CUDA(cudaStreamSynchronize(st));
    if (err) return fail(FTLM_EINTERNAL, "tridiagonal eigensolve did not converge");
    for (int t = 0; t < n_T; ++t) {
        if (lnZ) lnZ[t] = out[t];
        if (E) E[t] = out[n_T + t];
        if (C) C[t] = out[2 * n_T + t];
        if (chi) chi[t] = out[3 * n_T + t];
    }
    if (E0) *E0 = e0;
    return FTLM_OK;
}

}  // extern "C"
