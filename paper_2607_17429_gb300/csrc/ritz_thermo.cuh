// Ritz pairs and thermal sums on the GPU (Section 2.2, Eqs. 5-7 with the Eq. 14 weights):
// device code shared by the entry points that run them.
#pragma once

#include <float.h>
#include <math.h>

#include "common.cuh"

namespace ftlm {

constexpr int kThermoThreads = 256;

// ---------------------------------------------------------------- tridiagonal eigensolve (implicit QL, FP64)

// Eigenvalues of the symmetric tridiagonal matrix (diag d[0..n-1], off-diagonal
// e[i] between i and i+1) and the first row z of its orthonormal eigenvector
// matrix.  Implicit QL sweeps with the shift taken from the leading 2x2 block;
// each Givens rotation is also applied to z.  Returns false if a block does not
// converge within 60 sweeps.
static __device__ bool tridiag_ql(int n, double *d, double *e, double *z) {
    for (int i = 0; i < n; ++i) z[i] = (i == 0) ? 1.0 : 0.0;
    if (n > 0) e[n - 1] = 0.0;
    for (int l = 0; l < n; ++l) {
        for (int sweep = 0;; ++sweep) {
            int m = l;
            for (; m < n - 1; ++m) {
                const double dd = fabs(d[m]) + fabs(d[m + 1]);
                if (fabs(e[m]) <= DBL_EPSILON * dd) break;
            }
            if (m == l) break;
            if (sweep == 60) return false;
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
            double s = 1.0, c = 1.0, p = 0.0;
            bool deflated = false;
            for (int i = m - 1; i >= l; --i) {
                const double f = s * e[i], bb = c * e[i];
                r = hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {
                    d[i + 1] -= p;
                    e[m] = 0.0;
                    deflated = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * bb;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - bb;
                const double zi = z[i], zi1 = z[i + 1];
                z[i + 1] = s * zi + c * zi1;
                z[i] = c * zi - s * zi1;
            }
            if (deflated) continue;
            d[l] -= p;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    return true;
}

// one thread per chain: theta, w (sorted ascending) from alpha/beta rows of length m[c]
static __global__ void ritz_kernel(int n_chains, int ld, const int *m, const double *alpha, const double *beta, double *theta,
                            double *w, int *err) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chains) return;
    const int n = m[c];
    double *d = theta + (size_t)c * ld, *z = w + (size_t)c * ld;
    double e[kMaxSteps];
    for (int i = 0; i < ld; ++i) {
        d[i] = 0.0;
        z[i] = 0.0;
    }
    if (n <= 0) return;
    if (n > ld || n > kMaxSteps) {
        atomicOr(err, 2);
        return;
    }
    for (int i = 0; i < n; ++i) {
        d[i] = alpha[(size_t)c * ld + i];
        e[i] = beta[(size_t)c * ld + i];
    }
    if (!tridiag_ql(n, d, e, z)) atomicOr(err, 1);
    for (int i = 0; i < n; ++i) z[i] *= z[i];
    for (int i = 1; i < n; ++i) {  // insertion sort by theta
        const double td = d[i], tz = z[i];
        int k = i - 1;
        while (k >= 0 && d[k] > td) {
            d[k + 1] = d[k];
            z[k + 1] = z[k];
            --k;
        }
        d[k + 1] = td;
        z[k + 1] = tz;
    }
}

// ---------------------------------------------------------------- thermal sums (Eqs. 5-7, 14)

struct ThermoIn {
    int n_chains, ld;
    const int *m;
    const double *theta, *w, *Wc, *Msq;
};

static __device__ double block_sum(double v) {
    __shared__ double s[kThermoThreads];
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = kThermoThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    const double r = s[0];
    __syncthreads();
    return r;
}

static __device__ double block_min(double v) {
    __shared__ double s[kThermoThreads];
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = kThermoThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] = fmin(s[threadIdx.x], s[threadIdx.x + o]);
        __syncthreads();
    }
    const double r = s[0];
    __syncthreads();
    return r;
}

static __global__ void ground_energy(ThermoIn in, double *E0) {
    double mn = INFINITY;
    const uint64_t n = (uint64_t)in.n_chains * in.ld;
    for (uint64_t t = threadIdx.x; t < n; t += blockDim.x) {
        const int c = (int)(t / in.ld), k = (int)(t % in.ld);
        if (k < in.m[c]) mn = fmin(mn, in.theta[t]);
    }
    mn = block_min(mn);
    if (threadIdx.x == 0) *E0 = mn;
}

static __global__ void thermo_kernel(ThermoIn in, const double *T, const double *E0p, double g, double *out /*[4][n_T]*/,
                              int n_T) {
    const int it = blockIdx.x;
    const double beta = 1.0 / T[it], E0 = *E0p;
    const uint64_t n = (uint64_t)in.n_chains * in.ld;
    double z = 0.0, ze = 0.0, zm = 0.0;
    for (uint64_t t = threadIdx.x; t < n; t += blockDim.x) {
        const int c = (int)(t / in.ld), k = (int)(t % in.ld);
        if (k >= in.m[c]) continue;
        const double bz = in.Wc[c] * in.w[t] * exp(-beta * (in.theta[t] - E0));
        z += bz;
        ze += bz * in.theta[t];
        zm += bz * in.Msq[c];
    }
    z = block_sum(z);
    ze = block_sum(ze);
    zm = block_sum(zm);
    const double Em = ze / z;
    double v = 0.0;
    for (uint64_t t = threadIdx.x; t < n; t += blockDim.x) {
        const int c = (int)(t / in.ld), k = (int)(t % in.ld);
        if (k >= in.m[c]) continue;
        const double bz = in.Wc[c] * in.w[t] * exp(-beta * (in.theta[t] - E0));
        const double dt = in.theta[t] - Em;
        v += bz * dt * dt;
    }
    v = block_sum(v);
    if (threadIdx.x == 0) {
        out[it] = log(z) - beta * E0;
        out[n_T + it] = Em;
        out[2 * n_T + it] = beta * beta * v / z;
        out[3 * n_T + it] = g * g * beta * zm / z;
    }
}

}  // namespace ftlm
