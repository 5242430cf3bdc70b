/*
 * CPU oracle (test infrastructure only): brute-force basis enumeration and the
 * plain symmetry-adapted Hamiltonian action.  FP64, no blocking, no tricks.
 *
 * Labels use the paper's base-d encoding, Eq. 2: n = sum_k a_k d^k with
 * a_k = m_k + s and d = 2s + 1.  A group element acts by moving the digit of
 * site k to site pi_g(k) (Section 2.3), so (U(g) n)_{pi_g(k)} = n_k.  An entry
 * pi_g(k) >= N marks an element of G x Z_2 that also applies the global spin
 * flip m -> -m (Section 2.2, M = 0): the digit of site k moves to site
 * pi_g(k) - N as 2s - a_k.
 *
 * or_enumerate: every label of the M sector (digit sum A), kept when it is the
 *   smallest label of its orbit (Section 2.3), with its stabilizer (Eq. 8).
 * or_min_rep:   smallest label of the orbit of one label and the first group
 *   element (canonical index) that reaches it.
 * or_hv_rows:   y = H x for the chosen output representatives, pull form of
 *   Eq. 15 (Hermitian transpose of the entry matrix, real irreps) plus Eq. 16:
 *     y[r,k] = J sum_<ij> m_i m_j x[r,k]
 *            + sum_{bond, sign} c_a sqrt(|Stab r'|/|Stab r|)
 *                  sum_k' [V_r^T rho(g_e) V_r']_{k,k'} x[r',k']
 *   with a the flipped label, c_a from Eq. 3, r' = min O(a), a = U(g_e) r'.
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load this library.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXN 64

static void decode(uint64_t n, int N, int d, int *a) {
    for (int k = 0; k < N; ++k) {
        a[k] = (int)(n % (uint64_t)d);
        n /= (uint64_t)d;
    }
}

static uint64_t encode(const int *a, int N, int d) {
    uint64_t n = 0;
    for (int k = N - 1; k >= 0; --k) n = n * (uint64_t)d + (uint64_t)a[k];
    return n;
}

/* b = digits of U(g) applied to digits a: b[pi_g(k)] = a[k] (b[pi_g(k) - N] = d - 1 - a[k] when flipped) */
static void act(const int32_t *pi, const int *a, int *b, int N, int d) {
    for (int k = 0; k < N; ++k) {
        if (pi[k] < N)
            b[pi[k]] = a[k];
        else
            b[pi[k] - N] = d - 1 - a[k];
    }
}

static uint64_t image(const int32_t *pi, const int *a, int N, int d) {
    int b[OR_MAXN];
    act(pi, a, b, N, d);
    return encode(b, N, d);
}

int or_min_rep(int N, int d, int G, const int32_t *perms, uint64_t label, uint64_t *rep, int32_t *gstar) {
    if (N > OR_MAXN) return -1;
    int a[OR_MAXN];
    decode(label, N, d, a);
    uint64_t best = UINT64_MAX;
    int32_t bg = -1;
    for (int g = 0; g < G; ++g) {
        uint64_t v = image(perms + (size_t)g * N, a, N, d);
        if (v < best) {
            best = v;
            bg = g;
        }
    }
    *rep = best;
    *gstar = bg;
    return 0;
}

/* Number of labels below d^N: the caller guarantees d^N fits in 63 bits. */
static uint64_t ipow(uint64_t d, int N) {
    uint64_t v = 1;
    for (int k = 0; k < N; ++k) v *= d;
    return v;
}

typedef struct {
    uint64_t *reps;
    uint64_t *stab;
    int64_t n, cap;
} chunk_out;

static void push(chunk_out *c, uint64_t r, const uint64_t *mask, int W) {
    if (c->n == c->cap) {
        c->cap = c->cap ? 2 * c->cap : 1024;
        c->reps = (uint64_t *)realloc(c->reps, (size_t)c->cap * sizeof(uint64_t));
        c->stab = (uint64_t *)realloc(c->stab, (size_t)c->cap * W * sizeof(uint64_t));
    }
    c->reps[c->n] = r;
    memcpy(c->stab + (size_t)c->n * W, mask, (size_t)W * sizeof(uint64_t));
    c->n++;
}

/*
 * Writes at most cap representatives (ascending) and their stabilizer masks
 * (W = ceil(G/64) words per representative, bit g set when U(g) r = r).
 * Returns the number of representatives, or -(number) when cap is too small,
 * or a value below -(1<<62) on bad arguments.
 */
int64_t or_enumerate(int N, int d, int A, int G, const int32_t *perms, uint64_t *reps, uint64_t *stab,
                     int64_t cap) {
    if (N > OR_MAXN || G > 64 * 8) return INT64_MIN;
    const int W = (G + 63) / 64;
    const uint64_t total = ipow((uint64_t)d, N);
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    const int nchunks = nthreads * 16;
    chunk_out *outs = (chunk_out *)calloc((size_t)nchunks, sizeof(chunk_out));
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < nchunks; ++c) {
        uint64_t lo = total / nchunks * c + (c < (int)(total % nchunks) ? c : total % nchunks);
        uint64_t hi = lo + total / nchunks + (c < (int)(total % nchunks) ? 1 : 0);
        int a[OR_MAXN], b[OR_MAXN];
        uint64_t mask[8];
        for (uint64_t n = lo; n < hi; ++n) {
            decode(n, N, d, a);
            int sum = 0;
            for (int k = 0; k < N; ++k) sum += a[k];
            if (sum != A) continue;
            int is_min = 1;
            memset(mask, 0, sizeof(mask));
            for (int g = 0; g < G; ++g) {
                act(perms + (size_t)g * N, a, b, N, d);
                uint64_t v = encode(b, N, d);
                if (v < n) {
                    is_min = 0;
                    break;
                }
                if (v == n) mask[g / 64] |= 1ull << (g % 64);
            }
            if (is_min) push(&outs[c], n, mask, W);
        }
    }
    int64_t n_total = 0;
    for (int c = 0; c < nchunks; ++c) n_total += outs[c].n;
    if (n_total <= cap) {
        int64_t pos = 0;
        for (int c = 0; c < nchunks; ++c) {
            if (outs[c].n) {
                memcpy(reps + pos, outs[c].reps, (size_t)outs[c].n * sizeof(uint64_t));
                if (stab) memcpy(stab + (size_t)pos * W, outs[c].stab, (size_t)outs[c].n * W * sizeof(uint64_t));
            }
            pos += outs[c].n;
        }
    }
    for (int c = 0; c < nchunks; ++c) {
        free(outs[c].reps);
        free(outs[c].stab);
    }
    free(outs);
    return n_total <= cap ? n_total : -n_total;
}

static int64_t find_rep(const uint64_t *reps, int64_t n, uint64_t key) {
    int64_t lo = 0, hi = n; /* std::lower_bound */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (reps[mid] < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < n && reps[lo] == key) ? lo : -1;
}

/*
 * Block tables (per representative i): n[i] = n_Gamma(r_i), off[i] = row offset,
 * sqrtS[i] = sqrt|Stab r_i|, V + vidx[i]*dG*dG = V_r (dG x dG, V[beta*dG + k],
 * first n[i] columns used).  rho[g*dG*dG + a*dG + b] = rho_Gamma(g)_{ab},
 * inv[g] = index of g^{-1}.  x, y are [dim][B] row-major.
 * rows: representative indices to compute (NULL: all).  Returns 0, or -1 when
 * a flipped state's representative is missing from the table.
 */
int or_hv_rows(int N, int d, int two_s, int G, const int32_t *perms, const int32_t *inv, int n_bonds,
               const int32_t *bonds, double J, int64_t n_reps, const uint64_t *reps, const int32_t *n,
               const int64_t *off, const double *sqrtS, const int64_t *vidx, const double *V, int dG,
               const double *rho, int B, const double *x, double *y, const int64_t *rows, int64_t n_rows) {
    const double s = 0.5 * two_s;
    const double ss1 = s * (s + 1.0);
    int err = 0;
    if (!rows) n_rows = n_reps;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : err)
    for (int64_t t = 0; t < n_rows; ++t) {
        const int64_t i = rows ? rows[t] : t;
        const int ni = n[i];
        if (ni == 0) continue;
        int a[OR_MAXN], f[OR_MAXN];
        decode(reps[i], N, d, a);
        double diag = 0.0;
        for (int e = 0; e < n_bonds; ++e) {
            const double mi = a[bonds[2 * e]] - s, mj = a[bonds[2 * e + 1]] - s;
            diag += J * mi * mj;
        }
        double *yi = y + (size_t)off[i] * B;
        const double *xi = x + (size_t)off[i] * B;
        for (int k = 0; k < ni; ++k)
            for (int b = 0; b < B; ++b) yi[(size_t)k * B + b] = diag * xi[(size_t)k * B + b];
        const double *Vi = V + (size_t)vidx[i] * dG * dG;
        for (int e = 0; e < n_bonds; ++e) {
            const int si = bonds[2 * e], sj = bonds[2 * e + 1];
            for (int sgn = +1; sgn >= -1; sgn -= 2) {
                /* sgn = +1: s_i^+ s_j^-, sgn = -1: s_i^- s_j^+ */
                const int ai = a[si] + sgn, aj = a[sj] - sgn;
                if (ai < 0 || ai > two_s || aj < 0 || aj > two_s) continue;
                const double mi = a[si] - s, mj = a[sj] - s;
                const double ca = 0.5 * J * sqrt(ss1 - mi * (mi + sgn)) * sqrt(ss1 - mj * (mj - sgn));
                memcpy(f, a, sizeof(int) * N);
                f[si] = ai;
                f[sj] = aj;
                uint64_t lab = encode(f, N, d), rp;
                int32_t gs;
                /* representative search: min over all g, first minimiser */
                {
                    uint64_t best = UINT64_MAX;
                    int32_t bg = -1;
                    for (int g = 0; g < G; ++g) {
                        uint64_t v = image(perms + (size_t)g * N, f, N, d);
                        if (v < best) {
                            best = v;
                            bg = g;
                        }
                    }
                    rp = best;
                    gs = bg;
                }
                (void)lab;
                const int64_t j = find_rep(reps, n_reps, rp);
                if (j < 0) {
                    err |= 1;
                    continue;
                }
                const int nj = n[j];
                if (nj == 0) continue;
                const int ge = inv[gs]; /* a = U(g_e) r', g_e = gs^{-1} */
                const double *R = rho + (size_t)ge * dG * dG;
                const double *Vj = V + (size_t)vidx[j] * dG * dG;
                const double fac = ca * sqrtS[j] / sqrtS[i];
                const double *xj = x + (size_t)off[j] * B;
                /* M = V_i^T rho(g_e) V_j  (ni x nj) */
                for (int k = 0; k < ni; ++k) {
                    for (int kp = 0; kp < nj; ++kp) {
                        double m = 0.0;
                        for (int al = 0; al < dG; ++al)
                            for (int be = 0; be < dG; ++be)
                                m += Vi[al * dG + k] * R[al * dG + be] * Vj[be * dG + kp];
                        for (int b = 0; b < B; ++b) yi[(size_t)k * B + b] += fac * m * xj[(size_t)kp * B + b];
                    }
                }
            }
        }
    }
    return err ? -1 : 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Stabilizer bitmask (W words) of one label: bit g set when U(g) n = n (Eq. 8). */
int or_stab(int N, int d, int G, const int32_t *perms, uint64_t label, uint64_t *mask) {
    if (N > OR_MAXN) return -1;
    int a[OR_MAXN];
    decode(label, N, d, a);
    const int W = (G + 63) / 64;
    for (int w = 0; w < W; ++w) mask[w] = 0;
    for (int g = 0; g < G; ++g)
        if (image(perms + (size_t)g * N, a, N, d) == label) mask[g / 64] |= 1ull << (g % 64);
    return 0;
}

/*
 * Off-diagonal entries generated by one representative r (Section 2.4): for
 * every bond and admissible sign, the flipped label's orbit minimum r', the
 * first minimising element g* (a = U(g*^{-1}) r') and c_a (Eq. 3).  Also the
 * diagonal energy J sum m_i m_j (Eq. 16).  Returns the entry count (<= cap).
 */
int or_flip_entries(int N, int d, int two_s, int G, const int32_t *perms, int n_bonds, const int32_t *bonds,
                    double J, uint64_t label, int cap, uint64_t *rp, int32_t *gstar, double *coef, double *diag) {
    if (N > OR_MAXN) return -1;
    const double s = 0.5 * two_s, ss1 = s * (s + 1.0);
    int a[OR_MAXN], f[OR_MAXN];
    decode(label, N, d, a);
    double dg = 0.0;
    int cnt = 0;
    for (int e = 0; e < n_bonds; ++e) {
        const int si = bonds[2 * e], sj = bonds[2 * e + 1];
        const double mi = a[si] - s, mj = a[sj] - s;
        dg += J * mi * mj;
        for (int sgn = +1; sgn >= -1; sgn -= 2) {
            const int ai = a[si] + sgn, aj = a[sj] - sgn;
            if (ai < 0 || ai > two_s || aj < 0 || aj > two_s) continue;
            if (cnt >= cap) return -2;
            memcpy(f, a, sizeof(int) * N);
            f[si] = ai;
            f[sj] = aj;
            uint64_t best = UINT64_MAX;
            int32_t bg = -1;
            for (int g = 0; g < G; ++g) {
                uint64_t v = image(perms + (size_t)g * N, f, N, d);
                if (v < best) {
                    best = v;
                    bg = g;
                }
            }
            rp[cnt] = best;
            gstar[cnt] = bg;
            coef[cnt] = 0.5 * J * sqrt(ss1 - mi * (mi + sgn)) * sqrt(ss1 - mj * (mj - sgn));
            ++cnt;
        }
    }
    *diag = dg;
    return cnt;
}
