// Host group module (Section 3 of arXiv 2607.17429): closure of site-permutation
// generators, bond-invariance check, real irreps computed from the regular
// representation, verification, and built-in cluster providers.
//
// Irreps: the left regular representation L(g) e_h = e_{gh} commutes with every
// right multiplication, so a random symmetric element S = sum_h c_h (R(h) + R(h)^T)
// of the right-regular commutant has L-invariant eigenspaces.  On the isotypic
// component of a real-type irrep (d copies of it) S acts on the multiplicity
// space only, as a generic symmetric d x d matrix, so each eigenspace of S is one
// irreducible copy: an orthonormal basis B of it gives real orthogonal matrices
// rho(g) = B^T L(g) B.  Eigenspaces with equal characters are copies of the same
// irrep; one is kept.  The Frobenius-Schur indicator of every irrep is checked.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"

namespace ftlm {

static thread_local std::string g_last_error;

ftlm_status fail(ftlm_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

void clear_error() { g_last_error.clear(); }

// ---------------------------------------------------------------- closure

ftlm_status build_group(int n_sites, int n_gens, const int32_t *gens, int n_bonds, const int32_t *bonds, double J,
                        GroupData &out) {
    if (n_sites < 1 || n_sites > 64) return fail(FTLM_EINVAL, "n_sites must be in 1..64");
    if (n_gens < 0 || (n_gens > 0 && !gens)) return fail(FTLM_EINVAL, "bad generator list");
    if (n_bonds < 0 || (n_bonds > 0 && !bonds)) return fail(FTLM_EINVAL, "bad bond list");
    const int N = n_sites;
    for (int g = 0; g < n_gens; ++g) {
        std::vector<int> seen(N, 0);
        for (int k = 0; k < N; ++k) {
            int v = gens[g * N + k];
            if (v < 0 || v >= N || seen[v]) return fail(FTLM_ENOTGROUP, "generator %d is not a permutation", g);
            seen[v] = 1;
        }
    }
    for (int e = 0; e < n_bonds; ++e) {
        int i = bonds[2 * e], j = bonds[2 * e + 1];
        if (i < 0 || j < 0 || i >= N || j >= N || i == j) return fail(FTLM_EINVAL, "bond %d is invalid", e);
    }
    // breadth-first closure: new elements are products gen * element
    std::map<std::vector<int32_t>, int> seen;
    std::vector<std::vector<int32_t>> elems;
    std::vector<int32_t> id(N);
    std::iota(id.begin(), id.end(), 0);
    seen[id] = 0;
    elems.push_back(id);
    for (size_t head = 0; head < elems.size(); ++head) {
        for (int g = 0; g < n_gens; ++g) {
            std::vector<int32_t> c(N);
            for (int k = 0; k < N; ++k) c[k] = gens[g * N + elems[head][k]];
            if (seen.find(c) == seen.end()) {
                if ((int)elems.size() >= kMaxGHost)
                    return fail(FTLM_ENOTGROUP, "group order exceeds %d", kMaxGHost);
                seen[c] = (int)elems.size();
                elems.push_back(c);
            }
        }
    }
    std::sort(elems.begin(), elems.end());  // canonical order: lexicographic, identity first
    const int G = (int)elems.size();
    std::map<std::vector<int32_t>, int> index;
    for (int g = 0; g < G; ++g) index[elems[g]] = g;
    out = GroupData();
    out.N = N;
    out.G = G;
    out.perms.resize((size_t)G * N);
    for (int g = 0; g < G; ++g) std::copy(elems[g].begin(), elems[g].end(), out.perms.begin() + (size_t)g * N);
    out.mult.resize((size_t)G * G);
    out.inv.resize(G);
    std::vector<int32_t> c(N);
    for (int g = 0; g < G; ++g)
        for (int h = 0; h < G; ++h) {
            for (int k = 0; k < N; ++k) c[k] = elems[g][elems[h][k]];
            int gh = index[c];
            out.mult[(size_t)g * G + h] = gh;
            if (gh == 0) out.inv[g] = h;
        }
    // bond invariance (Section 3)
    std::vector<std::pair<int, int>> bs;
    for (int e = 0; e < n_bonds; ++e)
        bs.emplace_back(std::min(bonds[2 * e], bonds[2 * e + 1]), std::max(bonds[2 * e], bonds[2 * e + 1]));
    std::sort(bs.begin(), bs.end());
    if (std::adjacent_find(bs.begin(), bs.end()) != bs.end()) return fail(FTLM_EINVAL, "duplicate bond");
    for (int g = 0; g < G; ++g) {
        std::vector<std::pair<int, int>> im;
        for (auto &b : bs) {
            int i = elems[g][b.first], j = elems[g][b.second];
            im.emplace_back(std::min(i, j), std::max(i, j));
        }
        std::sort(im.begin(), im.end());
        if (im != bs) return fail(FTLM_EBONDS, "bond list is not invariant under group element %d", g);
    }
    out.bonds.assign(bonds, bonds + 2 * n_bonds);
    out.J = J;
    return FTLM_OK;
}

// ---------------------------------------------------------------- symmetric eigensolver (cyclic Jacobi)

// A (n x n, row-major) is overwritten; on return w holds the eigenvalues and
// V (row-major) the eigenvectors as columns.
static void jacobi(int n, std::vector<double> &A, std::vector<double> &V, std::vector<double> &w) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    double scale = 0.0;
    for (double v : A) scale += v * v;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
        if (off <= 1e-32 * scale) break;
        for (int p = 0; p < n; ++p) {
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (fabs(apq) < 1e-300) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double th = (aqq - app) / (2.0 * apq);
                const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

// ---------------------------------------------------------------- irreps

static uint64_t splitmix(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static bool char_less(const Irrep &a, const Irrep &b) {
    if (a.dim != b.dim) return a.dim < b.dim;
    for (size_t g = 0; g < a.chars.size(); ++g) {
        long long x = llround(a.chars[g] * 1e8), y = llround(b.chars[g] * 1e8);
        if (x != y) return x > y;  // descending
    }
    return false;
}

ftlm_status canonicalise_and_verify_irreps(GroupData &g, std::vector<Irrep> &irreps, double tol) {
    const int G = g.G;
    std::stable_sort(irreps.begin(), irreps.end(), char_less);
    int sum = 0;
    // sum over the complex irreps of d^2: a real form of dimension d stands for d^2 / kappa of it
    for (auto &ir : irreps) {
        if ((ir.dim * ir.dim) % ir.kappa()) return fail(FTLM_EIRREP, "real form of odd dimension");
        sum += ir.dim * ir.dim / ir.kappa();
    }
    if (sum != G) return fail(FTLM_EIRREP, "sum of d^2 = %d differs from |G| = %d", sum, G);
    for (size_t a = 0; a < irreps.size(); ++a) {
        for (size_t b = 0; b < irreps.size(); ++b) {
            double s = 0.0;
            for (int h = 0; h < G; ++h) s += irreps[a].chars[h] * irreps[b].chars[h];
            s /= G;
            const double want = (a == b) ? (double)irreps[a].kappa() : 0.0;
            if (fabs(s - want) > tol) return fail(FTLM_EIRREP, "character orthogonality violated");
        }
    }
    for (auto &ir : irreps) {
        const int d = ir.dim;
        if (ir.rho.size() != (size_t)G * d * d) return fail(FTLM_EIRREP, "irrep without matrices");
        for (int x = 0; x < G; ++x) {
            const double *A = &ir.rho[(size_t)x * d * d];
            double tr = 0.0;
            for (int i = 0; i < d; ++i) tr += A[i * d + i];
            if (fabs(tr - ir.chars[x]) > tol) return fail(FTLM_EIRREP, "trace differs from character");
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) {
                    double s = 0.0;
                    for (int k = 0; k < d; ++k) s += A[i * d + k] * A[j * d + k];
                    if (fabs(s - (i == j)) > tol) return fail(FTLM_EIRREP, "matrix not orthogonal");
                }
            for (int y = 0; y < G; ++y) {
                const double *Bm = &ir.rho[(size_t)y * d * d];
                const double *C = &ir.rho[(size_t)g.mult[(size_t)x * G + y] * d * d];
                for (int i = 0; i < d; ++i)
                    for (int j = 0; j < d; ++j) {
                        double s = 0.0;
                        for (int k = 0; k < d; ++k) s += A[i * d + k] * Bm[k * d + j];
                        if (fabs(s - C[i * d + j]) > tol) return fail(FTLM_EIRREP, "not a homomorphism");
                    }
            }
        }
    }
    return FTLM_OK;
}

static ftlm_status irreps_from_regular(GroupData &g, uint64_t seed, std::vector<Irrep> &out) {
    const int G = g.G;
    std::vector<double> c(G);
    for (int h = 0; h < G; ++h) c[h] = (double)(splitmix(seed) >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    // S[x][y] = c[x^{-1} y] + c[y^{-1} x]
    std::vector<double> S((size_t)G * G), V, w;
    for (int x = 0; x < G; ++x)
        for (int y = 0; y < G; ++y) {
            int a = g.mult[(size_t)g.inv[x] * G + y], b = g.mult[(size_t)g.inv[y] * G + x];
            S[(size_t)x * G + y] = c[a] + c[b];
        }
    jacobi(G, S, V, w);
    std::vector<int> order(G);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return w[a] < w[b]; });
    double scale = 1.0;
    for (double v : w) scale = std::max(scale, fabs(v));
    out.clear();
    std::vector<std::vector<double>> seen_chars;
    size_t i0 = 0;
    while (i0 < (size_t)G) {
        size_t i1 = i0 + 1;
        while (i1 < (size_t)G && w[order[i1]] - w[order[i1 - 1]] < 1e-9 * scale) ++i1;
        const int m = (int)(i1 - i0);
        // basis of the eigenspace, column-major Bm[i][y]
        std::vector<double> Bm((size_t)m * G);
        for (int i = 0; i < m; ++i)
            for (int y = 0; y < G; ++y) Bm[(size_t)i * G + y] = V[(size_t)y * G + order[i0 + i]];
        // character chi(x) = sum_i sum_y B[y][i] B[x^{-1} y][i]
        std::vector<double> chi(G, 0.0);
        for (int x = 0; x < G; ++x) {
            const int xi = g.inv[x];
            double s = 0.0;
            for (int i = 0; i < m; ++i) {
                const double *b = &Bm[(size_t)i * G];
                for (int y = 0; y < G; ++y) s += b[y] * b[g.mult[(size_t)xi * G + y]];
            }
            chi[x] = s;
        }
        bool dup = false;
        for (auto &sc : seen_chars) {
            double diff = 0.0;
            for (int x = 0; x < G; ++x) diff = std::max(diff, fabs(sc[x] - chi[x]));
            if (diff < 1e-6) dup = true;
        }
        if (!dup) {
            seen_chars.push_back(chi);
            double norm = 0.0, fsum = 0.0;
            for (int x = 0; x < G; ++x) {
                norm += chi[x] * chi[x];
                fsum += chi[g.mult[(size_t)x * G + x]];
            }
            norm /= G;
            fsum /= G;
            // The eigenspace is one copy of a real-irreducible representation: an irrep of real
            // type (<chi, chi> = 1, Frobenius-Schur sum 1), or the real form of a complex pair
            // (<chi, chi> = 2, sum 0) or of a quaternionic irrep (<chi, chi> = 4, sum -2).
            Irrep ir;
            if (fabs(norm - 1.0) < 1e-6 && fabs(fsum - 1.0) < 1e-6)
                ir.fs = 1;
            else if (fabs(norm - 2.0) < 1e-6 && fabs(fsum) < 1e-6)
                ir.fs = 0;
            else if (fabs(norm - 4.0) < 1e-6 && fabs(fsum + 2.0) < 1e-6)
                ir.fs = -1;
            else
                return fail(FTLM_EIRREP, "eigenspace of dimension %d is not real-irreducible", m);
            ir.dim = m;
            ir.chars = chi;
            ir.rho.resize((size_t)G * m * m);
            for (int x = 0; x < G; ++x) {
                const int xi = g.inv[x];
                for (int a = 0; a < m; ++a)
                    for (int b = 0; b < m; ++b) {
                        double s = 0.0;
                        const double *ba = &Bm[(size_t)a * G], *bb = &Bm[(size_t)b * G];
                        for (int y = 0; y < G; ++y) s += ba[y] * bb[g.mult[(size_t)xi * G + y]];
                        ir.rho[((size_t)x * m + a) * m + b] = s;
                    }
            }
            out.push_back(std::move(ir));
        }
        i0 = i1;
    }
    return canonicalise_and_verify_irreps(g, out, 1e-9);
}

ftlm_status compute_irreps(GroupData &g) {
    ftlm_status st = FTLM_EIRREP;
    for (uint64_t attempt = 0; attempt < 4; ++attempt) {
        std::vector<Irrep> irr;
        st = irreps_from_regular(g, 0x5eed0000ull + attempt, irr);
        if (st == FTLM_OK) {
            g.irreps = std::move(irr);
            clear_error();
            return FTLM_OK;
        }
    }
    return st;
}

// ---------------------------------------------------------------- built-in clusters

namespace {
struct Vec3 {
    double x, y, z;
};
const double kPhi = (1.0 + sqrt(5.0)) / 2.0;

std::vector<Vec3> icosahedron() {
    std::vector<Vec3> v;
    for (double a : {1.0, -1.0})
        for (double b : {kPhi, -kPhi}) {
            v.push_back({0, a, b});
            v.push_back({a, b, 0});
            v.push_back({b, 0, a});
        }
    return v;
}
std::vector<Vec3> dodecahedron() {
    std::vector<Vec3> v;
    for (double x : {1.0, -1.0})
        for (double y : {1.0, -1.0})
            for (double z : {1.0, -1.0}) v.push_back({x, y, z});
    for (double a : {kPhi, -kPhi})
        for (double b : {1.0 / kPhi, -1.0 / kPhi}) {
            v.push_back({0, a, b});
            v.push_back({a, b, 0});
            v.push_back({b, 0, a});
        }
    return v;
}
double dist(const Vec3 &a, const Vec3 &b) {
    return sqrt((a.x - b.x) * (a.x - b.x) + (a.y - b.y) * (a.y - b.y) + (a.z - b.z) * (a.z - b.z));
}
std::vector<int32_t> nn_bonds(const std::vector<Vec3> &v) {
    double dmin = 1e300;
    for (size_t i = 0; i < v.size(); ++i)
        for (size_t j = i + 1; j < v.size(); ++j) dmin = std::min(dmin, dist(v[i], v[j]));
    std::vector<int32_t> b;
    for (size_t i = 0; i < v.size(); ++i)
        for (size_t j = i + 1; j < v.size(); ++j)
            if (fabs(dist(v[i], v[j]) - dmin) < 1e-9 * std::max(1.0, dmin)) {
                b.push_back((int32_t)i);
                b.push_back((int32_t)j);
            }
    return b;
}
std::vector<Vec3> icosidodecahedron() {
    auto ic = icosahedron();
    auto e = nn_bonds(ic);
    std::vector<Vec3> v;
    for (size_t t = 0; t < e.size(); t += 2) {
        const Vec3 &a = ic[e[t]], &b = ic[e[t + 1]];
        v.push_back({(a.x + b.x) / 2, (a.y + b.y) / 2, (a.z + b.z) / 2});
    }
    return v;
}
std::vector<Vec3> cuboctahedron() {
    std::vector<Vec3> v;
    for (double a : {1.0, -1.0})
        for (double b : {1.0, -1.0}) {
            v.push_back({a, b, 0});
            v.push_back({a, 0, b});
            v.push_back({0, a, b});
        }
    return v;
}
// rotation by angle about axis (Rodrigues), as a row-major 3x3 matrix
std::array<double, 9> rot(Vec3 u, double ang) {
    double n = sqrt(u.x * u.x + u.y * u.y + u.z * u.z);
    u = {u.x / n, u.y / n, u.z / n};
    double c = cos(ang), s = sin(ang), t = 1 - c;
    return {c + t * u.x * u.x,       t * u.x * u.y - s * u.z, t * u.x * u.z + s * u.y,
            t * u.x * u.y + s * u.z, c + t * u.y * u.y,       t * u.y * u.z - s * u.x,
            t * u.x * u.z - s * u.y, t * u.y * u.z + s * u.x, c + t * u.z * u.z};
}
bool perm_of(const std::array<double, 9> &R, const std::vector<Vec3> &v, std::vector<int32_t> &p) {
    p.assign(v.size(), -1);
    for (size_t k = 0; k < v.size(); ++k) {
        Vec3 w = {R[0] * v[k].x + R[1] * v[k].y + R[2] * v[k].z, R[3] * v[k].x + R[4] * v[k].y + R[5] * v[k].z,
                  R[6] * v[k].x + R[7] * v[k].y + R[8] * v[k].z};
        for (size_t j = 0; j < v.size(); ++j)
            if (dist(w, v[j]) < 1e-9) p[k] = (int32_t)j;
        if (p[k] < 0) return false;
    }
    return true;
}
}  // namespace

static ftlm_status polyhedron(const std::vector<Vec3> &v, const std::vector<std::array<double, 9>> &ops,
                              ftlm_group **out) {
    std::vector<int32_t> gens, p;
    for (auto &R : ops) {
        if (!perm_of(R, v, p)) return fail(FTLM_EINTERNAL, "built-in generator does not map the cluster");
        gens.insert(gens.end(), p.begin(), p.end());
    }
    auto b = nn_bonds(v);
    return ftlm_group_init((int)v.size(), (int)ops.size(), gens.data(), (int)b.size() / 2, b.data(), 1.0, out);
}

}  // namespace ftlm

using namespace ftlm;

extern "C" {

const char *ftlm_last_error(void) { return g_last_error.c_str(); }

ftlm_status ftlm_group_init(int n_sites, int n_gens, const int32_t *gens, int n_bonds, const int32_t *bonds,
                            double J, ftlm_group **out) {
    if (!out) return fail(FTLM_EINVAL, "out is NULL");
    *out = nullptr;
    ftlm_group *g = new (std::nothrow) ftlm_group();
    if (!g) return fail(FTLM_ENOMEM, "host allocation failed");
    ftlm_status st = build_group(n_sites, n_gens, gens, n_bonds, bonds, J, g->d);
    if (st == FTLM_OK) st = compute_irreps(g->d);
    if (st != FTLM_OK) {
        delete g;
        return st;
    }
    *out = g;
    return FTLM_OK;
}

ftlm_status ftlm_group_builtin(const char *name, ftlm_group **out) {
    if (!name || !out) return fail(FTLM_EINVAL, "NULL argument");
    const std::string n(name);
    const double pi = acos(-1.0);
    const std::array<double, 9> inv = {-1, 0, 0, 0, -1, 0, 0, 0, -1};
    if (n == "icosahedron" || n == "dodecahedron" || n == "icosidodecahedron") {
        auto v = n == "icosahedron" ? icosahedron() : n == "dodecahedron" ? dodecahedron() : icosidodecahedron();
        return polyhedron(v, {rot({0, 1, kPhi}, 2 * pi / 5), rot({1, 1, 1}, 2 * pi / 3), inv}, out);
    }
    if (n == "cuboctahedron")
        return polyhedron(cuboctahedron(), {rot({0, 0, 1}, pi / 2), rot({1, 1, 1}, 2 * pi / 3), inv}, out);
    if (n == "tetrahedron") {
        std::vector<Vec3> v = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
        std::array<double, 9> mirror = {0, 1, 0, 1, 0, 0, 0, 0, 1};
        return polyhedron(v, {rot({1, 1, 1}, 2 * pi / 3), rot({0, 0, 1}, pi), mirror}, out);
    }
    if (n == "dimer") {
        int32_t gens[2] = {1, 0}, bonds[2] = {0, 1};
        return ftlm_group_init(2, 1, gens, 1, bonds, 1.0, out);
    }
    if (n.rfind("ring:", 0) == 0) {
        int N = atoi(n.c_str() + 5);
        if (N < 3 || N > 64) return fail(FTLM_EINVAL, "ring needs 3..64 sites");
        std::vector<int32_t> gens(2 * N), bonds;
        for (int k = 0; k < N; ++k) {
            gens[k] = (k + 1) % N;
            gens[N + k] = (N - k) % N;
        }
        std::vector<std::pair<int, int>> bs;
        for (int k = 0; k < N; ++k) bs.emplace_back(std::min(k, (k + 1) % N), std::max(k, (k + 1) % N));
        std::sort(bs.begin(), bs.end());
        for (auto &b : bs) {
            bonds.push_back(b.first);
            bonds.push_back(b.second);
        }
        return ftlm_group_init(N, 2, gens.data(), N, bonds.data(), 1.0, out);
    }
    if (n.rfind("square:", 0) == 0) {
        int lx = 0, ly = 0;
        char pg[8] = "";
        int got = sscanf(n.c_str() + 7, "%dx%d:%7s", &lx, &ly, pg);
        if (got < 2 || lx < 3 || ly < 3 || lx * ly > 64) return fail(FTLM_EINVAL, "bad square lattice name");
        std::string p = got == 3 ? pg : (lx == ly ? "c4v" : "c2v");
        auto idx = [&](int x, int y) { return ((x % lx) + lx) % lx + lx * (((y % ly) + ly) % ly); };
        const int N = lx * ly;
        std::vector<int32_t> gens;
        auto add = [&](auto f) {
            for (int k = 0; k < N; ++k) {
                int x = k % lx, y = k / lx, u, v;
                f(x, y, u, v);
                gens.push_back(idx(u, v));
            }
        };
        add([](int x, int y, int &u, int &v) { u = x + 1, v = y; });
        add([](int x, int y, int &u, int &v) { u = x, v = y + 1; });
        if (p == "c4v") {
            if (lx != ly) return fail(FTLM_EINVAL, "c4v needs a square torus");
            add([](int x, int y, int &u, int &v) { u = -y, v = x; });
            add([](int x, int y, int &u, int &v) { u = -x, v = y; });
        } else if (p == "c2v") {
            add([](int x, int y, int &u, int &v) { u = -x, v = y; });
            add([](int x, int y, int &u, int &v) { u = x, v = -y; });
        } else if (p != "t") {
            return fail(FTLM_EINVAL, "unknown point group");
        }
        std::vector<std::pair<int, int>> bs;
        for (int y = 0; y < ly; ++y)
            for (int x = 0; x < lx; ++x) {
                int a = idx(x, y), b = idx(x + 1, y), c = idx(x, y + 1);
                bs.emplace_back(std::min(a, b), std::max(a, b));
                bs.emplace_back(std::min(a, c), std::max(a, c));
            }
        std::sort(bs.begin(), bs.end());
        bs.erase(std::unique(bs.begin(), bs.end()), bs.end());
        std::vector<int32_t> bonds;
        for (auto &b : bs) {
            bonds.push_back(b.first);
            bonds.push_back(b.second);
        }
        return ftlm_group_init(N, (int)gens.size() / N, gens.data(), (int)bs.size(), bonds.data(), 1.0, out);
    }
    return fail(FTLM_EINVAL, "unknown built-in cluster '%s'", name);
}

ftlm_status ftlm_group_info(const ftlm_group *g, int *n_sites, int *order, int *n_irreps, int *dims, int *fs,
                            double *chars) {
    if (!g) return fail(FTLM_EINVAL, "group is NULL");
    const GroupData &d = g->d;
    if (n_sites) *n_sites = d.N;
    if (order) *order = d.G;
    if (n_irreps) *n_irreps = (int)d.irreps.size();
    for (size_t i = 0; i < d.irreps.size(); ++i) {
        if (dims) dims[i] = d.irreps[i].dim;
        if (fs) fs[i] = d.irreps[i].fs;
        if (chars) std::copy(d.irreps[i].chars.begin(), d.irreps[i].chars.end(), chars + i * d.G);
    }
    return FTLM_OK;
}

ftlm_status ftlm_group_weights(const ftlm_group *g, int *weights) {
    if (!g || !weights) return fail(FTLM_EINVAL, "NULL argument");
    for (size_t i = 0; i < g->d.irreps.size(); ++i) weights[i] = g->d.irreps[i].weight();
    return FTLM_OK;
}

ftlm_status ftlm_group_irrep(const ftlm_group *g, int irrep, double *rho, int32_t *perms) {
    if (!g) return fail(FTLM_EINVAL, "group is NULL");
    const GroupData &d = g->d;
    if (perms) std::copy(d.perms.begin(), d.perms.end(), perms);
    if (rho) {
        if (irrep < 0 || irrep >= (int)d.irreps.size()) return fail(FTLM_EINVAL, "irrep index out of range");
        std::copy(d.irreps[irrep].rho.begin(), d.irreps[irrep].rho.end(), rho);
    }
    return FTLM_OK;
}

ftlm_status ftlm_group_bonds(const ftlm_group *g, int *n_bonds, int32_t *bonds, double *J) {
    if (!g) return fail(FTLM_EINVAL, "group is NULL");
    if (n_bonds) *n_bonds = g->d.n_bonds();
    if (bonds) std::copy(g->d.bonds.begin(), g->d.bonds.end(), bonds);
    if (J) *J = g->d.J;
    return FTLM_OK;
}

ftlm_status ftlm_group_set_irreps(ftlm_group *g, int n_irreps, const int *dims, const double *rho_all) {
    if (!g || n_irreps <= 0 || !dims || !rho_all) return fail(FTLM_EINVAL, "bad arguments");
    const int G = g->d.G;
    std::vector<Irrep> irr(n_irreps);
    size_t pos = 0;
    for (int i = 0; i < n_irreps; ++i) {
        const int d = dims[i];
        if (d < 1 || d > 64) return fail(FTLM_EINVAL, "irrep dimension out of range");
        irr[i].dim = d;
        irr[i].fs = 1;
        irr[i].rho.assign(rho_all + pos, rho_all + pos + (size_t)G * d * d);
        pos += (size_t)G * d * d;
        irr[i].chars.resize(G);
        double norm = 0.0;
        for (int x = 0; x < G; ++x) {
            double tr = 0.0;
            for (int a = 0; a < d; ++a) tr += irr[i].rho[((size_t)x * d + a) * d + a];
            irr[i].chars[x] = tr;
            norm += tr * tr;
        }
        // the type of a real-irreducible representation from <chi, chi> = 1, 2, 4
        norm /= G;
        irr[i].fs = norm < 1.5 ? 1 : (norm < 3.0 ? 0 : -1);
    }
    ftlm_status st = canonicalise_and_verify_irreps(g->d, irr, 1e-9);
    if (st != FTLM_OK) return st;
    g->d.irreps = std::move(irr);
    return FTLM_OK;
}

void ftlm_group_free(ftlm_group *g) { delete g; }

}  // extern "C"
