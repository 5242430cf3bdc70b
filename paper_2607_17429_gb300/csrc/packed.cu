// Packed sets (K irrep blocks of one sector, rows interleaved by representative
// in lifted coordinates) and the entry points of the packed H·v: ftlm_hv (one
// block), ftlm_hv_packed, ftlm_multiblock_pack / _unpack, ftlm_set_wait_limit.
//
// Construction (Section 3's two phases): the irrep-independent records of the
// sector (label, stabilizer id) get the segment offset r * W of every
// representative; per stabilizer id the set keeps n_k (Section 2.3), their sum,
// and the projector V_k V_k^T of every block (Eq. 11).  Lifting a block vector,
// x~_k(r) = V_k(r) x_k(r), and lowering it back, x_k(r) = V_k(r)^T x~_k(r), are
// the pack and unpack copies.
#include <stdio.h>
#include <string.h>

#include <string>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "hvp_ops.h"

namespace ftlm {

namespace {

struct ShapeDef {
    int K;
    int d[kPMaxK];
};
const ShapeDef kShapeDefs[kNumShapes] = {
    {1, {1}}, {1, {2}}, {1, {3}}, {1, {4}}, {1, {5}}, {1, {6}}, {1, {7}}, {1, {8}}, {1, {9}}, {1, {10}},
    {1, {11}}, {1, {12}},
    {10, {1, 1, 3, 3, 3, 3, 4, 4, 5, 5}},
    {10, {1, 1, 1, 1, 2, 2, 3, 3, 3, 3}},
    {5, {1, 1, 2, 3, 3}},
};

std::atomic<unsigned long long> g_wait_limit{kDrainCycles};

__global__ void fill_records(const uint64_t *labels, const uint16_t *stab_id, uint64_t n, int W, HvRec *rec) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    HvRec r;
    r.label = labels[i];
    r.off = (uint32_t)(i * (uint64_t)W);
    r.sid = stab_id[i];
    rec[i] = r;
}

struct LiftArgs {
    uint64_t n_reps;
    int K, W, B, to_packed;
    int dims[kPMaxK], zoff[kPMaxK];
    const uint8_t *ntab;
    const HvRec *rec;
    const uint64_t *boff[kPMaxK];
    const void *V[kPMaxK];
    void *blk[kPMaxK];
};

// packed (lifted) <-> per-block vectors: one thread per (representative, right-hand side)
template <typename VT>
__global__ void lift_rows(const __grid_constant__ LiftArgs a, VT *packed) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_reps * (uint64_t)a.B) return;
    const uint64_t rep = t / a.B;
    const int b = (int)(t % a.B), B = a.B;
    const HvRec r = a.rec[rep];
    for (int k = 0; k < a.K; ++k) {
        const int d = a.dims[k];
        const int n = a.ntab[r.sid * a.K + k];
        const VT *V = reinterpret_cast<const VT *>(a.V[k]) + (size_t)r.sid * d * d;
        VT *blk = reinterpret_cast<VT *>(a.blk[k]);
        const uint64_t o = a.boff[k][rep];
        VT *pk = packed + ((uint64_t)r.off + a.zoff[k]) * B + b;
        if (a.to_packed) {
            for (int gm = 0; gm < d; ++gm) {
                VT v = (VT)0;
                if (r.sid == 0)
                    v = blk[(o + gm) * B + b];
                else
                    for (int q = 0; q < n; ++q) v += V[gm * d + q] * blk[(o + q) * B + b];
                pk[(size_t)gm * B] = v;
            }
        } else {
            for (int q = 0; q < n; ++q) {
                VT v = (VT)0;
                if (r.sid == 0)
                    v = pk[(size_t)q * B];
                else
                    for (int gm = 0; gm < d; ++gm) v += V[gm * d + q] * pk[(size_t)gm * B];
                blk[(o + q) * B + b] = v;
            }
        }
    }
}

}  // namespace

int packed_shape_id(int K, const int *dims) {
    for (int s = 0; s < kNumShapes; ++s) {
        if (kShapeDefs[s].K != K) continue;
        bool eq = true;
        for (int k = 0; k < K; ++k) eq = eq && kShapeDefs[s].d[k] == dims[k];
        if (eq) return s;
    }
    return -1;
}

unsigned long long wait_limit_cycles() { return g_wait_limit.load(); }

void packed_set_free(PackedSet *ps) {
    if (!ps) return;
    cudaFree(ps->d_rec);
    cudaFree(ps->d_ntab);
    cudaFree(ps->d_wtab);
    for (int k = 0; k < kPMaxK; ++k) {
        cudaFree(ps->d_P[k]);
        cudaFree(ps->d_Pf[k]);
    }
    cudaFree(ps->d_rhoT);
    cudaFree(ps->d_rhoTf);
    delete ps;
}

ftlm_status packed_set_build(ftlm_sector *s, int K, const ftlm_basis *const *blocks, void *stream_v, PackedSet **out) {
    cudaStream_t stream = (cudaStream_t)stream_v;
    *out = nullptr;
    if (K < 1 || K > kPMaxK) return fail(FTLM_EINVAL, "packed set: 1..%d blocks", kPMaxK);
    PackedSet *ps = new (std::nothrow) PackedSet();
    if (!ps) return fail(FTLM_ENOMEM, "host allocation failed");
    struct Guard {
        PackedSet *p;
        ~Guard() { packed_set_free(p); }
    } guard{ps};
    ps->K = K;
    for (int k = 0; k < K; ++k) {
        ps->dims[k] = blocks[k]->d;
        ps->W += blocks[k]->d;
    }
    ps->shape = packed_shape_id(K, ps->dims);
    for (int k = 0; k < K; ++k)
        if (s->flip && (blocks[k]->irrep & 1)) ps->neg |= 1u << k;
    const size_t ns = s->stab_elems.size();
    std::vector<uint8_t> ntab(ns * K), wtab(ns);
    for (size_t t = 0; t < ns; ++t) {
        int o = 0;
        for (int k = 0; k < K; ++k) {
            ntab[t * K + k] = blocks[k]->h_ntab[t];
            o += blocks[k]->h_ntab[t];
        }
        wtab[t] = (uint8_t)o;
    }
    ps->h_wtab = wtab;
    // projectors P = V V^T per block and stabilizer id (FP64 from the FP64 V, then rounded)
    for (int k = 0; k < K; ++k) {
        const int d = blocks[k]->d;
        std::vector<double> V(ns * d * d), Pm(ns * d * d);
        FTLM_CUDA(cudaMemcpy(V.data(), blocks[k]->d_V, V.size() * 8, cudaMemcpyDeviceToHost));
        for (size_t t = 0; t < ns; ++t)
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) {
                    double acc = 0.0;
                    for (int q = 0; q < d; ++q) acc += V[(t * d + i) * d + q] * V[(t * d + j) * d + q];
                    Pm[(t * d + i) * d + j] = acc;
                }
        std::vector<float> Pf(Pm.begin(), Pm.end());
        FTLM_CUDA(cudaMalloc((void **)&ps->d_P[k], Pm.size() * 8));
        FTLM_CUDA(cudaMalloc((void **)&ps->d_Pf[k], Pf.size() * 4));
        FTLM_CUDA(cudaMemcpy(ps->d_P[k], Pm.data(), Pm.size() * 8, cudaMemcpyHostToDevice));
        FTLM_CUDA(cudaMemcpy(ps->d_Pf[k], Pf.data(), Pf.size() * 4, cudaMemcpyHostToDevice));
        ps->device_bytes += Pm.size() * 12;
    }
    // rho(g) tables of the blocks, concatenated (FP64 and FP32), rows padded as in contract.cuh
    std::vector<double> rho;
    std::vector<float> rhof;
    const int G = s->G;
    for (int k = 0; k < K; ++k) {
        const Irrep &ir = s->grp.irreps[blocks[k]->irrep];
        const int d = ir.dim, RP = rho_row(d);
        ps->rho_off[k] = (int)rho.size();
        ps->rho_offf[k] = (int)rhof.size();
        rho.resize(rho.size() + rho_table_elems<double>(G, d), 0.0);
        rhof.resize(rhof.size() + rho_table_elems<float>(G, d), 0.0f);
        for (int g = 0; g < G; ++g)  // rho(g) row-major, rows padded to RP: [g][gamma][beta]
            for (int ga = 0; ga < d; ++ga)
                for (int be = 0; be < d; ++be) {
                    const double v = ir.rho[((size_t)g * d + ga) * d + be];
                    rho[ps->rho_off[k] + ((size_t)g * d + ga) * RP + be] = v;
                    rhof[ps->rho_offf[k] + ((size_t)g * d + ga) * RP + be] = (float)v;
                }
    }
    ps->rho_total = (int)rho.size();
    ps->rho_totalf = (int)rhof.size();
    FTLM_CUDA(cudaMalloc((void **)&ps->d_ntab, ntab.size() + 1));
    FTLM_CUDA(cudaMalloc((void **)&ps->d_wtab, wtab.size() + 1));
    FTLM_CUDA(cudaMalloc((void **)&ps->d_rhoT, rho.size() * 8 + 16));
    FTLM_CUDA(cudaMalloc((void **)&ps->d_rhoTf, rhof.size() * 4 + 16));
    FTLM_CUDA(cudaMalloc((void **)&ps->d_rec, s->n_reps * sizeof(HvRec) + sizeof(HvRec)));
    ps->device_bytes += ntab.size() + wtab.size() + rho.size() * 8 + rhof.size() * 4 + s->n_reps * sizeof(HvRec);
    FTLM_CUDA(cudaMemcpyAsync(ps->d_ntab, ntab.data(), ntab.size(), cudaMemcpyHostToDevice, stream));
    FTLM_CUDA(cudaMemcpyAsync(ps->d_wtab, wtab.data(), wtab.size(), cudaMemcpyHostToDevice, stream));
    FTLM_CUDA(cudaMemcpyAsync(ps->d_rhoT, rho.data(), rho.size() * 8, cudaMemcpyHostToDevice, stream));
    FTLM_CUDA(cudaMemcpyAsync(ps->d_rhoTf, rhof.data(), rhof.size() * 4, cudaMemcpyHostToDevice, stream));
    const uint64_t rows = s->n_reps * (uint64_t)ps->W;
    if (rows >= 0xffffffffull)
        return fail(FTLM_EUNSUPPORTED, "packed set has %llu rows (limit 2^32 - 1)", (unsigned long long)rows);
    ps->rows = rows;
    if (s->n_reps) {
        count_launch();
        fill_records<<<(unsigned)((s->n_reps + 255) / 256), 256, 0, stream>>>(s->d_labels, s->d_stab_id, s->n_reps,
                                                                               ps->W, ps->d_rec);
        FTLM_CUDA(cudaGetLastError());
    }
    FTLM_CUDA(cudaStreamSynchronize(stream));
    guard.p = nullptr;
    *out = ps;
    return FTLM_OK;
}

// ---------------------------------------------------------------- launch assembly

// mode 0: on-the-fly search; 1: flips from the sector's entry table
template <typename VT>
const HvpOps<VT> *hvp_ops(int shape, int gpl, bool half, int esize, int mode);
template <>
const HvpOps<float> *hvp_ops<float>(int shape, int gpl, bool half, int esize, int mode) {
    if (shape_is_wide(shape))
        return esize == 2 ? hvp_ops_wide_f16(shape, half, mode) : hvp_ops_wide_f32(shape, half, mode);
    if (mode == 1) return esize == 2 ? hvp_ops_table_f16(shape) : hvp_ops_table_f32(shape);
    if (esize == 2)
        return shape <= kShapeD5 ? hvp_ops_single_f16(shape, gpl, half) : hvp_ops_multi_f16(shape, gpl, half);
    return shape <= kShapeD5 ? hvp_ops_single_f32(shape, gpl, half) : hvp_ops_multi_f32(shape, gpl, half);
}
template <>
const HvpOps<double> *hvp_ops<double>(int shape, int gpl, bool half, int esize, int mode) {
    if (esize != 8) return nullptr;
    if (shape_is_wide(shape)) return hvp_ops_wide_f64(shape, half, mode);
    if (mode == 1) return hvp_ops_table_f64(shape);
    return shape <= kShapeD5 ? hvp_ops_single_f64(shape, gpl, half) : hvp_ops_multi_f64(shape, gpl, half);
}

// Sector-wide part of the arguments (search tables, coefficients, irreps of the set).
template <typename VT>
void hvp_fill_common(const ftlm_sector *s, const PackedSet *ps, int B, int esize, HvpArgs<VT> &a) {
    memset(&a, 0, sizeof(a));
    a.N = s->N;
    a.G = s->G;
    a.n_bonds = s->grp.n_bonds();
    a.bits = s->bits;
    a.two_s = s->two_s;
    a.n_chunks = s->n_chunks2;
    a.J = (VT)s->grp.J;
    const double sp = 0.5 * s->two_s, ss1 = sp * (sp + 1.0);
    for (int i = 0; i < 8; ++i) {
        const double mm = i - sp;
        const double u = ss1 - mm * (mm + 1.0), dn = ss1 - mm * (mm - 1.0);
        a.up[i] = (VT)(u > 0 ? sqrt(u) : 0.0);
        a.dn[i] = (VT)(dn > 0 ? sqrt(dn) : 0.0);
    }
    a.flip = s->flip;
    a.flipc = s->flipc;
    a.neg = ps->neg;
    a.lut2 = s->d_lut2;
    a.pos = s->d_pos;
    a.dtab = s->d_dtab;
    a.bonds = s->d_bonds;
    if (sizeof(VT) == 4) {
        a.rhoT = reinterpret_cast<const VT *>(ps->d_rhoTf);
        a.rho_total = ps->rho_totalf;
        for (int k = 0; k < ps->K; ++k) a.rho_off[k] = ps->rho_offf[k];
    } else {
        a.rhoT = reinterpret_cast<const VT *>(ps->d_rhoT);
        a.rho_total = ps->rho_total;
        for (int k = 0; k < ps->K; ++k) a.rho_off[k] = ps->rho_off[k];
    }
    int bt = 1, lg = 0;
    while (bt < B) {
        bt <<= 1;
        ++lg;
    }
    a.B = B;
    a.BT = bt;
    a.lgBT = lg;
    a.esize = esize;
    const int per16 = 16 / esize;
    a.slot_elems = (ps->W * B + per16 - 1) / per16 * per16;
    // Pad the slot so that the Q flip groups' slots start in different bank windows: a contraction
    // load reads byte  fg * slot_bytes + row * B * esize + b * esize  in every lane (fg, b), and the
    // Q windows of bt * esize bytes then tile the 32 four-byte banks (slot_bytes an odd multiple of the
    // window; windows below 16 bytes keep the 16-byte slot alignment the bulk copies need).
    {
        const int unit = std::max(16, bt * esize);
        if (unit < 128)
            for (int i = 0; i < 16; ++i) {
                const int sb = a.slot_elems * esize;
                if (sb % unit == 0 && (sb / unit) % 2 == 1) break;
                a.slot_elems += per16;
            }
    }
    const int Q = 32 / bt;
    int st = Q * a.slot_elems;
    // the epilogue reuses the staging buffer for W x bt arithmetic values
    st = std::max(st, (int)((ps->W * bt * sizeof(VT) + esize - 1) / esize));
    a.stage_elems = (st + per16 - 1) / per16 * per16;
    a.wait_limit = wait_limit_cycles();
    a.err = s->d_err;
}

template <typename VT>
void hvp_part_of(const ftlm_sector *s, const PackedSet *ps, const ftlm_basis *const *blocks, const void *x, void *y,
                 HvpPart<VT> &p) {
    memset(&p, 0, sizeof(p));
    p.n_reps = s->n_reps;
    p.rec = ps->d_rec;
    p.bucket = s->d_bucket;
    p.n_buckets = s->n_buckets;
    p.bucket_shift = s->bucket_shift;
    p.n_sid = (int)s->stab_elems.size();
    p.wtab = ps->d_wtab;
    if (sizeof(VT) == 4) {
        p.sqrtS = reinterpret_cast<const VT *>(blocks[0]->d_sqrtSf);
        for (int k = 0; k < ps->K; ++k) p.Pj[k] = reinterpret_cast<const VT *>(ps->d_Pf[k]);
    } else {
        p.sqrtS = reinterpret_cast<const VT *>(blocks[0]->d_sqrtS);
        for (int k = 0; k < ps->K; ++k) p.Pj[k] = reinterpret_cast<const VT *>(ps->d_P[k]);
    }
    p.x = x;
    p.y = y;
    p.eoff = s->d_eoff;
    p.ent = s->d_ent;
}

// Geometry: the most warps (up to the kernel's bound) whose shared memory fits;
// at that warp count, rho tables in shared memory before reading them through
// L1 (FP32), the own-row prefetch before plain loads, and the most staging
// buffers in flight (bulk-copy path, up to kMaxBuf).  FTLM_HV_WARPS,
// FTLM_HV_NBUF, FTLM_HV_RHO (smem|l1) and FTLM_HV_OWN (0|1) override the choice.
template <typename VT>
ftlm_status hvp_choose_geom(const HvpOps<VT> *ops, HvpArgs<VT> a, bool tma, HvpGeom &geo) {
    int dev = 0, sms = kNumSMs;
    FTLM_CUDA(cudaGetDevice(&dev));
    FTLM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const char *ew = getenv("FTLM_HV_WARPS");
    const char *eb = getenv("FTLM_HV_NBUF");
    const char *er = getenv("FTLM_HV_RHO");
    const char *eo = getenv("FTLM_HV_OWN");
    const int max_warps = ops->max_threads / 32;
    const int want_warps = ew ? std::min(atoi(ew), max_warps) : 0;
    const int want_nbuf = eb ? std::max(1, std::min(atoi(eb), kMaxBuf)) : 0;
    std::vector<int> rho_opts = sizeof(VT) == 4 ? std::vector<int>{1, 0} : std::vector<int>{0};
    if (er && sizeof(VT) == 4) rho_opts = {strcmp(er, "l1") == 0 ? 0 : 1};
    std::vector<int> own_opts = tma ? std::vector<int>{1, 0} : std::vector<int>{0};
    if (eo && tma) own_opts = {atoi(eo) ? 1 : 0};
    a.tma = tma ? 1 : 0;
    for (int warps = max_warps; warps >= 2; warps -= 2) {
        if (want_warps > 0 && warps != want_warps) continue;
        for (int rho : rho_opts)
            for (int own : own_opts) {
                const int nb_hi = tma ? (want_nbuf ? want_nbuf : kMaxBuf) : 1;
                const int nb_lo = tma && want_nbuf ? want_nbuf : 1;
                for (int nbuf = nb_hi; nbuf >= nb_lo; --nbuf) {
                    a.rho_smem = rho;
                    a.own = own;
                    const int per_sm = ops->occupancy(a, warps, nbuf);
                    if (per_sm < 1) continue;
                    geo.warps = warps;
                    geo.nbuf = nbuf;
                    geo.tma = tma ? 1 : 0;
                    geo.rho_smem = rho;
                    geo.own = own;
                    geo.tile_reps = ops->tile_fixed ? ops->tile_fixed : warps * 4;
                    geo.grid = sms * per_sm;
                    return FTLM_OK;
                }
            }
    }
    return fail(FTLM_EUNSUPPORTED, "packed H·v does not fit in shared memory");
}

// ---------------------------------------------------------------- autotuner
//
// With autotuning on, the first plan of every (shape, elements per lane, label
// width, element type, B, gather path, log2 of the representative count) key
// times the candidate geometries on the plan's own buffers and keeps the
// fastest for the rest of the process: warps per CTA (the kernel's bound down
// to 4), staging buffers in flight (1..4 on the bulk-copy path), rho tables in
// shared memory or read through L1 (FP32), the own-row prefetch on or off, and
// the representatives per tile (2, 4 or 8 per warp).  Every candidate computes
// the same rows (one warp per representative, fixed flip order), so the choice
// changes timing only.

struct TuneKey {
    int shape, gpl, half, vt, B, tma, lg, mode;
    bool operator<(const TuneKey &o) const {
        return std::tie(shape, gpl, half, vt, B, tma, lg, mode) <
               std::tie(o.shape, o.gpl, o.half, o.vt, o.B, o.tma, o.lg, o.mode);
    }
};
struct TuneVal {
    HvpGeom geo;
    float ms, ms_default;
    int tried;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tuned;
std::atomic<int> g_autotune{0};

template <typename VT>
void hvp_retile(HvpPlan<VT> &plan, std::vector<HvpPart<VT>> &parts) {
    uint64_t tiles = 0;
    plan.tile0.clear();
    plan.ntile.clear();
    for (auto &p : parts) {
        p.tile0 = tiles;
        const uint64_t nt = (p.n_reps + plan.geo.tile_reps - 1) / plan.geo.tile_reps;
        plan.tile0.push_back(tiles);
        plan.ntile.push_back(nt);
        tiles += nt;
    }
    plan.geo.grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)plan.geo.grid, tiles));
    HvpArgs<VT> &a = plan.a;
    a.n_parts = (int)parts.size();
    a.n_tiles = tiles;
    a.tile_reps = plan.geo.tile_reps;
    a.nbuf = plan.geo.nbuf;
    a.tma = plan.geo.tma;
    a.rho_smem = plan.geo.rho_smem;
    a.own = plan.geo.own;
    if (parts.size() == 1) a.part0 = parts[0];
}

template <typename VT>
ftlm_status hvp_tune(HvpPlan<VT> &plan, std::vector<HvpPart<VT>> &parts, bool tma, cudaStream_t stream,
                     TuneVal &out) {
    int dev = 0, sms = kNumSMs;
    FTLM_CUDA(cudaGetDevice(&dev));
    FTLM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DevBuf<HvpPart<VT>> d_parts;
    if (parts.size() > 1) FTLM_CUDA(d_parts.alloc(parts.size()));
    cudaEvent_t e0, e1;
    FTLM_CUDA(cudaEventCreate(&e0));
    FTLM_CUDA(cudaEventCreate(&e1));
    auto time_geo = [&](const HvpGeom &g, float &ms) -> ftlm_status {
        plan.geo = g;
        hvp_retile<VT>(plan, parts);
        if (parts.size() > 1) {
            FTLM_CUDA(cudaMemcpyAsync(d_parts.p, parts.data(), parts.size() * sizeof(HvpPart<VT>),
                                      cudaMemcpyHostToDevice, stream));
            plan.a.parts = d_parts.p;
        }
        ftlm_status st = hvp_launch_plan<VT>(plan, nullptr, stream, false);  // warm-up
        if (st != FTLM_OK) return st;
        FTLM_CUDA(cudaEventRecord(e0, stream));
        st = hvp_launch_plan<VT>(plan, nullptr, stream, false);
        if (st != FTLM_OK) return st;
        FTLM_CUDA(cudaEventRecord(e1, stream));
        FTLM_CUDA(cudaEventSynchronize(e1));
        FTLM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        return FTLM_OK;
    };
    const HvpGeom def = plan.geo;
    float best_ms = 0.f;
    ftlm_status st = time_geo(def, best_ms);
    if (st != FTLM_OK) return st;
    out.geo = def;
    out.ms = out.ms_default = best_ms;
    out.tried = 1;
    const int max_warps = plan.ops->max_threads / 32;
    std::vector<int> rho_opts = sizeof(VT) == 4 ? std::vector<int>{1, 0} : std::vector<int>{0};
    std::vector<int> own_opts = tma ? std::vector<int>{0, 1} : std::vector<int>{0};
    for (int warps = max_warps; warps >= 4; warps -= 4)
        for (int rho : rho_opts)
            for (int own : own_opts)
                for (int nbuf = 1; nbuf <= (tma ? kMaxBuf : 1); ++nbuf)
                    for (int tr : {2, 4, 8}) {
                        HvpArgs<VT> a = plan.a;
                        a.tma = tma ? 1 : 0;
                        a.rho_smem = rho;
                        a.own = own;
                        const int per_sm = plan.ops->occupancy(a, warps, nbuf);
                        if (per_sm < 1) continue;
                        HvpGeom g{warps, nbuf, tma ? 1 : 0, warps * tr, sms * per_sm, rho, own};
                        if (g.warps == def.warps && g.nbuf == def.nbuf && g.rho_smem == def.rho_smem &&
                            g.own == def.own && g.tile_reps == def.tile_reps)
                            continue;
                        float ms = 0.f;
                        if ((st = time_geo(g, ms)) != FTLM_OK) return st;
                        ++out.tried;
                        if (ms < out.ms) {
                            out.ms = ms;
                            out.geo = g;
                        }
                    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    plan.geo = out.geo;
    plan.geo.grid = sms * std::max(1, plan.ops->occupancy([&] {
                                           HvpArgs<VT> a = plan.a;
                                           a.tma = out.geo.tma;
                                           a.rho_smem = out.geo.rho_smem;
                                           a.own = out.geo.own;
                                           return a;
                                       }(),
                                                           out.geo.warps, out.geo.nbuf));
    out.geo.grid = plan.geo.grid;
    return FTLM_OK;
}

// Plan of a packed H·v launch over parts that share the set's shape and group:
// arguments, geometry and tile order.  One part travels inside the kernel
// arguments; several need a device array of descriptors (HvpPlan::a.parts),
// filled by the caller before the launch and kept alive until it ends.
template <typename VT>
ftlm_status hvp_plan(const ftlm_sector *s, const PackedSet *ps, std::vector<HvpPart<VT>> &parts, int B, int esize,
                     HvpPlan<VT> &plan, cudaStream_t tune_stream) {
    if (ps->shape < 0) return fail(FTLM_EUNSUPPORTED, "no compiled packed kernel for this block set");
    HvpArgs<VT> &a = plan.a;
    hvp_fill_common<VT>(s, ps, B, esize, a);
    const int gpl = s->G <= 64 ? 2 : 4;
    int mode = 1;  // the entry-table path when every part's sector has a table
    for (auto &p : parts) mode = mode && p.eoff && p.ent;
    plan.mode = mode;
    plan.ops = hvp_ops<VT>(ps->shape, gpl, s->half, esize, mode);
    if (mode == 1 && ps->K == 1 && B == 1) {  // one thread per representative
        const HvpOps<VT> *lane = nullptr;
        if constexpr (sizeof(VT) == 8)
            lane = shape_is_wide(ps->shape) ? hvp_ops_wide_f64(ps->shape, s->half, 2) : hvp_ops_lane_f64(ps->shape);
        else if (shape_is_wide(ps->shape))
            lane = esize == 2 ? hvp_ops_wide_f16(ps->shape, s->half, 2) : hvp_ops_wide_f32(ps->shape, s->half, 2);
        else
            lane = esize == 2 ? hvp_ops_lane_f16(ps->shape) : hvp_ops_lane_f32(ps->shape);
        // its rho table lives in shared memory: keep the warp kernel when the table does not fit
        if (lane && lane->occupancy(a, lane->max_threads / 32, 1) > 0) plan.ops = lane;
    }
    if (!plan.ops)
        return fail(FTLM_EUNSUPPORTED, "no compiled packed kernel for shape %d with |G| = %d", ps->shape, s->G);
    bool tma = (B * esize) % 16 == 0;
    uint64_t n_reps_total = 0;
    for (auto &p : parts) {
        tma = tma && ((uintptr_t)p.x % 16) == 0;
        n_reps_total += p.n_reps;
    }
    const char *gm = getenv("FTLM_HV_GATHER");
    if (gm && strcmp(gm, "direct") == 0) tma = false;
    ftlm_status st = hvp_choose_geom<VT>(plan.ops, a, tma, plan.geo);
    if (st != FTLM_OK) return st;
    plan.rows_total = 0;
    if (g_autotune.load() && !plan.ops->tile_fixed && !getenv("FTLM_HV_WARPS") && !getenv("FTLM_HV_NBUF")) {
        int lg = 0;
        while ((1ull << lg) < n_reps_total) ++lg;
        const TuneKey key{ps->shape, gpl, s->half ? 1 : 0, esize, B, tma ? 1 : 0, lg, mode};
        std::unique_lock<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            plan.geo = it->second.geo;
        } else {
            lk.unlock();
            TuneVal tv;
            st = hvp_tune<VT>(plan, parts, tma, tune_stream, tv);
            if (st != FTLM_OK) return st;
            lk.lock();
            g_tuned[key] = tv;
        }
    }
    hvp_retile<VT>(plan, parts);
    const uint64_t tiles = a.n_tiles;
    if (getenv("FTLM_HV_VERBOSE"))
        fprintf(stderr, "ftlm hvp plan: shape %d B %d mode %d warps %d nbuf %d tma %d rho_smem %d own %d grid %d "
                        "tiles %llu tile_reps %d wait_limit %llu\n",
                ps->shape, B, mode, plan.geo.warps, plan.geo.nbuf, plan.geo.tma, plan.geo.rho_smem, plan.geo.own,
                plan.geo.grid, (unsigned long long)tiles, plan.geo.tile_reps, (unsigned long long)a.wait_limit);
    a.parts = nullptr;
    return FTLM_OK;
}

// Launch a plan (no host-device copies, so it can be captured in a graph).
template <typename VT>
ftlm_status hvp_launch_plan(const HvpPlan<VT> &plan, double *dot_part, cudaStream_t stream, bool timed) {
    if (plan.a.n_tiles == 0) return FTLM_OK;
    HvpArgs<VT> a = plan.a;
    a.dot_part = dot_part;
    a.flips = profiling_on() && plan.mode != 2 ? profile_flip_counter() : nullptr;  // H·v flips only
    if (a.n_parts > 1 && !a.parts) return fail(FTLM_EINVAL, "several parts need a device descriptor array");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed) hv_timer_begin(stream, &e0, &e1);
    ftlm_status st = plan.ops->launch(a, plan.geo, stream);
    if (timed) hv_timer_end(stream, e0, e1, plan.rows_total * (uint64_t)a.B);
    return st;
}

template <typename VT>
ftlm_status lift_impl(const ftlm_sector *s, const PackedSet *ps, const ftlm_basis *const *blocks, int B,
                      VT *const *blk, VT *packed, int to_packed, cudaStream_t stream) {
    LiftArgs la;
    memset(&la, 0, sizeof(la));
    la.n_reps = s->n_reps;
    la.K = ps->K;
    la.W = ps->W;
    la.B = B;
    la.to_packed = to_packed;
    la.ntab = ps->d_ntab;
    la.rec = ps->d_rec;
    int z = 0;
    for (int k = 0; k < ps->K; ++k) {
        la.dims[k] = ps->dims[k];
        la.zoff[k] = z;
        z += ps->dims[k];
        la.boff[k] = blocks[k]->d_off;
        la.V[k] = sizeof(VT) == 8 ? (const void *)blocks[k]->d_V : (const void *)blocks[k]->d_Vf;
        la.blk[k] = blk[k];
    }
    const uint64_t n = s->n_reps * (uint64_t)B;
    if (n) {
        count_launch();
        lift_rows<VT><<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(la, packed);
        FTLM_CUDA(cudaGetLastError());
    }
    return FTLM_OK;
}

// One block through the packed kernel: lift x, H·v, lower y (stream-ordered scratch).
template <typename VT>
ftlm_status hv_block(const ftlm_basis *b, int B, const VT *x, VT *y, cudaStream_t stream) {
    const PackedSet *ps = b->ps;
    const size_t n = ps->rows * (size_t)B;
    VT *xl = nullptr, *yl = nullptr;
    FTLM_CUDA(cudaMallocAsync((void **)&xl, std::max<size_t>(n, 1) * sizeof(VT), stream));
    cudaError_t e = cudaMallocAsync((void **)&yl, std::max<size_t>(n, 1) * sizeof(VT), stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(xl, stream);
        return fail(e == cudaErrorMemoryAllocation ? FTLM_ENOMEM : FTLM_ECUDA, "H·v scratch: %s", cudaGetErrorString(e));
    }
    const ftlm_basis *one[1] = {b};
    VT *xb[1] = {const_cast<VT *>(x)};
    VT *yb[1] = {y};
    ftlm_status st = lift_impl<VT>(b->sec, ps, one, B, xb, xl, 1, stream);
    if (st == FTLM_OK) {
        std::vector<HvpPart<VT>> parts(1);
        hvp_part_of<VT>(b->sec, ps, one, xl, yl, parts[0]);
        HvpPlan<VT> plan;
        st = hvp_plan<VT>(b->sec, ps, parts, B, (int)sizeof(VT), plan, stream);
        plan.rows_total = ps->rows;
        if (st == FTLM_OK) st = hvp_launch_plan<VT>(plan, nullptr, stream, true);
    }
    if (st == FTLM_OK) st = lift_impl<VT>(b->sec, ps, one, B, yb, yl, 0, stream);
    cudaFreeAsync(xl, stream);
    cudaFreeAsync(yl, stream);
    return st;
}

template <typename VT>
ftlm_status hvp_run_one(const ftlm_sector *s, const PackedSet *ps, const ftlm_basis *const *blocks, int B, int esize,
                        const void *x, void *y, cudaStream_t stream) {
    std::vector<HvpPart<VT>> parts(1);
    hvp_part_of<VT>(s, ps, blocks, x, y, parts[0]);
    HvpPlan<VT> plan;
    ftlm_status st = hvp_plan<VT>(s, ps, parts, B, esize, plan, stream);
    if (st != FTLM_OK) return st;
    plan.rows_total = ps->rows;
    return hvp_launch_plan<VT>(plan, nullptr, stream, true);
}

template ftlm_status hvp_plan<float>(const ftlm_sector *, const PackedSet *, std::vector<HvpPart<float>> &, int,
                                     int, HvpPlan<float> &, cudaStream_t);
template ftlm_status hvp_plan<double>(const ftlm_sector *, const PackedSet *, std::vector<HvpPart<double>> &, int,
                                      int, HvpPlan<double> &, cudaStream_t);
template void hvp_fill_common<float>(const ftlm_sector *, const PackedSet *, int, int, HvpArgs<float> &);
template ftlm_status hvp_choose_geom<float>(const HvpOps<float> *, HvpArgs<float>, bool, HvpGeom &);
template void hvp_retile<float>(HvpPlan<float> &, std::vector<HvpPart<float>> &);
template ftlm_status hvp_launch_plan<float>(const HvpPlan<float> &, double *, cudaStream_t, bool);
template ftlm_status hvp_launch_plan<double>(const HvpPlan<double> &, double *, cudaStream_t, bool);
template void hvp_part_of<float>(const ftlm_sector *, const PackedSet *, const ftlm_basis *const *, const void *,
                                 void *, HvpPart<float> &);
template void hvp_part_of<double>(const ftlm_sector *, const PackedSet *, const ftlm_basis *const *, const void *,
                                  void *, HvpPart<double> &);

template <typename VT>
ftlm_status pack_impl(const ftlm_multiblock *mb, int B, VT *const *blk, VT *packed, int to_packed,
                      cudaStream_t stream) {
    ftlm_status st = lift_impl<VT>(mb->sec, mb->ps, mb->blocks.data(), B, blk, packed, to_packed, stream);
    if (st != FTLM_OK) return st;
    FTLM_CUDA(cudaStreamSynchronize(stream));
    return FTLM_OK;
}

template ftlm_status lift_impl<float>(const ftlm_sector *, const PackedSet *, const ftlm_basis *const *, int,
                                      float *const *, float *, int, cudaStream_t);
template ftlm_status lift_impl<double>(const ftlm_sector *, const PackedSet *, const ftlm_basis *const *, int,
                                       double *const *, double *, int, cudaStream_t);

}  // namespace ftlm

using namespace ftlm;

extern "C" {

ftlm_status ftlm_hv(const ftlm_basis *b, ftlm_dtype dtype, int B, const void *x, void *y, void *cuda_stream) {
    if (!b || !x || !y) return fail(FTLM_EINVAL, "NULL argument");
    if (B < 1 || B > kMaxB) return fail(FTLM_EINVAL, "B must be in 1..%d", kMaxB);
    if (b->dim == 0) return FTLM_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (dtype == FTLM_F64) return hv_block<double>(b, B, (const double *)x, (double *)y, st);
    if (dtype == FTLM_F32) return hv_block<float>(b, B, (const float *)x, (float *)y, st);
    return fail(FTLM_EINVAL, "unknown dtype");
}

ftlm_status ftlm_multiblock_packed_rows(const ftlm_multiblock *mb, uint64_t *rows) {
    if (!mb || !rows) return fail(FTLM_EINVAL, "NULL argument");
    if (!mb->ps) return fail(FTLM_EUNSUPPORTED, "no packed layout for this block set");
    *rows = mb->ps->rows;
    return FTLM_OK;
}

ftlm_status ftlm_hv_packed(const ftlm_multiblock *mb, ftlm_dtype dtype, int B, const void *x, void *y,
                           void *cuda_stream) {
    if (!mb || !x || !y) return fail(FTLM_EINVAL, "NULL argument");
    if (B < 1 || B > kMaxB) return fail(FTLM_EINVAL, "B must be in 1..%d", kMaxB);
    if (!mb->ps) return fail(FTLM_EUNSUPPORTED, "no packed layout for this block set");
    if (mb->ps->rows == 0) return FTLM_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const ftlm_basis *const *bl = mb->blocks.data();
    if (dtype == FTLM_F64) return hvp_run_one<double>(mb->sec, mb->ps, bl, B, 8, x, y, st);
    if (dtype == FTLM_F32) return hvp_run_one<float>(mb->sec, mb->ps, bl, B, 4, x, y, st);
    if (dtype == FTLM_F16) return hvp_run_one<float>(mb->sec, mb->ps, bl, B, 2, x, y, st);
    return fail(FTLM_EINVAL, "unknown dtype");
}

ftlm_status ftlm_multiblock_pack(const ftlm_multiblock *mb, ftlm_dtype dtype, int B, const void *const *blocks,
                                 void *packed, void *cuda_stream) {
    if (!mb || !blocks || !packed) return fail(FTLM_EINVAL, "NULL argument");
    if (B < 1 || B > kMaxB) return fail(FTLM_EINVAL, "B must be in 1..%d", kMaxB);
    if (!mb->ps) return fail(FTLM_EUNSUPPORTED, "no packed layout for this block set");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (dtype == FTLM_F64) return pack_impl<double>(mb, B, (double *const *)blocks, (double *)packed, 1, st);
    if (dtype == FTLM_F32) return pack_impl<float>(mb, B, (float *const *)blocks, (float *)packed, 1, st);
    return fail(FTLM_EINVAL, "unknown dtype");
}

ftlm_status ftlm_multiblock_unpack(const ftlm_multiblock *mb, ftlm_dtype dtype, int B, const void *packed,
                                   void *const *blocks, void *cuda_stream) {
    if (!mb || !blocks || !packed) return fail(FTLM_EINVAL, "NULL argument");
    if (B < 1 || B > kMaxB) return fail(FTLM_EINVAL, "B must be in 1..%d", kMaxB);
    if (!mb->ps) return fail(FTLM_EUNSUPPORTED, "no packed layout for this block set");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (dtype == FTLM_F64)
        return pack_impl<double>(mb, B, (double *const *)blocks, const_cast<double *>((const double *)packed), 0, st);
    if (dtype == FTLM_F32)
        return pack_impl<float>(mb, B, (float *const *)blocks, const_cast<float *>((const float *)packed), 0, st);
    return fail(FTLM_EINVAL, "unknown dtype");
}

ftlm_status ftlm_set_autotune(int on) {
    g_autotune.store(on > 0 ? 1 : 0);
    if (on < 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned.clear();
    }
    return FTLM_OK;
}

ftlm_status ftlm_autotune_report(char *buf, size_t len) {
    if (!buf || len == 0) return fail(FTLM_EINVAL, "bad arguments");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::string s;
    char line[256];
    for (auto &kv : g_tuned) {
        const TuneKey &k = kv.first;
        const TuneVal &v = kv.second;
        snprintf(line, sizeof line,
                 "shape=%d gpl=%d half=%d esize=%d B=%d tma=%d log2reps=%d -> warps=%d nbuf=%d rho_smem=%d own=%d "
                 "tile_reps=%d grid=%d ms=%.4f default_ms=%.4f tried=%d\n",
                 k.shape, k.gpl, k.half, k.vt, k.B, k.tma, k.lg, v.geo.warps, v.geo.nbuf, v.geo.rho_smem, v.geo.own,
                 v.geo.tile_reps, v.geo.grid, v.ms, v.ms_default, v.tried);
        s += line;
    }
    if (s.size() + 1 > len) return fail(FTLM_EINVAL, "buffer of %zu bytes too small (%zu needed)", len, s.size() + 1);
    memcpy(buf, s.c_str(), s.size() + 1);
    return FTLM_OK;
}

ftlm_status ftlm_set_wait_limit(uint64_t cycles) {
    g_wait_limit.store(cycles ? (unsigned long long)cycles : kDrainCycles);
    return FTLM_OK;
}

}  // extern "C"
