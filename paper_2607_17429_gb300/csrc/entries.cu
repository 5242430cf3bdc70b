// Entry table of a sector: the paper's two-phase design (Section 3), where one
// preparation pass maps every ladder flip of every representative to its
// target representative, minimising element and stabilizer, and every later
// H·v reads that table instead of searching.  Here the table is optional and
// per sector (shared by all its irrep blocks and packed sets); the build pass
// is the search part of the packed H·v kernel (build mode), so a table-mode
// H·v processes the same flips in the same order as the search-mode one.
//
// Entries are 8 bytes: target representative index, g*, bond and sign, target
// stabilizer id (HvEntry).  A first pass counts the admissible flips of every
// representative (Eq. 3) and prefix-sums them into the entry offsets.
#include "hvp_ops.h"

namespace ftlm {
namespace {

// Admissible flips of representative i (Eq. 3): s_i^+ s_j^- needs a_i < 2s and
// a_j > 0, s_i^- s_j^+ needs a_i > 0 and a_j < 2s.
struct FlipCount {
    const uint64_t *labels;
    const uint8_t *bonds;
    int n_bonds, bits, two_s;
    __device__ uint64_t operator()(uint64_t i) const {
        const uint64_t lab = labels[i];
        const uint64_t mask = (1ull << bits) - 1;
        uint64_t n = 0;
        for (int e = 0; e < n_bonds; ++e) {
            const int ai = (int)((lab >> (bits * bonds[2 * e])) & mask);
            const int aj = (int)((lab >> (bits * bonds[2 * e + 1])) & mask);
            n += (ai < two_s && aj > 0) + (ai > 0 && aj < two_s);
        }
        return n;
    }
};

// Records {label, index, stabilizer id}: the lookup of the build pass returns the index.
__global__ void index_records(const uint64_t *labels, const uint16_t *stab_id, uint64_t n, HvRec *rec) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    HvRec r;
    r.label = labels[i];
    r.off = (uint32_t)i;
    r.sid = stab_id[i];
    rec[i] = r;
}

}  // namespace

ftlm_status entry_table_build(ftlm_sector *s, cudaStream_t stream) {
    if (s->d_ent) return FTLM_OK;
    const uint64_t n = s->n_reps;
    if (n >= (1ull << 32)) return fail(FTLM_EUNSUPPORTED, "entry tables index representatives with 32 bits");
    if (s->stab_elems.size() > 65535) return fail(FTLM_EUNSUPPORTED, "too many stabilizer classes for an entry");
    DevBuf<uint64_t> eoff;
    FTLM_CUDA(eoff.alloc(n + 1));
    uint64_t total = 0;
    FlipCount fc{s->d_labels, s->d_bonds, s->grp.n_bonds(), s->bits, s->two_s};
    ftlm_status st = exclusive_scan(fc, n, eoff.p, stream, &total);
    if (st != FTLM_OK) return st;
    DevBuf<HvEntry> ent;
    cudaError_t e = cudaMalloc((void **)&ent.p, std::max<uint64_t>(total, 1) * sizeof(HvEntry));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(FTLM_ENOMEM, "entry table of %llu entries: %s", (unsigned long long)total, cudaGetErrorString(e));
    }
    DevBuf<HvRec> rec;
    FTLM_CUDA(rec.alloc(std::max<uint64_t>(n, 1)));
    DevBuf<int> err;
    FTLM_CUDA(err.alloc(1));
    FTLM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), stream));
    if (n) {
        count_launch();
        index_records<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(s->d_labels, s->d_stab_id, n, rec.p);
        FTLM_CUDA(cudaGetLastError());
        // build-mode arguments: the search tables of the sector, no blocks, no vectors
        PackedSet ps;
        ps.K = 1;
        ps.W = 1;
        ps.dims[0] = 1;
        ps.rows = n;
        ps.d_rec = rec.p;
        HvpPlan<float> plan;
        plan.mode = 2;
        HvpArgs<float> &a = plan.a;
        hvp_fill_common<float>(s, &ps, 1, 4, a);
        a.err = err.p;
        HvpPart<float> part;
        memset(&part, 0, sizeof(part));
        part.n_reps = n;
        part.rec = rec.p;
        part.bucket = s->d_bucket;
        part.n_buckets = s->n_buckets;
        part.bucket_shift = s->bucket_shift;
        part.n_sid = (int)s->stab_elems.size();
        part.eoff = eoff.p;
        part.ent = ent.p;
        const int gpl = s->G <= 64 ? 2 : 4;
        plan.ops = hvp_ops_build(gpl, s->half);
        if (!plan.ops) return fail(FTLM_EUNSUPPORTED, "no build kernel for |G| = %d", s->G);
        st = hvp_choose_geom<float>(plan.ops, a, false, plan.geo);
        if (st != FTLM_OK) return st;
        std::vector<HvpPart<float>> parts{part};
        hvp_retile<float>(plan, parts);
        st = hvp_launch_plan<float>(plan, nullptr, stream, false);
        if (st != FTLM_OK) return st;
    }
    int h_err = 0;
    FTLM_CUDA(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, stream));
    FTLM_CUDA(cudaStreamSynchronize(stream));
    if (h_err) {
        if (h_err & kErrWaitTimeout) return fail(FTLM_ETIMEOUT, "a bounded device wait gave up building entries");
        return fail(FTLM_EINTERNAL, "entry table build: a flipped state has no representative (code %d)", h_err);
    }
    s->d_eoff = eoff.release();
    s->d_ent = ent.release();
    s->n_entries = total;
    s->entry_bytes = (n + 1) * sizeof(uint64_t) + total * sizeof(HvEntry);
    s->device_bytes += s->entry_bytes;
    return FTLM_OK;
}

void entry_table_free(ftlm_sector *s) {
    if (!s->d_ent) return;
    cudaFree(s->d_eoff);
    cudaFree(s->d_ent);
    s->d_eoff = nullptr;
    s->d_ent = nullptr;
    s->device_bytes -= s->entry_bytes;
    s->n_entries = 0;
    s->entry_bytes = 0;
}

}  // namespace ftlm

using namespace ftlm;

extern "C" {

ftlm_status ftlm_sector_build_entries(const ftlm_sector *s, void *cuda_stream, uint64_t *n_entries) {
    if (!s) return fail(FTLM_EINVAL, "sector is NULL");
    ftlm_sector *sm = const_cast<ftlm_sector *>(s);
    ftlm_status st = entry_table_build(sm, (cudaStream_t)cuda_stream);
    if (st != FTLM_OK) return st;
    if (n_entries) *n_entries = sm->n_entries;
    return FTLM_OK;
}

ftlm_status ftlm_sector_free_entries(const ftlm_sector *s) {
    if (!s) return fail(FTLM_EINVAL, "sector is NULL");
    entry_table_free(const_cast<ftlm_sector *>(s));
    return FTLM_OK;
}

}  // extern "C"
