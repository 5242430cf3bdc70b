// Serving loop for many independent FTLM jobs on one GPU (no counterpart in
// the paper beyond its batch width chosen from free memory, Section 3).
//
// A job is one block (M, Gamma) of one cluster with R Lanczos chains of
// n_steps steps (Section 2.2).  A scheduler thread admits jobs in arrival
// order while the device bytes they charge stay within the cap: resident
// sector tables (shared by every job on the same cluster, s and M) and block
// tables (shared by the jobs on the same block), plus the job's own Lanczos
// vectors.  Tables no admitted job references are evicted least recently used
// first.  Admitted jobs that share cluster, spin, irrep, R, precision,
// generator and seed run as the parts (one per job, possibly of different S^z
// sectors) of one packed Lanczos launch, a wave, on one of the worker threads'
// streams; each part stops at its own step limit.  A job's coefficients are
// those of ftlm_lanczos on the same block up to rounding: its chains' sums
// keep their order within the part.
#include <math.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>

#include "common.cuh"
#include "hvp_ops.h"
#include "lanczos_packed.h"

namespace ftlm {
namespace {

using Clock = std::chrono::steady_clock;

struct SecEnt;
struct BlkEnt {
    SecEnt *se = nullptr;
    int irrep = 0;
    ftlm_basis *blk = nullptr;
    size_t bytes = 0;
    int refs = 0;  // admitted jobs on this block, plus the scheduler while it builds
    uint64_t last = 0;
};

struct SecEnt {
    ftlm_sector *sec = nullptr;
    size_t bytes = 0;
    int pins = 0;  // the scheduler while it builds this sector or one of its blocks
    uint64_t last = 0;
    std::map<int, std::unique_ptr<BlkEnt>> blocks;
};

struct Job {
    uint64_t id = 0;
    ftlm_job spec{};
    uint64_t ghash = 0;
    ftlm_status status = FTLM_OK;
    std::string msg;
    bool done = false;
    double t_submit = 0, t_admit = -1, t_start = -1, t_done = -1;
    BlkEnt *be = nullptr;
    size_t vec_bytes = 0;
    int d_gamma = 0;
    uint64_t dim = 0;
    std::vector<double> alpha, beta;  // [R][n_steps]
    std::vector<int> steps;           // [R]
};

using SecKey = std::tuple<uint64_t, int, int>;

// FNV-1a over everything that defines the Hamiltonian and its irreps: jobs on
// equal groups share tables even when they come through different handles.
uint64_t group_hash(const GroupData &g) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void *p, size_t n) {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    };
    mix(&g.N, sizeof g.N);
    mix(&g.G, sizeof g.G);
    mix(g.perms.data(), g.perms.size() * sizeof(int32_t));
    mix(g.bonds.data(), g.bonds.size() * sizeof(int32_t));
    mix(&g.J, sizeof g.J);
    for (const Irrep &ir : g.irreps) {
        mix(&ir.dim, sizeof ir.dim);
        mix(ir.rho.data(), ir.rho.size() * sizeof(double));
    }
    return h;
}

// Number of states with sum_i m_i = M (digits a_i = m_i + s in 0..2s), as a
// double: the admission estimate of a sector before it is built.
double sector_dim_estimate(int N, int two_s, int two_M) {
    const int d = two_s + 1;
    const int twice = N * two_s + two_M;
    if (twice < 0 || twice % 2) return 0.0;
    const int A = twice / 2;
    if (A > N * two_s) return 0.0;
    std::vector<double> c((size_t)A + 1, 0.0);
    c[0] = 1.0;
    for (int i = 0; i < N; ++i) {
        std::vector<double> n((size_t)A + 1, 0.0);
        for (int a = 0; a <= A; ++a)
            if (c[a] != 0.0)
                for (int q = 0; q < d && a + q <= A; ++q) n[(size_t)a + q] += c[a];
        c.swap(n);
    }
    return c[A];
}

double now_s(Clock::time_point t0) { return std::chrono::duration<double>(Clock::now() - t0).count(); }

}  // namespace
}  // namespace ftlm

using namespace ftlm;

struct ftlm_server {
    size_t cap = 0;
    int n_workers = 1, max_parts = 64, device = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_sched, cv_work, cv_done;
    bool stop = false;
    uint64_t next_id = 1, tick = 0;
    std::map<uint64_t, std::unique_ptr<Job>> jobs;
    std::deque<Job *> queue;  // submitted, not yet admitted
    std::list<Job *> ready;   // admitted, waiting for a wave
    std::map<SecKey, std::unique_ptr<SecEnt>> sectors;
    size_t charged = 0;
    int running = 0;  // waves in flight
    ftlm_server_stats st{};
    std::thread sched;
    std::vector<std::thread> workers;
};

namespace ftlm {
namespace {

// Evict unreferenced tables (least recently used first) until `need` more
// bytes fit under the cap.  Caller holds the lock.
bool make_room(ftlm_server *S, size_t need) {
    for (;;) {
        if (S->charged + need <= S->cap) return true;
        BlkEnt *vb = nullptr;
        SecEnt *vs = nullptr;
        SecKey vkey{};
        for (auto &kv : S->sectors) {
            SecEnt *se = kv.second.get();
            for (auto &bk : se->blocks) {
                BlkEnt *be = bk.second.get();
                if (be->refs == 0 && be->blk && (!vb || be->last < vb->last)) vb = be;
            }
            if (se->pins == 0 && se->blocks.empty() && se->sec && (!vs || se->last < vs->last)) {
                vs = se;
                vkey = kv.first;
            }
        }
        if (vb && (!vs || vb->last <= vs->last)) {
            ftlm_basis_free(vb->blk);
            S->charged -= vb->bytes;
            SecEnt *se = vb->se;
            se->blocks.erase(vb->irrep);
            ++S->st.evictions;
            continue;
        }
        if (vs) {
            ftlm_sector_free(vs->sec);
            S->charged -= vs->bytes;
            S->sectors.erase(vkey);
            ++S->st.evictions;
            continue;
        }
        return false;
    }
}

void fail_job(ftlm_server *S, Job *J, ftlm_status st, const std::string &msg) {
    J->status = st;
    J->msg = msg;
    J->done = true;
    J->t_done = now_s(S->t0);
    ++S->st.failed;
    S->cv_done.notify_all();
}

// Bytes a job's Lanczos launch allocates: three packed vectors, the scale and
// coefficient state, and the per-CTA dot partials.
size_t vector_bytes(const ftlm_basis *b, const ftlm_job &j) {
    const size_t e = j.dtype == FTLM_F64 ? 8 : (j.dtype == FTLM_F16 ? 2 : 4);
    const size_t B = (size_t)std::min(j.R, kMaxB);
    const size_t rows = b->ps ? b->ps->rows : b->dim;
    return 3 * std::max<size_t>(rows, 1) * B * e + (2 * (size_t)j.n_steps + 16) * B * 8 + 4 * kNumSMs * B * 8 +
           (1u << 20);
}

// One step of admission for the head job.  Returns false when the scheduler
// must wait for running waves to release memory.  Caller holds the lock; the
// lock is released while tables are built.
bool admit_head(ftlm_server *S, std::unique_lock<std::mutex> &lk, cudaStream_t bs) {
    Job *J = S->queue.front();
    const ftlm_job &js = J->spec;
    // nothing admitted will release memory later (re-evaluated after every unlocked build)
    auto idle = [&] { return S->running == 0 && S->ready.empty(); };
    const SecKey key{J->ghash, js.two_s, js.two_M};
    auto it = S->sectors.find(key);
    if (it == S->sectors.end()) it = S->sectors.emplace(key, std::make_unique<SecEnt>()).first;
    SecEnt *se = it->second.get();
    se->last = ++S->tick;
    if (!se->sec) {
        const GroupData &g = js.group->d;
        const double dim = sector_dim_estimate(g.N, js.two_s, js.two_M);
        const size_t est = (size_t)(dim / std::max(1, g.G) * 1.1 * 24.0) + (8u << 20);
        if (!make_room(S, est)) {
            if (!idle()) return false;
            if (se->blocks.empty() && se->pins == 0) S->sectors.erase(key);
            S->queue.pop_front();
            fail_job(S, J, FTLM_ENOMEM, "sector tables do not fit under the admission cap");
            return true;
        }
        ++se->pins;
        lk.unlock();
        ftlm_sector *sec = nullptr;
        ftlm_status st = ftlm_build_sector(js.group, js.two_s, js.two_M, bs, &sec);
        std::string msg = st == FTLM_OK ? "" : ftlm_last_error();
        if (st == FTLM_OK && cudaStreamSynchronize(bs) != cudaSuccess) {
            st = FTLM_ECUDA;
            msg = "sector build failed on the device";
        }
        lk.lock();
        --se->pins;
        if (st != FTLM_OK) {
            if (sec) ftlm_sector_free(sec);
            if (se->blocks.empty() && se->pins == 0) S->sectors.erase(key);
            S->queue.pop_front();
            fail_job(S, J, st, msg);
            return true;
        }
        se->sec = sec;
        se->bytes = sec->device_bytes;
        S->charged += se->bytes;
        S->st.peak_charged = std::max(S->st.peak_charged, S->charged);
        ++S->st.sectors_built;
    } else {
        ++S->st.sector_hits;
    }
    auto bit = se->blocks.find(js.irrep);
    if (bit == se->blocks.end()) {
        auto be = std::make_unique<BlkEnt>();
        be->se = se;
        be->irrep = js.irrep;
        bit = se->blocks.emplace(js.irrep, std::move(be)).first;
    }
    BlkEnt *be = bit->second.get();
    be->last = ++S->tick;
    ++be->refs;  // pinned from here on; kept by the job once admitted
    if (!be->blk) {
        const size_t est = (size_t)se->sec->n_reps * 40 + (4u << 20);
        if (!make_room(S, est)) {
            --be->refs;
            if (!idle()) return false;
            S->queue.pop_front();
            fail_job(S, J, FTLM_ENOMEM, "block tables do not fit under the admission cap");
            return true;
        }
        ++se->pins;
        lk.unlock();
        ftlm_basis *blk = nullptr;
        ftlm_status st = ftlm_build_block(se->sec, js.irrep, bs, &blk);
        std::string msg = st == FTLM_OK ? "" : ftlm_last_error();
        if (st == FTLM_OK && cudaStreamSynchronize(bs) != cudaSuccess) {
            st = FTLM_ECUDA;
            msg = "block build failed on the device";
        }
        if (st == FTLM_OK && !blk->ps) {
            st = FTLM_EUNSUPPORTED;
            msg = "no packed H·v for this block shape";
        }
        lk.lock();
        --se->pins;
        if (st != FTLM_OK) {
            if (blk) ftlm_basis_free(blk);
            --be->refs;
            se->blocks.erase(js.irrep);
            S->queue.pop_front();
            fail_job(S, J, st, msg);
            return true;
        }
        be->blk = blk;
        be->bytes = blk->device_bytes + blk->ps->device_bytes;
        S->charged += be->bytes;
        S->st.peak_charged = std::max(S->st.peak_charged, S->charged);
        ++S->st.blocks_built;
    } else {
        ++S->st.block_hits;
    }
    const size_t need = vector_bytes(be->blk, js);
    if (!make_room(S, need)) {
        --be->refs;
        if (!idle()) return false;
        S->queue.pop_front();
        fail_job(S, J, FTLM_ENOMEM, "the job's vectors do not fit under the admission cap");
        return true;
    }
    S->charged += need;
    S->st.peak_charged = std::max(S->st.peak_charged, S->charged);
    J->vec_bytes = need;
    J->be = be;
    J->d_gamma = be->blk->sec->grp.irreps[be->blk->irrep].weight();
    J->dim = be->blk->dim;
    J->t_admit = now_s(S->t0);
    S->queue.pop_front();
    S->ready.push_back(J);
    S->cv_work.notify_one();
    return true;
}

void scheduler_main(ftlm_server *S) {
    cudaSetDevice(S->device);
    cudaStream_t bs = nullptr;
    cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_sched.wait(lk, [&] { return S->stop || !S->queue.empty(); });
        if (S->stop) break;
        if (!admit_head(S, lk, bs)) S->cv_sched.wait(lk);  // woken when a wave releases memory
    }
    lk.unlock();
    if (bs) cudaStreamDestroy(bs);
}

bool same_wave(const Job *a, const Job *b) {
    const ftlm_job &x = a->spec, &y = b->spec;
    return a->ghash == b->ghash && x.two_s == y.two_s && x.irrep == y.irrep && x.R == y.R && x.dtype == y.dtype &&
           x.rng == y.rng && x.seed == y.seed;
}

void worker_main(ftlm_server *S) {
    cudaSetDevice(S->device);
    cudaStream_t ws = nullptr;
    cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_work.wait(lk, [&] { return S->stop || !S->ready.empty(); });
        if (S->stop) break;
        std::vector<Job *> wave;
        Job *J0 = S->ready.front();
        for (auto it = S->ready.begin(); it != S->ready.end() && (int)wave.size() < S->max_parts;) {
            if (same_wave(J0, *it)) {
                wave.push_back(*it);
                it = S->ready.erase(it);
            } else {
                ++it;
            }
        }
        ++S->running;
        const double t_start = now_s(S->t0);
        for (Job *J : wave) J->t_start = t_start;
        lk.unlock();

        const ftlm_job &js = J0->spec;
        const int P = (int)wave.size(), R = js.R;
        int nmax = 0;
        std::vector<const ftlm_basis *> blks(P);
        std::vector<LzSetIn> sets(P);
        for (int p = 0; p < P; ++p) {
            blks[p] = wave[p]->be->blk;
            sets[p] = LzSetIn{blks[p]->sec, blks[p]->ps, &blks[p], &wave[p]->spec.block_id, wave[p]->spec.n_steps};
            nmax = std::max(nmax, wave[p]->spec.n_steps);
        }
        std::vector<double> A((size_t)P * R * nmax), Bt((size_t)P * R * nmax);
        std::vector<int> Sd((size_t)P * R);
        ftlm_status st =
            js.dtype == FTLM_F64
                ? lanczos_packed<double>(sets, R, nmax, js.seed, js.rng, ws, A.data(), Bt.data(), Sd.data(), 8)
                : lanczos_packed<float>(sets, R, nmax, js.seed, js.rng, ws, A.data(), Bt.data(), Sd.data(),
                                        js.dtype == FTLM_F16 ? 2 : 4);
        const std::string msg = st == FTLM_OK ? "" : ftlm_last_error();

        lk.lock();
        const double t_done = now_s(S->t0);
        for (int p = 0; p < P; ++p) {
            Job *J = wave[p];
            const int n = J->spec.n_steps;
            J->alpha.assign((size_t)R * n, 0.0);
            J->beta.assign((size_t)R * n, 0.0);
            J->steps.assign(R, 0);
            for (int r = 0; r < R; ++r) {
                J->steps[r] = Sd[(size_t)p * R + r];
                for (int j = 0; j < n; ++j) {
                    J->alpha[(size_t)r * n + j] = A[((size_t)p * R + r) * nmax + j];
                    J->beta[(size_t)r * n + j] = Bt[((size_t)p * R + r) * nmax + j];
                }
            }
            J->status = st;
            J->msg = msg;
            J->done = true;
            J->t_done = t_done;
            S->charged -= J->vec_bytes;
            J->vec_bytes = 0;
            --J->be->refs;
            J->be->last = ++S->tick;
            J->be->se->last = S->tick;
            J->be = nullptr;
            if (st == FTLM_OK)
                ++S->st.completed;
            else
                ++S->st.failed;
        }
        ++S->st.waves;
        S->st.parts += (uint64_t)P;
        --S->running;
        S->cv_done.notify_all();
        S->cv_sched.notify_all();
    }
    lk.unlock();
    if (ws) cudaStreamDestroy(ws);
}

}  // namespace
}  // namespace ftlm

extern "C" {

ftlm_status ftlm_server_create(size_t cap_bytes, int n_workers, int max_parts, ftlm_server **out) {
    if (!out) return fail(FTLM_EINVAL, "NULL argument");
    *out = nullptr;
    if (cap_bytes == 0 || n_workers < 1 || n_workers > 16 || max_parts < 1 || max_parts > kPMaxParts)
        return fail(FTLM_EINVAL, "cap > 0, 1 <= n_workers <= 16 and 1 <= max_parts <= %d", kPMaxParts);
    ftlm_server *S = new (std::nothrow) ftlm_server();
    if (!S) return fail(FTLM_ENOMEM, "host allocation failed");
    S->cap = cap_bytes;
    S->n_workers = n_workers;
    S->max_parts = max_parts;
    S->st.cap = cap_bytes;
    S->t0 = Clock::now();
    cudaError_t e = cudaGetDevice(&S->device);
    if (e != cudaSuccess) {
        delete S;
        return fail(FTLM_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    }
    S->sched = std::thread(scheduler_main, S);
    for (int i = 0; i < n_workers; ++i) S->workers.emplace_back(worker_main, S);
    *out = S;
    return FTLM_OK;
}

ftlm_status ftlm_server_submit(ftlm_server *S, const ftlm_job *job, uint64_t *job_id) {
    if (!S || !job || !job_id) return fail(FTLM_EINVAL, "NULL argument");
    if (!job->group) return fail(FTLM_EINVAL, "job without a group");
    if (job->R < 1 || job->R > kMaxB) return fail(FTLM_EINVAL, "R must be in 1..%d", kMaxB);
    if (job->n_steps < 1 || job->n_steps > kMaxSteps) return fail(FTLM_EINVAL, "n_steps must be in 1..%d", kMaxSteps);
    if (job->dtype != FTLM_F32 && job->dtype != FTLM_F64 && job->dtype != FTLM_F16)
        return fail(FTLM_EINVAL, "unknown dtype");
    if (job->rng != FTLM_GAUSS && job->rng != FTLM_RADEMACHER) return fail(FTLM_EINVAL, "unknown rng");
    const GroupData &g = job->group->d;
    if (job->irrep < 0 || job->irrep >= (int)g.irreps.size())
        return fail(FTLM_EINVAL, "irrep %d out of range", job->irrep);
    if (job->two_s < 1 || job->two_s > 7 || job->two_M < 0 || (g.N * job->two_s + job->two_M) % 2)
        return fail(FTLM_EINVAL, "2s in 1..7 and 2M >= 0 with N s + M an integer");
    auto J = std::make_unique<Job>();
    J->spec = *job;
    J->ghash = group_hash(g);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return fail(FTLM_EINVAL, "server is stopping");
    J->id = S->next_id++;
    J->t_submit = now_s(S->t0);
    *job_id = J->id;
    S->queue.push_back(J.get());
    S->jobs.emplace(J->id, std::move(J));
    ++S->st.submitted;
    S->cv_sched.notify_one();
    return FTLM_OK;
}

ftlm_status ftlm_server_wait(ftlm_server *S, uint64_t job_id, double timeout_s, ftlm_job_info *info,
                             double *alpha, double *beta, int *steps_done) {
    if (!S) return fail(FTLM_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(job_id);
    if (it == S->jobs.end()) return fail(FTLM_EINVAL, "unknown job id %llu", (unsigned long long)job_id);
    Job *J = it->second.get();
    auto pred = [&] { return J->done; };
    if (timeout_s < 0)
        S->cv_done.wait(lk, pred);
    else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
        return fail(FTLM_ETIMEOUT, "job %llu not finished within %.3f s", (unsigned long long)job_id, timeout_s);
    if (info) {
        memset(info, 0, sizeof(*info));
        info->status = J->status;
        info->d_gamma = J->d_gamma;
        info->dim = J->dim;
        info->t_submit = J->t_submit;
        info->t_admit = J->t_admit;
        info->t_start = J->t_start;
        info->t_done = J->t_done;
    }
    const size_t n = (size_t)J->spec.R * J->spec.n_steps;
    if (J->status == FTLM_OK) {
        if (alpha) memcpy(alpha, J->alpha.data(), n * sizeof(double));
        if (beta) memcpy(beta, J->beta.data(), n * sizeof(double));
        if (steps_done) memcpy(steps_done, J->steps.data(), (size_t)J->spec.R * sizeof(int));
    }
    const ftlm_status st = J->status;
    const std::string msg = J->msg;
    S->jobs.erase(it);
    if (st != FTLM_OK) return fail(st, "job %llu: %s", (unsigned long long)job_id, msg.c_str());
    return FTLM_OK;
}

ftlm_status ftlm_server_stats_get(ftlm_server *S, ftlm_server_stats *out) {
    if (!S || !out) return fail(FTLM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    out->charged = S->charged;
    out->queued = (int)S->queue.size();
    out->ready = (int)S->ready.size();
    out->running_waves = S->running;
    size_t res = 0;
    for (auto &kv : S->sectors) {
        res += kv.second->sec ? kv.second->bytes : 0;
        for (auto &bk : kv.second->blocks) res += bk.second->blk ? bk.second->bytes : 0;
    }
    out->resident_table_bytes = res;
    return FTLM_OK;
}

void ftlm_server_free(ftlm_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_sched.notify_all();
        S->cv_work.notify_all();
    }
    if (S->sched.joinable()) S->sched.join();
    for (auto &t : S->workers)
        if (t.joinable()) t.join();
    for (auto &kv : S->sectors) {
        for (auto &bk : kv.second->blocks)
            if (bk.second->blk) ftlm_basis_free(bk.second->blk);
        if (kv.second->sec) ftlm_sector_free(kv.second->sec);
    }
    delete S;
}

}  // extern "C"
