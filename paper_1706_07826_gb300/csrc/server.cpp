// Request loop for serving Multi-start SPVAR (Alg. 2) on a stream of problems
// of mixed sizes, with continuous batching.
//
// Requests are admitted in arrival order whenever a request slot is free and
// their device workspace fits the memory budget (first-fit arena).  Every
// engine step runs one sweep chunk (sweeps_per_step sweeps, or a whole phase)
// of Alg. 2 for every admitted start of every request in one persistent launch
// sequence (the same kernels as the plans, captured once as a CUDA graph over
// the whole slot table); a start whose chunk completes its phase's sample
// also runs the persistence pass in that step.  A request that arrives while
// others are running therefore joins at the next step and its work overlaps
// theirs on the device.  Finished requests are copied back and
// their memory released at once.  All state -- problems, samples, reduced
// problems, fix maps -- stays on the device between steps.  Results do not
// depend on what else is in flight: randomness is keyed by (seed, start,
// phase, sweep, spin, replica) only.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "spvar_internal.h"

using namespace spvar;

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// First-fit allocator over one device allocation (offsets only).
class Arena {
public:
    void reset(size_t bytes)
    {
        free_.clear();
        if (bytes) free_[0] = bytes;
    }
    bool alloc(size_t bytes, size_t *off)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

private:
    std::map<size_t, size_t> free_;
};

struct Request {
    int64_t id = 0;
    HostProblem hp;
    uint64_t seed = 0;
    int state = 0;  // 0 queued, 1 running, 2 done
    int rslot = -1;
    size_t off = 0, bytes = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    // results (host)
    std::vector<int64_t> energies, best_e;
    std::vector<int32_t> counts, nfree;
    std::vector<int8_t> fixed, best_state;
};

}  // namespace

struct spvar_server {
    spvar_server_config cfg{};
    int device = 0, ns = 1, P = 2, Smax = 1, nslots = 0, sms = 1;
    cudaStream_t st = nullptr, cap_st = nullptr;
    void *arena_mem = nullptr;
    Arena arena;
    void *fixed_mem = nullptr;
    Slot *d_slots = nullptr;
    std::vector<Slot> h_slots;
    int32_t *d_modes = nullptr, *h_modes = nullptr;
    PhaseEngine E{};  // the engine sized for the largest admissible problem
    // Size tiers: the same engine sized for max_n, max_n / 2, max_n / 4 and
    // max_n / 8 spins (shared memory per CTA, hence CTAs per SM, follow the size),
    // each with its persistent grid and captured phase graph; a step launches the
    // smallest tier that holds every problem in flight.
    struct Tier {
        int max_n = 0, grid = 1;
        PhaseEngine E{};
        cudaGraphExec_t graph = nullptr;
    };
    std::vector<Tier> tiers;  // ascending max_n
    std::mutex mu;
    std::condition_variable cv;
    std::deque<int64_t> queue;
    std::map<int64_t, std::unique_ptr<Request>> reqs;
    std::vector<int64_t> rslot_owner;  // request id per request slot, -1 free
    int64_t next_id = 1;
    std::thread worker;
    bool running = false, stop = false;
    bool failed = false;  // the background engine stopped on an error
    int64_t attempts_done = 0, requests_done = 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};  // recorded around every step's sweep launch
    double sweep_ms = 0.0;                   // sum of the sweep launches' durations
    int64_t sweep_launches = 0;
};

namespace {

size_t request_bytes(const spvar_server *S, const HostProblem &hp)
{
    const size_t pb = a256(prob_blob_bytes(hp.cap_n, hp.cap_nnz, hp.md));
    const int n0 = hp.cap_n;
    size_t per = 2 * pb;
    per += a256(4 * (size_t)S->Smax * ceil_div(n0, 32));
    per += 2 * a256(4 * (size_t)n0) + a256(4 * (size_t)S->Smax) + a256(4 * (size_t)n0) + a256((size_t)n0) +
           a256(4 * (size_t)n0) + a256(4 * slot_scratch_ints(n0));
    per += a256(8 * (size_t)S->P * S->Smax) + 2 * a256(4 * (size_t)S->P) + a256(4) + a256(8) + 2 * a256((size_t)n0);
    per += boost_slot_bytes(S->cfg.params.component_boost, n0, S->Smax, ceil_div(n0, 32));
    per += tree_slot_bytes(S->cfg.params.tree_preprocess, n0);
    return pb + (size_t)S->ns * per;
}

// Lays out a request's workspace in the arena, uploads its problem and fills
// its slot entries (host mirror).  Called without the lock: the request's
// arena range and request slot are reserved, and only the engine thread
// touches the slot table.
int place_request(spvar_server *S, Request &R)
{
    char *base = static_cast<char *>(S->arena_mem) + R.off;
    size_t o = 0;
    auto take = [&](size_t b) { char *r = base + o; o += a256(b); return r; };
    const HostProblem &hp = R.hp;
    const size_t pbytes = prob_blob_bytes(hp.cap_n, hp.cap_nnz, hp.md);
    void *orig_blob = take(pbytes);
    DevProb hdr;
    int rc = host_problem_upload(hp, orig_blob, S->st, &hdr);
    if (rc) return rc;
    const int n0 = hp.cap_n;
    std::vector<DevProb> bufs;
    std::vector<DevProb *> dsts;
    for (int k = 0; k < S->ns; ++k) {
        Slot &s = S->h_slots[(size_t)R.rslot * S->ns + k];
        std::memset(&s, 0, sizeof(Slot));
        for (int b = 0; b < 2; ++b) {
            void *blob = take(pbytes);
            DevProb d;
            std::memset(&d, 0, sizeof(d));
            prob_carve(&d, blob, hp.cap_n, hp.cap_nnz, hp.md);
            bufs.push_back(d);
            dsts.push_back((DevProb *)blob);
            s.buf[b] = (DevProb *)blob;
        }
        s.orig_prob = (const DevProb *)orig_blob;
        s.cur = s.orig_prob;
        s.n0 = hp.hdr.n;
        s.W0 = ceil_div(n0, 32);
        s.seed = R.seed;
        s.start = (uint32_t)(S->cfg.params.start_offset + k);
        s.spins = (uint32_t *)take(4 * (size_t)S->Smax * s.W0);
        s.orig[0] = (int32_t *)take(4 * (size_t)n0);
        s.orig[1] = (int32_t *)take(4 * (size_t)n0);
        s.elite = (int32_t *)take(4 * (size_t)S->Smax);
        s.counts = (int32_t *)take(4 * (size_t)n0);
        s.fixed = (int8_t *)take((size_t)n0);
        s.old_of_new = (int32_t *)take(4 * (size_t)n0);
        s.scratch = (int32_t *)take(4 * slot_scratch_ints(n0));
        s.rec_e = (int64_t *)take(8 * (size_t)S->P * S->Smax);
        s.rec_count = (int32_t *)take(4 * (size_t)S->P);
        s.rec_nfree = (int32_t *)take(4 * (size_t)S->P);
        s.nphases = (int32_t *)take(4);
        s.best_e = (int64_t *)take(8);
        s.fmap = (int8_t *)take((size_t)n0);
        s.best_state = (int8_t *)take((size_t)n0);
        if (S->cfg.params.component_boost)
            boost_slot_carve(s, take(boost_slot_bytes(1, n0, S->Smax, s.W0)), n0, S->Smax, s.W0);
        if (S->cfg.params.tree_preprocess) tree_slot_carve(s, take(tree_slot_bytes(1, n0)), n0);
        s.mode = kDone;  // activated by the init kernel below
    }
    // the header copies must outlive the asynchronous uploads: synchronise here
    bool ok = true;
    for (size_t k = 0; k < bufs.size() && ok; ++k)
        ok = cudaMemcpyAsync(dsts[k], &bufs[k], sizeof(DevProb), cudaMemcpyHostToDevice, S->st) == cudaSuccess;
    Slot *d = S->d_slots + (size_t)R.rslot * S->ns;
    if (ok)
        ok = cudaMemcpyAsync(d, &S->h_slots[(size_t)R.rslot * S->ns], sizeof(Slot) * S->ns, cudaMemcpyHostToDevice,
                             S->st) == cudaSuccess;
    SolveConsts C = S->E.C;
    C.nslots = S->ns;
    if (ok) ok = launch_slots_init(d, C, n0, S->st) == cudaSuccess;
    if (ok) ok = cudaStreamSynchronize(S->st) == cudaSuccess;
    return ok ? SPVAR_OK : SPVAR_ECUDA;
}

int retire_request(spvar_server *S, Request &R)
{
    const int ns = S->ns, n = R.hp.hdr.n, P = S->P, Smax = S->Smax;
    R.energies.assign((size_t)ns * P * Smax, 0);
    R.counts.assign((size_t)ns * P, 0);
    R.nfree.assign((size_t)ns * P, 0);
    R.best_e.assign(ns, 0);
    R.fixed.assign((size_t)ns * std::max(n, 1), 0);
    R.best_state.assign((size_t)ns * std::max(n, 1), 0);
    bool ok = true;
    auto dn = [&](void *dst, const void *src, size_t b) {
        if (ok && b) ok = cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToHost, S->st) == cudaSuccess;
    };
    for (int k = 0; k < ns; ++k) {
        const Slot &s = S->h_slots[(size_t)R.rslot * ns + k];
        dn(&R.energies[(size_t)k * P * Smax], s.rec_e, 8 * (size_t)P * Smax);
        dn(&R.counts[(size_t)k * P], s.rec_count, 4 * (size_t)P);
        dn(&R.nfree[(size_t)k * P], s.rec_nfree, 4 * (size_t)P);
        dn(&R.best_e[k], s.best_e, 8);
        dn(&R.fixed[(size_t)k * n], s.fmap, (size_t)n);
        dn(&R.best_state[(size_t)k * n], s.best_state, (size_t)n);
    }
    if (ok) ok = cudaStreamSynchronize(S->st) == cudaSuccess;
    return ok ? SPVAR_OK : SPVAR_ECUDA;
}

int64_t request_attempts(const spvar_server *S, const Request &R)
{
    int64_t a = 0;
    // SQA: every Trotter slice of every run is swept
    const int64_t per = (int64_t)S->cfg.params.num_sweeps *
                        (S->cfg.params.sampler == SPVAR_SAMPLER_SQA ? S->cfg.params.sqa_slices : 1);
    for (size_t i = 0; i < R.counts.size(); ++i) a += (int64_t)R.counts[i] * R.nfree[i] * per;
    return a;
}

// One engine iteration: admit, run one phase for everything in flight, retire.
int server_step(spvar_server *S, int32_t *active_out)
{
    // admission (arrival order): reserve a request slot and an arena range under
    // the lock, then upload without it so that submit, wait and stats never wait
    // for a copy
    std::vector<Request *> admitted;
    {
        std::lock_guard<std::mutex> g(S->mu);
        while (!S->queue.empty()) {
            Request &R = *S->reqs[S->queue.front()];
            int rs = -1;
            for (size_t r = 0; r < S->rslot_owner.size(); ++r)
                if (S->rslot_owner[r] < 0) { rs = (int)r; break; }
            if (rs < 0) break;
            size_t off;
            if (!S->arena.alloc(R.bytes, &off)) break;
            R.off = off;
            R.rslot = rs;
            S->rslot_owner[rs] = R.id;
            S->queue.pop_front();
            admitted.push_back(&R);
        }
    }
    for (size_t a = 0; a < admitted.size(); ++a) {
        Request &R = *admitted[a];
        const int rc = place_request(S, R);
        std::lock_guard<std::mutex> g(S->mu);
        if (rc) {
            // give back what this and the later admissions reserved; they queue again in order
            for (size_t b = admitted.size(); b-- > a;) {
                Request &Q = *admitted[b];
                S->arena.release(Q.off, Q.bytes);
                S->rslot_owner[Q.rslot] = -1;
                Q.rslot = -1;
                S->queue.push_front(Q.id);
            }
            return rc;
        }
        R.state = 1;
        R.t_admit = now_s();
    }
    int active = 0;
    for (int64_t o : S->rslot_owner) active += (o >= 0);
    if (active_out) *active_out = active;
    if (!active) return SPVAR_OK;
    // the smallest size tier that holds every problem in flight
    int maxn = 0;
    {
        std::lock_guard<std::mutex> g(S->mu);
        for (int64_t o : S->rslot_owner)
            if (o >= 0) maxn = std::max(maxn, S->reqs[o]->hp.hdr.n);
    }
    const spvar_server::Tier *tier = &S->tiers.back();
    for (const spvar_server::Tier &t : S->tiers)
        if (t.max_n >= maxn) { tier = &t; break; }
    if (tier->graph) {
        SPVAR_CUDA_TRY(cudaGraphLaunch(tier->graph, S->st));
    } else {
        SPVAR_CUDA_TRY(engine_phase(tier->E, S->d_slots, S->nslots, S->cfg.params.num_sweeps, tier->grid, S->st,
                                    false, false));
    }
    SPVAR_CUDA_TRY(launch_gather_modes(S->d_slots, S->nslots, S->d_modes, S->st));
    SPVAR_CUDA_TRY(cudaMemcpyAsync(S->h_modes, S->d_modes, 4 * (size_t)S->nslots, cudaMemcpyDeviceToHost, S->st));
    SPVAR_CUDA_TRY(cudaStreamSynchronize(S->st));
    if (S->ev[0]) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, S->ev[0], S->ev[1]) == cudaSuccess) {
            std::lock_guard<std::mutex> g(S->mu);
            S->sweep_ms += ms;
            S->sweep_launches += 1;
        }
        cudaGetLastError();
    }
    // retirement
    std::vector<int64_t> finished;
    for (size_t r = 0; r < S->rslot_owner.size(); ++r) {
        if (S->rslot_owner[r] < 0) continue;
        bool done = true;
        for (int k = 0; k < S->ns; ++k) done &= S->h_modes[r * S->ns + k] == kDone;
        if (done) finished.push_back(S->rslot_owner[r]);
    }
    for (int64_t id : finished) {
        Request *R;
        {
            std::lock_guard<std::mutex> g(S->mu);
            R = S->reqs[id].get();
        }
        int rc = retire_request(S, *R);
        if (rc) return rc;
        std::lock_guard<std::mutex> g(S->mu);
        S->arena.release(R->off, R->bytes);
        S->rslot_owner[R->rslot] = -1;
        R->state = 2;
        R->t_done = now_s();
        S->attempts_done += request_attempts(S, *R);
        S->requests_done += 1;
        active -= 1;
    }
    if (!finished.empty()) S->cv.notify_all();
    if (active_out) *active_out = active;
    return SPVAR_OK;
}

void worker_loop(spvar_server *S)
{
    cudaSetDevice(S->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            bool idle = S->queue.empty();
            for (int64_t o : S->rslot_owner) idle &= (o < 0);
            if (S->stop) return;
            if (idle) {
                S->cv.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
        }
        if (server_step(S, nullptr) != SPVAR_OK) {
            std::lock_guard<std::mutex> g(S->mu);
            S->failed = true;
            S->stop = true;
            S->cv.notify_all();
            return;
        }
    }
}

void server_free(spvar_server *S)
{
    if (!S) return;
    for (spvar_server::Tier &t : S->tiers)
        if (t.graph) cudaGraphExecDestroy(t.graph);
    if (S->cap_st) cudaStreamDestroy(S->cap_st);
    for (cudaEvent_t e : S->ev)
        if (e) cudaEventDestroy(e);
    if (S->st) cudaStreamDestroy(S->st);
    if (S->arena_mem) cudaFree(S->arena_mem);
    if (S->fixed_mem) cudaFree(S->fixed_mem);
    if (S->h_modes) cudaFreeHost(S->h_modes);
    delete S;
}

}  // namespace

extern "C" {

int spvar_server_create(const spvar_server_config *cfg, spvar_server **out)
{
    if (!out || !cfg) return SPVAR_EINVAL;
    *out = nullptr;
    const spvar_params &p = cfg->params;
    if (p.num_starts < 1 || p.fixing_sample_size < 1 || p.solving_sample_size < 0 || p.num_sweeps < 0 ||
        p.max_fix_phases < 1 || p.fix_num <= 0 || p.fix_den <= 0 || p.fix_num > p.fix_den ||
        !(p.elite_threshold > 0.0) || !(p.elite_threshold <= 1.0) || !(p.beta0 > 0.0) || !(p.beta1 > 0.0) ||
        p.canon < -1 || p.canon > 1 || p.start_offset < 0 || p.component_boost < 0 || p.component_boost > 1 || p.tree_preprocess < 0 || p.tree_preprocess > 1 || cfg->max_n < 1 || cfg->max_nnz < 0 ||
        cfg->max_degree < 1 || cfg->max_dmax < 0 || cfg->energy_scale < 1 || cfg->max_requests < 1 ||
        cfg->budget_bytes == 0 || check_corr_params(p) != SPVAR_OK || check_sampler_params(p) != SPVAR_OK ||
        cfg->sweeps_per_step < 0 || (p.sampler == SPVAR_SAMPLER_SQA && cfg->sweeps_per_step > 0) ||
        p.sampler == SPVAR_SAMPLER_PTICM)
        return SPVAR_EINVAL;
    const int Smax = std::max(std::max(p.fixing_sample_size, p.solving_sample_size), p.corr_sample_size);
    if (cfg->max_n > SPVAR_MAX_N || cfg->max_degree > SPVAR_MAX_DEGREE || Smax > SPVAR_MAX_SAMPLES ||
        p.num_sweeps > SPVAR_MAX_SWEEPS || p.max_fix_phases + 2 > SPVAR_MAX_PHASE)
        return SPVAR_ELIMIT;
    spvar_server *S = new (std::nothrow) spvar_server();
    if (!S) return SPVAR_ENOMEM;
    S->cfg = *cfg;
    cudaGetDevice(&S->device);
    cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->device);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, S->device);
    S->ns = p.num_starts;
    S->P = p.max_fix_phases + 1 + (p.corr_sample_size > 0 ? 1 : 0);
    S->Smax = Smax;
    S->nslots = cfg->max_requests * S->ns;
    if (cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
        server_free(S);
        return SPVAR_ECUDA;
    }
    // fixed structures: slot table, jobs, work items, counters, modes, table
    const int T = p.num_sweeps, stride = cfg->max_dmax + 1;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off += a256(b); return o; };
    const size_t o_slots = take(sizeof(Slot) * S->nslots);
    const size_t o_jobs = take(sizeof(SweepJob) * S->nslots);
    const size_t o_items = take(sizeof(WorkItem) * (size_t)S->nslots * ceil_div(Smax, 4));
    const size_t o_ctr = take(16);
    const size_t o_modes = take(4 * (size_t)S->nslots);
    const size_t o_thr = take(4 * (size_t)std::max(T, 1) * stride);
    // SQA: acceptance entries [T][3][W] of the path-integral sweep
    const bool sqa = p.sampler == SPVAR_SAMPLER_SQA;
    const int sqa_W = 2 * (cfg->max_dmax / 2) + 1;
    const size_t o_ent = take(sqa ? 8 * (size_t)std::max(T, 1) * 3 * sqa_W : 0);
    if (cudaMalloc(&S->fixed_mem, off) != cudaSuccess || cudaMalloc(&S->arena_mem, cfg->budget_bytes) != cudaSuccess ||
        cudaMallocHost(&S->h_modes, 4 * (size_t)S->nslots) != cudaSuccess) {
        cudaGetLastError();
        server_free(S);
        return SPVAR_ENOMEM;
    }
    S->arena.reset(cfg->budget_bytes);
    char *w = static_cast<char *>(S->fixed_mem);
    S->d_slots = (Slot *)(w + o_slots);
    S->d_modes = (int32_t *)(w + o_modes);
    std::vector<double> beta(std::max(T, 1));
    std::vector<uint32_t> thr((size_t)std::max(T, 1) * stride, 0u);
    if (T > 0) {
        spvar_beta_geometric(T, p.beta0, p.beta1, beta.data());
        spvar_thresholds(T, beta.data(), cfg->max_dmax, cfg->energy_scale, thr.data());
    }
    std::vector<uint64_t> ent;
    if (sqa) {
        // constant beta, transverse field linear from gamma0 to gamma1 (as the plans)
        ent.assign((size_t)std::max(T, 1) * 3 * sqa_W, 0ull);
        std::vector<double> sb(std::max(T, 1), p.sqa_beta), sg(std::max(T, 1));
        if (T > 0) {
            spvar_gamma_linear(T, p.sqa_gamma0, p.sqa_gamma1, sg.data());
            spvar_sqa_table(T, p.sqa_slices, sb.data(), sg.data(), cfg->max_dmax, cfg->energy_scale, ent.data());
        }
    }
    // every slot starts free (done): the phase kernels skip it
    S->h_slots.assign(S->nslots, Slot());
    for (Slot &s : S->h_slots) {
        std::memset(&s, 0, sizeof(Slot));
        s.mode = kDone;
    }
    S->rslot_owner.assign(cfg->max_requests, -1);
    bool ok = cudaMemcpyAsync(w + o_thr, thr.data(), 4 * thr.size(), cudaMemcpyHostToDevice, S->st) == cudaSuccess &&
              (!sqa ||
               cudaMemcpyAsync(w + o_ent, ent.data(), 8 * ent.size(), cudaMemcpyHostToDevice, S->st) == cudaSuccess) &&
              cudaMemcpyAsync(S->d_slots, S->h_slots.data(), sizeof(Slot) * S->nslots, cudaMemcpyHostToDevice,
                              S->st) == cudaSuccess &&
              cudaStreamSynchronize(S->st) == cudaSuccess;
    if (!ok) { server_free(S); return SPVAR_ECUDA; }

    // engine: consts and sweep shape (general kernel; layout staged in shared memory when it fits)
    PhaseEngine &E = S->E;
    fill_solve_consts(p, E.C);
    E.C.nslots = S->nslots;
    E.C.max_n0 = cfg->max_n;
    int Q = p.replicas_per_block > 0 ? p.replicas_per_block / 4 : 1;
    const int blk = p.sweep_block ? p.sweep_block : 512;
    E.shape = SweepShape{0, blk, Q, 1, 0, 0};
    if (sweep_shape_smem(E.shape, cfg->max_n, stride, cfg->max_degree) > (size_t)optin) E.shape.stage = 0;
    // +-1-only servers: the streaming +-1 kernel (one quad per CTA, per-spin data
    // staged once per CTA), or with SPVAR_SWEEP_PM1Q the quad-group +-1 kernel
    // (work items of Q quads of the largest admissible problem, more quads of
    // smaller ones).  Measured at a request's 20 starts x 250 samples of 3D +-J
    // problems, the streaming kernel leads at every size (L = 8: 3.3e11 against
    // 2.7e11 attempts/s; L = 12: 6.3e11 against 4.8e11; L = 20: 6.9e11 against
    // 4.0e11): the quad-group kernel pays off only when a problem has hundreds of
    // quads to group.
    const int md = cfg->max_degree <= 6 ? 6 : 8;
    const bool pm1_only = p.sweep_kernel == SPVAR_SWEEP_PM1 || p.sweep_kernel == SPVAR_SWEEP_PM1S ||
                          p.sweep_kernel == SPVAR_SWEEP_PM1Q;
    const bool want_quads = p.sweep_kernel == SPVAR_SWEEP_PM1Q;
    bool chosen = false;
    if (pm1_only && want_quads && cfg->max_degree <= 8 && cfg->max_dmax <= 30) {
        const int qb = (p.sweep_block == 128 || p.sweep_block == 256) ? p.sweep_block : 512;
        SweepShape sh{6, qb, Q, 0, 0, md};
        if (pm1q_shape_ok(qb, md, cfg->max_n, Q) && sweep_shape_smem(sh, cfg->max_n, stride, cfg->max_degree) <= (size_t)optin) {
            E.shape = sh;
            chosen = true;
        }
    }
    if (!chosen && pm1_only && cfg->max_degree <= 8 && cfg->max_dmax <= 254 && pm1s_shape_ok(blk, md, cfg->max_n, 1)) {
        SweepShape sh{2, blk, 1, 0, 0, md};
        if (sweep_shape_smem(sh, cfg->max_n, stride, cfg->max_degree) <= (size_t)optin) {
            E.shape = sh;
            Q = 1;
        }
    }
    if (sqa) {
        // SQA: one quad (four runs, all slices in shared memory) per CTA, the item walk
        // over (slice, spin) (any problem that fits, +-1 or general couplers)
        const int sb = (p.sweep_block == 128 || p.sweep_block == 256 || p.sweep_block == 512) ? p.sweep_block : 256;
        SweepShape sh{5, sb, 1, pm1_only ? 1 : 0, sqa_W, cfg->max_degree};
        sh.slices = p.sqa_slices;
        if (!sqa_shape_ok(sh.stage, sb, cfg->max_n, cfg->max_degree, p.sqa_slices, sqa_W, 0) ||
            sweep_shape_smem(sh, cfg->max_n, stride, cfg->max_degree) > (size_t)optin) {
            server_free(S);
            return SPVAR_ELIMIT;
        }
        E.shape = sh;
        E.ent = (const unsigned long long *)(w + o_ent);
        E.P = p.sqa_slices;
        E.W = sqa_W;
    }
    E.C.Q = E.shape.Q;
    E.C.chunk = (cfg->sweeps_per_step > 0 && cfg->sweeps_per_step < T) ? cfg->sweeps_per_step : 0;
    E.sweep_smem = sweep_shape_smem(E.shape, cfg->max_n, stride, cfg->max_degree);
    if (E.sweep_smem > (size_t)optin) { server_free(S); return SPVAR_ELIMIT; }
    // +-1-only servers use the byte-wise local field; otherwise general couplers
    E.pm1 = pm1_only;
    E.max_n0 = cfg->max_n;
    E.max_deg = cfg->max_degree;
    E.thr_stride = stride;
    E.thr = (const uint32_t *)(w + o_thr);
    E.jobs = (SweepJob *)(w + o_jobs);
    E.items = (WorkItem *)(w + o_items);
    E.ctr = (int32_t *)(w + o_ctr);
    // events around the sweep launch of every step (the serving roofline's kernel time)
    if (cudaEventCreate(&S->ev[0]) != cudaSuccess || cudaEventCreate(&S->ev[1]) != cudaSuccess) {
        cudaGetLastError();
        for (cudaEvent_t &e : S->ev) {
            if (e) cudaEventDestroy(e);
            e = nullptr;
        }
    }
    E.ev_sweep[0] = S->ev[0];
    E.ev_sweep[1] = S->ev[1];
    E.ev_post = nullptr;
    // size tiers, smallest first; each captures one phase step over the whole slot table
    for (int k = 3; k >= 0; --k) {
        const int tn = cfg->max_n >> k;
        if (k > 0 && (tn < 256 || (!S->tiers.empty() && S->tiers.back().max_n == tn))) continue;
        spvar_server::Tier t;
        t.max_n = tn;
        t.E = E;
        t.E.max_n0 = tn;
        t.E.C.max_n0 = tn;
        t.E.sweep_smem = sweep_shape_smem(E.shape, tn, stride, cfg->max_degree);
        const int occ = std::max(1, sweep_shape_occupancy(t.E.shape, t.E.pm1, t.E.sweep_smem));
        t.grid = occ * S->sms;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(S->cap_st, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
            cudaError_t e = engine_phase(t.E, S->d_slots, S->nslots, T, t.grid, S->cap_st, false, true);
            cudaError_t e2 = cudaStreamEndCapture(S->cap_st, &g);
            if (e == cudaSuccess && e2 == cudaSuccess && g && cudaGraphInstantiate(&t.graph, g, 0) != cudaSuccess)
                t.graph = nullptr;
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
        S->tiers.push_back(t);
    }
    *out = S;
    return SPVAR_OK;
}

int spvar_server_submit(spvar_server *S, int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *val,
                        const int32_t *h, int64_t offset, uint64_t seed, int64_t *id)
{
    if (!S || !id) return SPVAR_EINVAL;
    std::unique_ptr<Request> R(new (std::nothrow) Request());
    if (!R) return SPVAR_ENOMEM;
    int rc = host_problem_build(n, row_ptr, col, val, h, offset, S->cfg.energy_scale, R->hp);
    if (rc) return rc;
    const DevProb &H = R->hp.hdr;
    if (S->E.pm1 && !H.pm1) return SPVAR_EINVAL;
    if (H.n > S->cfg.max_n || H.nnz > S->cfg.max_nnz || H.maxdeg > S->cfg.max_degree || H.dmax > S->cfg.max_dmax)
        return SPVAR_ELIMIT;
    R->bytes = request_bytes(S, R->hp);
    if (R->bytes > S->cfg.budget_bytes) return SPVAR_EBUDGET;
    R->seed = seed;
    R->t_submit = now_s();
    std::lock_guard<std::mutex> g(S->mu);
    R->id = S->next_id++;
    *id = R->id;
    S->queue.push_back(R->id);
    S->reqs[R->id] = std::move(R);
    S->cv.notify_all();
    return SPVAR_OK;
}

int spvar_server_step(spvar_server *S, int32_t *active)
{
    if (!S) return SPVAR_EINVAL;
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->running) return SPVAR_EINVAL;  // the background engine owns the loop
    }
    return server_step(S, active);
}

int spvar_server_start(spvar_server *S)
{
    if (!S) return SPVAR_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    if (S->running) return SPVAR_OK;
    S->stop = false;
    S->failed = false;
    S->running = true;
    S->worker = std::thread(worker_loop, S);
    return SPVAR_OK;
}

int spvar_server_stop(spvar_server *S)
{
    if (!S) return SPVAR_EINVAL;
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (!S->running) return SPVAR_OK;
        S->stop = true;
        S->cv.notify_all();
    }
    S->worker.join();
    std::lock_guard<std::mutex> g(S->mu);
    S->running = false;
    return SPVAR_OK;
}

int spvar_server_wait(spvar_server *S, int64_t id, double timeout_s, spvar_request_info *info)
{
    if (!S) return SPVAR_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return SPVAR_EINVAL;
    Request &R = *it->second;
    if (timeout_s > 0 && R.state != 2) {
        const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
        S->cv.wait_until(lk, until, [&] { return R.state == 2 || S->stop || S->failed; });
    }
    if (info) {
        info->state = R.state;
        info->n = R.hp.hdr.n;
        info->best_energy = R.state == 2 ? *std::min_element(R.best_e.begin(), R.best_e.end()) : 0;
        info->latency_s = R.state == 2 ? R.t_done - R.t_submit : -1.0;
        info->queue_s = R.state >= 1 ? R.t_admit - R.t_submit : -1.0;
        info->attempts = R.state == 2 ? request_attempts(S, R) : 0;
    }
    // an engine error fails every wait; a clean stop leaves unfinished requests timed out
    if (R.state != 2) return S->failed ? SPVAR_ECUDA : SPVAR_ETIMEOUT;
    return SPVAR_OK;
}

int spvar_server_result(spvar_server *S, int64_t id, int64_t *best_energy, int8_t *best_state, int8_t *fixed,
                        int64_t *energies, int32_t *counts, int32_t *nfree)
{
    if (!S) return SPVAR_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end() || it->second->state != 2) return SPVAR_EINVAL;
    const Request &R = *it->second;
    auto cp = [](void *dst, const void *src, size_t b) { if (dst && b) std::memcpy(dst, src, b); };
    cp(best_energy, R.best_e.data(), 8 * R.best_e.size());
    cp(best_state, R.best_state.data(), (size_t)S->ns * R.hp.hdr.n);
    cp(fixed, R.fixed.data(), (size_t)S->ns * R.hp.hdr.n);
    cp(energies, R.energies.data(), 8 * R.energies.size());
    cp(counts, R.counts.data(), 4 * R.counts.size());
    cp(nfree, R.nfree.data(), 4 * R.nfree.size());
    return SPVAR_OK;
}

int spvar_server_release(spvar_server *S, int64_t id)
{
    if (!S) return SPVAR_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end() || it->second->state != 2) return SPVAR_EINVAL;
    S->reqs.erase(it);
    return SPVAR_OK;
}

int spvar_server_sweep_time(spvar_server *S, double *total_ms, int64_t *launches)
{
    if (!S) return SPVAR_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    if (total_ms) *total_ms = S->sweep_ms;
    if (launches) *launches = S->sweep_launches;
    return SPVAR_OK;
}

int spvar_server_stats(spvar_server *S, int64_t *requests_done, int64_t *attempts_done, int32_t *queued,
                       int32_t *running)
{
    if (!S) return SPVAR_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    if (requests_done) *requests_done = S->requests_done;
    if (attempts_done) *attempts_done = S->attempts_done;
    if (queued) *queued = (int32_t)S->queue.size();
    if (running) {
        int a = 0;
        for (int64_t o : S->rslot_owner) a += (o >= 0);
        *running = a;
    }
    return SPVAR_OK;
}

void spvar_server_destroy(spvar_server *S)
{
    if (!S) return;
    spvar_server_stop(S);
    server_free(S);
}

}  // extern "C"
