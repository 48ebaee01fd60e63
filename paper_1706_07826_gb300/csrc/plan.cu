// Multi-start SPVAR driver (Alg. 2; ISPVAR when iterate is set).
//
// A plan owns one device workspace for every start of every problem
// ("slots"): two problem buffers of the original capacity for the reductions,
// the sample buffer, the recorded energies and the fix maps.  One phase of all
// slots is five launches -- plan (work list), persistent sweep, elite,
// count/fix, fold/compact -- captured once into a CUDA graph and replayed;
// control (which starts still fix, solve or are done, how large each reduced
// problem is) stays on the device.  The plain form runs the same kernels one
// start at a time without the graph, which is the comparison baseline.
// A small autotuner times the sweep on the plan's own first phase for a few
// (block, quads-per-CTA, staging) shapes; every shape gives bit-identical
// results because randomness is keyed by logical coordinates only.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <list>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "spvar_internal.h"

using namespace spvar;

namespace spvar {

cudaError_t engine_phase(const PhaseEngine &E, Slot *slots, int nslots, int T, int grid, cudaStream_t st,
                         bool count_active, bool capturing)
{
    // inside stream capture an event record only becomes a graph node when external
    auto record = [&](cudaEvent_t ev) {
        return capturing ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal) : cudaEventRecord(ev, st);
    };
    SolveConsts C = E.C;
    C.nslots = nslots;
    C.Q = E.shape.Q;
    C.fit_block = E.shape.kind == 1 ? E.shape.block : 0;
    C.fit_nslot = E.shape.kind == 1 ? E.shape.nslot : 0;
    C.fit_words = E.shape.kind == 6 ? 2 * E.shape.Q * (E.max_n0 + 1) : 0;
    C.grid = grid;
    C.T = T;
    cudaError_t e = launch_plan(slots, C, E.jobs, E.items, E.ctr + 0, E.ctr + 1, E.ctr + 2, st);
    if (e != cudaSuccess) return e;
    SweepLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.jobs = E.jobs;
    L.items = E.items;
    L.nitems = E.ctr + 0;
    L.queue = E.ctr + 1;
    L.thr = E.thr;
    L.thr_stride = E.thr_stride;
    L.T = T;
    L.Q = E.shape.Q;
    L.stage_ell = E.shape.stage;
    L.max_n = E.max_n0;
    L.max_deg = E.max_deg;
    L.ent = E.ent;
    L.P = E.P;
    L.W = E.W;
    if (E.ev_sweep[0] && (e = record(E.ev_sweep[0])) != cudaSuccess) return e;
    // the sampler: persistent sweep launch over the work items, or one PTICM run per start
    e = E.pt_R > 0 ? launch_pticm_slots(slots, nslots, C.Smax, E.pt_thr, E.thr_stride, E.pt_xthr, E.pt_dx, E.pt_R, T,
                                        E.pt_K, E.pt_smem, st)
                   : launch_sweep_shape(L, E.shape, E.pm1, grid, E.sweep_smem, st);
    if (e != cudaSuccess) return e;
    if (E.ev_sweep[1] && (e = record(E.ev_sweep[1])) != cudaSuccess) return e;
    if ((e = launch_boost(slots, C, st)) != cudaSuccess) return e;
    int32_t *nactive = count_active ? E.ctr + 2 : nullptr;
    if (C.tree) {
        // one CTA per start for each step, the tree step after the fold/compact
        if ((e = launch_elite_slots(slots, C, st)) != cudaSuccess) return e;
        if ((e = launch_count_slots(slots, C, E.max_n0, st)) != cudaSuccess) return e;
        e = launch_reduce_slots(slots, C, nactive, st);
    } else {
        // the whole pass in one launch, one thread-block cluster per start
        e = launch_pass_slots(slots, C, nactive, st);
    }
    if (e != cudaSuccess) return e;
    // end of the persistence pass (boosting, elite, counts and fixing, fold/compact)
    if (E.ev_post && (e = record(E.ev_post)) != cudaSuccess) return e;
    return cudaSuccess;
}

}  // namespace spvar

struct spvar_plan {
    int device = 0;
    std::vector<const Problem *> probs;
    std::vector<int> starts_of;  // slot -> problem
    spvar_params prm{};
    SolveConsts C{};
    int T = 0, thr_stride = 1, max_n0 = 0, max_deg = 1, iters_max = 1;
    int ncol_max = 0, class_max = 0;  // most colour classes and largest class of any problem
    int jabs_max = 0;                 // largest coupler magnitude of any problem
    bool pm1 = true;
    bool ujs = true;      // every problem has one coupler magnitude per spin
    uint64_t sig = 0;     // structure signature of the problems (autotune cache key)
    void *ws = nullptr;
    size_t ws_bytes = 0;
    Slot *d_slots = nullptr;
    std::vector<Slot> h_slots;
    Slot *h_slots_pinned = nullptr;
    uint32_t *d_thr = nullptr;
    unsigned long long *d_ent = nullptr;  // SQA acceptance entries
    int sqa_P = 0, sqa_W = 0;             // SQA slices and table width (0: SA)
    // PTICM as the sampler: temperatures, kept states per list, exchange-table width, tables
    int pt_R = 0, pt_K = 0, pt_dx = 0;
    uint32_t *d_pt_thr = nullptr, *d_pt_xthr = nullptr;
    size_t pt_smem = 0;
    bool sqa_ent32 = false;               // SQA: no acceptance entry is 2^32 (32-bit entries suffice)
    SweepJob *d_jobs = nullptr;
    WorkItem *d_items = nullptr;
    int32_t *d_ctr = nullptr;       // [0] nitems, [1] queue, [2] nactive, [3] phases run by the loop graph
    int32_t *h_nactive = nullptr;   // pinned
    int64_t *d_rec_e = nullptr;
    int32_t *d_rec_count = nullptr, *d_rec_nfree = nullptr, *d_nphases = nullptr;
    int64_t *d_best_e = nullptr;
    int8_t *d_fmap = nullptr, *d_best = nullptr;
    size_t fmap_total = 0;
    SweepShape shape{0, 256, 1, 0, 0, 0};
    int sweep_grid = 1, sms = 1, dmax = 0;
    size_t sweep_smem = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;       // one batched phase
    cudaGraphExec_t graph_loop = nullptr;  // every phase of a run: a device-side while loop over `graph`'s body
    cudaEvent_t ev_sweep[2] = {nullptr, nullptr};  // recorded around every sweep launch
    cudaEvent_t ev_post = nullptr;                 // end of each phase's persistence pass
    double post_ms = 0.0;
    int profiling = 0;
    double sweep_ms = 0.0;
    int32_t sweep_launches = 0;
};

namespace {

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct TuneKey {
    int max_n, max_deg, pm1, S, nslots, form, thr_stride, sqa_P;
    uint64_t sig;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(max_n, max_deg, pm1, S, nslots, form, thr_stride, sqa_P, sig) <
               std::tie(o.max_n, o.max_deg, o.pm1, o.S, o.nslots, o.form, o.thr_stride, o.sqa_P, o.sig);
    }
};
std::map<TuneKey, SweepShape> g_tune_cache;
std::mutex g_tune_mu;

void plan_free(spvar_plan *pl);

// Plans spvar_solve keeps between calls, most recent first.  A plan depends on
// its problem only through the fields in solve_key (sizes, capacities, colour
// classes, coupler kind, dmax and scale decide its workspace, tables and
// sweep shape); the problem's own data is read on the device through the
// starts' problem pointers, which are rebound before each run.  A plan is
// taken out of the cache while it runs, so concurrent calls never share one.
constexpr size_t kSolveCacheMax = 4;
constexpr size_t kSolveCacheBytes = size_t(256) << 20;  // larger workspaces are freed after the call
std::list<std::pair<std::vector<int64_t>, spvar_plan *>> g_solve_cache;
std::mutex g_solve_mu;

void solve_key(const Problem *P, const spvar_params &prm, std::vector<int64_t> &key)
{
    int dev = 0;
    cudaGetDevice(&dev);
    const DevProb &H = P->hdr;
    key = {dev, H.n, H.nnz, H.cap_n, H.cap_nnz, H.maxdeg, H.dmax, H.scale, H.ncol, H.pm1, H.ujs, H.hzero,
           P->jabs_max};
    for (int c = 0; c < H.ncol && c < kMaxColours; ++c) key.push_back(P->csize[c]);
    // the parameters bytewise (padding included: a mismatch there only misses the cache)
    unsigned char raw[sizeof(spvar_params)];
    std::memcpy(raw, &prm, sizeof(prm));
    for (size_t i = 0; i < sizeof(raw); i += 8) {
        int64_t w = 0;
        std::memcpy(&w, raw + i, std::min<size_t>(8, sizeof(raw) - i));
        key.push_back(w);
    }
}

spvar_plan *solve_cache_take(const std::vector<int64_t> &key)
{
    std::lock_guard<std::mutex> g(g_solve_mu);
    for (auto it = g_solve_cache.begin(); it != g_solve_cache.end(); ++it)
        if (it->first == key) {
            spvar_plan *pl = it->second;
            g_solve_cache.erase(it);
            return pl;
        }
    return nullptr;
}

void solve_cache_put(std::vector<int64_t> key, spvar_plan *pl)
{
    if (pl->ws_bytes > kSolveCacheBytes) {
        plan_free(pl);
        return;
    }
    spvar_plan *evict = nullptr;
    {
        std::lock_guard<std::mutex> g(g_solve_mu);
        g_solve_cache.emplace_front(std::move(key), pl);
        if (g_solve_cache.size() > kSolveCacheMax) {
            evict = g_solve_cache.back().second;
            g_solve_cache.pop_back();
        }
    }
    if (evict) plan_free(evict);
}

int grid_for(const spvar_plan *pl, int items)
{
    const int occ = std::max(1, sweep_shape_occupancy(pl->shape, pl->pm1, pl->sweep_smem));
    const int full = occ * pl->sms;
    if (!pl->shape.balance || items <= full) return std::max(1, std::min(items, full));
    return ceil_div(items, ceil_div(items, full));
}

PhaseEngine engine_of(const spvar_plan *pl)
{
    PhaseEngine E;
    E.shape = pl->shape;
    E.sweep_smem = pl->sweep_smem;
    E.pm1 = pl->pm1;
    E.max_n0 = pl->max_n0;
    E.max_deg = pl->max_deg;
    E.thr_stride = pl->thr_stride;
    E.thr = pl->d_thr;
    E.ent = pl->d_ent;
    E.P = pl->sqa_P;
    E.W = pl->sqa_W;
    E.jobs = pl->d_jobs;
    E.items = pl->d_items;
    E.ctr = pl->d_ctr;
    E.ev_sweep[0] = pl->ev_sweep[0];
    E.ev_sweep[1] = pl->ev_sweep[1];
    E.ev_post = pl->ev_post;
    E.C = pl->C;
    E.pt_R = pl->pt_R;
    E.pt_K = pl->pt_K;
    E.pt_dx = pl->pt_dx;
    E.pt_thr = pl->d_pt_thr;
    E.pt_xthr = pl->d_pt_xthr;
    E.pt_smem = pl->pt_smem;
    return E;
}

// One phase of the given slots (all of them in the batched form).  timed =
// false leaves out the event records (a conditional graph body takes none).
cudaError_t launch_phase(spvar_plan *pl, Slot *slots, int nslots, int T, int grid, cudaStream_t st,
                         bool count_active, bool capturing = false, bool timed = true)
{
    PhaseEngine E = engine_of(pl);
    if (!timed) E.ev_sweep[0] = E.ev_sweep[1] = E.ev_post = nullptr;
    return engine_phase(E, slots, nslots, T, grid, st, count_active, capturing);
}

// Sweep launches of a whole run: every phase takes launches_per_phase launches.
int plan_steps(const spvar_plan *pl) { return pl->iters_max * launches_per_phase(pl->T, pl->C.chunk); }

// Loop condition of the whole-run graph: run another phase while phases
// remain and (ISPVAR) some start is still active.
__global__ void k_loop_cond(cudaGraphConditionalHandle h, int32_t *ctr, int iters_max, int iterate)
{
    const int it = ++ctr[3];
    const bool more = it < iters_max && (!iterate || ctr[2] > 0);
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

// Captures every phase of a batched run as one graph: a conditional while
// node whose body is one phase followed by k_loop_cond, so the whole Alg. 2
// loop (ISPVAR included) runs without the host.  Returns false if the graph
// could not be built (the per-phase graph is used then).
bool build_loop_graph(spvar_plan *pl, int nslots)
{
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return false;
    bool ok = true;
    cudaGraphConditionalHandle h;
    ok = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (ok) ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
    if (ok) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        ok = cudaStreamBeginCaptureToGraph(pl->cap_stream, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeRelaxed) == cudaSuccess;
        if (ok) {
            cudaError_t e = launch_phase(pl, pl->d_slots, nslots, pl->T, pl->sweep_grid, pl->cap_stream, true, true,
                                         false);
            if (e == cudaSuccess) {
                k_loop_cond<<<1, 1, 0, pl->cap_stream>>>(h, pl->d_ctr, plan_steps(pl), pl->prm.iterate ? 1 : 0);
                e = cudaGetLastError();
            }
            cudaGraph_t out = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(pl->cap_stream, &out);
            ok = e == cudaSuccess && e2 == cudaSuccess;
        }
    }
    if (ok) ok = cudaGraphInstantiate(&pl->graph_loop, g, 0) == cudaSuccess;
    if (!ok) pl->graph_loop = nullptr;
    cudaGraphDestroy(g);
    cudaGetLastError();
    return ok;
}

int upload_slots(spvar_plan *pl, const uint64_t *seeds, cudaStream_t st)
{
    for (size_t s = 0; s < pl->h_slots.size(); ++s) {
        Slot x = pl->h_slots[s];
        x.seed = seeds ? seeds[pl->starts_of[s]] : 0;
        pl->h_slots_pinned[s] = x;
    }
    SPVAR_CUDA_TRY(cudaMemcpyAsync(pl->d_slots, pl->h_slots_pinned, sizeof(Slot) * pl->h_slots.size(),
                                   cudaMemcpyHostToDevice, st));
    return SPVAR_OK;
}

// Register-kernel slot count covering every problem of the plan (0 if none).
int plan_nslot(const spvar_plan *pl, int Q, int block)
{
    int ns = 2;
    for (const Problem *P : pl->probs) {
        const int x = pm1_nslot(P, Q, block);
        if (x == 0) return 0;
        ns = std::max(ns, x);
    }
    return ns;
}

// Candidate sweep shapes for a plan: the general kernel with and without the
// staged layout, and (for +-1 problems) the register-resident kernel.
// SQA sweep shape of a variant (0 general, 1 +-1 walk, 2 +-1 register form)
// and block size, or kind -1 if it does not apply or the slices do not fit.
SweepShape sqa_shape(const spvar_plan *pl, int block, int optin, int variant)
{
    SweepShape sh{5, block, 1, variant, pl->sqa_W, pl->max_deg};
    sh.slices = pl->sqa_P;
    sh.ncls = variant >= 2 ? sqa_reg_ncls(pl->ncol_max, pl->class_max, block, pl->sqa_P) : 0;
    sh.ent32 = variant >= 2 && pl->sqa_ent32 ? 1 : 0;
    const bool kind_ok = variant == 0 || (variant == 3 ? sqa_si_eligible(pl->jabs_max, pl->dmax, pl->max_deg)
                                                       : pl->pm1);
    const bool ok = kind_ok && (variant < 2 || sh.ncls > 0) &&
                    sqa_shape_ok(variant, block, pl->max_n0, pl->max_deg, pl->sqa_P, pl->sqa_W, sh.ncls) &&
                    sweep_shape_smem(sh, pl->max_n0, pl->thr_stride, pl->max_deg) <= (size_t)optin;
    if (!ok) sh.kind = -1;
    return sh;
}

std::vector<SweepShape> candidate_shapes(const spvar_plan *pl, int optin)
{
    std::vector<SweepShape> out;
    if (pl->sqa_P > 0) {
        for (int b : {128, 256, 512}) {
            const SweepShape sh = sqa_shape(pl, b, optin, pl->pm1 ? 1 : 0);
            if (sh.kind == 5) out.push_back(sh);
        }
        for (int b : {256, 512, 1024}) {
            const SweepShape sh = sqa_shape(pl, b, optin, 2);
            if (sh.kind == 5) out.push_back(sh);
        }
        if (!pl->pm1) {
            const SweepShape sh = sqa_shape(pl, 256, optin, 3);
            if (sh.kind == 5) out.push_back(sh);
        }
        return out;
    }
    if (pm1_kernel_eligible(pl->pm1, pl->dmax, pl->max_deg)) {
        const int md = pl->max_deg <= 6 ? 6 : 8;
        for (int w : {2, 4, 8, 16})
            for (int K : {2, 4}) {
                SweepShape sh{4, 32 * w, w, 0, K, md};
                if (pm1w_shape_ok(w, md, pl->max_n0, K) &&
                    sweep_shape_smem(sh, pl->max_n0, pl->thr_stride, pl->max_deg) <= (size_t)optin)
                    out.push_back(sh);
            }
    }
    if (pm1r_kernel_eligible(pl->pm1, pl->dmax, pl->max_deg)) {
        // quad-group kernel: Q quads of the largest problem per item (more for smaller ones)
        const int md = pl->max_deg <= 6 ? 6 : 8;
        for (int b : {128, 256, 512})
            for (int Q : {1, 2, 4, 8}) {
                SweepShape sh{6, b, Q, 0, 0, md};
                if (pm1q_shape_ok(b, md, pl->max_n0, Q) &&
                    sweep_shape_smem(sh, pl->max_n0, pl->thr_stride, pl->max_deg) <= (size_t)optin)
                    out.push_back(sh);
            }
    }
    const int blocks[3] = {128, 256, 512};
    const int qs[4] = {1, 2, 4, 8};
    const int quads = ceil_div(pl->C.S_fix, 4);
    for (int bi = 0; bi < 3; ++bi)
        for (int qi = 0; qi < 4; ++qi) {
            const int Q = qs[qi];
            if (Q > 1 && quads < Q) continue;
            for (int stg = 1; stg >= 0; --stg) {
                SweepShape sh{0, blocks[bi], Q, stg, 0, 0};
                if (sweep_shape_smem(sh, pl->max_n0, pl->thr_stride, pl->max_deg) <= (size_t)optin) out.push_back(sh);
            }
            if (Q == 1 && pm1_kernel_eligible(pl->pm1, pl->dmax, pl->max_deg)) {
                const int md = pl->max_deg <= 6 ? 6 : 8;
                for (int sb : {128, 256, 512, 1024}) {
                    if (sb != blocks[bi] && !(bi == 2 && sb == 1024)) continue;
                    SweepShape sh{2, sb, 1, 0, 0, md};
                    if (pm1s_shape_ok(sb, md, pl->max_n0, 1) &&
                        sweep_shape_smem(sh, pl->max_n0, pl->thr_stride, pl->max_deg) <= (size_t)optin)
                        out.push_back(sh);
                }
            }
            if (pm1r_kernel_eligible(pl->pm1, pl->dmax, pl->max_deg)) {
                const int ns = plan_nslot(pl, Q, blocks[bi]);
                const int md = pl->max_deg <= 6 ? 6 : 8;
                SweepShape sh{1, blocks[bi], Q, 0, ns, md};
                if (ns > 0 && pm1_shape_ok(blocks[bi], ns, md, 0) &&
                    sweep_shape_smem(sh, pl->max_n0, pl->thr_stride, pl->max_deg) <= (size_t)optin)
                    out.push_back(sh);
            }
        }
    const int mode16 = pm1r_kernel_eligible(pl->pm1, pl->dmax, pl->max_deg)          ? 0
                       : ujr_kernel_eligible(pl->ujs, pl->dmax, pl->max_deg)       ? 1
                       : sir_kernel_eligible(pl->jabs_max, pl->dmax, pl->max_deg) ? 2
                                                                                   : 0;
    if (mode16 != 0) {
        // one coupler magnitude per spin, or small integer couplers: the register
        // kernel's 16-bit-lane variants
        const int md = pl->max_deg <= 6 ? 6 : 8;
        for (int blk : {128, 256, 512, 576, 1024})
            for (int Q : {1, 2, 4}) {
                if (Q > 1 && quads < Q) continue;
                int ns = plan_nslot(pl, Q, blk);
                if (ns == 3) ns = 4;
                SweepShape sh{1, blk, Q, mode16, ns, md};
                if (ns > 0 && pm1_shape_ok(blk, ns, md, mode16) &&
                    sweep_shape_smem(sh, pl->max_n0, pl->thr_stride, pl->max_deg) <= (size_t)optin)
                    out.push_back(sh);
            }
    }
    return out;
}

// Times a short run of the plan's phases (at most 4, at most 64 sweeps each;
// the best of two repetitions after an untimed one, and one discarded trial
// before the first candidate) for every candidate shape and keeps the fastest;
// results are cached per problem/plan geometry.
void autotune(spvar_plan *pl, cudaStream_t st, int optin)
{
    const TuneKey key{pl->max_n0, pl->max_deg, pl->pm1 ? 1 : 0, pl->C.S_fix, pl->C.nslots,
                      pl->prm.form, pl->thr_stride, pl->sqa_P, pl->sig};
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            pl->shape = it->second;
            // 32-bit acceptance entries are a property of this plan's table, not of the geometry
            if (pl->shape.kind == 5 && pl->shape.stage >= 2) pl->shape.ent32 = pl->sqa_ent32 ? 1 : 0;
            pl->sweep_smem = sweep_shape_smem(pl->shape, pl->max_n0, pl->thr_stride, pl->max_deg);
            return;
        }
    }
    const int Tt = std::min(pl->T, 64);
    float best = 1e30f;
    SweepShape pick{0, 256, 1, 0, 0, 0};
    bool found = false;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    std::vector<SweepShape> cands;
    for (SweepShape sh : candidate_shapes(pl, optin)) {
        cands.push_back(sh);
        sh.balance = 1;
        if (pl->prm.form != SPVAR_FORM_PLAIN) cands.push_back(sh);
    }
    // a short run of the plan's phases (fixing, and solving on the problems it
    // reduced), so that shapes that suit the full problem but not the reduced
    // ones are not picked; chunk_t > 0 splits every phase into sweep launches
    auto trial = [&](const SweepShape &sh, int chunk_t) -> float {
        pl->shape = sh;
        pl->sweep_smem = sweep_shape_smem(sh, pl->max_n0, pl->thr_stride, pl->max_deg);
        if (sweep_shape_occupancy(sh, pl->pm1, pl->sweep_smem) < 1) return 1e30f;
        const int nslots = (pl->prm.form == SPVAR_FORM_PLAIN) ? 1 : pl->C.nslots;
        pl->C.Q = sh.Q;
        pl->C.chunk = chunk_t;
        SolveConsts C = pl->C;
        C.nslots = nslots;
        const int items = nslots * ceil_div(ceil_div(pl->C.Smax, 4), sh.Q);
        const int grid = (pl->prm.form == SPVAR_FORM_PLAIN) ? items : grid_for(pl, items);
        const int launches = std::min(pl->iters_max, 4) * launches_per_phase(Tt, chunk_t);
        float ms = 1e30f;
        bool ok = true;
        for (int rep = 0; rep < 3 && ok; ++rep) {
            ok = launch_slots_init(pl->d_slots, C, pl->max_n0, st) == cudaSuccess;
            cudaEventRecord(a, st);
            for (int it = 0; it < launches && ok; ++it)
                ok = launch_phase(pl, pl->d_slots, nslots, Tt, grid, st, false) == cudaSuccess;
            cudaEventRecord(b, st);
            if (!ok || cudaEventSynchronize(b) != cudaSuccess) { ok = false; break; }
            float m = 0.f;
            cudaEventElapsedTime(&m, a, b);
            if (rep > 0) ms = std::min(ms, m);  // the first repetition includes one-time setup
        }
        pl->C.chunk = 0;
        if (!ok) { cudaGetLastError(); return 1e30f; }
        return ms;
    };
    // one discarded trial first: clocks and caches settle before the timed candidates
    if (!cands.empty()) trial(cands.front(), 0);
    for (const SweepShape &sh : cands) {
        const float ms = trial(sh, 0);
        if (ms < best) {
            best = ms;
            pick = sh;
            found = true;
        }
    }
    // sweeps per launch: the whole phase in one launch against four launches per
    // phase (each resumes from the states the previous one wrote)
    if (found && pl->sqa_P == 0 && Tt >= 8) {
        const float ms4 = trial(pick, ceil_div(Tt, 4));
        if (ms4 < best) pick.lpp = 4;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (!found) pick = SweepShape{0, 256, 1, 0, 0, 0};
    pl->shape = pick;
    pl->sweep_smem = sweep_shape_smem(pl->shape, pl->max_n0, pl->thr_stride, pl->max_deg);
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[key] = pick;
}

void plan_free(spvar_plan *pl)
{
    if (!pl) return;
    if (pl->graph) cudaGraphExecDestroy(pl->graph);
    if (pl->graph_loop) cudaGraphExecDestroy(pl->graph_loop);
    for (int i = 0; i < 2; ++i)
        if (pl->ev_sweep[i]) cudaEventDestroy(pl->ev_sweep[i]);
    if (pl->ev_post) cudaEventDestroy(pl->ev_post);
    if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
    if (pl->ws) cudaFree(pl->ws);
    if (pl->h_slots_pinned) cudaFreeHost(pl->h_slots_pinned);
    if (pl->h_nactive) cudaFreeHost(pl->h_nactive);
    delete pl;
}

}  // namespace

extern "C" {

int spvar_plan_create(const spvar_problem *const *problems, int32_t nproblems,
                      const spvar_params *prm, size_t budget_bytes, void *stream, spvar_plan **out)
{
    if (!out) return SPVAR_EINVAL;
    *out = nullptr;
    if (!problems || nproblems < 1 || !prm) return SPVAR_EINVAL;
    const spvar_params &p = *prm;
    if (p.num_starts < 1 || p.fixing_sample_size < 1 || p.solving_sample_size < 0 || p.num_sweeps < 0 ||
        p.max_fix_phases < 1 || p.fix_num <= 0 || p.fix_den <= 0 || p.fix_num > p.fix_den ||
        !(p.elite_threshold > 0.0) || !(p.elite_threshold <= 1.0) || !(p.beta0 > 0.0) || !(p.beta1 > 0.0) ||
        p.canon < -1 || p.canon > 1 || (p.form != SPVAR_FORM_BATCHED && p.form != SPVAR_FORM_PLAIN) ||
        p.replicas_per_block < 0 || (p.replicas_per_block % 4) != 0 || p.sweep_kernel < 0 ||
        p.sweep_kernel > 5 || p.start_offset < 0 || p.component_boost < 0 || p.component_boost > 1 || p.tree_preprocess < 0 || p.tree_preprocess > 1 || (p.sweep_block != 0 && p.sweep_block != 128 && p.sweep_block != 256 &&
                               p.sweep_block != 512 && p.sweep_block != 1024 &&
                               !(p.sweep_block == 576 && p.sweep_kernel == SPVAR_SWEEP_PM1 &&
                                 p.sampler == SPVAR_SAMPLER_SA)) ||
        check_corr_params(p) != SPVAR_OK || check_sampler_params(p) != SPVAR_OK || p.sweeps_per_launch < 0 ||
        (p.sampler != SPVAR_SAMPLER_SA && p.sweeps_per_launch != 0))
        return SPVAR_EINVAL;
    const int Smax = std::max(std::max(p.fixing_sample_size, p.solving_sample_size), p.corr_sample_size);
    if (Smax > SPVAR_MAX_SAMPLES || p.num_sweeps > SPVAR_MAX_SWEEPS ||
        p.max_fix_phases + 2 > SPVAR_MAX_PHASE)
        return SPVAR_ELIMIT;
    spvar_plan *pl = new (std::nothrow) spvar_plan();
    if (!pl) return SPVAR_ENOMEM;
    cudaGetDevice(&pl->device);
    cudaDeviceGetAttribute(&pl->sms, cudaDevAttrMultiProcessorCount, pl->device);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->device);
    pl->prm = p;
    int dmax = 0, scale = 0;
    for (int i = 0; i < nproblems; ++i) {
        if (!problems[i]) { delete pl; return SPVAR_EINVAL; }
        const Problem *P = reinterpret_cast<const Problem *>(problems[i]);
        if (i == 0) scale = P->hdr.scale;
        if (P->hdr.scale != scale) { delete pl; return SPVAR_EINVAL; }
        pl->probs.push_back(P);
        dmax = std::max(dmax, P->hdr.dmax);
        pl->max_n0 = std::max(pl->max_n0, P->hdr.n);
        pl->max_deg = std::max(pl->max_deg, P->hdr.maxdeg);
        pl->ncol_max = std::max(pl->ncol_max, P->hdr.ncol);
        for (int c = 0; c < P->hdr.ncol && c < kMaxColours; ++c) pl->class_max = std::max(pl->class_max, P->csize[c]);
        if (!P->hdr.pm1) pl->pm1 = false;
        if (!P->hdr.ujs) pl->ujs = false;
        pl->jabs_max = std::max(pl->jabs_max, P->jabs_max);
        // colour classes, coupler kind and dmax decide which shapes are valid
        auto mix = [&](uint64_t v) { pl->sig = (pl->sig ^ v) * 1099511628211ull; };
        mix((uint64_t)P->hdr.ncol);
        for (int c = 0; c < P->hdr.ncol; ++c) mix((uint64_t)P->csize[c]);
        mix((uint64_t)P->hdr.pm1 << 1 | (uint64_t)P->hdr.ujs);
        mix((uint64_t)P->jabs_max);
        mix((uint64_t)P->hdr.dmax);
    }
    pl->T = p.num_sweeps;
    pl->thr_stride = dmax + 1;
    pl->dmax = dmax;
    if (p.sampler == SPVAR_SAMPLER_SQA) {
        pl->sqa_P = p.sqa_slices;
        pl->sqa_W = 2 * (dmax / 2) + 1;
    }
    if (p.sampler == SPVAR_SAMPLER_PTICM) {
        // every problem's replicas, tables and search queues in one CTA; the exchange
        // table covers energy differences up to n dmax (>= max E - min E of every problem)
        pl->pt_R = p.pticm_temps;
        pl->pt_K = p.pticm_keep;
        for (const Problem *P : pl->probs) {
            if (P->hdr.n > pticm_max_n() || p.pticm_temps > pticm_max_r()) { delete pl; return SPVAR_ELIMIT; }
            pl->pt_smem = std::max(pl->pt_smem, pticm_smem_bytes(P->hdr.n, p.pticm_temps, P->hdr.dmax));
            pl->pt_dx = std::max(pl->pt_dx, (int)std::min<long long>((long long)P->hdr.n * P->hdr.dmax, 1 << 30));
        }
        pl->pt_smem = std::max(pl->pt_smem, pticm_smem_bytes(pl->max_n0, p.pticm_temps, dmax));
        pl->pt_dx = std::max(pl->pt_dx, 1);
        if (pl->pt_smem > (size_t)optin) { delete pl; return SPVAR_ELIMIT; }
    }
    const int nslots = nproblems * p.num_starts;
    SolveConsts &C = pl->C;
    fill_solve_consts(p, C);
    const int P_slots = C.P;
    C.Q = 1;
    C.nslots = nslots;
    C.max_n0 = pl->max_n0;
    pl->iters_max = (p.corr_sample_size > 0 ? 1 : 0) + (p.iterate ? p.max_fix_phases : 1) +
                    (p.solving_sample_size > 0 ? 1 : 0);

    // workspace layout
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
    const size_t o_slots = take(sizeof(Slot) * nslots);
    const size_t o_jobs = take(sizeof(SweepJob) * nslots);
    const size_t max_items = (size_t)nslots * ceil_div(Smax, 4);
    const size_t o_items = take(sizeof(WorkItem) * max_items);
    const size_t o_ctr = take(16);
    const size_t o_thr = take(4 * (size_t)std::max(pl->T, 1) * pl->thr_stride);
    const size_t o_ent = take(pl->sqa_P > 0 ? 8 * (size_t)std::max(pl->T, 1) * 3 * pl->sqa_W : 0);
    const size_t o_pt_thr = take(pl->pt_R > 0 ? 4 * (size_t)pl->pt_R * pl->thr_stride : 0);
    const size_t o_pt_xthr = take(pl->pt_R > 0 ? 4 * (size_t)(pl->pt_R - 1) * ((size_t)pl->pt_dx + 1) : 0);
    const size_t o_rec = take(8 * (size_t)nslots * P_slots * Smax);
    const size_t o_rc = take(4 * (size_t)nslots * P_slots);
    const size_t o_rn = take(4 * (size_t)nslots * P_slots);
    const size_t o_nph = take(4 * (size_t)nslots);
    const size_t o_be = take(8 * (size_t)nslots);
    size_t fm_total = 0;
    for (int s = 0; s < nslots; ++s) fm_total += (size_t)pl->probs[s / p.num_starts]->hdr.n;
    pl->fmap_total = fm_total;
    const size_t o_fmap = take(std::max<size_t>(fm_total, 1));
    const size_t o_best = take(std::max<size_t>(fm_total, 1));
    std::vector<size_t> o_slot(nslots);
    for (int s = 0; s < nslots; ++s) {
        const DevProb &H = pl->probs[s / p.num_starts]->hdr;
        const int n0 = std::max(H.n, 1);
        const size_t pb = prob_blob_bytes(H.cap_n, H.cap_nnz, H.maxdeg);
        size_t b = 2 * align256(pb);
        b += align256(4 * (size_t)Smax * ceil_div(n0, 32));
        b += 2 * align256(4 * (size_t)n0);  // orig[2]
        b += align256(4 * (size_t)Smax);    // elite
        b += align256(4 * (size_t)n0);      // counts
        b += align256((size_t)n0);          // fixed
        b += align256(4 * (size_t)n0);      // old_of_new
        b += align256(4 * slot_scratch_ints(H.cap_n)); // scratch
        b += boost_slot_bytes(p.component_boost, n0, Smax, ceil_div(n0, 32));
        b += tree_slot_bytes(p.tree_preprocess, n0);
        o_slot[s] = take(b);
    }
    pl->ws_bytes = off;
    if (budget_bytes > 0 && off > budget_bytes) { plan_free(pl); return SPVAR_EBUDGET; }
    if (cudaMalloc(&pl->ws, off) != cudaSuccess) { cudaGetLastError(); plan_free(pl); return SPVAR_ENOMEM; }
    if (cudaMallocHost(&pl->h_slots_pinned, sizeof(Slot) * nslots) != cudaSuccess ||
        cudaMallocHost(&pl->h_nactive, sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        plan_free(pl);
        return SPVAR_ENOMEM;
    }
    if (cudaEventCreate(&pl->ev_sweep[0]) != cudaSuccess || cudaEventCreate(&pl->ev_sweep[1]) != cudaSuccess ||
        cudaEventCreate(&pl->ev_post) != cudaSuccess) {
        cudaGetLastError();
        plan_free(pl);
        return SPVAR_ECUDA;
    }
    char *w = static_cast<char *>(pl->ws);
    pl->d_slots = (Slot *)(w + o_slots);
    pl->d_jobs = (SweepJob *)(w + o_jobs);
    pl->d_items = (WorkItem *)(w + o_items);
    pl->d_ctr = (int32_t *)(w + o_ctr);
    pl->d_thr = (uint32_t *)(w + o_thr);
    if (pl->sqa_P > 0) pl->d_ent = (unsigned long long *)(w + o_ent);
    if (pl->pt_R > 0) {
        pl->d_pt_thr = (uint32_t *)(w + o_pt_thr);
        pl->d_pt_xthr = (uint32_t *)(w + o_pt_xthr);
    }
    pl->d_rec_e = (int64_t *)(w + o_rec);
    pl->d_rec_count = (int32_t *)(w + o_rc);
    pl->d_rec_nfree = (int32_t *)(w + o_rn);
    pl->d_nphases = (int32_t *)(w + o_nph);
    pl->d_best_e = (int64_t *)(w + o_be);
    pl->d_fmap = (int8_t *)(w + o_fmap);
    pl->d_best = (int8_t *)(w + o_best);

    cudaStream_t st = as_stream(stream);
    // acceptance table
    {
        std::vector<double> beta(std::max(pl->T, 1));
        std::vector<uint32_t> thr((size_t)std::max(pl->T, 1) * pl->thr_stride, 0u);
        if (pl->T > 0) {
            spvar_beta_geometric(pl->T, p.beta0, p.beta1, beta.data());
            spvar_thresholds(pl->T, beta.data(), dmax, scale, thr.data());
        }
        std::vector<uint64_t> ent;
        if (pl->sqa_P > 0) {
            // SQA: constant beta, linear transverse field
            ent.assign((size_t)std::max(pl->T, 1) * 3 * pl->sqa_W, 0ull);
            std::vector<double> sb(std::max(pl->T, 1), p.sqa_beta), sg(std::max(pl->T, 1));
            if (pl->T > 0) {
                spvar_gamma_linear(pl->T, p.sqa_gamma0, p.sqa_gamma1, sg.data());
                spvar_sqa_table(pl->T, pl->sqa_P, sb.data(), sg.data(), dmax, scale, ent.data());
            }
            pl->sqa_ent32 = std::all_of(ent.begin(), ent.end(), [](uint64_t v) { return (v >> 32) == 0; });
        }
        std::vector<uint32_t> pt_thr, pt_xthr;
        if (pl->pt_R > 0) {
            // PTICM: the temperatures' Metropolis rows and the exchange rows (beta_{k+1} - beta_k)
            std::vector<double> bt(pl->pt_R), db(std::max(pl->pt_R - 1, 1));
            spvar_beta_geometric(pl->pt_R, p.pticm_beta0, p.pticm_beta1, bt.data());
            for (int k = 0; k + 1 < pl->pt_R; ++k) db[k] = bt[k + 1] - bt[k];
            pt_thr.assign((size_t)pl->pt_R * pl->thr_stride, 0u);
            pt_xthr.assign((size_t)(pl->pt_R - 1) * ((size_t)pl->pt_dx + 1), 0u);
            spvar_thresholds(pl->pt_R, bt.data(), dmax, scale, pt_thr.data());
            spvar_thresholds(pl->pt_R - 1, db.data(), pl->pt_dx, scale, pt_xthr.data());
        }
        if ((pl->pt_R > 0 &&
             (cudaMemcpyAsync(pl->d_pt_thr, pt_thr.data(), 4 * pt_thr.size(), cudaMemcpyHostToDevice, st) !=
                  cudaSuccess ||
              cudaMemcpyAsync(pl->d_pt_xthr, pt_xthr.data(), 4 * pt_xthr.size(), cudaMemcpyHostToDevice, st) !=
                  cudaSuccess)) ||
            cudaMemcpyAsync(pl->d_thr, thr.data(), 4 * thr.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            (pl->sqa_P > 0 &&
             cudaMemcpyAsync(pl->d_ent, ent.data(), 8 * ent.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            plan_free(pl);
            return SPVAR_ECUDA;
        }
    }
    // slots and their problem buffers
    pl->h_slots.resize(nslots);
    pl->starts_of.resize(nslots);
    std::vector<DevProb> hdrs;
    std::vector<DevProb *> hdr_dst;
    size_t fm_off = 0;
    for (int s = 0; s < nslots; ++s) {
        const int pi = s / p.num_starts;
        const Problem *P = pl->probs[pi];
        const DevProb &H = P->hdr;
        const int n0 = std::max(H.n, 1);
        Slot &S = pl->h_slots[s];
        std::memset(&S, 0, sizeof(Slot));
        pl->starts_of[s] = pi;
        char *b = w + o_slot[s];
        size_t o = 0;
        auto carve = [&](size_t bytes) { char *r = b + o; o += align256(bytes); return r; };
        const size_t pb = prob_blob_bytes(H.cap_n, H.cap_nnz, H.maxdeg);
        for (int k = 0; k < 2; ++k) {
            void *blob = carve(pb);
            DevProb hd;
            std::memset(&hd, 0, sizeof(hd));
            prob_carve(&hd, blob, H.cap_n, H.cap_nnz, H.maxdeg);
            hdrs.push_back(hd);
            hdr_dst.push_back((DevProb *)blob);
            S.buf[k] = (DevProb *)blob;
        }
        S.orig_prob = P->dev;
        S.cur = P->dev;
        S.n0 = H.n;
        S.W0 = ceil_div(n0, 32);
        S.start = (uint32_t)(p.start_offset + s % p.num_starts);
        S.spins = (uint32_t *)carve(4 * (size_t)Smax * S.W0);
        S.orig[0] = (int32_t *)carve(4 * (size_t)n0);
        S.orig[1] = (int32_t *)carve(4 * (size_t)n0);
        S.elite = (int32_t *)carve(4 * (size_t)Smax);
        S.counts = (int32_t *)carve(4 * (size_t)n0);
        S.fixed = (int8_t *)carve((size_t)n0);
        S.old_of_new = (int32_t *)carve(4 * (size_t)n0);
        S.scratch = (int32_t *)carve(4 * slot_scratch_ints(H.cap_n));
        if (p.component_boost)
            boost_slot_carve(S, carve(boost_slot_bytes(1, n0, Smax, S.W0)), n0, Smax, S.W0);
        if (p.tree_preprocess) tree_slot_carve(S, carve(tree_slot_bytes(1, n0)), n0);
        S.rec_e = pl->d_rec_e + (size_t)s * P_slots * Smax;
        S.rec_count = pl->d_rec_count + (size_t)s * P_slots;
        S.rec_nfree = pl->d_rec_nfree + (size_t)s * P_slots;
        S.nphases = pl->d_nphases + s;
        S.best_e = pl->d_best_e + s;
        S.fmap = pl->d_fmap + fm_off;
        S.best_state = pl->d_best + fm_off;
        fm_off += (size_t)H.n;
    }
    bool ok = true;
    for (size_t k = 0; k < hdrs.size() && ok; ++k)
        ok = cudaMemcpyAsync(hdr_dst[k], &hdrs[k], sizeof(DevProb), cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (ok) ok = upload_slots(pl, nullptr, st) == SPVAR_OK;
    if (ok) ok = cudaStreamSynchronize(st) == cudaSuccess;
    if (!ok) { cudaGetLastError(); plan_free(pl); return SPVAR_ECUDA; }

    // sweep shape (PTICM: none, its runs replace the sweep launch)
    if (pl->pt_R > 0) {
        pl->shape = SweepShape{0, 256, 1, 0, 0, 0};
        pl->sweep_smem = 0;
    } else if (p.replicas_per_block > 0) {
        // requested shape: replicas per CTA, kernel and block size
        const int Q = p.replicas_per_block / 4;
        const int blk = p.sweep_block ? p.sweep_block : 256;
        const bool elig = pm1_kernel_eligible(pl->pm1, pl->dmax, pl->max_deg);
        SweepShape sh{0, blk, Q, 1, 0, 0};
        if (pl->sqa_P > 0) {
            // SQA: one quad per CTA; the register form (else the walk) for +-1 couplers unless the
            // walk or the general path is asked for
            if (p.sweep_kernel == SPVAR_SWEEP_GENERAL) sh = sqa_shape(pl, blk, optin, 0);
            else if (p.sweep_kernel == SPVAR_SWEEP_PM1S) sh = sqa_shape(pl, blk, optin, 1);
            else if (p.sweep_kernel == SPVAR_SWEEP_PM1W || p.sweep_kernel == SPVAR_SWEEP_PM1Q) sh.kind = -1;
            else if (!pl->pm1) {
                if (p.sweep_kernel == SPVAR_SWEEP_PM1) sh = sqa_shape(pl, blk, optin, 3);
                if (sh.kind != 5) sh = sqa_shape(pl, blk, optin, 0);
            }
            else {
                sh = sqa_shape(pl, blk, optin, 2);
                if (sh.kind != 5) sh = sqa_shape(pl, blk, optin, 1);
            }
            if (Q != 1 || sh.kind != 5) { plan_free(pl); return SPVAR_ELIMIT; }
        } else if (p.sweep_kernel == SPVAR_SWEEP_PM1 || (p.sweep_kernel == SPVAR_SWEEP_AUTO && elig)) {
            const int md = pl->max_deg <= 6 ? 6 : 8;
            // byte-lane register kernel, else (one coupler magnitude per spin) its
            // 16-bit-lane variant, else the streaming +-1 kernel
            const int ns = pm1r_kernel_eligible(pl->pm1, pl->dmax, pl->max_deg) ? plan_nslot(pl, Q, blk) : 0;
            const int mu = ujr_kernel_eligible(pl->ujs, pl->dmax, pl->max_deg)          ? 1
                           : sir_kernel_eligible(pl->jabs_max, pl->dmax, pl->max_deg) ? 2
                                                                                       : 0;
            int nsu = mu ? plan_nslot(pl, Q, blk) : 0;
            if (nsu == 3) nsu = 4;
            const SweepShape cu{1, blk, Q, mu, nsu, md};
            if (ns > 0 && pm1_shape_ok(blk, ns, md, 0)) sh = SweepShape{1, blk, Q, 0, ns, md};
            else if (nsu > 0 && pm1_shape_ok(blk, nsu, md, mu) &&
                     sweep_shape_smem(cu, pl->max_n0, pl->thr_stride, pl->max_deg) <= (size_t)optin)
                sh = cu;
            else if (elig && pm1s_shape_ok(blk, md, pl->max_n0, Q)) sh = SweepShape{2, blk, Q, 0, 0, md};
            else { plan_free(pl); return SPVAR_ELIMIT; }
            if (blk == 576 && (sh.kind != 1 || sh.stage == 0)) {  // the 16-bit-lane register kernel only
                plan_free(pl);
                return SPVAR_ELIMIT;
            }
        } else if (p.sweep_kernel == SPVAR_SWEEP_PM1Q) {
            const int md = pl->max_deg <= 6 ? 6 : 8;
            if (!pm1r_kernel_eligible(pl->pm1, pl->dmax, pl->max_deg) || !pm1q_shape_ok(blk, md, pl->max_n0, Q)) {
                plan_free(pl);
                return SPVAR_ELIMIT;
            }
            sh = SweepShape{6, blk, Q, 0, 0, md};
        } else if (p.sweep_kernel == SPVAR_SWEEP_PM1W) {
            const int md = pl->max_deg <= 6 ? 6 : 8;
            if (!elig || !pm1w_shape_ok(Q, md, pl->max_n0, 4)) { plan_free(pl); return SPVAR_ELIMIT; }
            sh = SweepShape{4, 32 * Q, Q, 0, 4, md};
        } else if (p.sweep_kernel == SPVAR_SWEEP_PM1S) {
            const int md = pl->max_deg <= 6 ? 6 : 8;
            if (!elig || !pm1s_shape_ok(blk, md, pl->max_n0, Q)) { plan_free(pl); return SPVAR_ELIMIT; }
            sh = SweepShape{2, blk, Q, 0, 0, md};
        } else if (sweep_shape_smem(sh, pl->max_n0, pl->thr_stride, pl->max_deg) > (size_t)optin) {
            sh.stage = 0;
        }
        pl->shape = sh;
        pl->sweep_smem = sweep_shape_smem(sh, pl->max_n0, pl->thr_stride, pl->max_deg);
        if (pl->sweep_smem > (size_t)optin) { plan_free(pl); return SPVAR_ELIMIT; }
    } else {
        autotune(pl, st, optin);
        if (pl->sweep_smem > (size_t)optin) { plan_free(pl); return SPVAR_ELIMIT; }
    }
    pl->C.Q = pl->shape.Q;
    // sweeps per launch: requested, else the autotuner's choice (one launch per phase by default)
    if (p.sweeps_per_launch > 0) pl->C.chunk = p.sweeps_per_launch < pl->T ? p.sweeps_per_launch : 0;
    else if (p.replicas_per_block == 0 && pl->shape.lpp > 1) pl->C.chunk = ceil_div(std::max(pl->T, 1), pl->shape.lpp);
    else pl->C.chunk = 0;
    const int items = nslots * ceil_div(ceil_div(Smax, 4), pl->shape.Q);
    pl->sweep_grid = grid_for(pl, items);

    // capture one batched phase as a CUDA graph
    if (p.form == SPVAR_FORM_BATCHED) {
        if (cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking) == cudaSuccess) {
            cudaGraph_t g = nullptr;
            bool cap = cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeRelaxed) == cudaSuccess;
            if (cap) {
                cudaError_t e =
                    launch_phase(pl, pl->d_slots, nslots, pl->T, pl->sweep_grid, pl->cap_stream, true, true);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(pl->h_nactive, pl->d_ctr + 2, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                        pl->cap_stream);
                cudaError_t e2 = cudaStreamEndCapture(pl->cap_stream, &g);
                if (e == cudaSuccess && e2 == cudaSuccess && g) {
                    if (cudaGraphInstantiate(&pl->graph, g, 0) != cudaSuccess) pl->graph = nullptr;
                }
                if (g) cudaGraphDestroy(g);
            }
            cudaGetLastError();
            build_loop_graph(pl, nslots);
        }
    }
    *out = pl;
    return SPVAR_OK;
}

size_t spvar_plan_workspace_bytes(const spvar_plan *plan) { return plan ? plan->ws_bytes : 0; }

int spvar_plan_run(spvar_plan *pl, const uint64_t *seeds, const spvar_result *res, void *stream)
{
    if (!pl || !seeds) return SPVAR_EINVAL;
    cudaStream_t st = as_stream(stream);
    const int nslots = pl->C.nslots;
    int rc = upload_slots(pl, seeds, st);
    if (rc) return rc;
    SPVAR_CUDA_TRY(launch_slots_init(pl->d_slots, pl->C, pl->max_n0, st));
    const bool iterate = pl->prm.iterate != 0;
    pl->sweep_ms = 0.0;
    pl->post_ms = 0.0;
    pl->sweep_launches = 0;
    // profiling: wait for each phase and add up the sweep kernel's event time
    auto profile_phase = [&]() -> int {
        if (!pl->profiling) return SPVAR_OK;
        SPVAR_CUDA_TRY(cudaEventSynchronize(pl->ev_sweep[1]));
        float ms = 0.f;
        SPVAR_CUDA_TRY(cudaEventElapsedTime(&ms, pl->ev_sweep[0], pl->ev_sweep[1]));
        pl->sweep_ms += ms;
        pl->sweep_launches += 1;
        SPVAR_CUDA_TRY(cudaEventSynchronize(pl->ev_post));
        SPVAR_CUDA_TRY(cudaEventElapsedTime(&ms, pl->ev_sweep[1], pl->ev_post));
        pl->post_ms += ms;
        return SPVAR_OK;
    };
    if (pl->prm.form == SPVAR_FORM_BATCHED && pl->graph_loop && !pl->profiling) {
        // the whole run on the device: phases loop inside the graph
        SPVAR_CUDA_TRY(cudaMemsetAsync(pl->d_ctr + 3, 0, sizeof(int32_t), st));
        SPVAR_CUDA_TRY(cudaGraphLaunch(pl->graph_loop, st));
    } else if (pl->prm.form == SPVAR_FORM_BATCHED) {
        const int steps = plan_steps(pl);
        for (int it = 0; it < steps; ++it) {
            if (pl->graph) {
                SPVAR_CUDA_TRY(cudaGraphLaunch(pl->graph, st));
            } else {
                SPVAR_CUDA_TRY(launch_phase(pl, pl->d_slots, nslots, pl->T, pl->sweep_grid, st, true));
                SPVAR_CUDA_TRY(cudaMemcpyAsync(pl->h_nactive, pl->d_ctr + 2, sizeof(int32_t),
                                               cudaMemcpyDeviceToHost, st));
            }
            if ((rc = profile_phase()) != SPVAR_OK) return rc;
            if (iterate && it + 1 < steps) {
                SPVAR_CUDA_TRY(cudaStreamSynchronize(st));
                if (*pl->h_nactive == 0) break;
            }
        }
    } else {
        const int grid = ceil_div(ceil_div(pl->C.Smax, 4), pl->shape.Q);
        const int steps = plan_steps(pl);
        for (int s = 0; s < nslots; ++s) {
            for (int it = 0; it < steps; ++it) {
                SPVAR_CUDA_TRY(launch_phase(pl, pl->d_slots + s, 1, pl->T, grid, st, iterate));
                if ((rc = profile_phase()) != SPVAR_OK) return rc;
                if (iterate && it + 1 < steps) {
                    SPVAR_CUDA_TRY(cudaMemcpyAsync(pl->h_nactive, pl->d_ctr + 2, sizeof(int32_t),
                                                   cudaMemcpyDeviceToHost, st));
                    SPVAR_CUDA_TRY(cudaStreamSynchronize(st));
                    if (*pl->h_nactive == 0) break;
                }
            }
        }
    }
    if (res) {
        const cudaMemcpyKind kind = res->device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        const size_t P_slots = pl->C.P, Smax = pl->C.Smax;
        auto cp = [&](void *dst, const void *src, size_t bytes) -> bool {
            return !dst || !bytes || cudaMemcpyAsync(dst, src, bytes, kind, st) == cudaSuccess;
        };
        bool ok = cp(res->energies, pl->d_rec_e, 8 * nslots * P_slots * Smax) &&
                  cp(res->counts, pl->d_rec_count, 4 * nslots * P_slots) &&
                  cp(res->nfree, pl->d_rec_nfree, 4 * nslots * P_slots) &&
                  cp(res->nphases, pl->d_nphases, 4 * (size_t)nslots) &&
                  cp(res->fixed, pl->d_fmap, pl->fmap_total) &&
                  cp(res->best_energy, pl->d_best_e, 8 * (size_t)nslots) &&
                  cp(res->best_state, pl->d_best, pl->fmap_total);
        if (!ok) return SPVAR_ECUDA;
        if (!res->device) SPVAR_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return SPVAR_OK;
}

int spvar_plan_set_profiling(spvar_plan *plan, int32_t on)
{
    if (!plan) return SPVAR_EINVAL;
    plan->profiling = on ? 1 : 0;
    return SPVAR_OK;
}

int spvar_plan_sweep_time(const spvar_plan *plan, double *total_ms, int32_t *launches)
{
    if (!plan) return SPVAR_EINVAL;
    if (total_ms) *total_ms = plan->sweep_ms;
    if (launches) *launches = plan->sweep_launches;
    return SPVAR_OK;
}

int spvar_plan_post_time(const spvar_plan *plan, double *total_ms)
{
    if (!plan) return SPVAR_EINVAL;
    if (total_ms) *total_ms = plan->post_ms;
    return SPVAR_OK;
}

int spvar_plan_shape(const spvar_plan *plan, int32_t *block, int32_t *replicas_per_block,
                     int32_t *staged, int32_t *grid)
{
    if (!plan) return SPVAR_EINVAL;
    if (block) *block = plan->shape.block;
    if (replicas_per_block) *replicas_per_block = 4 * plan->shape.Q;
    if (staged) {
        const int k = plan->shape.kind;
        *staged = k == 1 ? 2 : k == 2 ? 3 : k == 4 ? 4 : k == 5 ? (plan->shape.stage >= 2 ? 6 : 5) : k == 6 ? 7
                                                                                                 : plan->shape.stage;
    }
    if (grid) *grid = plan->sweep_grid;
    return SPVAR_OK;
}

int spvar_plan_sweeps_per_launch(const spvar_plan *plan, int32_t *sweeps)
{
    if (!plan || !sweeps) return SPVAR_EINVAL;
    *sweeps = plan->C.chunk > 0 ? plan->C.chunk : plan->T;
    return SPVAR_OK;
}

int spvar_plan_stats(const spvar_plan *plan, int64_t *attempts, int32_t *phases)
{
    if (!plan) return SPVAR_EINVAL;
    spvar_plan *pl = const_cast<spvar_plan *>(plan);
    const size_t n = (size_t)pl->C.nslots * pl->C.P;
    std::vector<int32_t> cnt(n), nf(n);
    if (cudaMemcpy(cnt.data(), pl->d_rec_count, 4 * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(nf.data(), pl->d_rec_nfree, 4 * n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return SPVAR_ECUDA;
    int64_t a = 0;
    int32_t ph = 0;
    const int64_t per = (int64_t)pl->T * (pl->sqa_P > 0 ? pl->sqa_P : 1);  // SQA: every slice is swept
    for (size_t i = 0; i < n; ++i) {
        // PTICM: a phase is one run, every one of its 2R replicas swept T times
        a += pl->pt_R > 0 ? (cnt[i] > 0 ? 2ll * pl->pt_R * nf[i] * pl->T : 0) : (int64_t)cnt[i] * nf[i] * per;
        if (cnt[i] > 0) ++ph;
    }
    if (attempts) *attempts = a;
    if (phases) *phases = ph;
    return SPVAR_OK;
}

void spvar_plan_destroy(spvar_plan *plan) { plan_free(plan); }

int spvar_solve(const spvar_problem *p, const spvar_params *prm, uint64_t seed, const spvar_result *res,
                void *stream)
{
    if (!p || !prm) return SPVAR_EINVAL;
    const Problem *P = reinterpret_cast<const Problem *>(p);
    std::vector<int64_t> key;
    solve_key(P, *prm, key);
    spvar_plan *pl = solve_cache_take(key);
    if (pl) {
        // a plan built for a problem of the same structure: point its starts at this one
        pl->probs[0] = P;
        for (Slot &S : pl->h_slots) {
            S.orig_prob = P->dev;
            S.cur = P->dev;
        }
    } else {
        const spvar_problem *arr[1] = {p};
        const int rc = spvar_plan_create(arr, 1, prm, 0, stream, &pl);
        if (rc) return rc;
    }
    const int rc = spvar_plan_run(pl, &seed, res, stream);
    if (rc == SPVAR_OK) solve_cache_put(std::move(key), pl);
    else plan_free(pl);
    return rc;
}

void spvar_solve_cache_release(void)
{
    std::list<std::pair<std::vector<int64_t>, spvar_plan *>> drop;
    {
        std::lock_guard<std::mutex> g(g_solve_mu);
        drop.swap(g_solve_cache);
    }
    for (auto &e : drop) plan_free(e.second);
}

}  // extern "C"
