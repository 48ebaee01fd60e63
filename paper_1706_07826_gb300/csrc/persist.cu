// Persistence pass (Alg. 1: elite sample, mean value of each variable,
// fixing rule), fold/compact (Alg. 1: update J and h) and the per-start state
// machine of Multi-start SPVAR (Alg. 2).
//
// Elite selection bounds the k lowest (energy, index) keys of one sample set
// by a histogram and places the candidates by rank in shared memory; the
// counts read only the k elite rows of the bit-packed sample, a lane per word,
// into bit-sliced counters; fold/compact writes the new CSR, the inherited
// colour classes and the sweep layout of the smaller problem.  In the
// multi-start driver one thread-block cluster per start runs all of it in one
// launch; the standalone entry points and the tree step use one CTA per call.
#include <algorithm>
#include <climits>

#include <cooperative_groups.h>

#include "persist.cuh"

namespace cg = cooperative_groups;

namespace spvar {

__device__ void reduce_core(const DevProb *S, DevProb *D, const int8_t *fixed, int32_t *old_of_new,
                            int32_t *scratch, bool fold)
{
    __shared__ int s_warp[32];
    __shared__ unsigned long long s_off;
    __shared__ int s_hnz;
    __shared__ long long s_rho_key;
    const int tid = threadIdx.x, B = blockDim.x;
    const int n = S->n;
    int32_t *new_of_old = scratch;          // [n]
    int32_t *rowcnt = scratch + S->cap_n;   // [n']
    if (tid == 0) {
        s_off = 0ull;
        s_hnz = 0;
        s_rho_key = -1;
    }
    __syncthreads();

    // free spins keep their order: new index = exclusive count of free spins before
    int carry = 0;
    for (int base = 0; base < n; base += B) {
        const int i = base + tid;
        const int f = (i < n && fixed[i] == 0) ? 1 : 0;
        int tot;
        const int ex = block_scan_excl(f, s_warp, &tot);
        if (i < n) {
            new_of_old[i] = f ? carry + ex : -1;
            if (f) old_of_new[carry + ex] = i;
        }
        carry += tot;
    }
    const int m = carry;
    __syncthreads();

    // h'_i = h_i + sum_{j fixed} J_ij v_j ;  offset' = offset + sum_{i fixed} h_i v_i
    //        + sum_{i<j both fixed} J_ij v_i v_j
    long long off_part = 0;
    for (int i = tid; i < n; i += B) {
        const int vi = fixed[i];
        long long hf = S->h[i];
        int nfree = 0;
        for (int p = S->row_ptr[i]; p < S->row_ptr[i + 1]; ++p) {
            const int j = S->col[p];
            const int vj = fixed[j];
            if (vi) {
                if (fold && vj && j > i) off_part += (long long)S->val[p] * vi * vj;
            } else {
                if (!vj) ++nfree;
                else if (fold) hf += (long long)S->val[p] * vj;
            }
        }
        if (vi) {
            if (fold) off_part += (long long)S->h[i] * vi;
        } else {
            const int a = new_of_old[i];
            D->h[a] = (int32_t)hf;
            rowcnt[a] = nfree;
            if (hf != 0) atomicOr(&s_hnz, 1);
        }
    }
    atomicAdd(&s_off, (unsigned long long)off_part);
    __syncthreads();

    // row pointers of the free-free couplers
    carry = 0;
    for (int base = 0; base < m; base += B) {
        const int a = base + tid;
        const int c = (a < m) ? rowcnt[a] : 0;
        int tot;
        const int ex = block_scan_excl(c, s_warp, &tot);
        if (a < m) D->row_ptr[a] = carry + ex;
        carry += tot;
    }
    const int nnz2 = carry;
    if (tid == 0) D->row_ptr[m] = nnz2;
    __syncthreads();

    for (int a = tid; a < m; a += B) {
        const int i = old_of_new[a];
        int q = D->row_ptr[a];
        for (int p = S->row_ptr[i]; p < S->row_ptr[i + 1]; ++p) {
            const int j = S->col[p];
            if (fixed[j] == 0) {
                D->col[q] = new_of_old[j];
                D->val[q] = S->val[p];
                ++q;
            }
        }
        D->colour[a] = S->colour[i];
    }
    __syncthreads();

    // inherited colour classes -> positions (class by class, increasing index)
    const int ncol = S->ncol;
    int cbase = 0;
    for (int c = 0; c < ncol; ++c) {
        if (tid == 0) D->cptr[c] = cbase;
        int cc = 0;
        for (int base = 0; base < m; base += B) {
            const int a = base + tid;
            const int f = (a < m && D->colour[a] == c) ? 1 : 0;
            int tot;
            const int ex = block_scan_excl(f, s_warp, &tot);
            if (f) {
                const int pos = cbase + cc + ex;
                D->pos_of_idx[a] = pos;
                D->idx_of_pos[pos] = a;
            }
            cc += tot;
        }
        cbase += cc;
    }
    if (tid == 0) D->cptr[ncol] = cbase;
    __syncthreads();

    // sweep layout: meta (h, degree) and ELL by position
    const int cap = D->cap_n;
    long long rk = -1;
    for (int a = tid; a < m; a += B) {
        const int pos = D->pos_of_idx[a];
        const int r0 = D->row_ptr[a];
        const int deg = D->row_ptr[a + 1] - r0;
        D->meta[pos] = ((uint32_t)(D->h[a] & 0xFFFF) << 16) | (uint32_t)deg;
        for (int d = 0; d < deg; ++d) {
            const int j = D->col[r0 + d];
            D->ell[(size_t)d * cap + pos] =
                ((uint32_t)D->pos_of_idx[j] & 0xFFFFu) | ((uint32_t)(D->val[r0 + d] & 0xFFFF) << 16);
        }
        // reference spin: largest degree, lowest index among those
        const long long key = ((long long)deg << 32) | (long long)(0x7FFFFFFF - a);
        rk = max(rk, key);
    }
    atomicMax(&s_rho_key, rk);
    __syncthreads();
    if (tid == 0) {
        D->n = m;
        D->nnz = nnz2;
        D->ncol = ncol;
        D->maxdeg = S->maxdeg;
        D->dmax = S->dmax;
        D->hzero = s_hnz ? 0 : 1;
        D->pm1 = S->pm1;
        D->ujs = S->ujs;
        D->rho = (m > 0) ? (0x7FFFFFFF - (int)(s_rho_key & 0xFFFFFFFFll)) : -1;
        D->offset = S->offset + (long long)s_off;
        D->scale = S->scale;
    }
    __syncthreads();
}

// Tree pre-processing of P in place (Sec. II.C), rounds as in the oracle:
// every active spin of active degree 0, and of active degree 1 except the
// lower-index end of an isolated coupler, is eliminated at once.  Writes
// code[i] (0 kept, +1/-1 fixed, 2 inferred), folds into P->h / P->offset,
// records fixings in fmap and inferences in the slot's log (original indices
// through orig).  deg: scratch [n].  One CTA; contains __syncthreads.
__device__ void tree_core(DevProb *P, int8_t *code, int32_t *scratch, int8_t *fmap, const int32_t *orig,
                          int32_t *log_child, int32_t *log_parent, int8_t *log_sigma, int32_t *nlog)
{
    __shared__ int s_any;
    __shared__ unsigned long long s_off;
    __shared__ int s_log;
    const int n = P->n, tid = threadIdx.x, B = blockDim.x;
    int32_t *deg = scratch;          // active degree (pass 1)
    int32_t *nb = scratch + P->cap_n; // this round's pick: -2 none, -1 degree 0, else the neighbour
    for (int i = tid; i < n; i += B) code[i] = 0;
    if (tid == 0) {
        s_off = 0ull;
        s_log = *nlog;
    }
    __syncthreads();
    for (;;) {
        // pass 1: active degrees
        for (int i = tid; i < n; i += B) {
            int d = 0;
            if (code[i] == 0)
                for (int p = P->row_ptr[i]; p < P->row_ptr[i + 1]; ++p) d += code[P->col[p]] == 0;
            deg[i] = d;
        }
        if (tid == 0) s_any = 0;
        __syncthreads();
        // pass 2: this round's leaves (codes are not modified in this pass)
        for (int i = tid; i < n; i += B) {
            int pick = -2;
            if (code[i] == 0 && deg[i] == 0) {
                pick = -1;
            } else if (code[i] == 0 && deg[i] == 1) {
                int j = -1;
                for (int p = P->row_ptr[i]; p < P->row_ptr[i + 1]; ++p)
                    if (code[P->col[p]] == 0) j = P->col[p];
                if (!(deg[j] == 1 && i < j)) pick = j;  // isolated coupler: the higher end goes first
            }
            nb[i] = pick;
            if (pick != -2) s_any = 1;
        }
        __syncthreads();
        if (!s_any) break;
        // pass 3: eliminate; a picked spin's neighbour is never picked, so the
        // updates of a shared neighbour only add up
        long long off = 0;
        for (int i = tid; i < n; i += B) {
            const int j = nb[i];
            if (j == -2) continue;
            const int h = P->h[i];
            if (j == -1) {
                const int v = h > 0 ? -1 : 1;
                off += (long long)h * v;
                code[i] = (int8_t)v;
                fmap[orig[i]] = (int8_t)v;
                continue;
            }
            int J = 0;
            for (int p = P->row_ptr[i]; p < P->row_ptr[i + 1]; ++p)
                if (P->col[p] == j) J = P->val[p];
            if (abs(J) <= abs(h)) {
                const int v = h > 0 ? -1 : 1;
                off += (long long)h * v;
                atomicAdd(&P->h[j], J * v);
                code[i] = (int8_t)v;
                fmap[orig[i]] = (int8_t)v;
            } else {
                const int sJ = J > 0 ? 1 : -1;
                off -= abs(J);
                atomicAdd(&P->h[j], -sJ * h);
                code[i] = 2;
                const int q = atomicAdd(&s_log, 1);
                log_child[q] = orig[i];
                log_parent[q] = orig[j];
                log_sigma[q] = (int8_t)(-sJ);
            }
        }
        atomicAdd(&s_off, (unsigned long long)off);
        __syncthreads();
    }
    if (tid == 0) {
        P->offset += (long long)s_off;
        *nlog = s_log;
    }
    __syncthreads();
}

namespace {

// ---------------------------------------------------------------- standalone
__global__ void __launch_bounds__(kBigBlock) k_elite_single(const int64_t *energies, int S, int k,
                                                            int32_t *elite)
{
    extern __shared__ __align__(16) unsigned long long s_key[];
    elite_fast(energies, S, k, elite, s_key);
}

__global__ void __launch_bounds__(kCountBlock)
    k_count_single(const DevProb *P, const uint32_t *spins, int W, const int32_t *elite, int k,
                   int canon, int fix_num, int fix_den, int32_t *counts, int8_t *fixed,
                   int32_t *nfixed)
{
    __shared__ CountSmem sm;
    count_bs_core(P, spins, W, elite, k, canon, fix_num, fix_den, counts, fixed, nfixed, nullptr, nullptr, blockIdx.x, sm);
}

__global__ void __launch_bounds__(kBigBlock) k_reduce_single(const DevProb *src, DevProb *dst,
                                                             const int8_t *fixed,
                                                             int32_t *old_of_new, int32_t *scratch)
{
    reduce_core(src, dst, fixed, old_of_new, scratch);
}

// ----------------------------------------------------------- multi-start slots
__global__ void __launch_bounds__(256) k_slots_init(Slot *slots, SolveConsts C)
{
    Slot &s = slots[blockIdx.x];
    for (int i = threadIdx.x; i < s.n0; i += blockDim.x) {
        s.orig[0][i] = i;
        s.fmap[i] = 0;
        s.best_state[i] = 0;
    }
    for (int p = threadIdx.x; p < C.P; p += blockDim.x) {
        s.rec_count[p] = 0;
        s.rec_nfree[p] = 0;
    }
    if (threadIdx.x == 0) {
        s.cur = s.orig_prob;
        s.next = 0;
        s.ocur = 0;
        s.mode = (C.S_corr > 0 && s.orig_prob->hzero) ? kCorr : kFixing;
        s.phase = 0;
        s.fix_done = 0;
        s.nfixed = 0;
        s.nlog = 0;
        s.tsw = 0;
        *s.best_e = LLONG_MAX;
        *s.nphases = 0;
    }
}

// Quads per work item of a start whose current problem is P and who runs
// nquads quads: C.Q; for the quad-group kernel the most that the launch's
// shared memory holds; for the register kernel the most that its slots hold
// (every colour class fills ceil(size * q / block) whole slots; at most
// block * nslot / 4 quads so that the per-item energy sums fit), but no more
// than leaves about two items per CTA of the launch (starts of similar size).
__device__ __forceinline__ int item_quads(const DevProb *P, const SolveConsts &C, int nquads)
{
    const int cap = max(1, (int)(((long long)nquads * C.nslots) / (2ll * max(C.grid, 1))));
    if (C.fit_words > 0) {
        // quad-group kernel: as many quads as the launch's spin words hold, at most 64
        const int fit = C.fit_words / (2 * (P->n + 1));
        return max(1, min(min(fit, 64), cap));
    }
    if (C.fit_block <= 0) return C.Q;
    const int ncol = P->ncol;
    auto need = [&](int q) {
        int s = 0;
        for (int c = 0; c < ncol; ++c) s += ceil_div((P->cptr[c + 1] - P->cptr[c]) * q, C.fit_block);
        return s;
    };
    int lo = 1, hi = max(1, min(cap, (C.fit_block * C.fit_nslot + 1) / 4));
    if (need(lo) > C.fit_nslot) return 1;  // cannot happen for a shape the host chose
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (need(mid) <= C.fit_nslot) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Builds this phase's sweep jobs and work items (one item = item_quads quads
// of one start) for every start that is not done, and resets the queue cursor.
// One thread per start sizes its items; the items are then written by one warp
// per start, a lane per item.
__global__ void __launch_bounds__(kBigBlock)
    k_plan(Slot *slots, SolveConsts C, SweepJob *jobs, WorkItem *items, int32_t *nitems,
           int32_t *queue, int32_t *nactive)
{
    __shared__ int s_warp[32];
    __shared__ int s_off[kBigBlock], s_groups[kBigBlock], s_qn[kBigBlock], s_nquads[kBigBlock];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int carry = 0;
    for (int base = 0; base < C.nslots; base += blockDim.x) {
        const int si = base + threadIdx.x;
        int groups = 0, qn = 1, nquads = 0;
        if (si < C.nslots) {
            Slot &s = slots[si];
            if (s.mode != kDone) {
                const int S = phase_samples(C, s.mode);
                // this launch's sweep range; a later chunk resumes from the states the
                // previous one wrote (every work item reads its own rows before it writes them)
                const int t0 = s.tsw;
                const int t1 = C.chunk > 0 ? min(C.T, t0 + C.chunk) : C.T;
                SweepJob j;
                j.prob = s.cur;
                j.spins = s.spins;
                j.energies = s.rec_e + (size_t)s.phase * C.Smax;
                j.seed = s.seed;
                j.S = S;
                j.W = s.W0;
                j.start = s.start;
                j.phase = (uint32_t)s.phase;
                j.init = t0 > 0 ? s.spins : nullptr;
                j.t0 = t0;
                j.t1 = t1;
                jobs[si] = j;
                nquads = ceil_div(S, 4);
                qn = item_quads(s.cur, C, nquads);
                groups = ceil_div(nquads, qn);
                if (t0 == 0) {
                    s.rec_count[s.phase] = S;
                    s.rec_nfree[s.phase] = s.cur->n;
                    s.nfixed = 0;
                }
                s.tsw = t1;
            }
        }
        int tot;
        const int ex = block_scan_excl(groups, s_warp, &tot);
        s_off[threadIdx.x] = carry + ex;
        s_groups[threadIdx.x] = groups;
        s_qn[threadIdx.x] = qn;
        s_nquads[threadIdx.x] = nquads;
        __syncthreads();
        const int nb = min((int)blockDim.x, C.nslots - base);
        for (int k = warp; k < nb; k += (int)(blockDim.x >> 5)) {
            const int g_n = s_groups[k], q_n = s_qn[k], nq = s_nquads[k], o = s_off[k];
            for (int g = lane; g < g_n; g += 32) {
                WorkItem w;
                w.job = base + k;
                w.quad0 = g * q_n;
                w.nq = min(q_n, nq - g * q_n);
                w.pad = 0;
                items[o + g] = w;
            }
        }
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *nitems = carry;
        *queue = 0;
        if (nactive) *nactive = 0;  // the persistence pass counts the starts still active
    }
}

// The per-step kernels of the persistence pass, one CTA per start, used when
// tree pre-processing follows each fold/compact (k_pass_slots does all of it
// otherwise).
// Elite sample of each active start; also keeps the start's best assignment
// (lifted to the original variables through its fix map).
__global__ void __launch_bounds__(kBigBlock) k_elite_slots(Slot *slots, SolveConsts C)
{
    extern __shared__ __align__(16) unsigned long long s_key[];
    __shared__ int s_better;
    Slot &s = slots[blockIdx.x];
    if (s.mode == kDone || !sample_complete(s, C)) return;
    // PTICM: the sample is the states its run kept
    const int S = C.pticm ? s.rec_count[s.phase] : phase_samples(C, s.mode);
    const int k = (s.mode == kFixing) ? (C.pticm ? elite_count_hd(C.elite, S) : C.k_fix)
                  : (s.mode == kCorr) ? C.k_corr : 1;
    const int64_t *e = s.rec_e + (size_t)s.phase * C.Smax;
    elite_fast(e, S, k, s.elite, s_key);
    const int rbest = s.elite[0];
    const int64_t eb = e[rbest];
    if (threadIdx.x == 0) {
        s_better = eb < *s.best_e;
        if (s_better) *s.best_e = eb;
    }
    __syncthreads();
    if (!s_better) return;
    for (int o = threadIdx.x; o < s.n0; o += blockDim.x) s.best_state[o] = s.fmap[o];
    __syncthreads();
    const int n = s.cur->n;
    const int32_t *orig = s.orig[s.ocur];
    const uint32_t *row = s.spins + (size_t)rbest * s.W0;
    for (int a = threadIdx.x; a < n; a += blockDim.x)
        s.best_state[orig[a]] = ((row[a >> 5] >> (a & 31)) & 1u) ? 1 : -1;
    if (C.tree) {
        // spins removed by tree inference, latest first: s_child = sigma s_parent
        __syncthreads();
        if (threadIdx.x == 0)
            for (int q = s.nlog - 1; q >= 0; --q)
                s.best_state[s.log_child[q]] = (int8_t)(s.log_sigma[q] * s.best_state[s.log_parent[q]]);
    }
}

__global__ void __launch_bounds__(kCountBlock) k_count_slots(Slot *slots, SolveConsts C)
{
    __shared__ CountSmem sm;
    Slot &s = slots[blockIdx.y];
    if ((s.mode != kFixing && s.mode != kCorr) || !sample_complete(s, C)) return;
    const DevProb *P = s.cur;
    if ((int)(blockIdx.x * 1024) >= P->n) return;
    if (s.mode == kCorr) {
        // correlation fixing: elite rows multiplied by their value at rho, then the
        // rule with the correlation threshold
        count_bs_core(P, s.spins, s.W0, s.elite, C.k_corr, 1, C.corr_num, C.corr_den, s.counts, s.fixed,
                      &s.nfixed, s.fmap, s.orig[s.ocur], blockIdx.x, sm);
        return;
    }
    const int canon = (C.canon < 0) ? P->hzero : C.canon;
    const int k = C.pticm ? elite_count_hd(C.elite, s.rec_count[s.phase]) : C.k_fix;
    count_bs_core(P, s.spins, s.W0, s.elite, k, canon, C.fix_num, C.fix_den, s.counts, s.fixed, &s.nfixed, s.fmap,
                  s.orig[s.ocur], blockIdx.x, sm);
}

// Stall rule, fold/compact into the spare buffer, and the phase transition.
__global__ void __launch_bounds__(kBigBlock) k_reduce_slots(Slot *slots, SolveConsts C)
{
    Slot &s = slots[blockIdx.x];
    const int mode = s.mode;
    if (mode == kDone || !sample_complete(s, C)) return;
    __syncthreads();  // every thread has read the slot's state before thread 0 moves it on
    if (mode == kSolving) {
        if (threadIdx.x == 0) {
            s.phase += 1;
            *s.nphases = s.phase;
            s.mode = kDone;
            s.tsw = 0;
        }
        return;
    }
    const DevProb *P = s.cur;
    const int n = P->n;
    const int32_t *orig = s.orig[s.ocur];
    if (threadIdx.x == 0 && mode == kFixing && C.iterate && s.nfixed == 0 && n > 0) {
        // nothing fixed: fix the lowest-index spin to its value in the best
        // elite sample so that every SPVAR phase makes progress
        const uint32_t w = s.spins[(size_t)s.elite[0] * s.W0];
        const int8_t v = (w & 1u) ? 1 : -1;
        s.fixed[0] = v;
        s.fmap[orig[0]] = v;
    }
    __syncthreads();
    DevProb *D = s.buf[s.next];
    reduce_core(P, D, s.fixed, s.old_of_new, s.scratch);
    int m = D->n;
    int32_t *orig2 = s.orig[s.ocur ^ 1];
    for (int a = threadIdx.x; a < m; a += blockDim.x) orig2[a] = orig[s.old_of_new[a]];
    __syncthreads();
    DevProb *cur2 = D;
    int next2 = s.next ^ 1, ocur2 = s.ocur ^ 1;
    if (C.tree && m > 0) {
        // exact tree reduction of the new problem (in place), then drop what it removed
        tree_core(D, s.fixed, s.scratch, s.fmap, orig2, s.log_child, s.log_parent, s.log_sigma, &s.nlog);
        DevProb *E2 = s.buf[s.next ^ 1];  // the problem sampled this phase is no longer needed
        reduce_core(D, E2, s.fixed, s.old_of_new, s.scratch, false);
        m = E2->n;
        int32_t *orig3 = s.orig[s.ocur];  // the start's map before this phase is no longer needed
        for (int a = threadIdx.x; a < m; a += blockDim.x) orig3[a] = orig2[s.old_of_new[a]];
        __syncthreads();
        cur2 = E2;
        next2 = s.next;
        ocur2 = s.ocur;
    }
    if (threadIdx.x == 0) {
        s.cur = cur2;
        s.next = next2;
        s.ocur = ocur2;
        s.phase += 1;
        s.tsw = 0;
        *s.nphases = s.phase;
        if (mode == kCorr) {
            s.mode = kFixing;  // the SPVAR phases follow the correlation phase
        } else {
            s.fix_done += 1;
            if (C.iterate && m > 0 && s.fix_done < C.max_fix) s.mode = kFixing;
            else s.mode = (C.S_solve > 0) ? kSolving : kDone;
        }
    }
}

// ------------------------------------------- the persistence pass, fused (Alg. 1)
// After a start's sample is complete, one thread-block cluster of
// kPassCluster CTAs runs the whole of Alg. 1 for it in one launch:
//   1. elite sample (rank 0 selects it; every other CTA finds only the best
//      sample and, after the first barrier, copies rank 0's list from its
//      shared memory over the cluster), and the start's best assignment;
//   2. persistence counts and the fixing rule, 1024 spins per count chunk;
//   3. the stall rule (ISPVAR), then the update of J and h spread over chunks
//      of kFoldChunk spins:
//        fold_count  per spin: folded bias, free-free row length, energy of
//                    the fixed spins; per chunk: the totals fold_index offsets by;
//        fold_index  new indices, h', row pointers, inherited colours and
//                    sweep positions (each chunk adds the totals of the chunks
//                    before it), and the new header (chunk 0);
//        fold_fill   CSR columns and values and the ELL layout of the free spins;
//   4. the phase transition and the count of active starts.
// Chunks are dealt to the cluster's CTAs round-robin, and a cluster barrier
// stands where one stage reads what another CTA wrote in the stage before.
// Each stage issues its global loads for all of a CTA's chunks (up to two,
// or kIndexBatch for the index stage) before it uses any of them.  A
// neighbour's fixing, and then its new index and position packed in one word,
// are single global loads; these per-start arrays (n bytes and 4n bytes) stay
// in L1 and L2, which measured faster than reading them from the owning CTA's
// shared memory over the cluster.  The result is the one the per-start
// kernels (elite, count_bs_core, reduce_core) compute: free spins keep their
// order, couplers between free spins keep theirs, colour classes are inherited.
constexpr int kPassCluster = 8;
constexpr int kPassBlock = kFoldChunk;  // one spin per thread in a fold chunk
constexpr int kFoldGather = 4;          // CSR entries of each row a thread loads at once
constexpr int kIndexBatch = 4;          // fold chunks a CTA indexes after one round of loads
// Four resident CTAs per SM (64 registers): 64 starts (512 CTAs) run in one wave.
constexpr int kPassMinBlocks = 4;
static_assert(kPassBlock == kCountBlock, "the count chunks run on the pass CTAs");
static_assert(SPVAR_MAX_N <= 32768, "new index and position are packed in 16 bits each");

// Cluster barrier: its arrive releases and its wait acquires at cluster
// scope, so every write (global or shared) a CTA makes before it is visible to
// the cluster's other CTAs after it.
__device__ __forceinline__ void pass_barrier() { cg::this_cluster().sync(); }

// New index | position << 16 of every old spin (~0 if fixed), in the slot's
// scratch area (the one-CTA reduction keeps its new indices there).
__device__ __forceinline__ uint32_t *npos_of(const Slot &s) { return reinterpret_cast<uint32_t *>(s.scratch); }

// Chunks ch[0..G) of the CTA (-1: none) at once, so that the loads of all of
// them are in flight together.
template <int G>
__device__ __forceinline__ void fold_count(Slot &s, const int (&ch)[G])
{
    __shared__ int s_cls[G][kMaxColours];
    __shared__ int s_free[G], s_nnz[G], s_hnz[G];
    __shared__ unsigned long long s_key[G], s_off[G];
    const DevProb *P = s.cur;
    const int n = P->n, cap = P->cap_n, tid = threadIdx.x;
    for (int x = tid; x < G * kMaxColours; x += kPassBlock) s_cls[x / kMaxColours][x % kMaxColours] = 0;
    if (tid < G) {
        s_free[tid] = s_nnz[tid] = s_hnz[tid] = 0;
        s_key[tid] = 0ull;
        s_off[tid] = 0ull;
    }
    __syncthreads();
    int32_t *rowcnt = s.scratch + cap, *hfold = s.scratch + 2 * cap;
    int i[G], vi[G], p0[G], p1[G], nf[G], h0[G], cl[G];
    long long hf[G], off[G];
    bool ok[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        i[g] = ch[g] * kFoldChunk + tid;
        ok[g] = ch[g] >= 0 && i[g] < n;
        vi[g] = ok[g] ? s.fixed[i[g]] : 0;
        h0[g] = ok[g] ? P->h[i[g]] : 0;
        cl[g] = ok[g] ? P->colour[i[g]] : -1;
        p0[g] = ok[g] ? P->row_ptr[i[g]] : 0;
        p1[g] = ok[g] ? P->row_ptr[i[g] + 1] : 0;
        hf[g] = h0[g];
        nf[g] = 0;
        off[g] = 0;
    }
    int len = 0;
#pragma unroll
    for (int g = 0; g < G; ++g) len = max(len, p1[g] - p0[g]);
    for (int d0 = 0; d0 < len; d0 += kFoldGather) {
        // kFoldGather entries of every row: all loads issued before any is used
        int jj[G][kFoldGather], vv[G][kFoldGather], fj[G][kFoldGather];
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int d = 0; d < kFoldGather; ++d) {
                const bool in = p0[g] + d0 + d < p1[g];
                jj[g][d] = in ? P->col[p0[g] + d0 + d] : -1;
                vv[g][d] = in ? P->val[p0[g] + d0 + d] : 0;
            }
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int d = 0; d < kFoldGather; ++d) fj[g][d] = jj[g][d] >= 0 ? s.fixed[jj[g][d]] : 0;
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int d = 0; d < kFoldGather; ++d) {
                if (jj[g][d] < 0) continue;
                if (vi[g]) {
                    if (fj[g][d] && jj[g][d] > i[g]) off[g] += (long long)vv[g][d] * vi[g] * fj[g][d];
                } else if (fj[g][d]) {
                    hf[g] += (long long)vv[g][d] * fj[g][d];
                } else {
                    ++nf[g];
                }
            }
    }
    const unsigned full = 0xFFFFFFFFu;
    const int lane = tid & 31;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        int nfree = 0, nnz = 0, hnz = 0, col = -1;
        unsigned long long key = 0ull;
        long long o = 0;
        if (ok[g]) {
            if (vi[g]) {
                o = off[g] + (long long)h0[g] * vi[g];
            } else {
                hfold[i[g]] = (int32_t)hf[g];
                rowcnt[i[g]] = nf[g];
                nfree = 1;
                nnz = nf[g];
                hnz = hf[g] != 0;
                col = cl[g];
                // reference spin of the new problem: largest degree, lowest index
                key = ((unsigned long long)nf[g] << 32) | (unsigned long long)(0x7FFFFFFF - i[g]);
            }
        }
        // one shared atomic per warp (and per colour class present in the warp)
        const unsigned same = __match_any_sync(full, col);
        if (col >= 0 && lane == __ffs(same) - 1) atomicAdd(&s_cls[g][col], __popc(same));
        nfree = __reduce_add_sync(full, nfree);
        nnz = __reduce_add_sync(full, nnz);
        hnz = __reduce_or_sync(full, hnz);
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) {
            key = max(key, __shfl_xor_sync(full, key, sh));
            o += __shfl_xor_sync(full, o, sh);
        }
        if (lane == 0 && ch[g] >= 0) {
            atomicAdd(&s_free[g], nfree);
            atomicAdd(&s_nnz[g], nnz);
            if (hnz) atomicOr(&s_hnz[g], 1);
            atomicMax(&s_key[g], key);
            atomicAdd(&s_off[g], (unsigned long long)o);
        }
    }
    __syncthreads();
    int32_t *tab = s.scratch + fold_table_offset(cap);
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (ch[g] < 0 || ch[g] * kFoldChunk >= n) continue;
        int32_t *e = tab + ch[g] * kFoldStride;
        if (tid == 0) {
            e[0] = s_free[g];
            e[1] = s_nnz[g];
            e[2] = s_hnz[g];
            e[3] = (int32_t)(s_key[g] >> 32);
            e[4] = (int32_t)(s_key[g] & 0xFFFFFFFFull);
            atomicAdd(reinterpret_cast<unsigned long long *>(tab + kFoldMaxChunks * kFoldStride), s_off[g]);
        }
        for (int c = tid; c < P->ncol; c += kPassBlock) e[6 + c] = s_cls[g][c];
    }
    __syncthreads();  // the shared totals are reset by this CTA's next chunks
}

constexpr int kScanCols = 6;  // colour classes ranked per multi-value scan

// Chunks ch[0..CB) of the CTA (-1: none).  The spins' own values and the
// table of chunk totals are loaded once for all of them, so the chunks' scans
// follow one another without a global load in between.
template <int CB>
__device__ __forceinline__ void fold_index(Slot &s, const int (&ch)[CB])
{
    __shared__ int s_w[32 * (2 + kScanCols)];
    __shared__ int s_base_cls[CB][kMaxColours], s_tot_cls[kMaxColours], s_cptr[kMaxColours + 1];
    __shared__ int s_base[CB][2], s_tot[2], s_hnz;
    const DevProb *P = s.cur;
    DevProb *D = s.buf[s.next];
    const int n = P->n, cap = P->cap_n, ncol = P->ncol, tid = threadIdx.x;
    const int nch = (n + kFoldChunk - 1) / kFoldChunk;
    const int32_t *tab = s.scratch + fold_table_offset(cap);
    // a chunk takes part if it holds spins; chunk 0 also writes the header, even for n = 0
    bool on[CB];
#pragma unroll
    for (int b = 0; b < CB; ++b) on[b] = ch[b] >= 0 && (ch[b] == 0 || ch[b] * kFoldChunk < n);
    // the spins' own values first (they do not wait for the table)
    const int32_t *rowcnt = s.scratch + cap, *hfold = s.scratch + 2 * cap;
    const int32_t *orig = s.orig[s.ocur];
    bool f[CB], valid[CB];
    int rc[CB], colv[CB], h[CB], oi[CB];
#pragma unroll
    for (int b = 0; b < CB; ++b) {
        const int i = ch[b] * kFoldChunk + tid;
        valid[b] = on[b] && i < n;
        f[b] = valid[b] && s.fixed[i] == 0;
        rc[b] = valid[b] ? rowcnt[i] : 0;
        colv[b] = valid[b] ? P->colour[i] : -1;
        h[b] = valid[b] ? hfold[i] : 0;
        oi[b] = valid[b] ? orig[i] : 0;
    }
    // offsets of each chunk (totals of the chunks before it) and the totals of all:
    // field f (0 free spins, 1 free-free entries, 2 + c spins of class c) summed by a warp
    {
        const int lane = tid & 31, warp = tid >> 5;
        for (int fld = warp; fld < 3 + ncol; fld += kPassBlock / 32) {
            const int fo = fld < 3 ? fld : 6 + (fld - 3);  // table column (2: nonzero-bias flag)
            int bs[CB], t = 0;
#pragma unroll
            for (int b = 0; b < CB; ++b) bs[b] = 0;
            for (int q = lane; q < nch; q += 32) {
                const int v = tab[q * kFoldStride + fo];
                t += fld == 2 ? (v != 0) : v;
#pragma unroll
                for (int b = 0; b < CB; ++b) bs[b] += q < ch[b] ? v : 0;
            }
#pragma unroll
            for (int b = 0; b < CB; ++b) bs[b] = __reduce_add_sync(0xFFFFFFFFu, bs[b]);
            t = __reduce_add_sync(0xFFFFFFFFu, t);
            if (lane == 0) {
                if (fld < 2) {
                    s_tot[fld] = t;
#pragma unroll
                    for (int b = 0; b < CB; ++b) s_base[b][fld] = bs[b];
                } else if (fld == 2) {
                    s_hnz = t;
                } else {
                    s_tot_cls[fld - 3] = t;
#pragma unroll
                    for (int b = 0; b < CB; ++b) s_base_cls[b][fld - 3] = bs[b];
                }
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        int c0 = 0;
        for (int c = 0; c < ncol; ++c) {
            s_cptr[c] = c0;
            c0 += s_tot_cls[c];
        }
        s_cptr[ncol] = c0;
    }
    __syncthreads();
    if (ch[0] == 0 && tid <= ncol) D->cptr[tid] = s_cptr[tid];
    if (ch[0] == 0 && tid == 0) {
        const int m = s_tot[0], nnz2 = s_tot[1];
        D->n = m;
        D->nnz = nnz2;
        D->ncol = ncol;
        D->maxdeg = P->maxdeg;
        D->dmax = P->dmax;
        D->hzero = s_hnz ? 0 : 1;
        D->pm1 = P->pm1;
        D->ujs = P->ujs;
        D->scale = P->scale;
        D->offset = P->offset +
                    (long long)*reinterpret_cast<const unsigned long long *>(tab + kFoldMaxChunks * kFoldStride);
        D->row_ptr[m] = nnz2;
    }
    // the output arrays in locals: a store through one of them cannot change where the others are
    int32_t *__restrict__ orig2 = s.orig[s.ocur ^ 1];
    int32_t *__restrict__ oon = s.old_of_new;
    uint32_t *__restrict__ npos = npos_of(s);
    int32_t *__restrict__ dh = D->h, *__restrict__ dcolour = D->colour, *__restrict__ drow = D->row_ptr;
    int32_t *__restrict__ dpos = D->pos_of_idx, *__restrict__ didx = D->idx_of_pos;
    uint32_t *__restrict__ dmeta = D->meta;
#pragma unroll
    for (int b = 0; b < CB; ++b) {
        if (!on[b] || ch[b] * kFoldChunk >= n) continue;  // uniform over the CTA
        const int i = ch[b] * kFoldChunk + tid;
        const int col = f[b] ? colv[b] : -1;
        // new index, row pointer and rank among the chunk's free spins of the same
        // colour class: one multi-value scan per group of kScanCols classes
        int exf = 0, exr = 0, rank = 0;
        for (int cb = 0; cb < max(ncol, 1); cb += kScanCols) {
            int v[2 + kScanCols], ex[2 + kScanCols], tot[2 + kScanCols];
            v[0] = cb == 0 && f[b] ? 1 : 0;
            v[1] = cb == 0 && f[b] ? rc[b] : 0;
#pragma unroll
            for (int q = 0; q < kScanCols; ++q) v[2 + q] = col == cb + q ? 1 : 0;
            block_scan_multi<2 + kScanCols>(v, ex, tot, s_w);
            if (cb == 0) {
                exf = ex[0];
                exr = ex[1];
            }
#pragma unroll
            for (int q = 0; q < kScanCols; ++q)
                if (col == cb + q) rank = s_base_cls[b][col] + ex[2 + q];
        }
        const int a = s_base[b][0] + exf;
        const int pos = f[b] ? s_cptr[col] + rank : 0;
        if (valid[b]) npos[i] = f[b] ? (uint32_t)a | ((uint32_t)pos << 16) : ~0u;
        if (f[b]) {
            oon[a] = i;
            orig2[a] = oi[b];
            dh[a] = h[b];
            dcolour[a] = col;
            drow[a] = s_base[b][1] + exr;
            dpos[a] = pos;
            didx[pos] = a;
            dmeta[pos] = ((uint32_t)(h[b] & 0xFFFF) << 16) | (uint32_t)rc[b];
        }
    }
    __syncthreads();  // the shared offsets are rewritten by this CTA's next chunks
}

template <int G>
__device__ __forceinline__ void fold_fill(Slot &s, const int (&ch)[G])
{
    const uint32_t *__restrict__ npos = npos_of(s);
    const DevProb *P = s.cur;
    DevProb *D = s.buf[s.next];
    const int n = P->n, cap = P->cap_n, tid = threadIdx.x;
    // the arrays in locals: a store through one of them cannot change where the others are
    const int32_t *__restrict__ prow = P->row_ptr, *__restrict__ pcol = P->col, *__restrict__ pval = P->val;
    const int32_t *__restrict__ drow = D->row_ptr;
    int32_t *__restrict__ dcol = D->col, *__restrict__ dval = D->val;
    uint32_t *__restrict__ dell = D->ell;
    if (ch[0] == 0 && tid == 0) {
        // the reference spin: the chunks' candidates, largest degree then lowest index
        const int32_t *tab = s.scratch + fold_table_offset(cap);
        unsigned long long best = 0ull;
        bool any = false;
        for (int q = 0; q * kFoldChunk < n; ++q) {
            const int32_t *e = tab + q * kFoldStride;
            if (e[0] == 0) continue;
            const unsigned long long k = ((unsigned long long)(uint32_t)e[3] << 32) | (uint32_t)e[4];
            best = max(best, k);
            any = true;
        }
        D->rho = any ? (int)(npos[0x7FFFFFFF - (int)(best & 0xFFFFFFFFull)] & 0xFFFFu) : -1;
    }
    int p0[G], p1[G], q[G], pos[G], d[G];
    uint32_t own[G];
    // the spin's new index and position, and its row bounds (which do not wait for them)
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int i = ch[g] * kFoldChunk + tid;
        const bool ok = ch[g] >= 0 && i < n;
        own[g] = ok ? npos[i] : ~0u;  // ~0: fixed
        p0[g] = ok ? prow[i] : 0;
        p1[g] = ok ? prow[i + 1] : 0;
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const bool free = own[g] != ~0u;  // free spins only
        if (!free) p1[g] = p0[g];
        q[g] = free ? drow[own[g] & 0xFFFFu] : 0;
        pos[g] = (int)(own[g] >> 16);
        d[g] = 0;
    }
    int len = 0;
#pragma unroll
    for (int g = 0; g < G; ++g) len = max(len, p1[g] - p0[g]);
    for (int d0 = 0; d0 < len; d0 += kFoldGather) {
        // kFoldGather entries of every row: each dependent step loads for all of them
        int vv[G][kFoldGather];
        uint32_t np[G][kFoldGather];
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int e = 0; e < kFoldGather; ++e) {
                const bool in = p0[g] + d0 + e < p1[g];
                np[g][e] = in ? (uint32_t)pcol[p0[g] + d0 + e] : ~0u;
                vv[g][e] = in ? pval[p0[g] + d0 + e] : 0;
            }
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int e = 0; e < kFoldGather; ++e)
                np[g][e] = np[g][e] != ~0u ? npos[np[g][e]] : ~0u;
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int e = 0; e < kFoldGather; ++e) {
                if (np[g][e] == ~0u) continue;
                const uint32_t b = np[g][e] & 0xFFFFu, pp = np[g][e] >> 16;
                dcol[q[g]] = (int32_t)b;
                dval[q[g]] = vv[g][e];
                dell[(size_t)d[g] * cap + pos[g]] = pp | ((uint32_t)(vv[g][e] & 0xFFFF) << 16);
                ++q[g];
                ++d[g];
            }
    }
}

// Dynamic shared memory of the pass: the elite list (Smax entries), then one
// region that holds in turn the elite's candidate keys and energies and a
// count chunk's counters.
__host__ __device__ inline size_t pass_list_bytes(int Smax) { return ((size_t)Smax * 4 + 15) & ~(size_t)15; }
__host__ __device__ inline size_t pass_smem(int Smax)
{
    size_t u = (size_t)elite_key_words(Smax) * 8;
    if (u < (size_t)(kEliteRankMax + Smax) * 8) u = (size_t)(kEliteRankMax + Smax) * 8;  // keys, then energies
    if (u < sizeof(CountSmem)) u = sizeof(CountSmem);
    return pass_list_bytes(Smax) + u;
}

// The grid is kPassCluster x nslots with one cluster per row, so blockIdx.x
// is the CTA's rank in its cluster and every CTA of a cluster reads the same
// slot.  The slot's state is read by every CTA before the first barrier and
// changed only by rank 0 after the last one, so all CTAs of a cluster take
// the same path through the barriers.
__global__ void __cluster_dims__(kPassCluster, 1, 1) __launch_bounds__(kPassBlock, kPassMinBlocks)
    k_pass_slots(Slot *slots, SolveConsts C, int32_t *nactive)
{
    extern __shared__ __align__(16) unsigned long long s_dyn[];
    Slot &s = slots[blockIdx.y];
    const int rank = blockIdx.x, tid = threadIdx.x;
    const int mode = s.mode;
    if (mode == kDone || !sample_complete(s, C)) {
        // a start whose sample is still running stays active
        if (nactive && mode != kDone && rank == 0 && tid == 0) atomicAdd(nactive, 1);
        return;
    }
    int32_t *s_elite = reinterpret_cast<int32_t *>(s_dyn);
    unsigned char *s_reg = reinterpret_cast<unsigned char *>(s_dyn) + pass_list_bytes(C.Smax);
    // 1. elite sample (PTICM: of the states its run kept) and the best assignment
    const int S = C.pticm ? s.rec_count[s.phase] : phase_samples(C, mode);
    const int k = (mode == kFixing) ? (C.pticm ? elite_count_hd(C.elite, S) : C.k_fix)
                  : (mode == kCorr) ? C.k_corr : 1;
    const int64_t *e = s.rec_e + (size_t)s.phase * C.Smax;
    // rank 0 selects the whole elite, which the other CTAs copy from its shared
    // memory after the barrier; they need only its best sample before it
    elite_fast(e, S, rank == 0 ? k : 1, s_elite, reinterpret_cast<unsigned long long *>(s_reg),
               reinterpret_cast<int64_t *>(s_reg) + kEliteRankMax);
    const DevProb *P = s.cur;
    const int n = P->n;
    const int32_t *orig = s.orig[s.ocur];
    const int rbest = s_elite[0];
    const int64_t eb = e[rbest];
    const bool better = eb < *s.best_e;  // every CTA reads it before rank 0 may change it
    constexpr int kStride = kPassCluster * kPassBlock;
    int8_t *__restrict__ bstate = s.best_state;
    if (better) {
        // spins fixed in earlier phases, before this phase adds its fixings to fmap
        // (four loads in flight per thread)
        const int n0 = s.n0;
        const int8_t *__restrict__ fm = s.fmap;
        for (int o0 = rank * kPassBlock + tid; o0 < n0; o0 += 4 * kStride) {
            int8_t v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = o0 + u * kStride < n0 ? fm[o0 + u * kStride] : 0;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (v[u]) bstate[o0 + u * kStride] = v[u];
        }
    }
    if (rank == 0) {
        for (int q = tid; q < k; q += kPassBlock) s.elite[q] = s_elite[q];
        if (tid == 0 && mode != kSolving)
            *reinterpret_cast<unsigned long long *>(s.scratch + fold_table_offset(P->cap_n) +
                                                    kFoldMaxChunks * kFoldStride) = 0ull;
    }
    pass_barrier();
    if (rank != 0 && k > 1) {
        const int32_t *r0 = cg::this_cluster().map_shared_rank(s_elite, 0);
        for (int q = tid; q < k; q += kPassBlock) s_elite[q] = r0[q];
        __syncthreads();
    }
    if (better) {
        if (rank == 0 && tid == 0) *s.best_e = eb;
        const uint32_t *row = s.spins + (size_t)rbest * s.W0;
        for (int a0 = rank * kPassBlock + tid; a0 < n; a0 += 4 * kStride) {
            int o[4];
            uint32_t w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int a = a0 + u * kStride;
                o[u] = a < n ? orig[a] : -1;
                w[u] = a < n ? row[a >> 5] : 0u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (o[u] >= 0) bstate[o[u]] = ((w[u] >> ((a0 + u * kStride) & 31)) & 1u) ? 1 : -1;
        }
    }
    if (mode == kSolving) {
        if (rank == 0 && tid == 0) {
            s.phase += 1;
            *s.nphases = s.phase;
            s.mode = kDone;
            s.tsw = 0;
        }
        return;
    }
    // 2. counts and the fixing rule (correlation fixing: rows times their value at rho)
    const bool corr = mode == kCorr;
    const int canon = corr ? 1 : (C.canon < 0 ? P->hzero : C.canon);
    for (int c = rank; c * 1024 < n; c += kPassCluster)
        count_bs_core(P, s.spins, s.W0, s_elite, k, canon, corr ? C.corr_num : C.fix_num,
                      corr ? C.corr_den : C.fix_den, s.counts, s.fixed, &s.nfixed, s.fmap, orig, c,
                      *reinterpret_cast<CountSmem *>(s_reg));
    pass_barrier();
    // 3. stall rule: nothing fixed in an ISPVAR phase fixes the lowest-index spin
    //    to its value in the best elite sample, so that every phase makes progress
    if (mode == kFixing && C.iterate && s.nfixed == 0 && n > 0) {
        if (rank == 0 && tid == 0) {
            const int8_t v = (s.spins[(size_t)s_elite[0] * s.W0] & 1u) ? 1 : -1;
            s.fixed[0] = v;
            s.fmap[orig[0]] = v;
        }
        pass_barrier();
    }
    const int nch = max(1, (n + kFoldChunk - 1) / kFoldChunk);
    // this CTA's chunks rank, rank + kPassCluster, ..., two at a time in the gather stages
    for (int c = rank; c < nch; c += 2 * kPassCluster) {
        const int ch[2] = {c, c + kPassCluster < nch ? c + kPassCluster : -1};
        fold_count<2>(s, ch);
    }
    pass_barrier();
    for (int c = rank; c < nch; c += kIndexBatch * kPassCluster) {
        int ch[kIndexBatch];
#pragma unroll
        for (int b = 0; b < kIndexBatch; ++b) ch[b] = c + b * kPassCluster < nch ? c + b * kPassCluster : -1;
        fold_index<kIndexBatch>(s, ch);
    }
    pass_barrier();
    for (int c = rank; c < nch; c += 2 * kPassCluster) {
        const int ch[2] = {c, c + kPassCluster < nch ? c + kPassCluster : -1};
        fold_fill<2>(s, ch);
    }
    pass_barrier();
    // 4. the phase transition
    if (rank == 0 && tid == 0) {
        DevProb *D = s.buf[s.next];
        const int m = D->n;
        s.cur = D;
        s.next ^= 1;
        s.ocur ^= 1;
        if (corr) {
            s.mode = kFixing;  // the SPVAR phases follow the correlation phase
        } else {
            s.fix_done += 1;
            if (C.iterate && m > 0 && s.fix_done < C.max_fix) s.mode = kFixing;
            else s.mode = (C.S_solve > 0) ? kSolving : kDone;
        }
        s.phase += 1;
        s.tsw = 0;
        *s.nphases = s.phase;
        if (nactive && s.mode != kDone) atomicAdd(nactive, 1);
    }
}

__global__ void k_count_active(const Slot *slots, int nslots, int32_t *nactive)
{
    __shared__ int s_n;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    int c = 0;
    for (int i = threadIdx.x; i < nslots; i += blockDim.x) c += (slots[i].mode != kDone) ? 1 : 0;
    atomicAdd(&s_n, c);
    __syncthreads();
    if (threadIdx.x == 0) *nactive = s_n;
}

// ------------------------------------------------ component boosting (Sec. II.C)
// Components of the current problem by min-label propagation with pointer
// jumping; numbered in increasing order of their lowest spin index.
__global__ void __launch_bounds__(kBigBlock) k_boost_components(Slot *slots, SolveConsts C)
{
    __shared__ int s_warp[32];
    __shared__ int s_changed;
    Slot &s = slots[blockIdx.x];
    if (s.mode != kSolving || !sample_complete(s, C)) return;
    const DevProb *P = s.cur;
    const int n = P->n;
    int32_t *lab = s.comp;
    for (int i = threadIdx.x; i < n; i += blockDim.x) lab[i] = i;
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) s_changed = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            int m = lab[i];
            for (int p = P->row_ptr[i]; p < P->row_ptr[i + 1]; ++p) m = min(m, lab[P->col[p]]);
            if (m < lab[i]) {
                atomicMin(&lab[i], m);
                s_changed = 1;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            int l = lab[i];
            while (lab[l] != l) l = lab[l];
            lab[i] = l;
        }
        __syncthreads();
        const int ch = s_changed;
        __syncthreads();
        if (!ch) break;
    }
    // rank of each root (a root is the lowest index of its component)
    int32_t *rank = s.scratch;
    int carry = 0;
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int f = (i < n && lab[i] == i) ? 1 : 0;
        int tot;
        const int ex = block_scan_excl(f, s_warp, &tot);
        if (f) rank[i] = carry + ex;
        carry += tot;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) lab[i] = rank[lab[i]];
    if (threadIdx.x == 0) s.ncomp = carry;
}

// Twice the partial energy of sample r on every component (one CTA per sample).
__global__ void __launch_bounds__(256) k_boost_partial(Slot *slots, SolveConsts C)
{
    extern __shared__ int s_acc[];
    Slot &s = slots[blockIdx.y];
    const int r = blockIdx.x;
    if (s.mode != kSolving || !sample_complete(s, C) || r >= C.S_solve) return;
    const DevProb *P = s.cur;
    const int n = P->n, m = s.ncomp;
    for (int c = threadIdx.x; c < m; c += blockDim.x) s_acc[c] = 0;
    __syncthreads();
    const uint32_t *row = s.spins + (size_t)r * s.W0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int si = ((row[i >> 5] >> (i & 31)) & 1u) ? 1 : -1;
        int v = 2 * P->h[i] * si;
        for (int p = P->row_ptr[i]; p < P->row_ptr[i + 1]; ++p) {
            const int j = P->col[p];
            const int sj = ((row[j >> 5] >> (j & 31)) & 1u) ? 1 : -1;
            v += P->val[p] * si * sj;
        }
        atomicAdd(&s_acc[s.comp[i]], v);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < m; c += blockDim.x) s.part[(size_t)r * s.n0 + c] = s_acc[c];
}

// Each component's samples ordered by (partial energy, sample index).
__global__ void __launch_bounds__(kBigBlock) k_boost_sort(Slot *slots, SolveConsts C)
{
    extern __shared__ __align__(16) unsigned long long s_key[];
    Slot &s = slots[blockIdx.y];
    const int c = blockIdx.x;
    if (s.mode != kSolving || !sample_complete(s, C) || c >= s.ncomp) return;
    const int S = C.S_solve;
    int N2 = 1;
    while (N2 < S) N2 <<= 1;
    for (int r = threadIdx.x; r < N2; r += blockDim.x)
        s_key[r] = (r < S) ? (((unsigned long long)((unsigned)s.part[(size_t)r * s.n0 + c] ^ 0x80000000u) << 32) |
                              (unsigned)r)
                           : ~0ull;
    __syncthreads();
    for (int size = 2; size <= N2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < N2; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const unsigned long long a = s_key[i], b = s_key[j];
                    if ((a > b) == ((i & size) == 0)) {
                        s_key[i] = b;
                        s_key[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int r = threadIdx.x; r < S; r += blockDim.x) s.perm[(size_t)c * C.Smax + r] = (int)(s_key[r] & 0xFFFFFFFFull);
}

// Rank r of the merged sample: each component's r-th partial state; its
// energy (with offset) replaces the recorded one.  One CTA per rank.
__global__ void __launch_bounds__(256) k_boost_merge(Slot *slots, SolveConsts C)
{
    __shared__ long long s_e;
    Slot &s = slots[blockIdx.y];
    const int r = blockIdx.x;
    if (s.mode != kSolving || !sample_complete(s, C) || r >= C.S_solve) return;
    const DevProb *P = s.cur;
    const int n = P->n, m = s.ncomp;
    if (threadIdx.x == 0) s_e = 0;
    __syncthreads();
    long long e = 0;
    for (int c = threadIdx.x; c < m; c += blockDim.x) e += s.part[(size_t)s.perm[(size_t)c * C.Smax + r] * s.n0 + c];
    atomicAdd((unsigned long long *)&s_e, (unsigned long long)e);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Wn = (n + 31) >> 5;
    for (int w = warp; w < Wn; w += blockDim.x / 32) {
        const int i = 32 * w + lane;
        unsigned b = 0;
        if (i < n) {
            const int src = s.perm[(size_t)s.comp[i] * C.Smax + r];
            b = (s.spins[(size_t)src * s.W0 + w] >> lane) & 1u;
        }
        const unsigned bits = __ballot_sync(0xFFFFFFFFu, b);
        if (lane == 0) s.spins2[(size_t)r * s.W0 + w] = bits;
    }
    __syncthreads();
    if (threadIdx.x == 0) s.rec_e[(size_t)s.phase * C.Smax + r] = s_e / 2 + P->offset;
}

__global__ void __launch_bounds__(256) k_boost_copy(Slot *slots, SolveConsts C)
{
    Slot &s = slots[blockIdx.y];
    const int r = blockIdx.x;
    if (s.mode != kSolving || !sample_complete(s, C) || r >= C.S_solve) return;
    const int Wn = (s.cur->n + 31) >> 5;
    for (int w = threadIdx.x; w < Wn; w += blockDim.x) s.spins[(size_t)r * s.W0 + w] = s.spins2[(size_t)r * s.W0 + w];
}

__global__ void k_gather_modes(const Slot *slots, int nslots, int32_t *modes)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nslots; i += gridDim.x * blockDim.x)
        modes[i] = slots[i].mode;
}

size_t elite_smem(int S) { return (size_t)elite_key_words(S) * 8; }


}  // namespace

cudaError_t launch_boost(Slot *slots, const SolveConsts &C, cudaStream_t st)
{
    if (!C.boost || C.S_solve <= 0 || C.nslots <= 0) return cudaSuccess;
    k_boost_components<<<C.nslots, kBigBlock, 0, st>>>(slots, C);
    const size_t acc = 4 * (size_t)std::max(C.max_n0, 1);
    cudaFuncSetAttribute(k_boost_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)acc);
    k_boost_partial<<<dim3(C.S_solve, C.nslots), 256, acc, st>>>(slots, C);
    const size_t keys = elite_smem(C.S_solve);
    cudaFuncSetAttribute(k_boost_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)keys);
    k_boost_sort<<<dim3(std::max(C.max_n0, 1), C.nslots), kBigBlock, keys, st>>>(slots, C);
    k_boost_merge<<<dim3(C.S_solve, C.nslots), 256, 0, st>>>(slots, C);
    k_boost_copy<<<dim3(C.S_solve, C.nslots), 256, 0, st>>>(slots, C);
    return cudaGetLastError();
}

cudaError_t launch_gather_modes(const Slot *slots, int nslots, int32_t *modes, cudaStream_t st)
{
    if (nslots <= 0) return cudaSuccess;
    k_gather_modes<<<ceil_div(nslots, 256), 256, 0, st>>>(slots, nslots, modes);
    return cudaGetLastError();
}

int elite_max_samples() { return SPVAR_MAX_SAMPLES; }

cudaError_t launch_elite_single(const int64_t *energies, int S, int k, int32_t *elite,
                                cudaStream_t stream)
{
    const size_t smem = elite_smem(S);
    cudaFuncSetAttribute(k_elite_single, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_elite_single<<<1, kBigBlock, smem, stream>>>(energies, S, k, elite);
    return cudaGetLastError();
}

cudaError_t launch_count_single(const DevProb *prob, int n_host, const uint32_t *spins, int W,
                                const int32_t *elite, int k, int canon, int fix_num, int fix_den,
                                int32_t *counts, int8_t *fixed, int32_t *nfixed, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(nfixed, 0, sizeof(int32_t), stream);
    if (e != cudaSuccess) return e;
    if (n_host <= 0) return cudaSuccess;
    k_count_single<<<ceil_div(n_host, 1024), kCountBlock, 0, stream>>>(
        prob, spins, W, elite, k, canon, fix_num, fix_den, counts, fixed, nfixed);
    return cudaGetLastError();
}

cudaError_t launch_reduce_single(const DevProb *src, DevProb *dst, const int8_t *fixed,
                                 int32_t *old_of_new, int32_t *scratch, cudaStream_t stream)
{
    k_reduce_single<<<1, kBigBlock, 0, stream>>>(src, dst, fixed, old_of_new, scratch);
    return cudaGetLastError();
}

cudaError_t launch_slots_init(Slot *slots, const SolveConsts &C, int, cudaStream_t st)
{
    k_slots_init<<<C.nslots, 256, 0, st>>>(slots, C);
    return cudaGetLastError();
}

cudaError_t launch_plan(Slot *slots, const SolveConsts &C, SweepJob *jobs, WorkItem *items,
                        int32_t *nitems, int32_t *queue, int32_t *nactive, cudaStream_t st)
{
    k_plan<<<1, kBigBlock, 0, st>>>(slots, C, jobs, items, nitems, queue, nactive);
    return cudaGetLastError();
}

cudaError_t launch_elite_slots(Slot *slots, const SolveConsts &C, cudaStream_t st)
{
    const size_t smem = elite_smem(C.Smax);
    cudaFuncSetAttribute(k_elite_slots, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_elite_slots<<<C.nslots, kBigBlock, smem, st>>>(slots, C);
    return cudaGetLastError();
}

cudaError_t launch_count_slots(Slot *slots, const SolveConsts &C, int max_n0, cudaStream_t st)
{
    if (max_n0 <= 0) return cudaSuccess;
    dim3 grid(ceil_div(max_n0, 1024), C.nslots);
    k_count_slots<<<grid, kCountBlock, 0, st>>>(slots, C);
    return cudaGetLastError();
}

cudaError_t launch_pass_slots(Slot *slots, const SolveConsts &C, int32_t *nactive, cudaStream_t st)
{
    if (C.nslots <= 0) return cudaSuccess;
    const size_t smem = pass_smem(C.Smax);
    cudaError_t e = cudaFuncSetAttribute(k_pass_slots, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // the kernel's cluster shape (kPassCluster x 1 x 1) makes each grid row one cluster
    k_pass_slots<<<dim3(kPassCluster, C.nslots), kPassBlock, smem, st>>>(slots, C, nactive);
    return cudaGetLastError();
}

cudaError_t launch_reduce_slots(Slot *slots, const SolveConsts &C, int32_t *nactive,
                                cudaStream_t st)
{
    k_reduce_slots<<<C.nslots, kBigBlock, 0, st>>>(slots, C);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !nactive) return e;
    k_count_active<<<1, 256, 0, st>>>(slots, C.nslots, nactive);
    return cudaGetLastError();
}

}  // namespace spvar
