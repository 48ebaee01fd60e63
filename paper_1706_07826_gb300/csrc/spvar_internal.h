// Internal declarations of the SPVAR CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "spvar.h"

namespace spvar {

// Colour classes are bounded by a first-fit colouring: <= max degree + 1.
constexpr int kMaxColours = SPVAR_MAX_DEGREE + 1;
constexpr uint32_t kSweepBits = 20;                 // counter word 1 = phase << 20 | sweep
constexpr uint32_t kInitSlot = (1u << kSweepBits) - 1u;

// Device-resident problem: CSR in index order plus the sweep layout.
// "Positions" order the spins colour class by colour class, increasing index
// inside a class; the sweep kernels work in positions so that one colour is
// one contiguous range.  Everything lives in one device allocation with fixed
// capacities (cap_n, cap_nnz, maxdeg) so that reductions can be written in
// place of a buffer of the same capacity.
struct DevProb {
    int32_t n, nnz, ncol, maxdeg;  // maxdeg: ELL rows (an upper bound on every row length)
    int32_t dmax, hzero, pm1, rho; // rho: lowest-index spin of maximum degree (-1 if n == 0)
    int64_t offset;
    int32_t cap_n, cap_nnz, scale;
    int32_t ujs;         // 1: the couplers of every spin share one magnitude
    int32_t *row_ptr;    // [cap_n + 1]
    int32_t *col;        // [cap_nnz]
    int32_t *val;        // [cap_nnz]
    int32_t *h;          // [cap_n]
    int32_t *colour;     // [cap_n]
    int32_t *cptr;       // [kMaxColours + 1] position range of each colour
    int32_t *idx_of_pos; // [cap_n]
    int32_t *pos_of_idx; // [cap_n]
    uint32_t *meta;      // [cap_n] (h as int16) << 16 | degree, by position
    uint32_t *ell;       // [maxdeg][cap_n] (neighbour position) | (J as int16) << 16, by position
};

// Host handle of a problem: the device blob and a host copy of its header.
struct Problem {
    DevProb hdr;        // host copy (pointers are device pointers)
    int32_t csize[kMaxColours];  // colour class sizes
    int32_t jabs_max = 0;        // largest coupler magnitude
    DevProb *dev;       // device copy of the header (inside the blob)
    void *blob;
    size_t blob_bytes;
    int device;
};

// A validated problem with its sweep layout, built on the host.
struct HostProblem {
    DevProb hdr;  // scalar fields (pointers unset)
    int cap_n = 1, cap_nnz = 1, md = 1;
    std::vector<int32_t> row_ptr, col, val, h, colour, cptr, idx_of_pos, pos_of_idx;
    std::vector<uint32_t> meta, ell;  // ell: [md][cap_n]
};
// Validates a host CSR problem and builds colours and layout (SPVAR_* code).
int host_problem_build(int n, const int32_t *row_ptr, const int32_t *col, const int32_t *val, const int32_t *h,
                       int64_t offset, int scale, HostProblem &out);
// Uploads into a blob of prob_blob_bytes(cap_n, cap_nnz, md) bytes (stream-ordered;
// the host arrays must stay alive until the stream reaches the copies).
int host_problem_upload(const HostProblem &hp, void *blob, cudaStream_t st, DevProb *hdr_out);

size_t prob_blob_bytes(int cap_n, int cap_nnz, int maxdeg);
// Carve a blob into a header with device pointers; the header itself sits at blob offset 0.
void prob_carve(DevProb *hdr, void *blob, int cap_n, int cap_nnz, int maxdeg);

// One sample job: anneal replicas [0, S) of one problem.
struct SweepJob {
    const DevProb *prob;
    uint32_t *spins;    // [S][W] bit-packed output (W = words per row)
    int64_t *energies;  // [S] output (with offset)
    uint64_t seed;
    int32_t S, W;
    uint32_t start, phase;
    const uint32_t *init;  // [S][W] states to continue from, or null: the initial state
    int32_t t0;            // first sweep to run
    int32_t t1;            // end of the sweep range (exclusive); 0: the launch's T.  The launch runs
                           // sweeps t0 .. min(t1, T) - 1 of this job
};

// A unit of sweep work: quads [quad0, quad0 + nq) of job `job`.
struct WorkItem {
    int32_t job, quad0, nq, pad;
};

struct SweepLaunch {
    const SweepJob *jobs;   // device array, or nullptr: use `single`
    const WorkItem *items;  // device array (persistent queue), or nullptr: item = blockIdx.x
    const int32_t *nitems;  // device counter of items (queue mode)
    int32_t *queue;         // device atomic cursor (queue mode)
    SweepJob single;
    const uint32_t *thr;
    int32_t thr_stride, T, Q, stage_ell;
    int32_t max_n;          // largest n of any job (shared-memory carve-up)
    int32_t max_deg;        // largest maxdeg of any job (staged ELL size)
    // simulated quantum annealing: acceptance entries [T][3][W], Trotter slices, chosen slice per sample
    const unsigned long long *ent;
    int32_t P, W;
    int32_t *slice_out;
};

// Per-start state of the multi-start driver (Alg. 2), in device memory.
enum SlotMode : int32_t { kFixing = 0, kSolving = 1, kDone = 2, kCorr = 3 };

struct Slot {
    const DevProb *orig_prob;  // original problem (read-only, shared by its starts)
    const DevProb *cur;        // problem sampled in the current phase
    DevProb *buf[2];           // reduction targets (capacity of the original)
    int32_t next;              // buffer the next reduction writes
    int32_t mode, phase, fix_done;
    int32_t nfixed, n0, W0, ocur;
    uint64_t seed;
    uint32_t start;
    int32_t tsw;               // sweeps of the current phase's sample issued so far (chunked phases)
    uint32_t *spins;           // [Smax][W0] current sample
    int64_t *rec_e;            // [P][Smax] recorded full-problem energies
    int32_t *rec_count;        // [P]
    int32_t *rec_nfree;        // [P]
    int32_t *nphases;          // [1]
    int64_t *best_e;           // [1]
    int8_t *fmap;              // [n0] fix map in original order
    int8_t *best_state;        // [n0]
    int32_t *orig[2];          // [n0] original index of each current spin (double-buffered)
    int32_t *elite;            // [Smax]
    int32_t *counts;           // [n0]
    int8_t *fixed;             // [n0]
    int32_t *old_of_new;       // [n0]
    int32_t *scratch;          // slot_scratch_ints(cap_n) ints: the fold/compact's working arrays
    // component boosting of the solving sample (Sec. II.C); null when off
    int32_t *comp;             // [n0] component of each current spin
    int32_t *part;             // [Smax][n0] twice the partial energy of sample r on component c
    int32_t *perm;             // [n0][Smax] sample of rank r on component c
    uint32_t *spins2;          // [Smax][W0] merged sample
    int32_t ncomp, nlog;
    // tree pre-processing (Sec. II.C): inferred spins s_child = sigma s_parent, in
    // elimination order (original indices); null when off
    int32_t *log_child;        // [n0]
    int32_t *log_parent;       // [n0]
    int8_t *log_sigma;         // [n0]
};

struct SolveConsts {
    int32_t S_fix, S_solve, k_fix, iterate;
    int32_t max_fix, canon, fix_num, fix_den;
    int32_t P, Smax, Q, nslots;
    int32_t boost, max_n0, tree, pad1;
    int32_t S_corr, k_corr, corr_num, corr_den;  // correlation phase (S_corr = 0: off)
    // register kernel: work items take as many quads as the slots hold (block
    // threads x nslot items per thread, colour classes in whole slots); 0: Q quads
    int32_t fit_block, fit_nslot, grid;  // grid: CTAs of the sweep launch
    int32_t fit_words;                   // quad-group kernel: spin words of the launch's shared memory
    // sweeps per phase, and sweeps per launch (0: the whole phase in one launch).  With
    // chunk > 0 a phase's sample is annealed over ceil(T / chunk) launches, each resuming
    // from the states the previous one wrote; the persistence pass runs after the last.
    int32_t T, chunk;
    // PTICM as the sampler: a phase's sample size is the number of states its run
    // kept (the slot's rec_count of the phase), and the elite is ceil(elite x that)
    int32_t pticm, pad2;
    double elite;
};
// Elite count k = ceil(elite * S), clamped to [1, S] (host and device).
__host__ __device__ inline int elite_count_hd(double elite, int S)
{
    const double x = ceil(elite * (double)S);
    const int k = (x >= (double)S) ? S : (int)x;
    return k < 1 ? 1 : (k > S ? S : k);
}
// Samples and elite size of a slot's current phase.
__host__ __device__ inline int phase_samples(const SolveConsts &C, int mode)
{
    return mode == kCorr ? C.S_corr : mode == kFixing ? C.S_fix : C.S_solve;
}
// Elite count k = ceil(elite * S), clamped to [1, S].
inline int elite_count(double elite, int S)
{
    const double x = std::ceil(elite * (double)S);
    const int k = (x >= (double)S) ? S : (int)x;
    return std::max(1, std::min(k, S));
}
// Checks the correlation-step parameters (SPVAR_OK or SPVAR_EINVAL).
inline int check_corr_params(const spvar_params &p)
{
    if (p.corr_sample_size < 0) return SPVAR_EINVAL;
    if (p.corr_sample_size == 0) return SPVAR_OK;
    if (p.corr_num <= 0 || p.corr_den <= 0 || p.corr_num > p.corr_den || !(p.corr_elite_threshold > 0.0) ||
        !(p.corr_elite_threshold <= 1.0))
        return SPVAR_EINVAL;
    return SPVAR_OK;
}
// Checks the sampler choice (SPVAR_OK or SPVAR_EINVAL).
inline int check_sampler_params(const spvar_params &p)
{
    if (p.sampler == SPVAR_SAMPLER_SA) return SPVAR_OK;
    if (p.sampler == SPVAR_SAMPLER_PTICM) {
        const int R = p.pticm_temps, ntr = 2 * (p.pticm_temps - p.pticm_temps / 2);
        if (R < 2 || R > 64 || p.pticm_keep < 1 || p.pticm_keep > SPVAR_PTICM_MAX_KEEP ||
            p.fixing_sample_size != ntr * p.pticm_keep ||
            (p.solving_sample_size != 0 && p.solving_sample_size != ntr * p.pticm_keep) || p.num_sweeps < 1 ||
            p.corr_sample_size != 0 || p.component_boost != 0 || p.sweeps_per_launch != 0 ||
            !(p.pticm_beta0 > 0.0) || !(p.pticm_beta1 > 0.0))
            return SPVAR_EINVAL;
        return SPVAR_OK;
    }
    if (p.sampler != SPVAR_SAMPLER_SQA) return SPVAR_EINVAL;
    if (p.sqa_slices < 1 || (p.sqa_slices > 1 && (p.sqa_slices & 1)) || p.sqa_slices > SPVAR_SQA_MAX_SLICES ||
        !(p.sqa_beta > 0.0) || !(p.sqa_gamma0 > 0.0) || !(p.sqa_gamma1 > 0.0))
        return SPVAR_EINVAL;
    return SPVAR_OK;
}
// Phase-independent constants of the multi-start loop (Alg. 2) from the parameters.
inline void fill_solve_consts(const spvar_params &p, SolveConsts &C)
{
    C.S_fix = p.fixing_sample_size;
    C.S_solve = p.solving_sample_size;
    C.k_fix = elite_count(p.elite_threshold, p.fixing_sample_size);
    C.iterate = p.iterate ? 1 : 0;
    C.max_fix = p.max_fix_phases;
    C.canon = p.canon;
    C.fix_num = p.fix_num;
    C.fix_den = p.fix_den;
    C.S_corr = p.corr_sample_size;
    C.k_corr = p.corr_sample_size > 0 ? elite_count(p.corr_elite_threshold, p.corr_sample_size) : 0;
    C.corr_num = p.corr_num;
    C.corr_den = p.corr_den;
    C.P = p.max_fix_phases + 1 + (p.corr_sample_size > 0 ? 1 : 0);
    C.Smax = std::max(std::max(p.fixing_sample_size, p.solving_sample_size), p.corr_sample_size);
    C.boost = p.component_boost;
    C.tree = p.tree_preprocess;
    C.T = p.num_sweeps;
    C.chunk = 0;
    C.pticm = p.sampler == SPVAR_SAMPLER_PTICM ? 1 : 0;
    C.pad2 = 0;
    C.elite = p.elite_threshold;
}
// Sweep launches per phase: ceil(T / chunk), or 1 without chunking.
inline int launches_per_phase(int T, int chunk) { return (chunk > 0 && T > chunk) ? (T + chunk - 1) / chunk : 1; }
// True once the slot's current phase has its whole sample (every sweep issued).
__host__ __device__ inline bool sample_complete(const Slot &s, const SolveConsts &C) { return s.tsw >= C.T; }
// Bytes of the tree-inference log of one slot (0 when the tree step is off).
inline size_t tree_slot_bytes(int tree, int n0)
{
    if (!tree) return 0;
    auto a = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return 2 * a(4 * (size_t)n0) + a((size_t)n0);
}
inline void tree_slot_carve(Slot &s, char *base, int n0)
{
    auto a = [](size_t x) { return (x + 255) & ~(size_t)255; };
    s.log_child = (int32_t *)base;
    s.log_parent = (int32_t *)(base + a(4 * (size_t)n0));
    s.log_sigma = (int8_t *)(base + 2 * a(4 * (size_t)n0));
}
// Bytes of the boosting buffers of one slot (0 when boosting is off).
inline size_t boost_slot_bytes(int boost, int n0, int Smax, int W0)
{
    if (!boost) return 0;
    auto a = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return a(4 * (size_t)n0) + 2 * a(4 * (size_t)Smax * n0) + a(4 * (size_t)Smax * W0);
}
// Carves the boosting buffers of a slot out of `base` (boost_slot_bytes bytes).
inline void boost_slot_carve(Slot &s, char *base, int n0, int Smax, int W0)
{
    auto a = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t o = 0;
    s.comp = (int32_t *)(base + o);
    o += a(4 * (size_t)n0);
    s.part = (int32_t *)(base + o);
    o += a(4 * (size_t)Smax * n0);
    s.perm = (int32_t *)(base + o);
    o += a(4 * (size_t)Smax * n0);
    s.spins2 = (uint32_t *)(base + o);
}

// Multi-CTA fold/compact: chunks of kFoldChunk spins, one CTA each.  A slot's
// scratch holds new_of_old, the free-free row lengths and the folded biases
// (three [cap_n] arrays, by old index), then a table of kFoldStride ints per
// chunk (free spins, free-free entries, nonzero-bias flag, the chunk's
// reference-spin candidate, free spins per colour class) and the int64 sum of
// the fixed spins' energy.
constexpr int kFoldChunk = 256;
constexpr int kFoldMaxChunks = (SPVAR_MAX_N + kFoldChunk - 1) / kFoldChunk;
constexpr int kFoldStride = 40;  // >= 6 + kMaxColours
inline size_t slot_scratch_ints(int cap_n)
{
    const size_t base = (3 * (size_t)cap_n + 1) & ~(size_t)1;  // the table starts 8-byte aligned
    return base + (size_t)kFoldMaxChunks * kFoldStride + 2;
}
__host__ __device__ inline size_t fold_table_offset(int cap_n) { return (3 * (size_t)cap_n + 1) & ~(size_t)1; }

cudaError_t launch_slots_init(Slot *slots, const SolveConsts &C, int max_n0, cudaStream_t st);
// Work list of the phase's sweep launch; also zeroes *nactive (if not null),
// which the persistence pass then counts up.
cudaError_t launch_plan(Slot *slots, const SolveConsts &C, SweepJob *jobs, WorkItem *items,
                        int32_t *nitems, int32_t *queue, int32_t *nactive, cudaStream_t st);
// Tree pre-processing on: elite, counts, then fold/compact and the tree step,
// one CTA per slot (nactive != null: the count of slots still active).
cudaError_t launch_elite_slots(Slot *slots, const SolveConsts &C, cudaStream_t st);
cudaError_t launch_count_slots(Slot *slots, const SolveConsts &C, int max_n0, cudaStream_t st);
cudaError_t launch_reduce_slots(Slot *slots, const SolveConsts &C, int32_t *nactive,
                                cudaStream_t st);
// Tree pre-processing off: the whole persistence pass (elite, best state,
// counts and fixing, fold/compact, phase transition) of every slot whose phase
// sample is complete, one thread-block cluster per slot; nactive (zeroed by
// launch_plan) is counted up by the slots still active.
cudaError_t launch_pass_slots(Slot *slots, const SolveConsts &C, int32_t *nactive, cudaStream_t st);

size_t sweep_smem_bytes(int max_n, int Q, int thr_stride, int maxdeg, bool stage_ell);
cudaError_t launch_sweep(const SweepLaunch &L, bool pm1, int block, int grid, size_t smem,
                         cudaStream_t stream);
int sweep_max_active_blocks(bool pm1, int block, size_t smem, bool stage_ell);

// Register-resident +-1 sweep (sweep_pm1.cu).
// mode 0: +-1 couplers in byte lanes; 1: one coupler magnitude per spin, 16-bit
// lanes; 2: small integer couplers (|J| <= 15), weighted byte-wise neighbour
// sum, 16-bit lanes.
bool pm1_shape_ok(int block, int nslot, int maxd, int mode);
size_t pm1_smem_bytes(bool scaled, int thr_stride);
cudaError_t launch_sweep_pm1(const SweepLaunch &L, int block, int nslot, int maxd, int mode, int grid, size_t smem,
                             cudaStream_t st);
int pm1_max_active_blocks(int block, int nslot, int maxd, int mode, size_t smem);

// Simulated quantum annealing sweep (sweep_sqa.cu): one quad per work item, all
// Trotter slices in shared memory.
// Variants: 0 general couplers, 1 +-1 couplers (item walk), 2 +-1 couplers in
// register form (ncls = 2 or 4 colour-class slots per thread), 3 small integer
// couplers (|J| <= 15, dmax <= 254) in register form.
constexpr int kSqaMaxSlices = 1024;
bool sqa_shape_ok(int variant, int block, int max_n, int max_deg, int P, int W, int ncls = 0);
size_t sqa_smem_bytes(int max_n, int P, int maxdeg, int W, bool pm1);
cudaError_t launch_sweep_sqa(const SweepLaunch &L, int variant, int block, int ncls, bool ent32, int grid,
                             size_t smem, cudaStream_t st);
int sqa_max_active_blocks(int variant, int block, int max_deg, int ncls, bool ent32, size_t smem);
// The register form holds one spin of every colour class per thread: two or
// more slices, at most 4 classes, none larger than the block.  Colour-class
// slots it needs (2 or 4), 0 if it does not apply.
inline bool sqa_si_eligible(int jabs_max, int dmax, int maxdeg)
{
    return jabs_max >= 1 && jabs_max <= 15 && dmax <= 254 && maxdeg <= 8;
}
inline int sqa_reg_ncls(int ncol, int max_class, int block, int P)
{
    if (P < 2 || ncol > 4 || max_class > block) return 0;
    return ncol <= 2 ? 2 : 4;
}

// Quad-group +-1 sweep (sweep_pm1q.cu): up to 64 quads of one problem per work
// item, spin words only in shared memory (2 (n + 1) words per quad).
bool pm1q_shape_ok(int block, int maxd, int max_n, int Q);
size_t pm1q_smem_bytes(int max_n, int Q);
cudaError_t launch_sweep_pm1q(const SweepLaunch &L, int block, int maxd, int grid, size_t smem, cudaStream_t st);
int pm1q_max_active_blocks(int block, int maxd, size_t smem);

// PTICM sampler (sweep_pticm.cu): one CTA per run, every replica's spins in
// shared memory.
size_t pticm_smem_bytes(int n, int R, int dmax);
// PTICM runs of every start of a slot table (the sampler of Alg. 2 in a plan).
cudaError_t launch_pticm_slots(Slot *slots, int nslots, int Smax, const uint32_t *thr, int thr_stride,
                               const uint32_t *xthr, int dx, int R, int T, int K, size_t smem, cudaStream_t st);
int pticm_max_r();
int pticm_max_n();
cudaError_t launch_pticm(const DevProb *prob, const uint32_t *thr, int thr_stride, const uint32_t *xthr, int dx,
                         int R, int T, int icm_from, int keep_from, int K, int flags, uint64_t seed,
                         uint32_t start0, uint32_t phase, int runs, size_t smem, uint32_t *kept, int64_t *kept_e,
                         int32_t *nkept, uint32_t *final_bits, int64_t *final_e, cudaStream_t st);

// Streaming +-1 sweep (sweep_pm1s.cu): one quad per work item.
bool pm1s_shape_ok(int block, int maxd, int max_n, int Q);
size_t pm1s_smem_bytes(int max_n, int Q, int maxd);
cudaError_t launch_sweep_pm1s(const SweepLaunch &L, int block, int maxd, int grid, size_t smem, cudaStream_t st);
int pm1s_max_active_blocks(int block, int maxd, size_t smem);

// Warp-per-quad +-1 sweep (sweep_pm1w.cu): WARPS quads per work item.
bool pm1w_shape_ok(int warps, int maxd, int max_n, int K);
size_t pm1w_smem_bytes(int max_n, int warps, int maxd);
cudaError_t launch_sweep_pm1w(const SweepLaunch &L, int warps, int maxd, int K, int grid, size_t smem,
                              cudaStream_t st);
int pm1w_max_active_blocks(int warps, int maxd, int K, size_t smem);

// Launch shape of a sweep: kind 0 = general kernel (stage: layout staged in
// shared memory), kind 1 = register-resident kernel (nslot items per thread,
// maxd neighbour registers per item; stage = 1: the 16-bit-lane variant for
// one coupler magnitude per spin, stage = 2: its variant for small integer
// couplers), kind 2 = streaming +-1 kernel
// (maxd neighbour offsets per spin staged in shared memory, Q = 1), kind 4 =
// warp-per-quad +-1 kernel (Q = warps = block / 32; nslot = spins in flight per lane,
// 2 or 4), kind 5 = simulated
// quantum annealing (Q = 1).  A persistent grid holds
// every CTA the SMs can keep resident, or (balance) the fewest CTAs that still
// need the same number of waves of items, so that no last wave runs nearly empty.
struct SweepShape {
    int kind, block, Q, stage, nslot, maxd;
    int balance = 0;  // 1: grid sized so that every CTA runs the same number of items
    int slices = 0;   // kind 5 (SQA): Trotter slices; stage = the variant (0 general, 1 +-1 walk,
                      // 2 +-1 register form), nslot the acceptance-table width W, maxd the largest degree
    int ncls = 0;     // kind 5, variant 2: colour-class slots per thread (2 or 4)
    int ent32 = 0;    // kind 5, variant 2: 32-bit acceptance entries (no entry of the table is 2^32)
    int lpp = 1;      // sweep launches per phase (the autotuner's sweeps-per-launch axis)
};
// The streaming and warp-per-quad kernels apply to +-1 couplers, degree <= 8
// and dmax <= 254; the register kernel needs dmax <= 30.
inline bool pm1_kernel_eligible(bool pm1, int dmax, int maxdeg) { return pm1 && dmax <= 254 && maxdeg <= 8; }
inline bool pm1r_kernel_eligible(bool pm1, int dmax, int maxdeg) { return pm1 && dmax <= 30 && maxdeg <= 8; }
// The register kernel's 16-bit-lane variant: one coupler magnitude per spin, dmax <= 4094.
inline bool ujr_kernel_eligible(bool ujs, int dmax, int maxdeg) { return ujs && dmax <= 4094 && maxdeg <= 8; }
// Its small-integer variant: every |J| <= 15 (four bits per neighbour), dmax <= 4094.
inline bool sir_kernel_eligible(int jabs_max, int dmax, int maxdeg)
{
    return jabs_max >= 1 && jabs_max <= 15 && dmax <= 4094 && maxdeg <= 8;
}
// Slots per thread the register kernel needs for problem P at Q quads per CTA
// (every colour class fills whole slots), rounded up to an instantiated count
// (2..4); 0 if more than 4.  Reductions only shrink classes, so the original
// problem's count covers all its phases.
inline int pm1_nslot(const Problem *P, int Q, int block)
{
    long long need = 0;
    for (int c = 0; c < P->hdr.ncol; ++c) need += ((long long)P->csize[c] * Q + block - 1) / block;
    if (need > 4) return 0;
    return need < 2 ? 2 : (int)need;
}
inline size_t sweep_shape_smem(const SweepShape &s, int max_n, int thr_stride, int max_deg)
{
    if (s.kind == 5) return sqa_smem_bytes(max_n, s.slices, max_deg, s.nslot, s.stage != 0);
    if (s.kind == 1) return pm1_smem_bytes(s.stage != 0, thr_stride);
    if (s.kind == 2) return pm1s_smem_bytes(max_n, s.Q, s.maxd);
    if (s.kind == 4) return pm1w_smem_bytes(max_n, s.Q, s.maxd);
    if (s.kind == 6) return pm1q_smem_bytes(max_n, s.Q);
    return sweep_smem_bytes(max_n, s.Q, thr_stride, max_deg, s.stage != 0);
}
inline cudaError_t launch_sweep_shape(const SweepLaunch &L, const SweepShape &s, bool pm1, int grid, size_t smem,
                                      cudaStream_t st)
{
    if (s.kind == 5) return launch_sweep_sqa(L, s.stage, s.block, s.ncls, s.ent32 != 0, grid, smem, st);
    if (s.kind == 1) return launch_sweep_pm1(L, s.block, s.nslot, s.maxd, s.stage, grid, smem, st);
    if (s.kind == 2) return launch_sweep_pm1s(L, s.block, s.maxd, grid, smem, st);
    if (s.kind == 4) return launch_sweep_pm1w(L, s.Q, s.maxd, s.nslot ? s.nslot : 2, grid, smem, st);
    if (s.kind == 6) return launch_sweep_pm1q(L, s.block, s.maxd, grid, smem, st);
    return launch_sweep(L, pm1, s.block, grid, smem, st);
}
inline int sweep_shape_occupancy(const SweepShape &s, bool pm1, size_t smem)
{
    if (s.kind == 5) return sqa_max_active_blocks(s.stage, s.block, s.maxd, s.ncls, s.ent32 != 0, smem);
    if (s.kind == 1) return pm1_max_active_blocks(s.block, s.nslot, s.maxd, s.stage, smem);
    if (s.kind == 2) return pm1s_max_active_blocks(s.block, s.maxd, smem);
    if (s.kind == 4) return pm1w_max_active_blocks(s.Q, s.maxd, s.nslot ? s.nslot : 2, smem);
    if (s.kind == 6) return pm1q_max_active_blocks(s.block, s.maxd, smem);
    return sweep_max_active_blocks(pm1, s.block, smem, s.stage != 0);
}

// Everything one Multi-start SPVAR phase needs besides the slots.
struct PhaseEngine {
    SweepShape shape;
    size_t sweep_smem;
    bool pm1;
    int max_n0, max_deg, thr_stride;
    const uint32_t *thr;
    const unsigned long long *ent;  // SQA acceptance entries (null for SA)
    int P, W;
    SweepJob *jobs;
    WorkItem *items;
    int32_t *ctr;  // [0] items, [1] queue cursor, [2] active slots
    cudaEvent_t ev_sweep[2];
    cudaEvent_t ev_post;  // recorded after each phase's persistence pass (null: none)
    SolveConsts C;
    // PTICM as the sampler (pt_R > 0): one run per start instead of the sweep launch
    int pt_R = 0, pt_K = 0, pt_dx = 0;
    const uint32_t *pt_thr = nullptr;   // [R][thr_stride]
    const uint32_t *pt_xthr = nullptr;  // [R - 1][pt_dx + 1]
    size_t pt_smem = 0;
};
// plan -> sweep -> elite -> count/fix -> fold/compact for `nslots` slots.
cudaError_t engine_phase(const PhaseEngine &E, Slot *slots, int nslots, int T, int grid, cudaStream_t st,
                         bool count_active, bool capturing);
cudaError_t launch_gather_modes(const Slot *slots, int nslots, int32_t *modes, cudaStream_t st);
// Disconnected-component boosting of every solving-phase slot (Sec. II.C).
cudaError_t launch_boost(Slot *slots, const SolveConsts &C, cudaStream_t st);

// Elite selection of one sample set (standalone form).
cudaError_t launch_elite_single(const int64_t *energies, int S, int k, int32_t *elite,
                                cudaStream_t stream);
cudaError_t launch_count_single(const DevProb *prob, int n_host, const uint32_t *spins, int W,
                                const int32_t *elite, int k, int canon, int fix_num, int fix_den,
                                int32_t *counts, int8_t *fixed, int32_t *nfixed, cudaStream_t stream);
cudaError_t launch_reduce_single(const DevProb *src, DevProb *dst, const int8_t *fixed,
                                 int32_t *old_of_new, int32_t *scratch, cudaStream_t stream);
int elite_max_samples();

__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

}  // namespace spvar

#define SPVAR_CUDA_TRY(expr)                                   \
    do {                                                       \
        cudaError_t _e = (expr);                               \
        if (_e != cudaSuccess) return SPVAR_ECUDA;             \
    } while (0)
