/*
 * spvar.h -- C ABI of the GB300 (sm_103a) library for sample-persistence
 * variable reduction with a simulated-annealing sampler.
 *
 * The method (Karimi, Rosenberg, Katzgraber, "Effective optimization using
 * sample persistence"): minimise the Ising energy of Sec. I,
 *
 *     E(s) = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i + offset,  s in {-1,+1}^N,
 *
 * by sampling low-energy states, fixing the variables that take the same
 * value across the lowest-energy part of the sample (SPVAR, Alg. 1) and
 * sampling the smaller problem that remains, over many independent starts
 * (Multi-start SPVAR, Alg. 2).  The sampler is simulated annealing: Metropolis
 * single-spin sweeps under an increasing inverse temperature (the SA solver
 * of Sec. III.A).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Return value: SPVAR_OK (0) or a negative SPVAR_E* code; spvar_strerror()
 *    names it.  On error nothing is written to outputs except where stated.
 *  - Integers only: couplers, biases and energies are integers (a real-valued
 *    problem is passed multiplied by an integer energy_scale), so every
 *    result is exact and reproducible bit for bit.
 *  - Problems are symmetric CSR: row i lists the neighbours j of spin i with
 *    J_ij; each coupler appears in both rows with the same value, columns
 *    strictly ascending, no diagonal, no zero-valued entries.
 *  - Spin samples are bit-packed rows: sample r occupies W = ceil(n/32)
 *    uint32 words; bit (i % 32) of word (i / 32) is 1 iff s_i = +1.
 *  - "device" pointers are CUDA device memory of the current device (for
 *    example torch tensor data_ptr()); "host" pointers are CPU memory.  The
 *    caller owns every buffer it passes; the library copies inputs and never
 *    retains caller pointers after a call returns.  Opaque objects are owned
 *    by the library until their *_destroy call.
 *  - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device-pointer outputs are written asynchronously on that stream; calls
 *    that return host data synchronise the stream before returning.
 *  - Randomness: Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit
 *    seed, counter (spin, phase * 2^20 + sweep, replica / 4, start), word
 *    replica % 4.  Results therefore depend only on the logical coordinates,
 *    never on launch shape, batching or scheduling.
 *
 * How these calls differ from a plain host-side statement of Alg. 1
 * -----------------------------------------------------------------
 *  - Samples are not library objects: spvar_sample writes spins and energies
 *    into device buffers the caller owns (e.g. torch tensors), so a phase
 *    allocates nothing and its output feeds spvar_persistence directly.
 *  - The acceptance table is a required device input, built once by
 *    spvar_thresholds from the beta schedule and reused by every call and
 *    start: the table (not beta) is what both this library and a checker
 *    evaluate, so results are bit-exact, and no call hides a host-to-device
 *    copy of a table per sample.
 *  - spvar_persistence writes the counts, the fixings and the number fixed to
 *    device memory and does not synchronise, so sample -> persistence ->
 *    reduction chain on the stream; only the elite size returns to the host.
 *  - spvar_reduce synchronises once, to learn the size of the new problem.
 *  - Problem sizes and the constant term are read through
 *    spvar_problem_get_info rather than one accessor each.
 */
#ifndef SPVAR_H
#define SPVAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPVAR_OK 0
#define SPVAR_EINVAL (-1)    /* invalid argument or malformed problem */
#define SPVAR_EOVERFLOW (-2) /* values would overflow the 32-bit energy arithmetic */
#define SPVAR_ENOMEM (-3)    /* host or device allocation failed */
#define SPVAR_EBUDGET (-4)   /* request does not fit the device-memory budget */
#define SPVAR_ETIMEOUT (-5)  /* a bounded device-side wait gave up */
#define SPVAR_ECUDA (-6)     /* a CUDA runtime call failed */
#define SPVAR_ELIMIT (-7)    /* size beyond a documented library limit */

/* Library limits (SPVAR_ELIMIT beyond them). */
#define SPVAR_MAX_N 32768        /* spins per problem (shared-memory spin state) */
#define SPVAR_MAX_DEGREE 32      /* couplers per spin */
#define SPVAR_MAX_SWEEPS 1048574 /* sweeps per sample: 2^20 - 2 (slot 2^20-1 = initial state) */
#define SPVAR_MAX_PHASE 4095     /* phase index < 2^12 */
#define SPVAR_MAX_SAMPLES 16384  /* samples per (problem, phase) */

const char *spvar_strerror(int code);

/* Number of CUDA devices visible, or a negative code.  Loads no kernel. */
int spvar_device_count(int *count);

/* ------------------------------------------------------------------ */
/* Problem (Sec. I)                                                    */
/* ------------------------------------------------------------------ */
typedef struct spvar_problem spvar_problem;

typedef struct spvar_problem_info {
    int32_t n;            /* spins */
    int32_t nnz;          /* CSR entries (2 x couplers) */
    int32_t ncol;         /* colour classes of the sweep order */
    int32_t maxdeg;       /* largest row length */
    int32_t dmax;         /* 2 * max_i (sum_j |J_ij| + |h_i|): largest flip cost */
    int32_t hzero;        /* 1 iff every h_i == 0 */
    int32_t pm1;          /* 1 iff every J_ij is -1 or +1 */
    int32_t energy_scale; /* integer energies = real energies x energy_scale */
    int64_t offset;       /* constant term */
} spvar_problem_info;

/* Host helper: edge list -> symmetric CSR with ascending columns.
 * ei, ej, J: host [m], 0 <= ei, ej < n, ei != ej, each pair at most once.
 * row_ptr: host [n+1]; col, val: host [2m].  SPVAR_EINVAL on a self loop,
 * an index out of range or a repeated pair. */
int spvar_csr_from_edges(int32_t n, int64_t m, const int32_t *ei, const int32_t *ej,
                         const int32_t *J, int32_t *row_ptr, int32_t *col, int32_t *val);

/* Create a problem on the current device from host CSR arrays
 * (row_ptr [n+1], col/val [row_ptr[n]], h [n]; all host, copied).
 * Validates symmetry, ordering, index ranges and the int32 energy range
 * (sum_ij |J_ij| + sum_i |h_i| < 2^30), computes the colour classes of the
 * sweep order (bipartite: BFS distance parity from the lowest index of each
 * component; otherwise first-fit greedy in index order) and uploads the
 * sweep layout.  energy_scale >= 1 only enters the acceptance table.
 * Errors: EINVAL, EOVERFLOW, ELIMIT (n > SPVAR_MAX_N, degree >
 * SPVAR_MAX_DEGREE, |J| > 32767), ENOMEM, ECUDA. */
int spvar_problem_create(int32_t n, const int32_t *row_ptr, const int32_t *col,
                         const int32_t *val, const int32_t *h, int64_t offset,
                         int32_t energy_scale, void *stream, spvar_problem **out);

void spvar_problem_destroy(spvar_problem *p);

int spvar_problem_get_info(const spvar_problem *p, spvar_problem_info *info);

/* Copy the problem back to host buffers (row_ptr [n+1], col/val [nnz],
 * h [n], colour [n]); any pointer may be NULL.  Synchronises the stream. */
int spvar_problem_download(const spvar_problem *p, int32_t *row_ptr, int32_t *col,
                           int32_t *val, int32_t *h, int32_t *colour, void *stream);

/* ------------------------------------------------------------------ */
/* Annealing schedule                                                  */
/* ------------------------------------------------------------------ */
/* Host: beta[t] = beta0 * (beta1/beta0)^(t/(T-1)), t = 0..T-1 (T = 1: beta0). */
int spvar_beta_geometric(int32_t T, double beta0, double beta1, double *beta);

/* Host: acceptance table thr [T][dmax+1],
 * thr[t][d] = min(2^32-1, floor(2^32 * exp(-beta[t] * d / energy_scale))),
 * computed in double.  A flip that raises the energy by d > 0 at sweep t is
 * accepted iff the flip's random word is < thr[t][d]. */
int spvar_thresholds(int32_t T, const double *beta, int32_t dmax, int32_t energy_scale,
                     uint32_t *thr);

/* ------------------------------------------------------------------ */
/* Sampler: simulated annealing (Sec. III.A; Alg. 1 "obtain sample")   */
/* ------------------------------------------------------------------ */
/* One independent annealing run per sample r < num_samples.
 * Initial state: s_i = +1 iff the top bit of the random word at sweep slot
 * 2^20-1 is set.  Sweep t = 0..num_sweeps-1 visits the colour classes in
 * increasing order and, inside a class (no two spins coupled), proposes
 * each spin once: dE = -2 s_i (h_i + sum_j J_ij s_j); accepted iff dE <= 0
 * or word < thr[t * thr_stride + dE].
 *   thr       device [num_sweeps][thr_stride], thr_stride >= dmax + 1
 *   spins     device [num_samples][ceil(n/32)] final states (bit-packed)
 *   energies  device [num_samples] final energies INCLUDING the offset
 * Errors: EINVAL (sizes, thr_stride <= dmax), ELIMIT, ECUDA. */
int spvar_sample(const spvar_problem *p, int32_t num_sweeps, const uint32_t *thr,
                 int32_t thr_stride, int32_t num_samples, uint64_t seed, uint32_t start,
                 uint32_t phase, uint32_t *spins, int64_t *energies, void *stream);

/* Checkpoint / resume of an anneal: runs sweeps sweep_begin .. sweep_end-1
 * of the same sample, starting from init_spins (device [num_samples][ceil(n/32)],
 * the spins a previous range wrote; NULL = the initial state, only with
 * sweep_begin = 0).  Because every random word is keyed by the absolute sweep
 * index, any split of [0, T) into consecutive ranges gives exactly the result
 * of one spvar_sample over T sweeps.  thr must hold rows up to sweep_end - 1;
 * init_spins must not alias spins.  Errors as spvar_sample, EINVAL for bad ranges. */
int spvar_sample_range(const spvar_problem *p, int32_t sweep_begin, int32_t sweep_end,
                       const uint32_t *thr, int32_t thr_stride, int32_t num_samples, uint64_t seed,
                       uint32_t start, uint32_t phase, const uint32_t *init_spins, uint32_t *spins,
                       int64_t *energies, void *stream);

/* ------------------------------------------------------------------ */
/* Simulated quantum annealing: a second sampler for Alg. 1 (Sec. III:  */
/* discrete-time path-integral Monte Carlo of the transverse-field     */
/* Ising model)                                                         */
/* ------------------------------------------------------------------ */

#define SPVAR_SQA_MAX_SLICES 1024

/* Acceptance entries of the path-integral sweep, host -> host.
 * P Trotter slices (1, or even), beta[T] and gamma[T] the inverse temperature
 * and transverse field of each sweep.  With bias = dmax / 2, W = 2 bias + 1,
 * Jp = -1/2 ln tanh(beta gamma / P) (0 when P = 1) and, for flip-cost index
 * k = dE/2 + bias and a = number of the spin's two slice neighbours equal to
 * it (a = 1 when P = 1),
 *   dA = (2 beta / P) (k - bias) / scale + 4 Jp (a - 1),
 *   ent[(t*3 + a)*W + k] = 2^32 - min(2^32, floor(2^32 exp(-dA)))   (double).
 * A move is accepted iff u + ent < 2^32 (u the 32-bit uniform).  ent: host
 * [T][3][W].  EINVAL on a bad P, T, dmax or scale, or gamma <= 0 with P > 1. */
int spvar_sqa_table(int32_t T, int32_t P, const double *beta, const double *gamma, int32_t dmax,
                    int32_t energy_scale, uint64_t *ent);

/* Linear transverse-field schedule gamma[t] = g0 + (g1 - g0) t / (T - 1)
 * (gamma[0] = g0 when T = 1), host -> host. */
int spvar_gamma_linear(int32_t T, double g0, double g1, double *gamma);

/* num_samples SQA runs of the problem (each returns its lowest-energy slice,
 * lowest slice index on ties).  ent: device [num_sweeps][3][W] from
 * spvar_sqa_table for a dmax >= the problem's (W = 2 (dmax/2) + 1).  Counters
 * as spvar_sample with spin word i | tau << 16 for slice tau; sweep = colour
 * classes in order, even slices then odd slices inside each.  spins: device
 * [num_samples][ceil(n/32)]; energies: device [num_samples] (with offset);
 * slice: device [num_samples] (chosen slice) or NULL.  Asynchronous on stream.
 * Errors: EINVAL (bad P or table width), ELIMIT (the P slices do not fit in
 * shared memory), ECUDA. */
int spvar_sqa_sample(const spvar_problem *p, int32_t num_sweeps, int32_t P, const uint64_t *ent, int32_t W,
                     int32_t num_samples, uint64_t seed, uint32_t start, uint32_t phase, uint32_t *spins,
                     int64_t *energies, int32_t *slice, void *stream);

/* ------------------------------------------------------------------ */
/* Third sampler: parallel tempering with isoenergetic cluster moves     */
/* (PTICM, Sec. III.D), with the paper's sample rule                     */
/* ------------------------------------------------------------------ */

#define SPVAR_PTICM_MAX_KEEP 64

/* num_runs independent PTICM runs of the problem (run j uses start word
 * start0 + j), one CTA each.  R inverse temperatures beta_0 < ... < beta_{R-1}
 * with two replicas each (replica r = 2k + c), initial states from the
 * initial-state words of spvar_sample (replica r = sample r).  Each of
 * num_sweeps sweeps: (1) a Metropolis sweep of every replica at its
 * temperature, thr: device [R][thr_stride] from spvar_thresholds of the betas
 * (thr_stride >= dmax + 1), random words as spvar_sample; (2) if flags & 2,
 * Houdayer's move at every temperature k >= icm_from whose two replicas
 * differ: the seed is element floor(u |D| / 2^32) of the differing set D in
 * index order (u: word 0 of Philox((0xFFFF0000 | k, phase 2^20 + t, 0,
 * start))), the cluster its connected component among the couplers inside
 * D, and both replicas flip on it; (3) if flags & 1, replica exchange between
 * temperatures k and k + 1 for k = t (mod 2), each copy: with
 * d = E(k) - E(k+1), accepted iff d <= 0 or u < xthr[k][d] (xthr: device
 * [R-1][dx+1] from spvar_thresholds of beta_{k+1} - beta_k, dx >= the range
 * max E - min E; u: word 0 of Philox((0xFFFE0000 | (2k + c), phase 2^20 + t,
 * 0, start))); (4) every replica of temperature k >= keep_from offers its
 * state to its list of the K lowest-energy distinct states seen (ordered by
 * energy, then first sight; a full list takes a state only below its highest
 * energy).  Outputs (device): kept [num_runs][2 (R - keep_from)][K][ceil(n/32)]
 * bit-packed in index order, kept_e [..][K] (with offset), nkept [num_runs][2
 * (R - keep_from)] (zeroed here), final_states [num_runs][2R][ceil(n/32)],
 * final_e [num_runs][2R] (with offset).  Asynchronous on stream.  Errors:
 * EINVAL (bad sizes or flags, missing buffers), ELIMIT (R > 64, K >
 * SPVAR_PTICM_MAX_KEEP, n > 2048, or the 2Rn + 4R(dmax + 1) + 32n bytes of
 * replicas, thresholds and search queues exceed the shared memory of one
 * CTA), ECUDA. */
int spvar_pticm_sample(const spvar_problem *p, int32_t R, int32_t num_sweeps, const uint32_t *thr,
                       int32_t thr_stride, const uint32_t *xthr, int32_t dx, int32_t icm_from, int32_t keep_from,
                       int32_t K, int32_t flags, int32_t num_runs, uint64_t seed, uint32_t start0, uint32_t phase,
                       uint32_t *kept, int64_t *kept_e, int32_t *nkept, uint32_t *final_states, int64_t *final_e,
                       void *stream);

/* ------------------------------------------------------------------ */
/* Persistence (Alg. 1: elite sample, mean value, fixing rule)          */
/* ------------------------------------------------------------------ */
/* k = ceil(elite_threshold * num_samples) (clamped to [1, num_samples])
 * lowest-energy samples, ordered by (energy, sample index), form the elite.
 * If canon is 1 (or -1 and every h is 0) each elite row is multiplied by
 * its value at the reference spin rho = the lowest-index spin of maximum
 * degree, which breaks the two-fold degeneracy of zero-bias problems
 * (Sec. II.C).  counts[i] = number of elite rows with s_i = +1;
 * fixed[i] = sign(2 counts[i] - k) if fix_den * |2 counts[i] - k| >=
 * fix_num * k (fixing_threshold = fix_num / fix_den, 0 < fix_num <= fix_den),
 * else 0.
 *   spins, energies  device, as written by spvar_sample
 *   elite            device [k] out: sample indices in elite order
 *   counts           device [n] out;  fixed  device int8 [n] out
 *   nfixed           device [1] out: number of fixed spins
 *   k_out            host, may be NULL: the elite size used */
int spvar_persistence(const spvar_problem *p, int32_t num_samples, const uint32_t *spins,
                      const int64_t *energies, double elite_threshold, int32_t fix_num,
                      int32_t fix_den, int32_t canon, int32_t *elite, int32_t *counts,
                      int8_t *fixed, int32_t *nfixed, int32_t *k_out, void *stream);

/* ------------------------------------------------------------------ */
/* Fold and compact (Alg. 1: update J and h)                            */
/* ------------------------------------------------------------------ */
/* New problem over the free spins (fixed[i] == 0), renumbered in increasing
 * old index: h'_i = h_i + sum_{j fixed} J_ij v_j, offset' = offset +
 * sum_{i fixed} h_i v_i + sum_{i<j both fixed} J_ij v_i v_j, couplers
 * between free spins kept, colour classes inherited.
 *   fixed       device int8 [n] (0, +1, -1)
 *   old_of_new  device [n] out: old index of each new spin (first n' used)
 * Synchronises the stream (the new size is read back). */
int spvar_reduce(const spvar_problem *p, const int8_t *fixed, int32_t *old_of_new,
                 void *stream, spvar_problem **out);

/* Allocation-free fold/compact.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc while they run (code
 * working inside a fully committed memory budget, or a host runtime that owns
 * every device allocation and forbids allocating calls after start-up).  It
 * computes the same reduction as spvar_reduce but allocates nothing: the
 * result goes to caller buffers as plain CSR, and the working arrays live in
 * a static device array of 2 * SPVAR_NOALLOC_MAX_N int32 (128 KB) that every
 * device loading the library keeps until the process exits.
 *   fixed            device int8 [n] (0, +1, -1)
 *   row_ptr          device [n+1] out (first n'+1 entries written)
 *   col, val         device [nnz] out (first row_ptr[n'] entries written)
 *   h                device [n] out; offset device int64 [1] out
 *   old_of_new       device [n] out; n_out device int32 [1] out (n')
 * Asynchronous on `stream`; returns SPVAR_ELIMIT when n > SPVAR_NOALLOC_MAX_N.
 * The first call on a device looks up the static array's device address
 * (make it before any stream capture).  All calls share the array: calls
 * that can overlap on the GPU race and must be serialised by the caller. */
#define SPVAR_NOALLOC_MAX_N 16384
int spvar_reduce_noalloc(const spvar_problem *p, const int8_t *fixed, int32_t *row_ptr, int32_t *col,
                         int32_t *val, int32_t *h, int64_t *offset, int32_t *old_of_new,
                         int32_t *n_out, void *stream);

/* ------------------------------------------------------------------ */
/* Multi-start SPVAR (Alg. 2) on one or many problems                   */
/* ------------------------------------------------------------------ */
typedef struct spvar_params {
    int32_t num_starts;          /* independent starts per problem */
    int32_t fixing_sample_size;  /* samples in each SPVAR phase */
    int32_t solving_sample_size; /* samples of the final reduced problem (0: none) */
    int32_t num_sweeps;          /* sweeps per annealing run */
    double beta0, beta1;         /* geometric schedule endpoints */
    double elite_threshold;      /* elite fraction */
    int32_t fix_num, fix_den;    /* fixing_threshold = fix_num / fix_den */
    int32_t iterate;             /* 1: repeat SPVAR while spins remain (ISPVAR) */
    int32_t max_fix_phases;      /* SPVAR phases per start, >= 1 */
    int32_t canon;               /* -1: when h == 0; 0: never; 1: always */
    int32_t form;                /* SPVAR_FORM_BATCHED or SPVAR_FORM_PLAIN */
    int32_t replicas_per_block;  /* 0: autotune the sweep shape; else a multiple of 4 */
    int32_t sweep_kernel;        /* with replicas_per_block > 0: SPVAR_SWEEP_* */
    int32_t sweep_block;         /* with replicas_per_block > 0: threads per CTA (128/256/512/1024), 0 = 256 */
    int32_t start_offset;        /* start s of a problem uses counter word start_offset + s (sharding) */
    int32_t component_boost;     /* 1: disconnected-component boosting of the solving sample (Sec. II.C):
                                    each connected component's partial samples are sorted by partial
                                    energy and merged rank by rank; recorded energies are the merged ones */
    int32_t tree_preprocess;     /* 1: exact tree elimination after every SPVAR reduction (Sec. II.C):
                                    degree-0/1 spins fixed by their bias or inferred from their neighbour,
                                    recursively; inferred spins are restored in best_state */
    int32_t corr_sample_size;    /* > 0: correlation fixing (Sec. II.C; Alg. 2 optional step) for a
                                    problem whose every h is 0: a first phase of this many samples; its
                                    corr_elite_threshold elite fixes the reference spin rho (lowest-index
                                    spin of maximum degree) to +1 and every spin j with
                                    |mean(s_rho s_j)| >= corr_num / corr_den to the sign of the mean.
                                    Skipped for a problem with some h != 0.  0: off */
    int32_t corr_num, corr_den;  /* correlation threshold corr_num / corr_den (the paper uses 1.0) */
    double corr_elite_threshold; /* elite fraction of the correlation phase */
    int32_t sampler;             /* SPVAR_SAMPLER_SA (beta0 -> beta1 anneal) or SPVAR_SAMPLER_SQA */
    int32_t sqa_slices;          /* SQA: Trotter slices P (1, or even, <= SPVAR_SQA_MAX_SLICES) */
    double sqa_beta;             /* SQA: inverse temperature, constant over the anneal */
    double sqa_gamma0, sqa_gamma1; /* SQA: transverse field, linear from gamma0 to gamma1 (both > 0) */
    int32_t sweeps_per_launch;   /* SA: sweeps of a phase's anneal per sweep launch; a phase then takes
                                    ceil(num_sweeps / sweeps_per_launch) launches, each resuming from the
                                    states the previous one wrote (results are identical: every random
                                    word is keyed by the absolute sweep).  0: the autotuner chooses
                                    between one launch per phase and four when replicas_per_block is 0,
                                    else one launch per phase.  Must be 0 with the SQA and PTICM
                                    samplers */
    int32_t pticm_temps;         /* PTICM: inverse temperatures R (2 .. 64), geometric from pticm_beta0
                                    to pticm_beta1; cluster moves and kept lists at k >= R / 2 */
    int32_t pticm_keep;          /* PTICM: lowest distinct states K kept per tracked replica (1 .. 64) */
    double pticm_beta0, pticm_beta1;
} spvar_params;

#define SPVAR_SAMPLER_SA 0  /* simulated annealing (Sec. III.A) */
#define SPVAR_SAMPLER_SQA 1 /* simulated quantum annealing: discrete-time path integral (Sec. III);
                               the sample of a run is its lowest-energy Trotter slice */
#define SPVAR_SAMPLER_PTICM 2 /* parallel tempering with isoenergetic cluster moves (Sec. III.D), one run
                                 per start and phase (as spvar_pticm_sample with exchanges and cluster
                                 moves on, icm_from = keep_from = R / 2, start word = the start, phase =
                                 the phase); the phase's sample is the kept lists, list after list, so
                                 its size is the number of states kept, at most 2 (R - R/2) K, and the
                                 elite is ceil(elite_threshold x that size).  fixing_sample_size must
                                 be 2 (R - R/2) K and solving_sample_size 0 or the same; num_sweeps
                                 >= 1; no correlation phase, no component boosting; every problem
                                 n <= 2048 and its 2Rn + 4R(dmax + 1) + 32n bytes in one CTA's
                                 shared memory (else SPVAR_ELIMIT).  Not taken by the server */

#define SPVAR_SWEEP_AUTO 0    /* register kernel when eligible, else general */
#define SPVAR_SWEEP_GENERAL 1 /* general integer-coupler kernel */
#define SPVAR_SWEEP_PM1 2     /* register-resident kernel (degree <= 8; |J| = 1 and dmax <= 30 in byte lanes, or
                                 one coupler magnitude per spin, or every |J| <= 15, with dmax <= 4094 in
                                 16-bit lanes), else the streaming +-1 kernel (|J| = 1, dmax <= 254) */
#define SPVAR_SWEEP_PM1S 3    /* streaming +-1 kernel (shared-memory neighbour offsets, 4 replicas per CTA) */
#define SPVAR_SWEEP_PM1W 4    /* warp-per-quad +-1 kernel: replicas_per_block / 4 warps, one quad each */
#define SPVAR_SWEEP_PM1Q 5    /* quad-group +-1 kernel (|J| = 1, degree <= 8, dmax <= 30): work items of
                                 replicas_per_block / 4 quads of the largest problem (more quads of smaller
                                 ones, at most 64), spin words alone in shared memory */
/* With the SQA sampler (replicas_per_block = 4): AUTO and PM1 take the register
 * form for +-1 couplers when it applies (two or more slices, at most 4 colour
 * classes, none larger than sweep_block; blocks 256/512/1024), else the item
 * walk (blocks 128/256/512); PM1 on small integer couplers (every |J| <= 15,
 * degree <= 8, dmax <= 254) takes their register form (block 256) when it
 * applies, else the general path; PM1S the item walk; GENERAL the general path;
 * PM1W and PM1Q are rejected (SPVAR_ELIMIT). */

#define SPVAR_FORM_BATCHED 0 /* every start of every problem in one persistent launch per phase */
#define SPVAR_FORM_PLAIN 1   /* one start at a time, one launch per kernel and start */

/* Output buffers; P = max_fix_phases + 1 phase slots (+1 when
 * corr_sample_size > 0: the correlation phase is slot 0), Smax = max sample
 * size, n_p = spins of problem p.  Rows are ordered problem-major then
 * start.  Any pointer may be NULL (not written).  device = 1: pointers are
 * device memory written on the stream without synchronising; device = 0:
 * host memory, the call synchronises. */
typedef struct spvar_result {
    int32_t device;
    int64_t *energies;    /* [starts][P][Smax] recorded full-problem energies */
    int32_t *counts;      /* [starts][P] samples recorded per phase slot */
    int32_t *nfree;       /* [starts][P] free spins when the phase sampled */
    int32_t *nphases;     /* [starts] phase slots used */
    int8_t *fixed;        /* [sum_p num_starts * n_p] final fix maps, original order */
    int64_t *best_energy; /* [starts] */
    int8_t *best_state;   /* [sum_p num_starts * n_p] best assignment (+1/-1) */
} spvar_result;

typedef struct spvar_plan spvar_plan;

/* Build an executable plan: device workspace for every start, acceptance
 * table, work queues and the captured per-phase CUDA graph.
 * problems: host array [nproblems] of handles (all on the current device);
 * the same table is used for all problems (dmax = largest dmax, scale of
 * problems[0]; every problem must share energy_scale).
 * Errors: EINVAL, ELIMIT, ENOMEM, EBUDGET (workspace > budget_bytes when
 * budget_bytes > 0), ECUDA. */
int spvar_plan_create(const spvar_problem *const *problems, int32_t nproblems,
                      const spvar_params *prm, size_t budget_bytes, void *stream,
                      spvar_plan **out);

/* Device bytes the plan holds. */
size_t spvar_plan_workspace_bytes(const spvar_plan *plan);

/* Run Alg. 2 for every start of every problem.  seeds: host [nproblems]
 * (problem p uses key seeds[p]; start s of it uses counter word start = s). */
int spvar_plan_run(spvar_plan *plan, const uint64_t *seeds, const spvar_result *res,
                   void *stream);

void spvar_plan_destroy(spvar_plan *plan);

/* Convenience: plan_create + plan_run for one problem.  The plan is kept
 * after the call and reused by a later call whose problem has the same
 * structure (n, nnz, capacities, degree bound, dmax, energy scale, colour
 * class sizes, coupler kind) and whose parameters are byte-for-byte the same:
 * that call skips plan creation (workspace allocation, autotuning lookup,
 * graph capture) and runs the kept plan on its own problem's data, with
 * results identical to a fresh plan.  At most 4 plans are kept, each holding
 * at most 256 MB of device memory (larger ones are freed after the call);
 * spvar_solve_cache_release frees them.  Safe to call from several threads
 * (a kept plan serves one call at a time).
 * Errors: as spvar_plan_create and spvar_plan_run. */
int spvar_solve(const spvar_problem *p, const spvar_params *prm, uint64_t seed,
                const spvar_result *res, void *stream);

/* Frees every plan spvar_solve keeps (their device memory and graphs).  Call
 * it with no spvar_solve in flight, e.g. before freeing the device. */
void spvar_solve_cache_release(void);

/* Work statistics of the last plan_run: spin-flip attempts (sum over
 * phases of samples x sweeps x free spins) and phases executed. */
int spvar_plan_stats(const spvar_plan *plan, int64_t *attempts, int32_t *phases);

/* Sweeps per sweep launch the plan uses (requested, or chosen by the
 * autotuner); num_sweeps when a phase is one launch. */
int spvar_plan_sweeps_per_launch(const spvar_plan *plan, int32_t *sweeps);

/* ------------------------------------------------------------------ */
/* Serving: a request loop with continuous batching                      */
/* ------------------------------------------------------------------ */
/* Requests (problems) are admitted in arrival order when a request slot is
 * free and their device workspace fits budget_bytes; each engine step runs
 * one phase of Alg. 2 for every admitted start of every request (one
 * persistent launch sequence, CUDA graph), so requests arriving while others
 * run join at the next phase boundary.  State stays on the device between
 * steps; results are copied back when a request finishes.  A request's
 * result is identical whether it ran alone or in any mix (randomness is
 * keyed by seed, start, phase, sweep, spin and replica only). */
typedef struct spvar_server spvar_server;

typedef struct spvar_server_config {
    spvar_params params;    /* Alg. 2 parameters of every request; sweep_kernel = SPVAR_SWEEP_PM1
                               restricts the server to +-1 couplers (faster sweep: the streaming
                               +-1 kernel; SPVAR_SWEEP_PM1Q: the quad-group kernel) */
    size_t budget_bytes;    /* device memory for admitted requests' workspaces */
    int32_t max_n;          /* largest request: spins, CSR entries, degree */
    int32_t max_nnz;
    int32_t max_degree;
    int32_t max_dmax;       /* acceptance table covers flip costs up to this */
    int32_t energy_scale;   /* shared by all requests */
    int32_t max_requests;   /* requests in flight at once */
    int32_t sweeps_per_step; /* sweeps of every in-flight anneal per engine step (0: a whole phase).  A
                                request that arrives is admitted at the next step, so smaller steps
                                shorten its wait; results do not depend on it.  Must be 0 with the
                                SQA sampler (params.sampler = SPVAR_SAMPLER_SQA: every request is
                                sampled by SQA, the item walk over (slice, spin)) */
} spvar_server_config;

typedef struct spvar_request_info {
    int32_t state;       /* 0 queued, 1 running, 2 done */
    int32_t n;
    int64_t best_energy; /* min over starts (done only) */
    double latency_s;    /* submit -> results on the host (done only) */
    double queue_s;      /* submit -> admission (admitted only) */
    int64_t attempts;    /* spin-flip attempts of the request (done only) */
} spvar_request_info;

/* Allocates the arena (budget_bytes), the slot table and the acceptance
 * table on the current device and captures the phase graph. */
int spvar_server_create(const spvar_server_config *cfg, spvar_server **out);
/* Host CSR problem (validated and laid out here), seed; returns its id.
 * ELIMIT beyond the configured sizes, EBUDGET if it can never fit. */
int spvar_server_submit(spvar_server *s, int32_t n, const int32_t *row_ptr, const int32_t *col,
                        const int32_t *val, const int32_t *h, int64_t offset, uint64_t seed,
                        int64_t *id);
/* One engine iteration on the calling thread: admit, one phase, retire.
 * *active = requests still in flight.  EINVAL while the background engine runs. */
int spvar_server_step(spvar_server *s, int32_t *active);
/* Background engine thread (steps while work exists). */
int spvar_server_start(spvar_server *s);
int spvar_server_stop(spvar_server *s);
/* Waits up to timeout_s (0: just query) for a request; ETIMEOUT if not done. */
int spvar_server_wait(spvar_server *s, int64_t id, double timeout_s, spvar_request_info *info);
/* Host copies of a finished request's results (layouts as spvar_result with
 * one problem; any pointer may be NULL). */
int spvar_server_result(spvar_server *s, int64_t id, int64_t *best_energy, int8_t *best_state,
                        int8_t *fixed, int64_t *energies, int32_t *counts, int32_t *nfree);
/* Forgets a finished request's host results. */
int spvar_server_release(spvar_server *s, int64_t id);
int spvar_server_stats(spvar_server *s, int64_t *requests_done, int64_t *attempts_done,
                       int32_t *queued, int32_t *running);
/* Sum of the sweep launches' durations (ms; CUDA events recorded around the
 * sweep of every engine step) and the number of steps timed, since creation. */
int spvar_server_sweep_time(spvar_server *s, double *total_ms, int64_t *launches);
void spvar_server_destroy(spvar_server *s);

/* Profiling: when on, plan_run waits for every phase and adds up the
 * duration of the sweep kernel (CUDA events recorded on the run's stream
 * around each sweep launch, also inside the captured graph). */
int spvar_plan_set_profiling(spvar_plan *plan, int32_t on);

/* Sum of sweep-kernel durations (ms) and sweep launches of the last
 * profiled plan_run. */
int spvar_plan_sweep_time(const spvar_plan *plan, double *total_ms, int32_t *launches);

/* Sum of the persistence-pass durations (ms) of the last profiled plan_run:
 * from the end of each sweep launch to the end of the phase's fold/compact
 * (boosting, elite, counts and fixing, fold and compact kernels). */
int spvar_plan_post_time(const spvar_plan *plan, double *total_ms);

/* The sweep launch shape the plan chose (autotuned or requested): threads
 * per CTA, replicas per CTA, kernel (0: general kernel reading its layout
 * from global memory, 1: general kernel with the layout staged in shared
 * memory, 2: register-resident +-1 kernel, 3: streaming +-1 kernel, 4:
 * warp-per-quad +-1 kernel, 5: simulated quantum annealing kernel walking
 * (spin, slice) items, 6: simulated quantum annealing kernel in register form:
 * each thread keeps one spin of every colour class in registers and sweeps a
 * fixed set of its slices, 7: quad-group +-1 kernel), persistent grid size. */
int spvar_plan_shape(const spvar_plan *plan, int32_t *block, int32_t *replicas_per_block,
                     int32_t *staged, int32_t *grid);

/* ------------------------------------------------------------------ */
/* Measurement: integer issue ceilings of the current GPU               */
/* ------------------------------------------------------------------ */
/* The paper has no counterpart: these probes give the measured ceilings that
 * the sweep kernels' rooflines divide by (the sweep is bound by 32-bit integer
 * instruction issue, not by memory).  One launch of `iters` iterations on
 * every CTA the SMs keep resident (256 threads each), each thread running 16
 * independent register chains of one instruction form:
 *   form 0  three-input logic (lop3)           form 1  three-input add
 *   form 2  32-bit multiply-add (mad.lo)       form 3  forms 0 and 2 alternating
 *   form 4  32x32->64 multiply (mul.wide) whose halves one lop3 folds
 *   form 5  whole Philox4x32-10 blocks
 * ops_per_s: thread-level operations per second of the timed launch (forms
 * 0-3 count every instruction of the form, form 4 the wide multiplies, form 5
 * the Philox blocks), timed with CUDA events on `stream` after one untimed
 * launch of iters/8 iterations; ms (may be NULL): the timed launch.
 * Synchronises the stream.  Errors: EINVAL (form outside 0-5, iters < 1, NULL
 * ops_per_s), ECUDA. */
int spvar_measure_issue_rate(int32_t form, int32_t iters, double *ops_per_s, double *ms, void *stream);

#ifdef __cplusplus
}
#endif
#endif
