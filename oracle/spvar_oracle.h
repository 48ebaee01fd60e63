/*
 * spvar_oracle.h -- plain, slow, single-threaded C restatement of the
 * sample-persistence variable reduction method (SPVAR, Alg. 1; Multi-start
 * SPVAR, Alg. 2, Sec. II.A-II.C) with simulated annealing as the sampler, and
 * the paper's other samplers of Sec. III: simulated quantum annealing and
 * parallel tempering with isoenergetic cluster moves (PTICM).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists so that tests, the
 * smoke check and the CPU baseline leg of the benchmark can check and time
 * the CUDA library.  The product path never links, loads or calls it, and it
 * shares no code, header, table or helper with the CUDA library.
 *
 * Conventions (Sec. I problem statement, readings listed in the design notes):
 *   E(s) = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i + offset,  s_i in {-1,+1}.
 *   Symmetric CSR: every coupler appears in both rows with the same value,
 *   columns strictly ascending inside a row, no diagonal entries.
 *   Spins are int8 values -1/+1; energies are int64.
 *
 * Return codes: 0 = ok, negative = invalid input (documented per function).
 */
#ifndef SPVAR_ORACLE_H
#define SPVAR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11):
 * out = philox(ctr, key).  Parity pinned against cuRAND's host generator. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Edge list (ei[e], ej[e], J[e]), e < m, i != j, no duplicates, J != 0
 * allowed to be any int32 -> symmetric CSR (row_ptr[n+1], col/val[2m]).
 * Returns 0, or -1 on a self loop / out-of-range index / duplicate pair. */
int or_csr_from_edges(int32_t n, int64_t m, const int32_t *ei, const int32_t *ej,
                      const int32_t *J, int32_t *row_ptr, int32_t *col, int32_t *val);

/* Colour classes used for the sweep order.  If the graph is bipartite each
 * connected component is 2-coloured by BFS distance parity from its
 * lowest-index vertex; otherwise first-fit greedy in index order.  Writes
 * colour[n], returns the number of colours (>= 1 for n >= 1, 0 for n == 0). */
int32_t or_colour(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t *colour);

/* Largest possible energy change of one flip:
 * dmax = 2 * max_i (sum_j |J_ij| + |h_i|). */
int64_t or_dmax(int32_t n, const int32_t *row_ptr, const int32_t *val, const int32_t *h);

/* Acceptance thresholds: thr[t*(dmax+1)+d] =
 * min(2^32-1, floor(2^32 * exp(-beta[t] * d / scale))), d = 0..dmax. */
void or_thresholds(int32_t T, const double *beta, int32_t dmax, int32_t scale, uint32_t *thr);

/* Geometric schedule beta_t = beta0 * (beta1/beta0)^(t/(T-1)), endpoints
 * included (T == 1 gives beta0). */
void or_beta_geometric(int32_t T, double beta0, double beta1, double *beta);

/* E(s) without the offset. */
int64_t or_energy(int32_t n, const int32_t *row_ptr, const int32_t *col,
                  const int32_t *val, const int32_t *h, const int8_t *s);

/* Simulated annealing sample (one independent run per replica r < S).
 * Random word for (spin i, sweep slot t, replica r): word (r & 3) of
 * philox(ctr = {i, phase*2^20 + t, r >> 2, start}, key = {seed lo, seed hi});
 * slot 2^20-1 is the initial state (s_i = +1 iff the top bit is set).
 * Replicas r0 .. r0+S-1 are computed (rows 0 .. S-1 of the output).
 * Sweep t visits colour 0 ascending index, colour 1, ...; a flip with
 * dE = -2 s_i (h_i + sum_j J_ij s_j) is accepted iff dE <= 0 or
 * word < thr[t][dE].  Writes spins[S*n] (row r = replica r) and e[S]
 * (energy without offset).  If incr_err != NULL, the running energy is
 * compared with a full recomputation after every sweep of every replica and
 * the largest absolute difference is stored there.
 * Returns 0, -1 on bad sizes (T >= 2^20-1, phase >= 2^12), -2 if a dE
 * exceeds dmax. */
int or_sample(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *val,
              const int32_t *h, const int32_t *colour, int32_t ncol,
              int32_t T, const uint32_t *thr, int32_t dmax,
              int32_t r0, int32_t S, uint64_t seed, uint32_t start, uint32_t phase,
              int8_t *spins, int64_t *e, int64_t *incr_err);

/* ---- Simulated quantum annealing (SQA, Sec. III: discrete-time path-integral
 * Monte Carlo of the transverse-field Ising model, a second sampler for Alg. 1).
 * P Trotter slices s^tau (tau = 0..P-1, periodic), weight exp(-A) with
 *   A(s) = (beta/P) sum_tau E(s^tau)/scale - Jp sum_tau sum_i s_i^tau s_i^(tau+1),
 *   Jp(t) = -1/2 ln tanh(beta Gamma_t / P);
 * P = 1 has no slice coupling (classical).  Flipping s_i^tau changes A by
 *   dA = (2 beta / P) (k - bias) / scale + 4 Jp (a - 1),
 * k = dE/2 + bias (bias = dmax/2; dE the classical flip cost in slice tau) and
 * a = number of the two slice neighbours equal to s_i^tau (a = 1 when P = 1).
 * Metropolis acceptance min(1, exp(-dA)) with a 32-bit uniform u, as a carry:
 *   ent[(t*3 + a)*W + k] = 2^32 - min(2^32, floor(2^32 exp(-dA)))   (W = 2 bias + 1)
 * and the move is accepted iff u + ent < 2^32 (ent = 0: always).
 * beta[T], gamma[T]: inverse temperature and transverse field of each sweep
 * (quantum annealing: beta constant, gamma falling). */
void or_sqa_table(int32_t T, int32_t P, const double *beta, const double *gamma, int32_t dmax, int32_t scale,
                  uint64_t *ent);

/* SQA samples of replicas r0..r0+S-1 (P even, or P = 1).  Random word of
 * spin i in slice tau: the SA counter with spin word i | tau << 16.  Sweep:
 * colour classes in order; inside a class the even slices, then the odd
 * slices; indices ascending.  The sample of a run is its lowest-energy slice
 * (lowest tau on ties): spins[S][n], e[S] (without offset), slice[S].
 * Returns 0, -1 on bad arguments, -2 if a flip cost exceeds dmax. */
int or_sqa_sample(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *val,
                  const int32_t *h, const int32_t *colour, int32_t ncol,
                  int32_t T, int32_t P, const uint64_t *ent, int32_t dmax,
                  int32_t r0, int32_t S, uint64_t seed, uint32_t start, uint32_t phase,
                  int8_t *spins, int64_t *e, int32_t *slice);

/* Isoenergetic cluster move between two replicas a and b of one temperature
 * (the cluster step of PTICM, Sec. III.D; Houdayer's move): D = the spins
 * where a and b differ; the cluster is the connected component of `seed_spin`
 * (which must be in D) in the graph of couplers restricted to D; both
 * replicas flip on it, which leaves E(a) + E(b) unchanged.  Returns the
 * cluster size, or -1 if seed_spin is out of range or not in D. */
int32_t or_icm_move(int32_t n, const int32_t *row_ptr, const int32_t *col, int8_t *a, int8_t *b,
                    int32_t seed_spin);

/* Parallel tempering with isoenergetic cluster moves (PTICM, Sec. III.D) as a
 * sampler of Alg. 1.  R inverse temperatures beta_0 < ... < beta_{R-1}, two
 * replicas per temperature (replica r = 2k + c, copy c of temperature k),
 * all started from the initial-state words of or_sample.  Each of T sweeps:
 *   1. a Metropolis sweep of every replica at its temperature: thr[k][dE]
 *      (or_thresholds of beta_k), random word of spin i of replica r as in
 *      or_sample with sweep t;
 *   2. if flags & 2, for every k >= icm_from with D non-empty, or_icm_move
 *      on the two copies, seeded at element floor(u |D| / 2^32) of D in index
 *      order, u = word 0 of Philox((0xFFFF0000 | k, phase 2^20 + t, 0, start));
 *   3. if flags & 1, replica exchange between temperatures k and k + 1 for
 *      every k = t (mod 2), copy 0 then copy 1: with d = E(k, c) - E(k+1, c),
 *      accepted iff d <= 0 or u < xthr[k][d] (xthr = or_thresholds of
 *      beta_{k+1} - beta_k over d = 1 .. dx), u = word 0 of
 *      Philox((0xFFFE0000 | (2k + c), phase 2^20 + t, 0, start)); accepted
 *      exchanges swap the two replicas' states and energies;
 *   4. for every temperature k >= keep_from and copy c, the current state is
 *      offered to that replica's list of the K lowest-energy distinct states
 *      seen (ordered by energy, then by first sight; a state already listed
 *      is not listed again; a full list takes a state only if its energy is
 *      below the list's highest, which then leaves).
 * Outputs: kept[2 (R - keep_from)][K][n], kept_e[..][K] (without offset),
 * nkept[2 (R - keep_from)] (replica order k = keep_from.., copy 0 then 1),
 * and the final states final[2R][n], final_e[2R].  Returns 0, -1 on bad
 * arguments, -2 if a flip cost exceeds dmax or an energy gap exceeds dx. */
int or_pticm_sample(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *val,
                    const int32_t *h, const int32_t *colour, int32_t ncol,
                    int32_t R, int32_t T, const uint32_t *thr, int32_t dmax, const uint32_t *xthr, int32_t dx,
                    int32_t icm_from, int32_t keep_from, int32_t K, int32_t flags,
                    uint64_t seed, uint32_t start, uint32_t phase,
                    int8_t *kept, int64_t *kept_e, int32_t *nkept, int8_t *final, int64_t *final_e);

/* Elite sample size k = ceil(elite * S), clamped to [1, S] (Alg. 1). */
int32_t or_elite_count(double elite, int32_t S);

/* Indices of the k lowest-energy samples ordered by (energy, index). */
void or_elite(int32_t S, const int64_t *e, int32_t k, int32_t *idx);

/* Persistence pass (Alg. 1, Sec. II.C).  Over the elite rows, optionally
 * multiplied by their value at the reference spin rho (the lowest-index spin
 * of maximum degree) when canon != 0, counts cnt[i] = #{+1}; fixes
 * v = sign(2cnt-k) when fix_den*|2cnt-k| >= fix_num*k.  Writes cnt[n],
 * fixed[n] (0 free, +1, -1) and *rho_out (-1 without canonicalisation).
 * Returns the number of fixed spins. */
int32_t or_persistence(int32_t n, const int32_t *row_ptr, int32_t S, const int8_t *spins,
                       const int64_t *e, int32_t k, int32_t fix_num, int32_t fix_den,
                       int32_t canon, int32_t *cnt, int8_t *fixed, int32_t *rho_out);

/* Fold and compact (Alg. 1 "update J and h").  Free spins keep their order;
 * h'_i = h_i + sum_{j fixed} J_ij v_j; offset' = offset + sum_{i fixed} h_i v_i
 * + sum_{i<j both fixed} J_ij v_i v_j; CSR of free-free couplers; colours
 * inherited.  Output arrays must hold n+1 / nnz / n entries.  Writes
 * *n_out, *offset_out, returns 0. */
int or_reduce(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *val,
              const int32_t *h, int64_t offset, const int32_t *colour, const int8_t *fixed,
              int32_t *n_out, int32_t *row_ptr_out, int32_t *col_out, int32_t *val_out,
              int32_t *h_out, int64_t *offset_out, int32_t *colour_out, int32_t *old_of_new);

/* Connected components (Sec. II.C boosting): comp[i] = index of i's
 * component, components numbered in increasing order of their lowest spin
 * index.  Returns the number of components. */
int32_t or_components(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t *comp);

/* Disconnected-component boosting of one sample (Sec. II.C): partial energy
 * of every sample on every component, each component's partial samples
 * sorted by (partial energy, sample index), merged rank by rank.  spins
 * [S*n] and e [S] (without offset) are replaced by the merged sample. */
int or_component_boost(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *val,
                       const int32_t *h, int32_t S, int8_t *spins, int64_t *e);

/* Tree pre-processing (Sec. II.C), in rounds.  In each round every active
 * spin of active degree 0, and every spin of active degree 1 except the
 * lower-index end of an isolated coupler, is eliminated at once:
 *   degree 0:              fixed to -sign(h) (+1 if h = 0);
 *   degree 1, |J| <= |h|:  fixed to -sign(h), J v folded into the neighbour;
 *   degree 1, |J| >  |h|:  inferred s_i = -sign(J) s_j: h_j -= sign(J) h_i,
 *                          offset -= |J|.
 * Biases and the constant are updated in place (h [n], *offset); code[i] is
 * 0 (kept), +1/-1 (fixed to that value) or 2 (inferred from parent[i]);
 * order[] lists the inferred spins in elimination order.  Returns the number
 * of eliminated spins; *ninfer gets the number of inferred ones. */
int32_t or_tree(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *val, int32_t *h,
                int64_t *offset, int8_t *code, int32_t *parent, int32_t *order, int32_t *ninfer);

/* Drops every spin with code != 0 and its couplers WITHOUT folding (the
 * tree step has folded already); colours inherited.  Same outputs as or_reduce. */
int or_compact(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *val,
               const int32_t *h, int64_t offset, const int32_t *colour, const int8_t *code,
               int32_t *n_out, int32_t *row_ptr_out, int32_t *col_out, int32_t *val_out,
               int32_t *h_out, int64_t *offset_out, int32_t *colour_out, int32_t *old_of_new);

/* Multi-start SPVAR (Alg. 2) with SA as the sampler. */
typedef struct or_params {
    int32_t num_starts;
    int32_t fixing_sample_size;
    int32_t solving_sample_size;   /* 0: no solving phase */
    int32_t num_sweeps;
    double elite_threshold;
    int32_t fix_num, fix_den;      /* fixing_threshold = fix_num / fix_den */
    int32_t iterate;               /* 1: repeat SPVAR until no free spin (ISPVAR) */
    int32_t max_fix_phases;        /* cap on SPVAR phases per start (>= 1) */
    int32_t canon;                 /* -1: when every h is 0; 0: never; 1: always */
    int32_t start0;                /* start st uses counter word start0 + st */
    int32_t boost;                 /* 1: component boosting of the solving sample (Sec. II.C) */
    int32_t tree;                  /* 1: tree pre-processing after every SPVAR reduction (Sec. II.C) */
    /* Correlation fixing (Sec. II.C, Alg. 2 optional step; sample split in the
     * appendix): for a problem with every h = 0, a first phase samples
     * corr_sample_size states, takes the corr_elite_threshold elite, fixes the
     * reference spin rho to +1 and fixes every spin j whose elite correlation
     * with rho has |mean(s_rho s_j)| >= corr_num / corr_den to sign(mean).
     * 0 = off; skipped when some h != 0. */
    int32_t corr_sample_size;
    int32_t corr_num, corr_den;
    double corr_elite_threshold;
    /* Sampler of every phase: 0 = SA with the table thr; 1 = SQA with
     * sqa_slices slices, constant sqa_beta and a transverse field linear from
     * sqa_gamma0 to sqa_gamma1 over the sweeps (or_gamma_linear); 2 = PTICM
     * (Sec. III.D): one run per start and phase with pticm_temps inverse
     * temperatures geometric from pticm_beta0 to pticm_beta1, exchanges and
     * cluster moves on, cluster moves and kept lists in the lower half of the
     * temperatures (k >= R / 2); the phase's sample is the kept lists
     * (pticm_keep lowest distinct states per tracked replica) in list order,
     * so its size is the number of states kept (at most 2 (R - R/2) K, which
     * fixing_sample_size must equal; solving_sample_size 0 or the same; no
     * correlation step, no boosting). */
    int32_t sampler, sqa_slices;
    double sqa_beta, sqa_gamma0, sqa_gamma1;
    int32_t energy_scale;          /* the problem's scale (SQA and PTICM tables; >= 1) */
    int32_t pticm_temps, pticm_keep;
    double pticm_beta0, pticm_beta1;
} or_params;

/* gamma[t] = g0 + (g1 - g0) t / (T - 1); gamma[0] = g0 when T = 1. */
void or_gamma_linear(int32_t T, double g0, double g1, double *gamma);

/* Outputs (caller-allocated, P = max_fix_phases + 1 (+1 with corr_sample_size > 0),
 * Smax = max sample size):
 *   energies[num_starts][P][Smax]  recorded full-problem energies
 *   counts[num_starts][P]          samples recorded in each phase slot
 *   nfree[num_starts][P]           free spins when that phase sampled
 *   nphases[num_starts]            phase slots used
 *   fixed[num_starts][n0]          final fix map in original indices
 *   best_e[num_starts], best_state[num_starts][n0] (+1/-1)
 * thr is the table for the original problem (dmax from or_dmax on it).
 * Returns 0 or a negative code from a step. */
int or_solve(int32_t n0, const int32_t *row_ptr0, const int32_t *col0, const int32_t *val0,
             const int32_t *h0, int64_t offset0, const or_params *prm,
             const uint32_t *thr, int32_t dmax, uint64_t seed,
             int64_t *energies, int32_t *counts, int32_t *nfree, int32_t *nphases,
             int8_t *fixed, int64_t *best_e, int8_t *best_state);

#ifdef __cplusplus
}
#endif
#endif
