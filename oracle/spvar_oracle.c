/*
 * spvar_oracle.c -- TEST INFRASTRUCTURE ONLY (see spvar_oracle.h).
 *
 * A plain single-threaded restatement of Alg. 1 (SPVAR) and Alg. 2
 * (Multi-start SPVAR) with simulated annealing as the sampler.  Every loop
 * follows the order the method states; nothing is blocked, fused or
 * reordered.  It is deliberately slow and shares nothing with the CUDA
 * library: tests compare the two element by element.
 */
#include "spvar_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64       */
/* multiplies with a Weyl-sequence key schedule.                            */
/* ---------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ---------------------------------------------------------------------- */
/* Problem construction                                                     */
/* ---------------------------------------------------------------------- */
int or_csr_from_edges(int32_t n, int64_t m, const int32_t *ei, const int32_t *ej,
                      const int32_t *J, int32_t *row_ptr, int32_t *col, int32_t *val)
{
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!deg) return -1;
    for (int64_t e = 0; e < m; ++e) {
        if (ei[e] < 0 || ei[e] >= n || ej[e] < 0 || ej[e] >= n || ei[e] == ej[e]) {
            free(deg);
            return -1;
        }
        deg[ei[e]]++;
        deg[ej[e]]++;
    }
    row_ptr[0] = 0;
    for (int32_t i = 0; i < n; ++i) row_ptr[i + 1] = (int32_t)(row_ptr[i] + deg[i]);
    /* place entries, then sort each row by column (insertion sort: rows are short) */
    int64_t *fill = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!fill) { free(deg); return -1; }
    for (int64_t e = 0; e < m; ++e) {
        int32_t a = ei[e], b = ej[e];
        int64_t pa = row_ptr[a] + fill[a]++;
        col[pa] = b; val[pa] = J[e];
        int64_t pb = row_ptr[b] + fill[b]++;
        col[pb] = a; val[pb] = J[e];
    }
    int rc = 0;
    for (int32_t i = 0; i < n && rc == 0; ++i) {
        for (int32_t p = row_ptr[i] + 1; p < row_ptr[i + 1]; ++p) {
            int32_t c = col[p], v = val[p];
            int32_t q = p - 1;
            while (q >= row_ptr[i] && col[q] > c) {
                col[q + 1] = col[q];
                val[q + 1] = val[q];
                --q;
            }
            col[q + 1] = c;
            val[q + 1] = v;
        }
        for (int32_t p = row_ptr[i] + 1; p < row_ptr[i + 1]; ++p)
            if (col[p] == col[p - 1]) rc = -1; /* duplicate pair */
    }
    free(deg);
    free(fill);
    return rc;
}

int32_t or_colour(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t *colour)
{
    if (n == 0) return 0;
    /* bipartite attempt: BFS from the lowest unvisited vertex, colour = parity */
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t i = 0; i < n; ++i) colour[i] = -1;
    for (int32_t root = 0; root < n; ++root) {
        if (colour[root] >= 0) continue;
        int32_t head = 0, tail = 0;
        colour[root] = 0;
        queue[tail++] = root;
        while (head < tail) {
            int32_t v = queue[head++];
            for (int32_t p = row_ptr[v]; p < row_ptr[v + 1]; ++p) {
                int32_t u = col[p];
                if (colour[u] < 0) {
                    colour[u] = 1 - colour[v];
                    queue[tail++] = u;
                }
            }
        }
    }
    free(queue);
    int bipartite = 1;
    int32_t used = 1;
    for (int32_t v = 0; v < n; ++v) {
        if (colour[v] == 1) used = 2;
        for (int32_t p = row_ptr[v]; p < row_ptr[v + 1]; ++p)
            if (colour[col[p]] == colour[v]) bipartite = 0;
    }
    if (bipartite) return used;

    /* first-fit greedy in index order: smallest colour no lower-index
       neighbour already has */
    int32_t *seen = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    for (int32_t c = 0; c <= n; ++c) seen[c] = -1;
    int32_t ncol = 0;
    for (int32_t v = 0; v < n; ++v) {
        for (int32_t p = row_ptr[v]; p < row_ptr[v + 1]; ++p) {
            int32_t u = col[p];
            if (u < v) seen[colour[u]] = v;
        }
        int32_t c = 0;
        while (seen[c] == v) ++c;
        colour[v] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(seen);
    return ncol;
}

int64_t or_dmax(int32_t n, const int32_t *row_ptr, const int32_t *val, const int32_t *h)
{
    int64_t best = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t s = llabs((long long)h[i]);
        for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) s += llabs((long long)val[p]);
        if (s > best) best = s;
    }
    return 2 * best;
}

void or_thresholds(int32_t T, const double *beta, int32_t dmax, int32_t scale, uint32_t *thr)
{
    for (int32_t t = 0; t < T; ++t) {
        for (int32_t d = 0; d <= dmax; ++d) {
            double x = ldexp(exp(-beta[t] * (double)d / (double)scale), 32);
            double f = floor(x);
            uint32_t v = (f >= 4294967295.0) ? 0xFFFFFFFFu : (uint32_t)f;
            thr[(int64_t)t * (dmax + 1) + d] = v;
        }
    }
}

void or_beta_geometric(int32_t T, double beta0, double beta1, double *beta)
{
    for (int32_t t = 0; t < T; ++t) {
        if (T == 1) { beta[t] = beta0; continue; }
        beta[t] = beta0 * pow(beta1 / beta0, (double)t / (double)(T - 1));
    }
}

int64_t or_energy(int32_t n, const int32_t *row_ptr, const int32_t *col,
                  const int32_t *val, const int32_t *h, const int8_t *s)
{
    int64_t e = 0;
    for (int32_t i = 0; i < n; ++i) {
        e += (int64_t)h[i] * s[i];
        for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
            if (col[p] > i) e += (int64_t)val[p] * s[i] * s[col[p]];
    }
    return e;
}

/* ---------------------------------------------------------------------- */
/* Simulated annealing                                                      */
/* ---------------------------------------------------------------------- */
#define SWEEP_BITS 20u
#define INIT_SLOT ((1u << SWEEP_BITS) - 1u)

static uint32_t rng_word(uint64_t seed, uint32_t start, uint32_t phase, uint32_t slot,
                         int32_t spin, int32_t replica)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)spin, (phase << SWEEP_BITS) + slot, (uint32_t)replica >> 2, start};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return out[replica & 3];
}

int or_sample(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *val,
              const int32_t *h, const int32_t *colour, int32_t ncol,
              int32_t T, const uint32_t *thr, int32_t dmax,
              int32_t r0, int32_t S, uint64_t seed, uint32_t start, uint32_t phase,
              int8_t *spins, int64_t *e, int64_t *incr_err)
{
    if (T < 0 || (uint32_t)T >= INIT_SLOT || phase >= (1u << 12) || S < 0 || r0 < 0) return -1;
    /* sweep order: colour classes in increasing colour, index ascending */
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t m = 0;
    for (int32_t c = 0; c < ncol; ++c)
        for (int32_t i = 0; i < n; ++i)
            if (colour[i] == c) order[m++] = i;
    if (m != n) { free(order); return -1; }
    int64_t worst = 0;
    int rc = 0;
    for (int32_t row = 0; row < S && rc == 0; ++row) {
        const int32_t r = r0 + row; /* replica index */
        int8_t *s = spins + (int64_t)row * n;
        for (int32_t i = 0; i < n; ++i)
            s[i] = (rng_word(seed, start, phase, INIT_SLOT, i, r) >> 31) ? 1 : -1;
        int64_t E = or_energy(n, row_ptr, col, val, h, s);
        for (int32_t t = 0; t < T && rc == 0; ++t) {
            const uint32_t *row = thr + (int64_t)t * (dmax + 1);
            for (int32_t q = 0; q < n; ++q) {
                int32_t i = order[q];
                int64_t f = h[i];
                for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) f += (int64_t)val[p] * s[col[p]];
                int64_t dE = -2 * (int64_t)s[i] * f;
                uint32_t u = rng_word(seed, start, phase, (uint32_t)t, i, r);
                int accept;
                if (dE <= 0) {
                    accept = 1;
                } else {
                    if (dE > dmax) { rc = -2; break; }
                    accept = u < row[dE];
                }
                if (accept) {
                    s[i] = (int8_t)-s[i];
                    E += dE;
                }
            }
            if (incr_err) {
                int64_t Er = or_energy(n, row_ptr, col, val, h, s);
                int64_t d = llabs((long long)(Er - E));
                if (d > worst) worst = d;
            }
        }
        e[row] = E;
    }
    if (incr_err) *incr_err = worst;
    free(order);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Simulated quantum annealing (discrete-time path integral)                */
/* ---------------------------------------------------------------------- */
void or_sqa_table(int32_t T, int32_t P, const double *beta, const double *gamma, int32_t dmax, int32_t scale,
                  uint64_t *ent)
{
    const int32_t bias = dmax / 2, W = 2 * bias + 1;
    for (int32_t t = 0; t < T; ++t) {
        /* slice coupling of this sweep (none for a single slice) */
        double jp = (P > 1) ? -0.5 * log(tanh(beta[t] * gamma[t] / (double)P)) : 0.0;
        for (int32_t a = 0; a < 3; ++a) {
            for (int32_t k = 0; k < W; ++k) {
                double dA = (2.0 * beta[t] / (double)P) * (double)(k - bias) / (double)scale +
                            4.0 * jp * (double)(a - 1);
                double x = floor(ldexp(exp(-dA), 32));
                uint64_t thr = (x >= 4294967296.0) ? (1ull << 32) : (uint64_t)x;
                ent[((int64_t)t * 3 + a) * W + k] = (1ull << 32) - thr;
            }
        }
    }
}

void or_gamma_linear(int32_t T, double g0, double g1, double *gamma)
{
    for (int32_t t = 0; t < T; ++t) gamma[t] = (T == 1) ? g0 : g0 + (g1 - g0) * (double)t / (double)(T - 1);
}

int or_sqa_sample(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *val,
                  const int32_t *h, const int32_t *colour, int32_t ncol,
                  int32_t T, int32_t P, const uint64_t *ent, int32_t dmax,
                  int32_t r0, int32_t S, uint64_t seed, uint32_t start, uint32_t phase,
                  int8_t *spins, int64_t *e, int32_t *slice)
{
    if (T < 0 || (uint32_t)T >= INIT_SLOT || phase >= (1u << 12) || S < 0 || r0 < 0 || P < 1 ||
        (P > 1 && (P & 1)) || P > 1024 || n >= (1 << 16))
        return -1;
    const int32_t bias = dmax / 2, W = 2 * bias + 1;
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *cstart = (int32_t *)malloc(sizeof(int32_t) * ((size_t)ncol + 2));
    int32_t m = 0;
    for (int32_t c = 0; c < ncol; ++c) {
        cstart[c] = m;
        for (int32_t i = 0; i < n; ++i)
            if (colour[i] == c) order[m++] = i;
    }
    cstart[ncol] = m;
    int8_t *x = (int8_t *)malloc((size_t)P * (size_t)n + 1); /* x[tau*n + i] */
    if (m != n) { free(order); free(cstart); free(x); return -1; }
    int rc = 0;
    for (int32_t row = 0; row < S && rc == 0; ++row) {
        const int32_t r = r0 + row;
        for (int32_t tau = 0; tau < P; ++tau)
            for (int32_t i = 0; i < n; ++i)
                x[(int64_t)tau * n + i] =
                    (rng_word(seed, start, phase, INIT_SLOT, i | (tau << 16), r) >> 31) ? 1 : -1;
        for (int32_t t = 0; t < T && rc == 0; ++t) {
            for (int32_t c = 0; c < ncol && rc == 0; ++c) {
                for (int32_t par = 0; par < (P > 1 ? 2 : 1) && rc == 0; ++par) {
                    for (int32_t tau = par; tau < P && rc == 0; tau += 2) {
                        int8_t *s = x + (int64_t)tau * n;
                        const int8_t *up = x + (int64_t)((tau + 1) % P) * n;
                        const int8_t *dn = x + (int64_t)((tau + P - 1) % P) * n;
                        for (int32_t q = cstart[c]; q < cstart[c + 1]; ++q) {
                            const int32_t i = order[q];
                            int64_t f = h[i];
                            for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
                                f += (int64_t)val[p] * s[col[p]];
                            const int64_t dE = -2 * (int64_t)s[i] * f;
                            if (dE > dmax || dE < -dmax) { rc = -2; break; }
                            const int32_t k = (int32_t)(dE / 2) + bias;
                            const int32_t a = (P > 1) ? (up[i] == s[i]) + (dn[i] == s[i]) : 1;
                            const uint64_t en = ent[((int64_t)t * 3 + a) * W + k];
                            const uint32_t u = rng_word(seed, start, phase, (uint32_t)t, i | (tau << 16), r);
                            if ((uint64_t)u + en < (1ull << 32)) s[i] = (int8_t)-s[i];
                        }
                    }
                }
            }
        }
        /* the run's sample: its lowest-energy slice */
        int64_t best = 0;
        int32_t bt = 0;
        for (int32_t tau = 0; tau < P; ++tau) {
            int64_t Et = or_energy(n, row_ptr, col, val, h, x + (int64_t)tau * n);
            if (tau == 0 || Et < best) { best = Et; bt = tau; }
        }
        memcpy(spins + (int64_t)row * n, x + (int64_t)bt * n, (size_t)n);
        e[row] = best;
        slice[row] = bt;
    }
    free(order);
    free(cstart);
    free(x);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Persistence (Alg. 1)                                                     */
/* ---------------------------------------------------------------------- */
/* ---------------------------------------------------------------------- */
/* Parallel tempering with isoenergetic cluster moves                       */
/* ---------------------------------------------------------------------- */

int32_t or_icm_move(int32_t n, const int32_t *row_ptr, const int32_t *col, int8_t *a, int8_t *b,
                    int32_t seed_spin)
{
    if (seed_spin < 0 || seed_spin >= n || a[seed_spin] == b[seed_spin]) return -1;
    /* breadth-first search over couplers between spins where the replicas differ */
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int8_t *in = (int8_t *)calloc((size_t)n, 1);
    int32_t head = 0, tail = 0;
    queue[tail++] = seed_spin;
    in[seed_spin] = 1;
    while (head < tail) {
        const int32_t i = queue[head++];
        for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            const int32_t j = col[p];
            if (!in[j] && a[j] != b[j]) {
                in[j] = 1;
                queue[tail++] = j;
            }
        }
    }
    for (int32_t q = 0; q < tail; ++q) {
        a[queue[q]] = (int8_t)-a[queue[q]];
        b[queue[q]] = (int8_t)-b[queue[q]];
    }
    free(in);
    free(queue);
    return tail;
}

static uint32_t rng_word0(uint64_t seed, uint32_t w0, uint32_t phase, uint32_t t, uint32_t start)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {w0, (phase << SWEEP_BITS) + t, 0u, start};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return out[0];
}

/* Offers state s (energy E) to a list of at most K distinct states ordered by
 * (energy, first sight). */
static void keep_offer(int32_t n, int32_t K, int8_t *list, int64_t *le, int32_t *cnt, const int8_t *s, int64_t E)
{
    if (*cnt == K && E >= le[K - 1]) return;
    for (int32_t q = 0; q < *cnt; ++q)
        if (le[q] == E && memcmp(list + (int64_t)q * n, s, (size_t)n) == 0) return;
    int32_t pos = *cnt;
    while (pos > 0 && le[pos - 1] > E) --pos; /* after every listed state of energy <= E */
    const int32_t last = *cnt < K ? *cnt : K - 1;
    for (int32_t q = last; q > pos; --q) {
        memcpy(list + (int64_t)q * n, list + (int64_t)(q - 1) * n, (size_t)n);
        le[q] = le[q - 1];
    }
    memcpy(list + (int64_t)pos * n, s, (size_t)n);
    le[pos] = E;
    if (*cnt < K) ++*cnt;
}

int or_pticm_sample(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *val,
                    const int32_t *h, const int32_t *colour, int32_t ncol,
                    int32_t R, int32_t T, const uint32_t *thr, int32_t dmax, const uint32_t *xthr, int32_t dx,
                    int32_t icm_from, int32_t keep_from, int32_t K, int32_t flags,
                    uint64_t seed, uint32_t start, uint32_t phase,
                    int8_t *kept, int64_t *kept_e, int32_t *nkept, int8_t *final, int64_t *final_e)
{
    if (n < 0 || R < 1 || T < 0 || (uint32_t)T >= INIT_SLOT || phase >= (1u << 12) || K < 1 ||
        keep_from < 0 || keep_from > R || icm_from < 0 || n >= 0xFFFF || R > 0x7FFF)
        return -1;
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t m = 0;
    for (int32_t c = 0; c < ncol; ++c)
        for (int32_t i = 0; i < n; ++i)
            if (colour[i] == c) order[m++] = i;
    if (m != n) { free(order); return -1; }
    const int32_t NR = 2 * R;
    int8_t *s = final; /* the replicas' current states, [2R][n] */
    int64_t *E = final_e;
    for (int32_t r = 0; r < NR; ++r) {
        for (int32_t i = 0; i < n; ++i)
            s[(int64_t)r * n + i] = (rng_word(seed, start, phase, INIT_SLOT, i, r) >> 31) ? 1 : -1;
        E[r] = or_energy(n, row_ptr, col, val, h, s + (int64_t)r * n);
    }
    const int32_t ntr = 2 * (R - keep_from);
    for (int32_t q = 0; q < ntr; ++q) nkept[q] = 0;
    int8_t *tmp = (int8_t *)malloc((size_t)n + 1);
    int rc = 0;
    for (int32_t t = 0; t < T && rc == 0; ++t) {
        /* 1. Metropolis sweep of every replica at its temperature */
        for (int32_t r = 0; r < NR && rc == 0; ++r) {
            const uint32_t *row = thr + (int64_t)(r / 2) * (dmax + 1);
            int8_t *x = s + (int64_t)r * n;
            for (int32_t q = 0; q < n; ++q) {
                const int32_t i = order[q];
                int64_t f = h[i];
                for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) f += (int64_t)val[p] * x[col[p]];
                const int64_t dE = -2 * (int64_t)x[i] * f;
                const uint32_t u = rng_word(seed, start, phase, (uint32_t)t, i, r);
                int accept;
                if (dE <= 0) {
                    accept = 1;
                } else {
                    if (dE > dmax) { rc = -2; break; }
                    accept = u < row[dE];
                }
                if (accept) {
                    x[i] = (int8_t)-x[i];
                    E[r] += dE;
                }
            }
        }
        if (rc) break;
        /* 2. isoenergetic cluster moves at the lower temperatures */
        if (flags & 2)
            for (int32_t k = icm_from; k < R; ++k) {
                int8_t *a = s + (int64_t)(2 * k) * n, *b = s + (int64_t)(2 * k + 1) * n;
                int32_t nd = 0;
                for (int32_t i = 0; i < n; ++i) nd += a[i] != b[i];
                if (nd == 0) continue;
                const uint32_t u = rng_word0(seed, 0xFFFF0000u | (uint32_t)k, phase, (uint32_t)t, start);
                const int32_t pick = (int32_t)(((uint64_t)u * (uint64_t)nd) >> 32);
                int32_t seen = 0, seed_spin = -1;
                for (int32_t i = 0; i < n && seed_spin < 0; ++i)
                    if (a[i] != b[i] && seen++ == pick) seed_spin = i;
                or_icm_move(n, row_ptr, col, a, b, seed_spin);
                E[2 * k] = or_energy(n, row_ptr, col, val, h, a);
                E[2 * k + 1] = or_energy(n, row_ptr, col, val, h, b);
            }
        /* 3. replica exchange between neighbouring temperatures */
        if (flags & 1)
            for (int32_t k = t & 1; k + 1 < R && rc == 0; k += 2)
                for (int32_t c = 0; c < 2; ++c) {
                    const int32_t lo = 2 * k + c, hi = 2 * (k + 1) + c;
                    const int64_t d = E[lo] - E[hi];
                    const uint32_t u = rng_word0(seed, 0xFFFE0000u | (uint32_t)lo, phase, (uint32_t)t, start);
                    int accept;
                    if (d <= 0) {
                        accept = 1;
                    } else {
                        if (d > dx) { rc = -2; break; }
                        accept = u < xthr[(int64_t)k * (dx + 1) + d];
                    }
                    if (accept) {
                        memcpy(tmp, s + (int64_t)lo * n, (size_t)n);
                        memcpy(s + (int64_t)lo * n, s + (int64_t)hi * n, (size_t)n);
                        memcpy(s + (int64_t)hi * n, tmp, (size_t)n);
                        const int64_t ex = E[lo];
                        E[lo] = E[hi];
                        E[hi] = ex;
                    }
                }
        /* 4. the lowest distinct states seen at the tracked replicas */
        for (int32_t k = keep_from; k < R; ++k)
            for (int32_t c = 0; c < 2; ++c) {
                const int32_t q = 2 * (k - keep_from) + c;
                keep_offer(n, K, kept + (int64_t)q * K * n, kept_e + (int64_t)q * K, nkept + q,
                           s + (int64_t)(2 * k + c) * n, E[2 * k + c]);
            }
    }
    free(tmp);
    free(order);
    return rc;
}

int32_t or_elite_count(double elite, int32_t S)
{
    double x = ceil(elite * (double)S);
    int32_t k = (x >= (double)S) ? S : (int32_t)x;
    if (k < 1) k = 1;
    if (k > S) k = S;
    return k;
}

static const int64_t *g_sort_e; /* single-threaded oracle: plain qsort context */
static int cmp_energy_index(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    if (g_sort_e[x] != g_sort_e[y]) return g_sort_e[x] < g_sort_e[y] ? -1 : 1;
    return x < y ? -1 : (x > y ? 1 : 0);
}

void or_elite(int32_t S, const int64_t *e, int32_t k, int32_t *idx)
{
    int32_t *all = (int32_t *)malloc(sizeof(int32_t) * ((size_t)S + 1));
    for (int32_t r = 0; r < S; ++r) all[r] = r;
    g_sort_e = e;
    qsort(all, (size_t)S, sizeof(int32_t), cmp_energy_index);
    for (int32_t q = 0; q < k; ++q) idx[q] = all[q];
    free(all);
}

int32_t or_persistence(int32_t n, const int32_t *row_ptr, int32_t S, const int8_t *spins,
                       const int64_t *e, int32_t k, int32_t fix_num, int32_t fix_den,
                       int32_t canon, int32_t *cnt, int8_t *fixed, int32_t *rho_out)
{
    int32_t *elite = (int32_t *)malloc(sizeof(int32_t) * ((size_t)k + 1));
    or_elite(S, e, k, elite);
    int32_t rho = -1;
    if (canon && n > 0) {
        int32_t bestdeg = -1;
        for (int32_t i = 0; i < n; ++i) {
            int32_t d = row_ptr[i + 1] - row_ptr[i];
            if (d > bestdeg) { bestdeg = d; rho = i; }
        }
    }
    for (int32_t i = 0; i < n; ++i) cnt[i] = 0;
    for (int32_t q = 0; q < k; ++q) {
        const int8_t *s = spins + (int64_t)elite[q] * n;
        int32_t sign = (rho >= 0) ? s[rho] : 1; /* multiply the row by s_rho */
        for (int32_t i = 0; i < n; ++i)
            if (s[i] * sign > 0) cnt[i]++;
    }
    int32_t nfixed = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t diff = 2 * (int64_t)cnt[i] - k; /* k * mean of s_i over the elite */
        int8_t v = 0;
        if (diff > 0 && (int64_t)fix_den * diff >= (int64_t)fix_num * k) v = 1;
        if (diff < 0 && (int64_t)fix_den * (-diff) >= (int64_t)fix_num * k) v = -1;
        fixed[i] = v;
        if (v) nfixed++;
    }
    if (rho_out) *rho_out = rho;
    free(elite);
    return nfixed;
}

/* ---------------------------------------------------------------------- */
/* Fold and compact (Alg. 1, update of J and h)                            */
/* ---------------------------------------------------------------------- */
int or_reduce(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *val,
              const int32_t *h, int64_t offset, const int32_t *colour, const int8_t *fixed,
              int32_t *n_out, int32_t *row_ptr_out, int32_t *col_out, int32_t *val_out,
              int32_t *h_out, int64_t *offset_out, int32_t *colour_out, int32_t *old_of_new)
{
    int32_t *new_of_old = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t m = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (fixed[i] == 0) {
            new_of_old[i] = m;
            old_of_new[m] = i;
            ++m;
        } else {
            new_of_old[i] = -1;
        }
    }
    /* constant: bias of fixed spins, couplers with both ends fixed (i<j once) */
    int64_t off = offset;
    for (int32_t i = 0; i < n; ++i) {
        if (fixed[i] == 0) continue;
        off += (int64_t)h[i] * fixed[i];
        for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            int32_t j = col[p];
            if (j > i && fixed[j] != 0) off += (int64_t)val[p] * fixed[i] * fixed[j];
        }
    }
    /* fields and free-free couplers, in the old order */
    int32_t nnz = 0;
    row_ptr_out[0] = 0;
    for (int32_t a = 0; a < m; ++a) {
        int32_t i = old_of_new[a];
        int64_t f = h[i];
        for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            int32_t j = col[p];
            if (fixed[j] != 0) {
                f += (int64_t)val[p] * fixed[j];
            } else {
                col_out[nnz] = new_of_old[j];
                val_out[nnz] = val[p];
                ++nnz;
            }
        }
        h_out[a] = (int32_t)f;
        colour_out[a] = colour[i];
        row_ptr_out[a + 1] = nnz;
    }
    *n_out = m;
    *offset_out = off;
    free(new_of_old);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Disconnected-component boosting (Sec. II.C)                              */
/* ---------------------------------------------------------------------- */
int32_t or_components(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t *comp)
{
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    for (int32_t i = 0; i < n; ++i) comp[i] = -1;
    int32_t m = 0;
    for (int32_t root = 0; root < n; ++root) {
        if (comp[root] >= 0) continue;
        int32_t head = 0, tail = 0;
        comp[root] = m;
        queue[tail++] = root;
        while (head < tail) {
            int32_t v = queue[head++];
            for (int32_t p = row_ptr[v]; p < row_ptr[v + 1]; ++p)
                if (comp[col[p]] < 0) {
                    comp[col[p]] = m;
                    queue[tail++] = col[p];
                }
        }
        ++m;
    }
    free(queue);
    return m;
}

static const int64_t *g_part_e; /* single-threaded oracle: plain qsort context */
static int32_t g_part_m, g_part_c;
static int cmp_partial(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    int64_t ex = g_part_e[(int64_t)x * g_part_m + g_part_c], ey = g_part_e[(int64_t)y * g_part_m + g_part_c];
    if (ex != ey) return ex < ey ? -1 : 1;
    return x < y ? -1 : (x > y ? 1 : 0);
}

int or_component_boost(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *val,
                       const int32_t *h, int32_t S, int8_t *spins, int64_t *e)
{
    if (n == 0 || S == 0) return 0;
    int32_t *comp = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t m = or_components(n, row_ptr, col, comp);
    /* partial energy of sample r on component c: couplers inside c once, biases of c */
    int64_t *pe = (int64_t *)calloc((size_t)S * m, sizeof(int64_t));
    for (int32_t r = 0; r < S; ++r) {
        const int8_t *s = spins + (int64_t)r * n;
        for (int32_t i = 0; i < n; ++i) {
            int64_t v = (int64_t)h[i] * s[i];
            for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
                if (col[p] > i) v += (int64_t)val[p] * s[i] * s[col[p]];
            pe[(int64_t)r * m + comp[i]] += v;
        }
    }
    /* each component's partial samples in (partial energy, sample index) order */
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)S * m);
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)S);
    for (int32_t c = 0; c < m; ++c) {
        for (int32_t r = 0; r < S; ++r) idx[r] = r;
        g_part_e = pe;
        g_part_m = m;
        g_part_c = c;
        qsort(idx, (size_t)S, sizeof(int32_t), cmp_partial);
        for (int32_t r = 0; r < S; ++r) perm[(int64_t)c * S + r] = idx[r];
    }
    /* merged sample: rank r of every component; energy = sum of the partials */
    int8_t *out = (int8_t *)malloc((size_t)S * n);
    for (int32_t r = 0; r < S; ++r) {
        int64_t E = 0;
        for (int32_t c = 0; c < m; ++c) E += pe[(int64_t)perm[(int64_t)c * S + r] * m + c];
        e[r] = E;
        for (int32_t i = 0; i < n; ++i)
            out[(int64_t)r * n + i] = spins[(int64_t)perm[(int64_t)comp[i] * S + r] * n + i];
    }
    memcpy(spins, out, (size_t)S * n);
    free(out); free(idx); free(perm); free(pe); free(comp);
    return m;
}

/* ---------------------------------------------------------------------- */
/* Tree pre-processing (Sec. II.C)                                          */
/* ---------------------------------------------------------------------- */
static int sgn(int64_t x) { return (x > 0) - (x < 0); }

int32_t or_tree(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *val, int32_t *h,
                int64_t *offset, int8_t *code, int32_t *parent, int32_t *order, int32_t *ninfer)
{
    int32_t *deg = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int8_t *pick = (int8_t *)malloc((size_t)n + 1);
    int32_t removed = 0, ni = 0;
    for (int32_t i = 0; i < n; ++i) { code[i] = 0; parent[i] = -1; }
    for (;;) {
        /* active degree of every active spin */
        for (int32_t i = 0; i < n; ++i) {
            deg[i] = 0;
            if (code[i]) continue;
            for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
                if (code[col[p]] == 0) deg[i]++;
        }
        /* this round's leaves */
        int32_t any = 0;
        for (int32_t i = 0; i < n; ++i) {
            pick[i] = 0;
            if (code[i] || deg[i] > 1) continue;
            if (deg[i] == 1) {
                int32_t j = -1;
                for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
                    if (code[col[p]] == 0) j = col[p];
                if (deg[j] == 1 && i < j) continue; /* isolated coupler: the higher end goes first */
            }
            pick[i] = 1;
            any = 1;
        }
        if (!any) break;
        /* eliminate them simultaneously (updates of a shared neighbour add up) */
        int32_t *hnew = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
        memcpy(hnew, h, sizeof(int32_t) * (size_t)n);
        for (int32_t i = 0; i < n; ++i) {
            if (!pick[i]) continue;
            if (deg[i] == 0) {
                int8_t v = h[i] > 0 ? -1 : 1;
                *offset += (int64_t)h[i] * v;
                code[i] = v;
            } else {
                int32_t j = -1, J = 0;
                for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
                    if (code[col[p]] == 0) { j = col[p]; J = val[p]; }
                if (llabs((long long)J) <= llabs((long long)h[i])) {
                    int8_t v = (int8_t)(-sgn(h[i]));
                    *offset += (int64_t)h[i] * v;
                    hnew[j] += J * v;
                    code[i] = v;
                } else {
                    *offset -= llabs((long long)J);
                    hnew[j] -= sgn(J) * h[i];
                    code[i] = 2;
                    parent[i] = j;
                    order[ni++] = i;
                }
            }
            removed++;
        }
        /* codes of this round were set in index order; active degrees of the next
           round are recomputed from scratch, so the order does not matter */
        memcpy(h, hnew, sizeof(int32_t) * (size_t)n);
        free(hnew);
    }
    free(deg);
    free(pick);
    if (ninfer) *ninfer = ni;
    return removed;
}

int or_compact(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *val,
               const int32_t *h, int64_t offset, const int32_t *colour, const int8_t *code,
               int32_t *n_out, int32_t *row_ptr_out, int32_t *col_out, int32_t *val_out,
               int32_t *h_out, int64_t *offset_out, int32_t *colour_out, int32_t *old_of_new)
{
    int32_t *new_of_old = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t m = 0;
    for (int32_t i = 0; i < n; ++i) {
        new_of_old[i] = code[i] == 0 ? m : -1;
        if (code[i] == 0) old_of_new[m++] = i;
    }
    int32_t nnz = 0;
    row_ptr_out[0] = 0;
    for (int32_t a = 0; a < m; ++a) {
        int32_t i = old_of_new[a];
        for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
            if (code[col[p]] == 0) {
                col_out[nnz] = new_of_old[col[p]];
                val_out[nnz] = val[p];
                ++nnz;
            }
        h_out[a] = h[i];
        colour_out[a] = colour[i];
        row_ptr_out[a + 1] = nnz;
    }
    *n_out = m;
    *offset_out = offset;
    free(new_of_old);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Multi-start SPVAR (Alg. 2)                                               */
/* ---------------------------------------------------------------------- */
static int all_zero(int32_t n, const int32_t *h)
{
    for (int32_t i = 0; i < n; ++i)
        if (h[i] != 0) return 0;
    return 1;
}

int or_solve(int32_t n0, const int32_t *row_ptr0, const int32_t *col0, const int32_t *val0,
             const int32_t *h0, int64_t offset0, const or_params *prm,
             const uint32_t *thr, int32_t dmax, uint64_t seed,
             int64_t *energies, int32_t *counts, int32_t *nfree, int32_t *nphases,
             int8_t *fixed, int64_t *best_e, int8_t *best_state)
{
    const int32_t P = prm->max_fix_phases + 1 + (prm->corr_sample_size > 0 ? 1 : 0);
    int32_t Smax = prm->fixing_sample_size > prm->solving_sample_size
                       ? prm->fixing_sample_size : prm->solving_sample_size;
    if (prm->corr_sample_size > Smax) Smax = prm->corr_sample_size;
    if (n0 < 0) return -1;
    const int64_t nnz0 = row_ptr0[n0];
    if (prm->max_fix_phases < 1 || prm->fix_den <= 0 || prm->fix_num <= 0 ||
        prm->fix_num > prm->fix_den || prm->fixing_sample_size < 1 || prm->solving_sample_size < 0 ||
        prm->corr_sample_size < 0 ||
        (prm->corr_sample_size > 0 && (prm->corr_den <= 0 || prm->corr_num <= 0 || prm->corr_num > prm->corr_den)))
        return -1;
    if (prm->sampler == 2) {
        /* PTICM: the sample of a phase is the kept lists, at most 2 (R - R/2) K states */
        const int32_t R = prm->pticm_temps, ntr = 2 * (prm->pticm_temps - prm->pticm_temps / 2);
        if (R < 2 || R > 0x7FFF || prm->pticm_keep < 1 || prm->fixing_sample_size != ntr * prm->pticm_keep ||
            (prm->solving_sample_size != 0 && prm->solving_sample_size != ntr * prm->pticm_keep) ||
            prm->corr_sample_size != 0 || prm->boost || !(prm->pticm_beta0 > 0.0) || !(prm->pticm_beta1 > 0.0))
            return -1;
    }

    int32_t *colour0 = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n0 + 1));
    int32_t ncol = or_colour(n0, row_ptr0, col0, colour0);

    /* current problem (two buffers, swapped after each reduction) */
    int32_t *rp[2], *cl[2], *vl[2], *hh[2], *co[2];
    for (int b = 0; b < 2; ++b) {
        rp[b] = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n0 + 1));
        cl[b] = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nnz0 + 1));
        vl[b] = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nnz0 + 1));
        hh[b] = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n0 + 1));
        co[b] = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n0 + 1));
    }
    int32_t *orig = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n0 + 1));
    int32_t *old_of_new = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n0 + 1));
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n0 + 1));
    int32_t *cnt = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n0 + 1));
    int8_t *fx = (int8_t *)malloc((size_t)n0 + 1);
    int8_t *spins = (int8_t *)malloc((size_t)Smax * (size_t)n0 + 1);
    int64_t *e = (int64_t *)malloc(sizeof(int64_t) * ((size_t)Smax + 1));
    int32_t *elite = (int32_t *)malloc(sizeof(int32_t) * ((size_t)Smax + 1));
    /* tree pre-processing: codes, parents, and the inference log in original indices */
    int8_t *tcode = (int8_t *)malloc((size_t)n0 + 1);
    int32_t *tpar = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n0 + 1));
    int32_t *tord = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n0 + 1));
    int32_t *log_child = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n0 + 1));
    int32_t *log_parent = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n0 + 1));
    int8_t *log_sigma = (int8_t *)malloc((size_t)n0 + 1);
    int rc = 0;
    /* SQA: its acceptance table for the original problem, and the chosen slices */
    uint64_t *ent = NULL;
    int32_t *slice = NULL;
    if (prm->sampler == 1) {
        const int32_t T = prm->num_sweeps, W = 2 * (dmax / 2) + 1;
        double *bt = (double *)malloc(sizeof(double) * ((size_t)T + 1));
        double *gt = (double *)malloc(sizeof(double) * ((size_t)T + 1));
        for (int32_t t = 0; t < T; ++t) bt[t] = prm->sqa_beta;
        or_gamma_linear(T, prm->sqa_gamma0, prm->sqa_gamma1, gt);
        ent = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)T * 3 * W + 1));
        or_sqa_table(T, prm->sqa_slices, bt, gt, dmax, prm->energy_scale > 0 ? prm->energy_scale : 1, ent);
        free(bt);
        free(gt);
        slice = (int32_t *)malloc(sizeof(int32_t) * ((size_t)Smax + 1));
    }
    /* PTICM: the temperatures' Metropolis tables and the exchange table of the
       original problem (reductions keep dmax and shrink the energy range), and
       room for one run's kept lists */
    uint32_t *pt_thr = NULL, *pt_xthr = NULL;
    int8_t *pt_kept = NULL, *pt_final = NULL;
    int64_t *pt_kept_e = NULL, *pt_final_e = NULL;
    int32_t *pt_nkept = NULL;
    int32_t pt_R = prm->pticm_temps, pt_K = prm->pticm_keep, pt_from = prm->pticm_temps / 2, pt_dx = 1;
    if (prm->sampler == 2) {
        const int32_t ntr = 2 * (pt_R - pt_from);
        const int32_t scale = prm->energy_scale > 0 ? prm->energy_scale : 1;
        double *bt = (double *)malloc(sizeof(double) * (size_t)pt_R);
        double *db = (double *)malloc(sizeof(double) * (size_t)pt_R);
        or_beta_geometric(pt_R, prm->pticm_beta0, prm->pticm_beta1, bt);
        for (int32_t k = 0; k + 1 < pt_R; ++k) db[k] = bt[k + 1] - bt[k];
        int64_t range = 0; /* max E - min E <= 2 (sum_{i<j} |J_ij| + sum_i |h_i|) */
        for (int64_t q = 0; q < nnz0; ++q) range += val0[q] < 0 ? -(int64_t)val0[q] : val0[q];
        for (int32_t i = 0; i < n0; ++i) range += 2 * (int64_t)(h0[i] < 0 ? -h0[i] : h0[i]);
        pt_dx = range > 1 ? (int32_t)range : 1;
        pt_thr = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)pt_R * ((size_t)dmax + 1));
        pt_xthr = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)pt_R * ((size_t)pt_dx + 1));
        or_thresholds(pt_R, bt, dmax, scale, pt_thr);
        or_thresholds(pt_R - 1, db, pt_dx, scale, pt_xthr);
        free(bt);
        free(db);
        pt_kept = (int8_t *)malloc((size_t)ntr * pt_K * ((size_t)n0 + 1));
        pt_kept_e = (int64_t *)malloc(sizeof(int64_t) * (size_t)ntr * pt_K);
        pt_nkept = (int32_t *)malloc(sizeof(int32_t) * (size_t)ntr);
        pt_final = (int8_t *)malloc((size_t)2 * pt_R * ((size_t)n0 + 1));
        pt_final_e = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)pt_R);
    }

    for (int32_t st = 0; st < prm->num_starts && rc == 0; ++st) {
        int b = 0;
        int32_t n = n0;
        int64_t off = offset0;
        memcpy(rp[0], row_ptr0, sizeof(int32_t) * ((size_t)n0 + 1));
        memcpy(cl[0], col0, sizeof(int32_t) * (size_t)nnz0);
        memcpy(vl[0], val0, sizeof(int32_t) * (size_t)nnz0);
        memcpy(hh[0], h0, sizeof(int32_t) * (size_t)n0);
        memcpy(co[0], colour0, sizeof(int32_t) * (size_t)n0);
        for (int32_t i = 0; i < n0; ++i) orig[i] = i;
        int8_t *fmap = fixed + (int64_t)st * n0;
        int8_t *bstate = best_state + (int64_t)st * n0;
        memset(fmap, 0, (size_t)n0);
        best_e[st] = INT64_MAX;
        int32_t phase = 0;    /* every phase: the RNG phase word and the record slot */
        int32_t fphase = 0;   /* SPVAR fixing phases done */
        int32_t nlog = 0;
        /* correlation step first, for a zero-bias problem */
        int corr = prm->corr_sample_size > 0 && all_zero(n, hh[0]);

        for (;;) {
            int fixing = corr || (fphase < prm->max_fix_phases && (fphase == 0 || (prm->iterate && n > 0)));
            int32_t S = corr ? prm->corr_sample_size : fixing ? prm->fixing_sample_size : prm->solving_sample_size;
            if (!fixing && S == 0) break;
            if (prm->sampler == 2) {
                rc = or_pticm_sample(n, rp[b], cl[b], vl[b], hh[b], co[b], ncol, pt_R, prm->num_sweeps, pt_thr, dmax,
                                     pt_xthr, pt_dx, pt_from, pt_from, pt_K, 3, seed, (uint32_t)(prm->start0 + st),
                                     (uint32_t)phase, pt_kept, pt_kept_e, pt_nkept, pt_final, pt_final_e);
                /* the sample: every tracked replica's kept states, in list order */
                S = 0;
                for (int32_t q = 0; q < 2 * (pt_R - pt_from) && rc == 0; ++q)
                    for (int32_t x = 0; x < pt_nkept[q]; ++x, ++S) {
                        memcpy(spins + (int64_t)S * n, pt_kept + ((int64_t)q * pt_K + x) * n, (size_t)n);
                        e[S] = pt_kept_e[(int64_t)q * pt_K + x];
                    }
            } else if (prm->sampler == 1)
                rc = or_sqa_sample(n, rp[b], cl[b], vl[b], hh[b], co[b], ncol, prm->num_sweeps, prm->sqa_slices,
                                   ent, dmax, 0, S, seed, (uint32_t)(prm->start0 + st), (uint32_t)phase, spins, e,
                                   slice);
            else
                rc = or_sample(n, rp[b], cl[b], vl[b], hh[b], co[b], ncol, prm->num_sweeps, thr, dmax,
                               0, S, seed, (uint32_t)(prm->start0 + st), (uint32_t)phase, spins, e, NULL);
            if (rc) break;
            if (!fixing && prm->boost) or_component_boost(n, rp[b], cl[b], vl[b], hh[b], S, spins, e);
            int64_t *rec = energies + ((int64_t)st * P + phase) * Smax;
            for (int32_t r = 0; r < S; ++r) rec[r] = e[r] + off;
            counts[st * P + phase] = S;
            nfree[st * P + phase] = n;

            /* best sample of this phase, lifted to the original variables */
            or_elite(S, e, 1, elite);
            if (e[elite[0]] + off < best_e[st]) {
                best_e[st] = e[elite[0]] + off;
                for (int32_t i = 0; i < n0; ++i) bstate[i] = fmap[i];
                for (int32_t a = 0; a < n; ++a) bstate[orig[a]] = spins[(int64_t)elite[0] * n + a];
                /* inferred spins, latest elimination first: s_child = sigma s_parent */
                for (int32_t q = nlog - 1; q >= 0; --q)
                    bstate[log_child[q]] = (int8_t)(log_sigma[q] * bstate[log_parent[q]]);
            }
            ++phase;
            if (!fixing) break;

            int32_t nf;
            if (corr) {
                /* correlation fixing: every elite row multiplied by its value at rho
                   (so rho itself has mean +1), then the rule with the correlation
                   threshold: |mean(s_rho s_j)| >= corr_num / corr_den */
                int32_t k = or_elite_count(prm->corr_elite_threshold, S);
                nf = or_persistence(n, rp[b], S, spins, e, k, prm->corr_num, prm->corr_den, 1, cnt, fx, NULL);
            } else {
                int32_t k = or_elite_count(prm->elite_threshold, S);
                int32_t canon = prm->canon < 0 ? all_zero(n, hh[b]) : prm->canon;
                nf = or_persistence(n, rp[b], S, spins, e, k, prm->fix_num, prm->fix_den, canon, cnt, fx, NULL);
            }
            if (!corr && nf == 0 && prm->iterate && n > 0) {
                /* stall rule: fix the lowest-index free spin to its value in
                   the best elite sample, so every SPVAR phase makes progress */
                or_elite(S, e, 1, elite);
                fx[0] = spins[(int64_t)elite[0] * n + 0];
            }
            if (corr) corr = 0;
            else ++fphase;
            for (int32_t a = 0; a < n; ++a)
                if (fx[a]) fmap[orig[a]] = fx[a];
            int32_t n2;
            int64_t off2;
            or_reduce(n, rp[b], cl[b], vl[b], hh[b], off, co[b], fx, &n2, rp[1 - b], cl[1 - b],
                      vl[1 - b], hh[1 - b], &off2, co[1 - b], old_of_new);
            for (int32_t a = 0; a < n2; ++a) tmp[a] = orig[old_of_new[a]];
            memcpy(orig, tmp, sizeof(int32_t) * (size_t)n2);
            n = n2;
            off = off2;
            b = 1 - b;
            if (prm->tree && n > 0) {
                int32_t ninf = 0;
                or_tree(n, rp[b], cl[b], vl[b], hh[b], &off, tcode, tpar, tord, &ninf);
                for (int32_t a = 0; a < n; ++a)
                    if (tcode[a] == 1 || tcode[a] == -1) fmap[orig[a]] = tcode[a];
                for (int32_t q = 0; q < ninf; ++q) {
                    int32_t a = tord[q], j = tpar[a], J = 0;
                    for (int32_t p = rp[b][a]; p < rp[b][a + 1]; ++p)
                        if (cl[b][p] == j) J = vl[b][p];
                    log_child[nlog] = orig[a];
                    log_parent[nlog] = orig[j];
                    log_sigma[nlog] = (int8_t)(J > 0 ? -1 : 1);
                    ++nlog;
                }
                or_compact(n, rp[b], cl[b], vl[b], hh[b], off, co[b], tcode, &n2, rp[1 - b], cl[1 - b],
                           vl[1 - b], hh[1 - b], &off2, co[1 - b], old_of_new);
                for (int32_t a = 0; a < n2; ++a) tmp[a] = orig[old_of_new[a]];
                memcpy(orig, tmp, sizeof(int32_t) * (size_t)n2);
                n = n2;
                off = off2;
                b = 1 - b;
            }
        }
        nphases[st] = phase;
    }

    for (int b = 0; b < 2; ++b) { free(rp[b]); free(cl[b]); free(vl[b]); free(hh[b]); free(co[b]); }
    free(colour0); free(orig); free(old_of_new); free(tmp); free(cnt); free(fx);
    free(spins); free(e); free(elite);
    free(tcode); free(tpar); free(tord); free(log_child); free(log_parent); free(log_sigma);
    free(ent); free(slice);
    free(pt_thr); free(pt_xthr); free(pt_kept); free(pt_kept_e); free(pt_nkept); free(pt_final); free(pt_final_e);
    return rc;
}
