// Device building blocks of the persistence pass (Alg. 1: elite sample, mean
// value per variable, fixing rule) and of the fold/compact step (Alg. 1:
// update J and h).  Shared by the standalone entry points and by the
// multi-start driver.
#pragma once
#include "spvar_internal.h"

namespace spvar {

constexpr int kBigBlock = 1024;  // elite / reduce CTAs
constexpr int kCountBlock = 256;

// Exclusive block-wide scan of one int per thread (blockDim.x == kBigBlock).
// s_warp: >= 32 ints of shared memory.  Returns the exclusive prefix and the
// block total through *total.  Contains __syncthreads: call uniformly.
__device__ __forceinline__ int block_scan_excl(int v, int *s_warp, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = (lane < (int)(blockDim.x >> 5)) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    const int prefix = (warp > 0 ? s_warp[warp - 1] : 0) + x - v;
    *total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return prefix;
}

// Exclusive block-wide scans of V ints per thread at once, with the three
// barriers of one scan.  s_w: >= 32 V ints of shared memory.  Contains
// __syncthreads: call uniformly.
template <int V>
__device__ __forceinline__ void block_scan_multi(const int (&v)[V], int (&ex)[V], int (&tot)[V], int *s_w)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    int x[V];
#pragma unroll
    for (int q = 0; q < V; ++q) x[q] = v[q];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, x[q], o);
            if (lane >= o) x[q] += y;
        }
    }
    if (lane == 31) {
#pragma unroll
        for (int q = 0; q < V; ++q) s_w[q * 32 + warp] = x[q];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < V; ++q) {
            int w = lane < nw ? s_w[q * 32 + lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xFFFFFFFFu, w, o);
                if (lane >= o) w += y;
            }
            s_w[q * 32 + lane] = w;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < V; ++q) {
        ex[q] = (warp > 0 ? s_w[q * 32 + warp - 1] : 0) + x[q] - v[q];
        tot[q] = s_w[q * 32 + nw - 1];
    }
    __syncthreads();
}

// Elite selection: indices of the k lowest (energy, index) pairs, in order.
// Bitonic sort of packed 64-bit keys (energy - min) << 32 | index in shared
// memory (s_key >= next power of two of S entries).  blockDim.x == kBigBlock.
__device__ __forceinline__ void elite_core(const int64_t *energies, int S, int k, int32_t *elite,
                                           unsigned long long *s_key)
{
    __shared__ long long s_min;
    const int tid = threadIdx.x;
    if (tid == 0) s_min = LLONG_MAX;
    __syncthreads();
    long long m = LLONG_MAX;
    for (int r = tid; r < S; r += blockDim.x) m = min(m, (long long)energies[r]);
    atomicMin(&s_min, m);
    __syncthreads();
    const long long emin = s_min;
    int N2 = 1;
    while (N2 < S) N2 <<= 1;
    for (int r = tid; r < N2; r += blockDim.x)
        s_key[r] = (r < S) ? (((unsigned long long)(energies[r] - emin) << 32) | (unsigned)r)
                           : ~0ull;
    __syncthreads();
    for (int size = 2; size <= N2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < N2; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const unsigned long long a = s_key[i], b = s_key[j];
                    const bool up = (i & size) == 0;
                    if ((a > b) == up) {
                        s_key[i] = b;
                        s_key[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int q = tid; q < k; q += blockDim.x) elite[q] = (int32_t)(s_key[q] & 0xFFFFFFFFull);
    __syncthreads();
}

// Elite selection without sorting the whole sample: the same k indices in the
// same order as elite_core.  The lowest energy and the spread give a
// histogram of (E - Emin) >> shift over kEliteBins bins; the bin holding the
// k-th lowest key bounds the candidates (every key in a lower or equal bin),
// which are compacted in index order and placed by rank (the number of
// candidate keys below each; keys are distinct because they carry the
// index).  k = 1 is a block-wide arg-min.  More than kEliteRankMax candidates
// (a crowded bin) fall back to elite_core.  Any block size; s_key as for
// elite_core.  s_e (optional, shared memory, S entries, apart from the first
// kEliteRankMax keys): the energies are read from global memory once and kept
// there for the later passes.
// Keys of elite_core's sort: the next power of two of S.
__host__ __device__ inline int elite_key_words(int S)
{
    int N2 = 1;
    while (N2 < S) N2 <<= 1;
    return N2;
}

constexpr int kEliteBins = 1024;
constexpr int kEliteRankMax = 512;
__device__ __forceinline__ void elite_fast(const int64_t *energies, int S, int k, int32_t *elite,
                                           unsigned long long *s_key, int64_t *s_e = nullptr)
{
    __shared__ long long s_min, s_max;
    __shared__ unsigned long long s_best;
    __shared__ int s_hist[kEliteBins];
    __shared__ int s_warp[32];
    __shared__ int s_bin, s_cand;
    const int tid = threadIdx.x, B = blockDim.x;
    if (tid == 0) {
        s_min = LLONG_MAX;
        s_max = LLONG_MIN;
        s_best = ~0ull;
    }
    for (int b = tid; b < kEliteBins; b += B) s_hist[b] = 0;
    __syncthreads();
    long long mn = LLONG_MAX, mx = LLONG_MIN;
    for (int r0 = tid; r0 < S; r0 += 4 * B) {
        // four loads in flight per thread
        long long ev[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) ev[u] = r0 + u * B < S ? (long long)energies[r0 + u * B] : 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = r0 + u * B;
            if (r < S) {
                if (s_e) s_e[r] = ev[u];
                mn = min(mn, ev[u]);
                mx = max(mx, ev[u]);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    }
    if ((tid & 31) == 0) {
        atomicMin(&s_min, mn);
        atomicMax(&s_max, mx);
    }
    __syncthreads();
    const long long emin = s_min;
    const int64_t *E = s_e ? s_e : energies;  // the later passes
    if (k == 1) {
        unsigned long long best = ~0ull;
        for (int r = tid; r < S; r += B)
            best = min(best, ((unsigned long long)(E[r] - emin) << 32) | (unsigned)r);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xFFFFFFFFu, best, o));
        if ((tid & 31) == 0) atomicMin(&s_best, best);
        __syncthreads();
        if (tid == 0) elite[0] = (int32_t)(s_best & 0xFFFFFFFFull);
        __syncthreads();
        return;
    }
    int shift = 0;
    while (((unsigned long long)(s_max - emin) >> shift) >= (unsigned long long)kEliteBins) ++shift;
    for (int r = tid; r < S; r += B) atomicAdd(&s_hist[(int)((unsigned long long)(E[r] - emin) >> shift)], 1);
    __syncthreads();
    // the bin holding the k-th lowest key (keys in bins below it number < k, with
    // it >= k): each thread scans a run of consecutive bins after one block scan
    {
        const int per = (kEliteBins + B - 1) / B, b0 = tid * per;
        int h = 0;
        for (int b = b0; b < b0 + per && b < kEliteBins; ++b) h += s_hist[b];
        int tot;
        int below = block_scan_excl(h, s_warp, &tot);
        for (int b = b0; b < b0 + per && b < kEliteBins; ++b) {
            const int hb = s_hist[b];
            if (below < k && below + hb >= k) {
                s_bin = b;
                s_cand = below + hb;
            }
            below += hb;
        }
    }
    __syncthreads();
    const int bstar = s_bin, C = s_cand;
    if (C > kEliteRankMax) {
        elite_core(energies, S, k, elite, s_key);
        return;
    }
    // candidates in index order: each thread takes a run of consecutive samples
    {
        const int per = (S + B - 1) / B, r0 = tid * per;
        int f = 0;
        for (int r = r0; r < r0 + per && r < S; ++r)
            f += (int)((unsigned long long)(E[r] - emin) >> shift) <= bstar;
        int tot;
        int o = block_scan_excl(f, s_warp, &tot);
        for (int r = r0; r < r0 + per && r < S; ++r) {
            const unsigned long long d = (unsigned long long)(E[r] - emin);
            if ((int)(d >> shift) <= bstar) s_key[o++] = (d << 32) | (unsigned)r;
        }
    }
    __syncthreads();
    for (int c = tid; c < C; c += B) {
        const unsigned long long key = s_key[c];
        int rank = 0;
        for (int j = 0; j < C; ++j) rank += s_key[j] < key;
        if (rank < k) elite[rank] = (int32_t)(key & 0xFFFFFFFFull);
    }
    __syncthreads();
}

// Persistence count and fixing rule, bit-sliced: one CTA of kCountBlock
// threads covers 32 words (1024 spins, chunk `chunk`) of the sample rows.
// Lane l of every warp owns word 32 chunk + l; the k elite rows are split over the 8
// warps, and each lane adds its rows' words (each multiplied by its value at
// rho when canon is set) into NB bit planes: plane b holds bit b of the
// running count of every spin of the word (a vertical counter, two logic
// operations per plane and row).  The warps' counters are then summed by a
// bit-sliced ripple adder and each spin's count read off its planes.
// counts[i] (if not null) is the number of elite rows with s_i = +1 (after
// the canonicalisation), fixed[i] the fixing rule's value (+1, -1 or 0),
// *nfixed grows by the spins fixed, and with fmap/orig the fixings are also
// recorded by original index.  NB: planes per warp (2^NB > rows per warp).
constexpr int kCountWarps = kCountBlock / 32;
constexpr int kCountPlanes = 12;  // 2^12 > 16384 / kCountWarps rows per warp
// Shared memory of one count chunk (callers place it, so the multi-start pass
// can overlay it on buffers of other steps).
struct CountSmem {
    uint32_t planes[kCountWarps][kCountPlanes + 3][32];
    uint32_t tot[kCountPlanes + 3][32];
    int row[1024];
    uint32_t flip[1024];
};
template <int NB>
__device__ __forceinline__ void count_planes(const uint32_t *spins, int W, const int32_t *elite, int k,
                                             int canon, int rho, uint32_t (*s_planes)[kCountPlanes + 3][32],
                                             int *s_row, uint32_t *s_flip, int chunk)
{
    constexpr int kChunk = 1024;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int word = chunk * 32 + lane;
    uint32_t c[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) c[b] = 0u;
    for (int c0 = 0; c0 < k; c0 += kChunk) {
        const int m = min(kChunk, k - c0);
        for (int q = threadIdx.x; q < m; q += blockDim.x) {
            const int r = elite[c0 + q];
            s_row[q] = r;
            uint32_t f = 0u;
            if (canon && rho >= 0) f = ((spins[(size_t)r * W + (rho >> 5)] >> (rho & 31)) & 1u) ? 0u : 0xFFFFFFFFu;
            s_flip[q] = f;
        }
        __syncthreads();
        if (word < W) {
#pragma unroll 8
            for (int q = warp; q < m; q += kCountWarps) {
                uint32_t carry = spins[(size_t)s_row[q] * W + word] ^ s_flip[q];
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const uint32_t t = c[b] & carry;
                    c[b] ^= carry;
                    carry = t;
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) s_planes[warp][b][lane] = c[b];
}

__device__ __forceinline__ void count_bs_core(const DevProb *P, const uint32_t *spins, int W, const int32_t *elite,
                                              int k, int canon, int fix_num, int fix_den, int32_t *counts,
                                              int8_t *fixed, int32_t *nfixed, int8_t *fmap, const int32_t *orig,
                                              int chunk, CountSmem &sm)
{
    uint32_t(*s_planes)[kCountPlanes + 3][32] = sm.planes;
    uint32_t(*s_tot)[32] = sm.tot;
    int *s_row = sm.row;
    uint32_t *s_flip = sm.flip;
    const int n = P->n, rho = P->rho;
    const int per_warp = (k + kCountWarps - 1) / kCountWarps;
    const int NB = per_warp < 16 ? 4 : per_warp < 64 ? 6 : per_warp < 256 ? 8 : per_warp < 1024 ? 10 : 12;
    if (NB == 4) count_planes<4>(spins, W, elite, k, canon, rho, s_planes, s_row, s_flip, chunk);
    else if (NB == 6) count_planes<6>(spins, W, elite, k, canon, rho, s_planes, s_row, s_flip, chunk);
    else if (NB == 8) count_planes<8>(spins, W, elite, k, canon, rho, s_planes, s_row, s_flip, chunk);
    else if (NB == 10) count_planes<10>(spins, W, elite, k, canon, rho, s_planes, s_row, s_flip, chunk);
    else count_planes<12>(spins, W, elite, k, canon, rho, s_planes, s_row, s_flip, chunk);
    __syncthreads();
    const int NT = NB + 3;  // the sum of 8 counters below 2^NB is below 2^(NB + 3)
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        uint32_t t[kCountPlanes + 3];
#pragma unroll
        for (int b = 0; b < kCountPlanes + 3; ++b) t[b] = 0u;
        for (int w = 0; w < kCountWarps; ++w) {
            uint32_t carry = 0u;
#pragma unroll
            for (int b = 0; b < kCountPlanes + 3; ++b) {
                if (b < NT) {
                    const uint32_t a = t[b], x = b < NB ? s_planes[w][b][lane] : 0u;
                    t[b] = a ^ x ^ carry;
                    carry = (a & x) | (carry & (a ^ x));
                }
            }
        }
#pragma unroll
        for (int b = 0; b < kCountPlanes + 3; ++b)
            if (b < NT) s_tot[b][lane] = t[b];
    }
    __syncthreads();
    for (int sp0 = threadIdx.x; sp0 < 1024; sp0 += 4 * blockDim.x) {
        // the original indices of four spins loaded before any store
        int oi[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = chunk * 1024 + sp0 + u * (int)blockDim.x;
            oi[u] = (fmap && sp0 + u * (int)blockDim.x < 1024 && i < n) ? orig[i] : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int sp = sp0 + u * (int)blockDim.x;
            if (sp >= 1024) break;
            const int i = chunk * 1024 + sp;
            const int wl = sp >> 5, bit = sp & 31;
            int8_t v = 0;
            if (i < n) {
                int cnt = 0;
                for (int b = 0; b < NT; ++b) cnt |= (int)((s_tot[b][wl] >> bit) & 1u) << b;
                const long long diff = 2ll * cnt - k;
                if (diff > 0 && (long long)fix_den * diff >= (long long)fix_num * k) v = 1;
                if (diff < 0 && (long long)fix_den * (-diff) >= (long long)fix_num * k) v = -1;
                if (counts) counts[i] = cnt;
                fixed[i] = v;
                if (v && fmap) fmap[oi[u]] = v;
            }
            const unsigned ball = __ballot_sync(0xFFFFFFFFu, v != 0);
            if ((threadIdx.x & 31) == 0 && ball) atomicAdd(nfixed, __popc(ball));
        }
    }
}

// Fold the fixed spins into h and the offset and compact the free spins into
// dst (same capacities as src).  old_of_new [n], scratch [2 * cap_n].
// blockDim.x == kBigBlock, one CTA per reduction.
// fold = false: spins with fixed[i] != 0 are only dropped (their values were
// already folded into h and the offset, e.g. by the tree step).
__device__ void reduce_core(const DevProb *src, DevProb *dst, const int8_t *fixed,
                            int32_t *old_of_new, int32_t *scratch, bool fold = true);

}  // namespace spvar
