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

// Persistence count and fixing rule for spins [i0, i0 + blockDim.x) of one
// sample set.  With canon, each elite row is multiplied by its value at
// prob->rho.  fmap/orig (optional): also record fixings in original order.
__device__ __forceinline__ void count_core(const DevProb *P, const uint32_t *spins, int W,
                                           const int32_t *elite, int k, int canon, int fix_num,
                                           int fix_den, int32_t *counts, int8_t *fixed,
                                           int32_t *nfixed, int8_t *fmap, const int32_t *orig)
{
    constexpr int kChunk = 512;
    __shared__ int s_row[kChunk];
    __shared__ unsigned s_flip[kChunk];
    const int n = P->n;
    const int rho = P->rho;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int word = i >> 5;
    const unsigned bit = (unsigned)(i & 31);
    int cnt = 0;
    for (int c0 = 0; c0 < k; c0 += kChunk) {
        const int m = min(kChunk, k - c0);
        for (int q = threadIdx.x; q < m; q += blockDim.x) {
            const int r = elite[c0 + q];
            s_row[q] = r;
            unsigned f = 0;
            if (canon && rho >= 0) {
                const unsigned b = (spins[(size_t)r * W + (rho >> 5)] >> (rho & 31)) & 1u;
                f = b ? 0u : 0xFFFFFFFFu;
            }
            s_flip[q] = f;
        }
        __syncthreads();
        if (i < n)
            for (int q = 0; q < m; ++q)
                cnt += (int)(((spins[(size_t)s_row[q] * W + word] ^ s_flip[q]) >> bit) & 1u);
        __syncthreads();
    }
    int8_t v = 0;
    if (i < n) {
        const long long diff = 2ll * cnt - k;
        if (diff > 0 && (long long)fix_den * diff >= (long long)fix_num * k) v = 1;
        if (diff < 0 && (long long)fix_den * (-diff) >= (long long)fix_num * k) v = -1;
        if (counts) counts[i] = cnt;
        fixed[i] = v;
        if (v && fmap) fmap[orig[i]] = v;
    }
    const unsigned ball = __ballot_sync(0xFFFFFFFFu, v != 0);
    if ((threadIdx.x & 31) == 0 && ball) atomicAdd(nfixed, __popc(ball));
}

// Fold the fixed spins into h and the offset and compact the free spins into
// dst (same capacities as src).  old_of_new [n], scratch [2 * cap_n].
// blockDim.x == kBigBlock, one CTA per reduction.
// fold = false: spins with fixed[i] != 0 are only dropped (their values were
// already folded into h and the offset, e.g. by the tree step).
__device__ void reduce_core(const DevProb *src, DevProb *dst, const int8_t *fixed,
                            int32_t *old_of_new, int32_t *scratch, bool fold = true);

}  // namespace spvar
