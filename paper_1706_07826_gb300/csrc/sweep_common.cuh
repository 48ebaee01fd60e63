// Parts shared by the sweep kernels: initial state, final energies and the
// bit-packed output of one work item.  Spins of quad q, position p live in
// shared memory at sw[q * n + p], one byte (0/1) per replica.
#pragma once
#include "philox.cuh"
#include "spvar_internal.h"

namespace spvar {

// Twice the energy contribution of one spin for the four replicas of a word:
// s_i (h_i + f_i) with f_i = h_i + sum_j J_ij s_j  (summed over i this is 2E).
template <bool PM1>
__device__ __forceinline__ void energy2(uint32_t own, uint32_t meta, const uint32_t *ell, int ld,
                                        int p, const uint32_t *swq, int out[4])
{
    const int deg = (int)(meta & 0xFFFFu);
    const int h = (int)meta >> 16;
    if (PM1) {
        // bond (i,j) satisfied (J s_i s_j = -1) iff b_i ^ b_j ^ [J < 0] = 1
        uint32_t acc = 0;
        for (int d = 0; d < deg; ++d) {
            const uint32_t e = ell[d * ld + p];
            acc += own ^ swq[e & 0xFFFFu] ^ ((e >> 31) ? 0x01010101u : 0u);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int s = 2 * (int)((own >> (8 * r)) & 1u) - 1;
            out[r] = 2 * s * h + deg - 2 * (int)((acc >> (8 * r)) & 0xFFu);
        }
    } else {
        int a[4] = {0, 0, 0, 0}, sumJ = 0;
        for (int d = 0; d < deg; ++d) {
            const uint32_t e = ell[d * ld + p];
            const int Jv = (int)e >> 16;
            const uint32_t w = swq[e & 0xFFFFu];
            sumJ += Jv;
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] += Jv * (int)((w >> (8 * r)) & 1u);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int s = 2 * (int)((own >> (8 * r)) & 1u) - 1;
            out[r] = s * (h + h - sumJ + 2 * a[r]);
        }
    }
}

// End (exclusive) of the sweep range a work item of `job` runs: the job's own
// t1 when it is set and below the launch's T, else T.
__device__ __forceinline__ int job_end(const SweepLaunch &L, const SweepJob &job)
{
    return (job.t1 > 0 && job.t1 < L.T) ? job.t1 : L.T;
}

// Word of spin i (position p) for quad q.  A fresh sample starts from
// s_i = +1 iff the top bit of the replica's random word at the initial-state
// slot is set; a resumed one (job.init) continues from bit-packed rows
// (replicas past the sample size read as 0 and are never output).
__device__ __forceinline__ uint32_t start_word(const DevProb *P, const SweepJob &job, int quad, int p)
{
    const uint32_t i = (uint32_t)P->idx_of_pos[p];
    if (job.init) {
        uint32_t w = 0;
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const int r = 4 * quad + rr;
            if (r < job.S) w |= ((job.init[(size_t)r * job.W + (i >> 5)] >> (i & 31)) & 1u) << (8 * rr);
        }
        return w;
    }
    const uint32_t k0 = (uint32_t)job.seed, k1 = (uint32_t)(job.seed >> 32);
    const uint32_t y = (job.phase << kSweepBits) | kInitSlot;
    const uint4 r = philox4x32_10(make_uint4(i, y, (uint32_t)quad, job.start), k0, k1);
    return (r.x >> 31) | ((r.y >> 31) << 8) | ((r.z >> 31) << 16) | ((r.w >> 31) << 24);
}

// Writes sw[q * n + p] for every quad and position (and, if sw_comp !=
// nullptr, the complemented copy).
__device__ __forceinline__ void init_spins(const DevProb *P, const SweepJob &job, int quad0, int nq,
                                           uint32_t *sw, uint32_t *sw_comp)
{
    const int n = P->n;
    for (int x = threadIdx.x; x < nq * n; x += blockDim.x) {
        const int q = x / n, p = x - q * n;
        const uint32_t w = start_word(P, job, quad0 + q, p);
        sw[x] = w;
        if (sw_comp) sw_comp[x] = w ^ 0x01010101u;
    }
}

// Final energies (with offset) and bit-packed states of the item's replicas.
// Quad q's words start at sw + q * qstride (qstride = n when the quads are
// packed back to back).  e2: 4 * nq ints of shared memory.  Contains
// __syncthreads.
template <bool PM1>
__device__ __forceinline__ void finish_item(const DevProb *P, const SweepJob &job, int quad0, int nq,
                                            const uint32_t *sw, int *e2, int qstride = -1)
{
    const int tid = threadIdx.x, B = blockDim.x;
    const int n = P->n;
    const int qs = qstride < 0 ? n : qstride;
    for (int x = tid; x < 4 * nq; x += B) e2[x] = 0;
    __syncthreads();
    for (int x = tid; x < nq * n; x += B) {
        const int q = x / n, p = x - q * n;
        int c2[4];
        energy2<PM1>(sw[q * qs + p], P->meta[p], P->ell, P->cap_n, p, sw + q * qs, c2);
#pragma unroll
        for (int r = 0; r < 4; ++r) atomicAdd(&e2[4 * q + r], c2[r]);
    }
    __syncthreads();
    for (int x = tid; x < 4 * nq; x += B) {
        const int r = 4 * quad0 + x;
        if (r < job.S) job.energies[r] = (int64_t)(e2[x] / 2) + P->offset;
    }
    // one warp per (quad, 32-spin word): ballot of each replica's bit
    const int lane = tid & 31, warp = tid >> 5;
    const int Wn = (n + 31) >> 5;
    for (int x = warp; x < nq * Wn; x += B / 32) {
        const int q = x / Wn, w = x - q * Wn;
        const int i = 32 * w + lane;
        const uint32_t word = (i < n) ? sw[q * qs + P->pos_of_idx[i]] : 0u;
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const uint32_t bits = __ballot_sync(0xFFFFFFFFu, (word >> (8 * rr)) & 1u);
            const int r = 4 * (quad0 + q) + rr;
            if (lane == 0 && r < job.S) job.spins[(size_t)r * job.W + w] = bits;
        }
    }
}

// Next work item of a sweep launch: queue mode pulls from the atomic
// cursor, single mode takes blockIdx.x once.  Returns false when done.
// Contains __syncthreads (uniform).
__device__ __forceinline__ bool next_item(const SweepLaunch &L, int iter, int *s_item, SweepJob &job,
                                          int &quad0, int &nq)
{
    if (L.items) {
        if (threadIdx.x == 0) *s_item = atomicAdd(L.queue, 1);
        __syncthreads();
        const int it = *s_item;
        if (it >= *L.nitems) return false;
        const WorkItem wi = L.items[it];
        job = L.jobs[wi.job];
        quad0 = wi.quad0;
        nq = wi.nq;
        return true;
    }
    if (iter > 0) return false;
    job = L.single;
    quad0 = blockIdx.x * L.Q;
    nq = min(L.Q, (job.S + 3) / 4 - quad0);
    return nq > 0;
}

}  // namespace spvar
