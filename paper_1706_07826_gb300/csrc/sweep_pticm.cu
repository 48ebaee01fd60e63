// Parallel tempering with isoenergetic cluster moves (PTICM, Sec. III.D) as
// a sampler of Alg. 1, with the paper's sample: the K lowest-energy distinct
// states seen at each replica of the lower half of the temperatures.
//
// One CTA runs one PTICM run (start = start0 + blockIdx.x).  R inverse
// temperatures, two replicas (copies) each, replica r = 2k + c; every replica's
// spins live in shared memory as bytes by position (bit 0 the spin; bit 1 of
// copy 0 marks cluster members during a cluster move).  A sweep:
//   1. a Metropolis sweep of every replica at its temperature: a warp takes a
//      quad of replicas (one Philox block per spin gives their four words, the
//      counter and word of the SA sweep) through the colour classes; with at
//      least as many quads as warps it owns the quad for the whole sweep and
//      only warp synchronisation separates the classes, otherwise several
//      warps share a quad between CTA barriers.  Energy changes add up in
//      registers and reach the replica energies once per sweep;
//   2. Houdayer's cluster move at every temperature k >= icm_from whose
//      copies differ somewhere, one warp per temperature: |D| and the seed
//      (element floor(u |D| / 2^32) of the differing set D in index order) by
//      ballots, then the cluster by breadth-first search from a queue in
//      shared memory; expanded spins flip in both copies, and the copies'
//      energies change by the boundary sum of the cluster (the couplers that
//      leave it end outside D), so no energy pass follows;
//   3. replica exchange between temperatures k and k + 1 for k = t (mod 2):
//      the pairs are disjoint, so every decision is taken at once from the
//      replicas' energies and an integer threshold table, and accepted pairs
//      swap their states;
//   4. a warp per tracked replica offers its state, bit-packed in index
//      order, to the replica's list of the K lowest distinct states seen.
// Every wait is a CTA or warp barrier that all of its threads reach.
#include <cstring>

#include "sweep_common.cuh"

namespace spvar {

namespace {

constexpr int kPtMaxR = 64;     // most temperatures
constexpr int kPtBlock = 512;   // threads per run: two runs (32 warps) per SM when shared memory allows
constexpr int kPtWarpWords = 64;  // packed words of one state a warp keeps (n <= 2048)

struct PticmArgs {
    const DevProb *prob;
    const uint32_t *thr;   // [R][thr_stride]: Metropolis thresholds of each temperature
    const uint32_t *xthr;  // [R - 1][dx + 1]: exchange thresholds
    int32_t R, T, thr_stride, dx, icm_from, keep_from, K, flags;
    uint64_t seed;
    uint32_t start0, phase;
    uint32_t *kept;        // [runs][ntr][K][W] bit-packed, index order
    int64_t *kept_e;       // [runs][ntr][K] (with offset)
    int32_t *nkept;        // [runs][ntr]
    uint32_t *final_bits;  // [runs][2R][W]
    int64_t *final_e;      // [runs][2R] (with offset)
    // slot mode (the sampler of Alg. 2 in a plan): CTA b runs start b of the slot
    // table with that start's current problem, seed and phase; the kept lists go
    // to its sample rows and recorded energies and are compacted there
    Slot *slots;
    int32_t Smax;
};

__device__ __forceinline__ uint32_t word0(uint32_t w0, uint32_t y, uint32_t start, uint32_t k0, uint32_t k1)
{
    return philox4x32_10(make_uint4(w0, y, 0u, start), k0, k1).x;
}

// Energies (without offset) of replicas r0 .. NR - 1 into E[r]: one warp per
// replica sums s_i (2 h_i + sum_j J_ij s_j) = 2E over its spins.  Contains
// __syncthreads.
template <int B>
__device__ void replica_energies(const DevProb *P, const uint8_t *s8, int r0, int NR, int *E)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n = P->n, cap_n = P->cap_n;
    for (int r = r0 + warp; r < NR; r += B / 32) {
        const uint8_t *s = s8 + (size_t)r * n;
        int acc = 0;
        for (int p = lane; p < n; p += 32) {
            const uint32_t meta = P->meta[p];
            const int deg = (int)(meta & 0xFFFFu);
            int f = 2 * ((int)meta >> 16);
            for (int d = 0; d < deg; ++d) {
                const uint32_t e = P->ell[(size_t)d * cap_n + p];
                f += ((int)e >> 16) * (2 * (int)s[e & 0xFFFFu] - 1);
            }
            acc += (2 * (int)s[p] - 1) * f;
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if (lane == 0) E[r] = acc / 2;
    }
    __syncthreads();
}

template <int B>
__global__ void __launch_bounds__(B, 2) k_pticm(const PticmArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_pt[];
    __shared__ int sE[2 * kPtMaxR], sAcc[kPtMaxR];
    __shared__ int s_cptr[kMaxColours + 1];
    __shared__ uint32_t sPack[B / 32][kPtWarpWords];
    __shared__ int32_t s_nk[2 * kPtMaxR];  // slot mode: the kept lists' lengths

    const int run = blockIdx.x;
    Slot *slot = A.slots ? A.slots + run : nullptr;
    if (slot && slot->mode == kDone) return;  // the whole CTA: a finished start
    const DevProb *P = slot ? slot->cur : A.prob;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = P->n, ncol = P->ncol, cap_n = P->cap_n, dmax = P->dmax;
    const int R = A.R, NR = 2 * R, T = A.T;
    const int nic = R - A.icm_from;            // temperatures with cluster moves
    const int ntr = 2 * (R - A.keep_from);     // tracked replicas
    const int W = (n + 31) >> 5;
    const uint64_t seed = slot ? slot->seed : A.seed;
    const uint32_t start = slot ? slot->start : A.start0 + (uint32_t)run;
    const uint32_t phase = slot ? (uint32_t)slot->phase : A.phase;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint32_t phase_hi = phase << kSweepBits;
    // kept lists: list q, entry j at kept_rows + (q K + j) kstride words, energy kept_en[q K + j], length nk[q]
    const size_t kstride = slot ? (size_t)slot->W0 : (size_t)W;
    uint32_t *kept_rows = slot ? slot->spins : A.kept + (size_t)run * ntr * A.K * W;
    int64_t *kept_en = slot ? slot->rec_e + (size_t)slot->phase * A.Smax : A.kept_e + (size_t)run * ntr * A.K;
    int32_t *nk = slot ? s_nk : A.nkept + (size_t)run * ntr;
    if (slot)
        for (int q = tid; q < ntr; q += B) s_nk[q] = 0;

    uint8_t *s8 = smem_pt;                                         // [2R][n]
    uint32_t *thr_s = reinterpret_cast<uint32_t *>(smem_pt + (((size_t)NR * n + 15) & ~(size_t)15));
    uint16_t *queue = reinterpret_cast<uint16_t *>(thr_s + (size_t)R * (dmax + 1));  // [B / 32][n]

    for (int c = tid; c <= ncol; c += B) s_cptr[c] = P->cptr[c];
    for (int x = tid; x < R * (dmax + 1); x += B) {
        const int k = x / (dmax + 1), d = x - k * (dmax + 1);
        thr_s[x] = A.thr[(size_t)k * A.thr_stride + d];
    }
    // initial states: the SA initial-state words of replica r
    for (int x = tid; x < NR * n; x += B) {
        const int r = x / n, p = x - r * n;
        const uint4 w = philox4x32_10(
            make_uint4((uint32_t)P->idx_of_pos[p], phase_hi | kInitSlot, (uint32_t)(r >> 2), start), k0, k1);
        const uint32_t u = (r & 3) == 0 ? w.x : (r & 3) == 1 ? w.y : (r & 3) == 2 ? w.z : w.w;
        s8[x] = (uint8_t)(u >> 31);
    }
    __syncthreads();
    replica_energies<B>(P, s8, 0, NR, sE);

    const int nq = (NR + 3) >> 2;
    constexpr int NW = B / 32;
    // Metropolis work split: with at least as many quads (four replicas) as warps a warp owns whole quads for
    // a sweep and walks the colour classes under warp synchronisation only; with fewer, gq warps share a
    // quad and a CTA barrier separates the classes
    const int gq = nq >= NW ? 1 : NW / nq;
    const int mslot = warp / gq, msub = warp - mslot * gq, nslots = NW / gq;
    for (int t = 0; t < T; ++t) {
        const uint32_t y = phase_hi | (uint32_t)t;
        // 1. Metropolis sweep of every replica, colour class by colour class
        for (int q0 = 0; q0 < nq; q0 += nslots) {
            const int q = q0 + mslot;
            const bool mine = mslot < nslots && q < nq;
            const int nr = min(4, NR - 4 * q);
            uint8_t *sq = s8 + (size_t)(4 * q) * n;
            int acc[4] = {0, 0, 0, 0};
            for (int c = 0; c < ncol; ++c) {
                if (mine) {
                    const int hi = s_cptr[c + 1];
                    for (int p = s_cptr[c] + 32 * msub + lane; p < hi; p += 32 * gq) {
                        const uint4 w =
                            philox4x32_10(make_uint4((uint32_t)P->idx_of_pos[p], y, (uint32_t)q, start), k0, k1);
                        const uint32_t uu[4] = {w.x, w.y, w.z, w.w};
                        const uint32_t meta = P->meta[p];
                        const int deg = (int)(meta & 0xFFFFu), h = (int)meta >> 16;
                        int f[4] = {h, h, h, h};
                        for (int d = 0; d < deg; ++d) {
                            const uint32_t e = P->ell[(size_t)d * cap_n + p];
                            const int j = (int)(e & 0xFFFFu), Jv = (int)e >> 16;
#pragma unroll
                            for (int rr = 0; rr < 4; ++rr)
                                if (rr < nr) f[rr] += Jv * (2 * (int)sq[(size_t)rr * n + j] - 1);
                        }
#pragma unroll
                        for (int rr = 0; rr < 4; ++rr) {
                            if (rr >= nr) break;
                            const int r = 4 * q + rr;
                            const int dE = -2 * (2 * (int)sq[(size_t)rr * n + p] - 1) * f[rr];
                            const bool accept =
                                dE <= 0 || uu[rr] < thr_s[(size_t)(r >> 1) * (dmax + 1) + min(dE, dmax)];
                            if (accept) {
                                sq[(size_t)rr * n + p] ^= 1u;
                                acc[rr] += dE;
                            }
                        }
                    }
                }
                if (gq > 1)
                    __syncthreads();
                else
                    __syncwarp();
            }
            if (mine) {
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) {
                    int v = acc[rr];
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
                    if (lane == 0 && rr < nr) atomicAdd(&sE[4 * q + rr], v);
                }
            }
        }
        __syncthreads();
        // 2. cluster moves at the lower temperatures, one warp per temperature: |D|, the seed (element
        //    floor(u |D| / 2^32) of D in index order), then the cluster by breadth-first search.  A step
        //    expands up to 32 queued spins, neighbour slot by neighbour slot; a spin found by several lanes in
        //    one slot is queued once (match) and marked before the next slot looks, so the queue never exceeds
        //    n.  Expanded spins flip in both copies (membership of D is unchanged by that), and the copies'
        //    energies change by -+2 (sum over the cluster of h_i a_i plus J_ij a_i a_j over couplers leaving it):
        //    every neighbour outside the cluster lies outside D
        if ((A.flags & 2) && nic > 0) {
            for (int kk = warp; kk < nic; kk += NW) {
                const int k = A.icm_from + kk;
                uint8_t *sa = s8 + (size_t)(2 * k) * n, *sb = sa + n;
                int cnt = 0;
                for (int base = 0; base < n; base += 32) {
                    const int p = base + lane;
                    cnt += __popc(__ballot_sync(0xFFFFFFFFu, p < n && ((sa[p] ^ sb[p]) & 1)));
                }
                if (cnt == 0) continue;
                const uint32_t u = word0(0xFFFF0000u | (uint32_t)k, y, start, k0, k1);
                const int pick = (int)(((uint64_t)u * (uint64_t)cnt) >> 32);
                int seedpos = -1, seen = 0;
                for (int base = 0; base < n && seedpos < 0; base += 32) {
                    const int i = base + lane;
                    int pos = -1;
                    bool dif = false;
                    if (i < n) {
                        pos = P->pos_of_idx[i];
                        dif = (sa[pos] ^ sb[pos]) & 1;
                    }
                    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, dif);
                    const int c = __popc(bal);
                    if (pick < seen + c) {
                        // the (pick - seen)-th set lane
                        const bool hit = dif && __popc(bal & ((1u << lane) - 1u)) == pick - seen;
                        seedpos = __shfl_sync(0xFFFFFFFFu, pos, __ffs(__ballot_sync(0xFFFFFFFFu, hit)) - 1);
                    }
                    seen += c;
                }
                uint16_t *qu = queue + (size_t)warp * n;
                if (lane == 0) {
                    qu[0] = (uint16_t)seedpos;
                    sa[seedpos] |= 2u;
                }
                __syncwarp();
                int head = 0, tail = 1, bsum = 0;
                while (head < tail) {
                    const int take = min(32, tail - head);
                    const int v = lane < take ? (int)qu[head + lane] : -1;
                    int deg = 0, av = 0;
                    if (v >= 0) {
                        const uint32_t meta = P->meta[v];
                        deg = (int)(meta & 0xFFFFu);
                        av = 2 * (int)(sa[v] & 1u) - 1;
                        bsum += ((int)meta >> 16) * av;
                    }
                    int maxdeg = deg;
                    for (int o = 16; o > 0; o >>= 1) maxdeg = max(maxdeg, __shfl_xor_sync(0xFFFFFFFFu, maxdeg, o));
                    for (int d = 0; d < maxdeg; ++d) {
                        int j = -1;
                        if (d < deg) {
                            const uint32_t e = P->ell[(size_t)d * cap_n + v];
                            const int cand = (int)(e & 0xFFFFu);
                            const int ac = sa[cand];
                            if ((ac ^ sb[cand]) & 1) {
                                if (!(ac & 2)) j = cand;
                            } else {
                                bsum += ((int)e >> 16) * av * (2 * (ac & 1) - 1);
                            }
                        }
                        // one lane per distinct new spin
                        const uint32_t same = __match_any_sync(0xFFFFFFFFu, j);
                        const bool first = j >= 0 && (__ffs(same) - 1) == lane;
                        const uint32_t add = __ballot_sync(0xFFFFFFFFu, first);
                        if (first) {
                            qu[tail + __popc(add & ((1u << lane) - 1u))] = (uint16_t)j;
                            sa[j] |= 2u;
                        }
                        tail += __popc(add);
                        __syncwarp();
                    }
                    if (v >= 0) {
                        sa[v] ^= 1u;
                        sb[v] ^= 1u;
                    }
                    __syncwarp();
                    head += take;
                }
                for (int o = 16; o > 0; o >>= 1) bsum += __shfl_xor_sync(0xFFFFFFFFu, bsum, o);
                if (lane == 0) {
                    sE[2 * k] -= 2 * bsum;
                    sE[2 * k + 1] += 2 * bsum;
                }
                for (int i = lane; i < tail; i += 32) sa[qu[i]] &= 1u;
                __syncwarp();
            }
            __syncthreads();
        }
        // 3. replica exchange between temperatures k and k + 1, k = t (mod 2)
        if (A.flags & 1) {
            const int npair = (R - 1 - (t & 1) + 1) / 2;  // k = (t & 1), (t & 1) + 2, ... < R - 1
            for (int z = tid; z < 2 * max(npair, 0); z += B) {
                const int k = (t & 1) + 2 * (z >> 1), c = z & 1;
                const int lo = 2 * k + c, hi = lo + 2;
                const int d = sE[lo] - sE[hi];
                const uint32_t u = word0(0xFFFE0000u | (uint32_t)lo, y, start, k0, k1);
                sAcc[z] = d <= 0 || u < A.xthr[(size_t)k * (A.dx + 1) + min(d, A.dx)];
            }
            __syncthreads();
            for (int x = tid; x < 2 * max(npair, 0) * n; x += B) {
                const int z = x / n, p = x - z * n;
                if (!sAcc[z]) continue;
                const int lo = 2 * ((t & 1) + 2 * (z >> 1)) + (z & 1), hi = lo + 2;
                const uint8_t a = s8[(size_t)lo * n + p];
                s8[(size_t)lo * n + p] = s8[(size_t)hi * n + p];
                s8[(size_t)hi * n + p] = a;
            }
            __syncthreads();
            for (int z = tid; z < 2 * max(npair, 0); z += B) {
                if (!sAcc[z]) continue;
                const int lo = 2 * ((t & 1) + 2 * (z >> 1)) + (z & 1), hi = lo + 2;
                const int e = sE[lo];
                sE[lo] = sE[hi];
                sE[hi] = e;
            }
            __syncthreads();
        }
        // 4. each tracked replica's list of the K lowest distinct states seen
        for (int q = warp; q < ntr; q += B / 32) {
            const int r = 2 * (A.keep_from + q / 2) + (q & 1);
            const int64_t E = (int64_t)sE[r] + P->offset;
            int32_t *cntp = nk + q;
            int64_t *le = kept_en + (size_t)q * A.K;
            uint32_t *lst = kept_rows + (size_t)q * A.K * kstride;
            const int cnt = *cntp;
            if (cnt == A.K && E >= le[A.K - 1]) continue;
            // the state, bit-packed in index order
            for (int w = 0; w < W; ++w) {
                const int i = 32 * w + lane;
                const bool b = i < n && s8[(size_t)r * n + P->pos_of_idx[i]];
                const uint32_t bits = __ballot_sync(0xFFFFFFFFu, b);
                if (lane == 0) sPack[warp][w] = bits;
            }
            __syncwarp();
            bool dup = false;
            for (int j = 0; j < cnt && !dup; ++j) {
                if (le[j] != E) continue;
                bool diff = false;
                for (int w = lane; w < W; w += 32) diff |= lst[(size_t)j * kstride + w] != sPack[warp][w];
                dup = !__any_sync(0xFFFFFFFFu, diff);
            }
            if (dup) continue;
            int pos = cnt;
            while (pos > 0 && le[pos - 1] > E) --pos;
            const int last = cnt < A.K ? cnt : A.K - 1;
            for (int j = last; j > pos; --j) {
                for (int w = lane; w < W; w += 32)
                    lst[(size_t)j * kstride + w] = lst[(size_t)(j - 1) * kstride + w];
                __syncwarp();
                if (lane == 0) le[j] = le[j - 1];
                __syncwarp();
            }
            for (int w = lane; w < W; w += 32) lst[(size_t)pos * kstride + w] = sPack[warp][w];
            if (lane == 0) {
                le[pos] = E;
                if (cnt < A.K) *cntp = cnt + 1;
            }
            __syncwarp();
        }
        __syncthreads();
    }
    if (slot) {
        // the phase's sample: the lists one after another.  List q moves down by
        // q K - (entries before it); rows are copied in waves of that distance, so
        // a wave never overwrites a row a later wave still reads
        int before = 0;
        for (int q = 0; q < ntr; ++q) {
            const int len = s_nk[q], shift = q * A.K - before;
            if (shift > 0)
                for (int j0 = 0; j0 < len; j0 += shift) {
                    const int jn = min(len, j0 + shift);
                    for (int x = tid; x < (jn - j0) * W; x += B) {
                        const int j = j0 + x / W, w = x - (x / W) * W;
                        kept_rows[(size_t)(before + j) * kstride + w] = kept_rows[(size_t)(q * A.K + j) * kstride + w];
                    }
                    for (int j = j0 + tid; j < jn; j += B) kept_en[before + j] = kept_en[q * A.K + j];
                    __syncthreads();
                }
            before += len;
        }
        if (tid == 0) slot->rec_count[slot->phase] = before;
        return;
    }
    // final states and energies of every replica
    for (int r = warp; r < NR; r += B / 32) {
        for (int w = 0; w < W; ++w) {
            const int i = 32 * w + lane;
            const bool b = i < n && s8[(size_t)r * n + P->pos_of_idx[i]];
            const uint32_t bits = __ballot_sync(0xFFFFFFFFu, b);
            if (lane == 0) A.final_bits[((size_t)run * NR + r) * W + w] = bits;
        }
        if (lane == 0) A.final_e[(size_t)run * NR + r] = (int64_t)sE[r] + P->offset;
    }
}

}  // namespace

size_t pticm_smem_bytes(int n, int R, int dmax)
{
    const size_t spins = (2 * (size_t)R * n + 15) & ~(size_t)15;
    return spins + 4 * (size_t)R * ((size_t)dmax + 1) + 2 * (size_t)(kPtBlock / 32) * n;  // + one queue per warp
}

int pticm_max_r() { return kPtMaxR; }
int pticm_max_n() { return 32 * kPtWarpWords; }

cudaError_t launch_pticm(const DevProb *prob, const uint32_t *thr, int thr_stride, const uint32_t *xthr, int dx,
                         int R, int T, int icm_from, int keep_from, int K, int flags, uint64_t seed,
                         uint32_t start0, uint32_t phase, int runs, size_t smem, uint32_t *kept, int64_t *kept_e,
                         int32_t *nkept, uint32_t *final_bits, int64_t *final_e, cudaStream_t st)
{
    PticmArgs A;
    A.prob = prob;
    A.thr = thr;
    A.xthr = xthr;
    A.R = R;
    A.T = T;
    A.thr_stride = thr_stride;
    A.dx = dx;
    A.icm_from = icm_from;
    A.keep_from = keep_from;
    A.K = K;
    A.flags = flags;
    A.seed = seed;
    A.start0 = start0;
    A.phase = phase;
    A.kept = kept;
    A.kept_e = kept_e;
    A.nkept = nkept;
    A.final_bits = final_bits;
    A.final_e = final_e;
    A.slots = nullptr;
    A.Smax = 0;
    void *k = reinterpret_cast<void *>(k_pticm<kPtBlock>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {&A};
    return cudaLaunchKernel(k, dim3(runs), dim3(kPtBlock), args, smem, st);
}

}  // namespace spvar

namespace spvar {

cudaError_t launch_pticm_slots(Slot *slots, int nslots, int Smax, const uint32_t *thr, int thr_stride,
                               const uint32_t *xthr, int dx, int R, int T, int K, size_t smem, cudaStream_t st)
{
    if (nslots <= 0) return cudaSuccess;
    PticmArgs A;
    std::memset(&A, 0, sizeof(A));
    A.thr = thr;
    A.xthr = xthr;
    A.R = R;
    A.T = T;
    A.thr_stride = thr_stride;
    A.dx = dx;
    A.icm_from = R / 2;
    A.keep_from = R / 2;
    A.K = K;
    A.flags = 3;
    A.slots = slots;
    A.Smax = Smax;
    void *k = reinterpret_cast<void *>(k_pticm<kPtBlock>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {&A};
    return cudaLaunchKernel(k, dim3(nslots), dim3(kPtBlock), args, smem, st);
}

}  // namespace spvar
