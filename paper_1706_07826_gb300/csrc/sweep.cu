// Simulated-annealing sweep kernel (the sampler of Sec. III.A, Alg. 1
// "obtain sample").
//
// One CTA anneals 4*nq replicas ("quads": the four replicas that share one
// Philox4x32-10 call) of one problem.  The spins of those replicas live in
// shared memory, one byte per replica and four replicas per 32-bit word, laid
// out by position (colour class by colour class).  A sweep visits the colour
// classes in order; inside a class no two spins are coupled, so every
// (spin, quad) item of the class is updated in parallel, and the result is the
// same as visiting the class in increasing index one spin at a time.  A
// __syncthreads separates classes.
//
// For +-1 couplers the local field of all four replicas is formed with byte-
// wise (SWAR) adds of "bond satisfied" bits; general integer couplers use one
// multiply-add per replica.  Acceptance compares the replica's Philox word
// with a row of the uint32 threshold table staged in shared memory.
//
// In queue mode the grid is persistent: each CTA pulls work items (job,
// quad range) from an atomic cursor until the list is exhausted, so jobs of
// uneven size share one launch.
#include "sweep_common.cuh"

namespace spvar {

size_t sweep_smem_bytes(int max_n, int Q, int thr_stride, int maxdeg, bool stage_ell)
{
    size_t words = (size_t)Q * max_n + 2 * (size_t)thr_stride + 4 * (size_t)Q;
    if (stage_ell) words += (size_t)(2 + maxdeg) * max_n;
    return words * 4;
}

namespace {

template <bool PM1>
__device__ __forceinline__ uint32_t flip_mask(uint32_t own, uint32_t meta, const uint32_t *ell,
                                              int ld, int p, const uint32_t *swq, uint4 rw,
                                              const uint32_t *th, int thr_w)
{
    const int deg = (int)(meta & 0xFFFFu);
    const int h = (int)meta >> 16;
    int dE[4];
    if (PM1) {
        // acc byte r = number of satisfied bonds of replica r:
        // bond (i,j) is satisfied (J s_i s_j = -1) iff b_i ^ b_j ^ [J < 0] = 1.
        uint32_t acc = 0;
        for (int d = 0; d < deg; ++d) {
            const uint32_t e = ell[d * ld + p];
            const uint32_t w = swq[e & 0xFFFFu];
            acc += own ^ w ^ ((e >> 31) ? 0x01010101u : 0u);
        }
        // dE = -2 s (h + sum_j J s_j) = 4 sat - 2 deg + 2h - 4h b   (s = 2b - 1)
        const int base = 2 * h - 2 * deg;
        const int h4 = 4 * h;
#pragma unroll
        for (int r = 0; r < 4; ++r)
            dE[r] = base + 4 * (int)((acc >> (8 * r)) & 0xFFu) - h4 * (int)((own >> (8 * r)) & 1u);
    } else {
        int a0 = 0, a1 = 0, a2 = 0, a3 = 0, sumJ = 0;
        for (int d = 0; d < deg; ++d) {
            const uint32_t e = ell[d * ld + p];
            const int Jv = (int)e >> 16;
            const uint32_t w = swq[e & 0xFFFFu];
            sumJ += Jv;
            a0 += Jv * (int)(w & 1u);
            a1 += Jv * (int)((w >> 8) & 1u);
            a2 += Jv * (int)((w >> 16) & 1u);
            a3 += Jv * (int)((w >> 24) & 1u);
        }
        // f = h + sum_j J s_j = h - sum_j J + 2 sum_j J b_j ;  dE = -2 s f
        const int hb = h - sumJ;
        const int a[4] = {a0, a1, a2, a3};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int f = hb + 2 * a[r];
            const int s = 2 * (int)((own >> (8 * r)) & 1u) - 1;
            dE[r] = -2 * s * f;
        }
    }
    const uint32_t u[4] = {rw.x, rw.y, rw.z, rw.w};
    uint32_t flip = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int idx = min(max(dE[r], 0), thr_w - 1);
        const bool acc = (dE[r] <= 0) | (u[r] < th[idx]);
        flip |= (uint32_t)acc << (8 * r);
    }
    return flip;
}

template <bool PM1, bool STAGE, int B>
__device__ void run_item(const SweepLaunch &L, const SweepJob &job, int quad0, int nq,
                         unsigned char *smem)
{
    const int tid = threadIdx.x;
    const DevProb *P = job.prob;
    const int n = P->n;
    const int ncol = P->ncol;
    const int maxdeg = P->maxdeg;
    const int cap_n = P->cap_n;
    const int thr_w = min(L.thr_stride, P->dmax + 1);
    const int64_t offset = P->offset;
    const uint32_t k0 = (uint32_t)job.seed, k1 = (uint32_t)(job.seed >> 32);
    const uint32_t phase_hi = job.phase << kSweepBits;
    const int T = job_end(L, job);

    uint32_t *sw = reinterpret_cast<uint32_t *>(smem);
    uint32_t *thr_s = sw + (size_t)L.Q * L.max_n;
    int *e2 = reinterpret_cast<int *>(thr_s + 2 * L.thr_stride);
    int32_t *s_idx = e2 + 4 * L.Q;
    uint32_t *s_meta = reinterpret_cast<uint32_t *>(s_idx + L.max_n);
    uint32_t *s_ell = s_meta + L.max_n;

    __shared__ int s_cptr[kMaxColours + 1];

    const int32_t *idx;
    const uint32_t *meta;
    const uint32_t *ell;
    int ld;
    if (STAGE) {
        for (int p = tid; p < n; p += B) {
            s_idx[p] = P->idx_of_pos[p];
            s_meta[p] = P->meta[p];
        }
        for (int d = 0; d < maxdeg; ++d)
            for (int p = tid; p < n; p += B) s_ell[d * n + p] = P->ell[(size_t)d * cap_n + p];
        idx = s_idx;
        meta = s_meta;
        ell = s_ell;
        ld = n;
    } else {
        idx = P->idx_of_pos;
        meta = P->meta;
        ell = P->ell;
        ld = cap_n;
    }
    for (int c = tid; c <= ncol; c += B) s_cptr[c] = P->cptr[c];
    for (int x = tid; x < 4 * nq; x += B) e2[x] = 0;

    // initial state (s_i = +1 iff the top bit of the word at the init slot is
    // set), or the state a resumed sample continues from
    init_spins(P, job, quad0, nq, sw, nullptr);
    const int t0 = job.t0;
    if (t0 < T)
        for (int d = tid; d < thr_w; d += B) thr_s[(t0 & 1) * L.thr_stride + d] = L.thr[(size_t)t0 * L.thr_stride + d];
    __syncthreads();

    for (int t = t0; t < T; ++t) {
        const uint32_t *th = thr_s + (t & 1) * L.thr_stride;
        const uint32_t ctr_y = phase_hi | (uint32_t)t;
        for (int c = 0; c < ncol; ++c) {
            if (c == 0 && t + 1 < T) {
                uint32_t *nxt = thr_s + ((t + 1) & 1) * L.thr_stride;
                const uint32_t *src = L.thr + (size_t)(t + 1) * L.thr_stride;
                for (int d = tid; d < thr_w; d += B) nxt[d] = src[d];
            }
            const int lo = s_cptr[c];
            const int nc = s_cptr[c + 1] - lo;
            if (nc > 0) {
                // flatten (q, k) over nq * nc items, k fastest
                int q = tid / nc, k = tid - q * nc;
                const int dq = B / nc, dk = B - dq * nc;
                while (q < nq) {
                    const int p = lo + k;
                    uint32_t *swq = sw + q * n;
                    const uint32_t own = swq[p];
                    const uint4 rw = philox4x32_10(
                        make_uint4((uint32_t)idx[p], ctr_y, (uint32_t)(quad0 + q), job.start), k0, k1);
                    const uint32_t flip = flip_mask<PM1>(own, meta[p], ell, ld, p, swq, rw, th, thr_w);
                    swq[p] = own ^ flip;
                    q += dq;
                    k += dk;
                    if (k >= nc) { k -= nc; ++q; }
                }
            }
            __syncthreads();
        }
    }

    // energies (2E accumulated per replica)
    for (int q = 0; q < nq; ++q) {
        const uint32_t *swq = sw + q * n;
        for (int p = tid; p < n; p += B) {
            int c2[4];
            energy2<PM1>(swq[p], meta[p], ell, ld, p, swq, c2);
#pragma unroll
            for (int r = 0; r < 4; ++r) atomicAdd(&e2[4 * q + r], c2[r]);
        }
    }
    __syncthreads();
    for (int x = tid; x < 4 * nq; x += B) {
        const int r = 4 * quad0 + x;
        if (r < job.S) job.energies[r] = (int64_t)(e2[x] / 2) + offset;
    }

    // bit-packed final states, one warp per (quad, word)
    const int lane = tid & 31, warp = tid >> 5;
    const int Wn = (n + 31) >> 5;
    for (int x = warp; x < nq * Wn; x += B / 32) {
        const int q = x / Wn, w = x - q * Wn;
        const int i = 32 * w + lane;
        const uint32_t word = (i < n) ? sw[q * n + P->pos_of_idx[i]] : 0u;
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const uint32_t bits = __ballot_sync(0xFFFFFFFFu, (word >> (8 * rr)) & 1u);
            const int r = 4 * (quad0 + q) + rr;
            if (lane == 0 && r < job.S) job.spins[(size_t)r * job.W + w] = bits;
        }
    }
}

template <bool PM1, bool STAGE, int B>
__global__ void __launch_bounds__(B) k_sweep(const SweepLaunch L)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    for (int iter = 0;; ++iter) {
        SweepJob job;
        int quad0, nq;
        if (L.items) {
            if (threadIdx.x == 0) s_item = atomicAdd(L.queue, 1);
            __syncthreads();
            const int it = s_item;
            if (it >= *L.nitems) break;
            const WorkItem wi = L.items[it];
            job = L.jobs[wi.job];
            quad0 = wi.quad0;
            nq = wi.nq;
        } else {
            if (iter > 0) break;
            job = L.single;
            quad0 = blockIdx.x * L.Q;
            nq = min(L.Q, (job.S + 3) / 4 - quad0);
            if (nq <= 0) break;
        }
        run_item<PM1, STAGE, B>(L, job, quad0, nq, smem);
        __syncthreads();
    }
}

template <bool PM1, bool STAGE>
cudaError_t launch_b(const SweepLaunch &L, int block, int grid, size_t smem, cudaStream_t st)
{
    switch (block) {
    case 128:
        cudaFuncSetAttribute(k_sweep<PM1, STAGE, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_sweep<PM1, STAGE, 128><<<grid, 128, smem, st>>>(L);
        break;
    case 256:
        cudaFuncSetAttribute(k_sweep<PM1, STAGE, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_sweep<PM1, STAGE, 256><<<grid, 256, smem, st>>>(L);
        break;
    case 512:
        cudaFuncSetAttribute(k_sweep<PM1, STAGE, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_sweep<PM1, STAGE, 512><<<grid, 512, smem, st>>>(L);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <bool PM1, bool STAGE>
int occ_b(int block, size_t smem)
{
    int nb = 0;
    switch (block) {
    case 128:
        cudaFuncSetAttribute(k_sweep<PM1, STAGE, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<PM1, STAGE, 128>, 128, smem);
        break;
    case 256:
        cudaFuncSetAttribute(k_sweep<PM1, STAGE, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<PM1, STAGE, 256>, 256, smem);
        break;
    case 512:
        cudaFuncSetAttribute(k_sweep<PM1, STAGE, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<PM1, STAGE, 512>, 512, smem);
        break;
    default:
        return 0;
    }
    return nb;
}

}  // namespace

cudaError_t launch_sweep(const SweepLaunch &L, bool pm1, int block, int grid, size_t smem,
                         cudaStream_t stream)
{
    if (grid <= 0) return cudaSuccess;
    if (pm1) return L.stage_ell ? launch_b<true, true>(L, block, grid, smem, stream)
                                : launch_b<true, false>(L, block, grid, smem, stream);
    return L.stage_ell ? launch_b<false, true>(L, block, grid, smem, stream)
                       : launch_b<false, false>(L, block, grid, smem, stream);
}

int sweep_max_active_blocks(bool pm1, int block, size_t smem, bool stage_ell)
{
    if (pm1) return stage_ell ? occ_b<true, true>(block, smem) : occ_b<true, false>(block, smem);
    return stage_ell ? occ_b<false, true>(block, smem) : occ_b<false, false>(block, smem);
}

}  // namespace spvar
