// Warp-per-quad simulated-annealing sweep for +-1 couplers (the sampler of
// Sec. III.A).  Same dynamics, random words and result as the other sweep
// kernels.
//
// A CTA takes WARPS quads (4 replicas each) of one problem; warp w anneals
// quad w alone, in its own region of shared memory (spin words as is, spin
// words with every replica bit inverted, a zero word).  A colour class is
// therefore closed by __syncwarp, not by a CTA barrier, and each lane walks
// many spins of the class, K (2 or 4) at a time.  What every quad needs is staged
// once per CTA: each spin's (h, degree), its neighbour word offsets (16-bit,
// J < 0 neighbours pointing into the inverted copy, missing neighbours at the
// zero word) and the parts of Philox rounds 1-3 that depend only on the spin
// and the start.  The parts that depend only on the quad and the sweep are
// computed once per warp and sweep, so an item pays two wide multiplies less.
// The flip-cost index of the four replicas is formed byte-wise (SWAR) and
// looked up in the warp's own row of the threshold table.
// Eligible when every |J| = 1, degree <= MAXD, dmax <= 254 and 2n + 1 < 65536.
#include "sweep_common.cuh"

namespace spvar {

namespace {

constexpr int kRowW = 128;  // one threshold row: entries for dE/2 = 1 .. bias (bias <= 127)

// Words of shared memory per CTA for a problem of at most max_n spins.
__host__ __device__ inline size_t pm1w_words(int max_n, int warps, int maxd)
{
    const size_t region = 2 * (size_t)max_n + 2;
    return 4 * (size_t)max_n + ((size_t)maxd * max_n + 1) / 2 + (size_t)warps * region + kRowW +
           (size_t)warps * 2 * kRowW + 4 * (size_t)warps + 2;
}

template <int MAXD>
__device__ __forceinline__ uint32_t update_spin(uint32_t *sw, const uint16_t *off, int n, int p, uint32_t meta,
                                                int bias, uint4 u, const uint32_t *th_adj)
{
    const uint32_t own = sw[p];
    uint32_t x = 0;
#pragma unroll
    for (int d = 0; d < MAXD; ++d) x += sw[off[d * n + p]];
    const int deg = (int)(meta & 0xFFFFu);
    const int h = (int)meta >> 16;
    const uint32_t c0 = (uint32_t)(bias - deg + h) * 0x01010101u;
    const uint32_t c1 = (uint32_t)(bias + deg - h) * 0x01010101u;
    // byte r: number of neighbours with b_j ^ [J_ij < 0] = 1; index dE/2 + bias
    const uint32_t m = own * 0xFFu;
    const uint32_t x2 = x + x;
    const uint32_t idx4 = ((x2 + c0) & ~m) | ((c1 - x2) & m);
    const uint32_t always = ((uint32_t)(bias + 0x80) * 0x01010101u - idx4) & 0x80808080u;
    uint32_t flip = always >> 7;
    const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int ir = (int)((idx4 >> (8 * r)) & 0xFFu);
        // th_adj[ir] is the threshold of dE = 2 (ir - bias) for ir > bias (lanes with ir <= bias
        // read a word of the preceding region and are accepted by `always` anyway)
        if (uu[r] < th_adj[ir]) flip |= 1u << (8 * r);
    }
    return own ^ flip;
}

template <int WARPS, int MAXD, int K>
__device__ void run_item_pm1w(const SweepLaunch &L, const SweepJob &job, int quad0, int nq, uint32_t *smem)
{
    constexpr int B = 32 * WARPS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const DevProb *P = job.prob;
    const int n = P->n;
    const int ncol = P->ncol;
    const int cap_n = P->cap_n;
    const int bias = P->dmax >> 1;
    const int T = job_end(L, job);
    const int max_n = L.max_n;
    const uint32_t k0 = (uint32_t)job.seed, k1 = (uint32_t)(job.seed >> 32);
    const uint32_t phase_hi = job.phase << kSweepBits;
    const int region = 2 * max_n + 2;

    uint32_t *meta_s = smem;
    uint32_t *l0k_s = meta_s + max_n;
    uint32_t *h2_s = l0k_s + max_n;
    uint32_t *d_s = h2_s + max_n;
    uint16_t *off = reinterpret_cast<uint16_t *>(d_s + max_n);
    uint32_t *regions = d_s + max_n + (MAXD * max_n + 1) / 2;
    // kRowW pad words before the rows: lookups of always-accepted lanes land up to
    // bias + 1 <= 128 words before a row and must stay inside this allocation
    uint32_t *rows = regions + WARPS * region + kRowW;
    int *e2 = reinterpret_cast<int *>(rows + WARPS * 2 * kRowW);
    __shared__ int s_cptr[kMaxColours + 1];

    // per-spin constants shared by every quad of the CTA
    for (int c = tid; c <= ncol; c += B) s_cptr[c] = P->cptr[c];
    for (int p = tid; p < n; p += B) {
        meta_s[p] = P->meta[p];
        uint32_t H0, L0, H2, L2;
        philox_mulhilo(kPhiloxM0, (uint32_t)P->idx_of_pos[p], H0, L0);
        const uint32_t Z = H0 ^ job.start ^ k1;  // round-1 counter word 2
        philox_mulhilo(kPhiloxM1, Z, H2, L2);              // its round-2 product
        l0k_s[p] = L0 ^ (k1 + kPhiloxW1);
        h2_s[p] = H2;
        d_s[p] = L2 ^ (k0 + 2 * kPhiloxW0);
    }
    for (int x = tid; x < MAXD * n; x += B) {
        const int d = x / n, p = x - d * n;
        const int deg = (int)(P->meta[p] & 0xFFFFu);
        uint16_t o = (uint16_t)(2 * n);
        if (d < deg) {
            const uint32_t e = P->ell[(size_t)d * cap_n + p];
            o = (uint16_t)(((e >> 31) ? n : 0) + (int)(e & 0xFFFFu));
        }
        off[x] = o;
    }
    __syncthreads();

    if (warp < nq) {
        uint32_t *sw = regions + warp * region;
        uint32_t *myrows = rows + warp * 2 * kRowW;
        const uint32_t q = (uint32_t)(quad0 + warp);
        // initial state of this quad (or the state a resumed sample continues from)
        for (int p = lane; p < n; p += 32) {
            const uint32_t w = start_word(P, job, (int)q, p);
            sw[p] = w;
            sw[n + p] = w ^ 0x01010101u;
        }
        if (lane == 0) sw[2 * n] = 0u;
        // quad constants of rounds 1-3
        uint32_t H1, L1;
        philox_mulhilo(kPhiloxM1, q, H1, L1);
        const uint32_t A = H1 ^ k0;                // round-1 word 0 = A ^ sweep word
        const uint32_t L1k = L1 ^ (k0 + kPhiloxW0);     // round-2 word 0 = H2 ^ L1k
        const PhiloxKeys<3> Kr = philox_keys<3>(k0, k1);
        const uint32_t k1_2 = k1 + 2 * kPhiloxW1;
        const int t0 = job.t0;
        if (t0 < T)
            for (int e = lane + 1; e <= bias; e += 32)
                myrows[(t0 & 1) * kRowW + e - 1] = L.thr[(size_t)t0 * L.thr_stride + 2 * e];
        __syncwarp();

        for (int t = t0; t < T; ++t) {
            const uint32_t *th_adj = myrows + (t & 1) * kRowW - (bias + 1);
            const uint32_t y = phase_hi | (uint32_t)t;
            // round-2 product of word 0: the same for every spin of the quad
            uint32_t hh, ll;
            philox_mulhilo(kPhiloxM0, A ^ y, hh, ll);
            const uint32_t lk = ll ^ k1_2;
            for (int c = 0; c < ncol; ++c) {
                if (c == 0 && t + 1 < T) {
                    uint32_t *nxt = myrows + ((t + 1) & 1) * kRowW;
                    const uint32_t *src = L.thr + (size_t)(t + 1) * L.thr_stride;
                    for (int e = lane + 1; e <= bias; e += 32) nxt[e - 1] = src[2 * e];
                }
                const int lo = s_cptr[c], hi = s_cptr[c + 1];
                for (int p1 = lo + lane; p1 < hi; p1 += 32 * K) {
                    // K spins of the class per lane, all loads and Philox blocks before any store
                    int pp[K];
                    bool valid[K];
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        valid[k] = p1 + 32 * k < hi;
                        pp[k] = valid[k] ? p1 + 32 * k : p1;
                    }
                    uint4 u[K];
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const int p = pp[k];
                        uint32_t h3, l3, HH, LL;
                        philox_mulhilo(kPhiloxM1, hh ^ l0k_s[p], h3, l3);        // round 2, word 2
                        philox_mulhilo(kPhiloxM0, h2_s[p] ^ L1k, HH, LL);        // round 3, word 0
                        u[k] = philox_rounds<3>(make_uint4(h3 ^ d_s[p], l3, HH ^ lk, LL), Kr);
                    }
                    uint32_t w[K];
#pragma unroll
                    for (int k = 0; k < K; ++k)
                        w[k] = update_spin<MAXD>(sw, off, n, pp[k], meta_s[pp[k]], bias, u[k], th_adj);
#pragma unroll
                    for (int k = 0; k < K; ++k)
                        if (valid[k]) {
                            sw[pp[k]] = w[k];
                            sw[n + pp[k]] = w[k] ^ 0x01010101u;
                        }
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    finish_item<true>(P, job, quad0, nq, regions, e2, region);
}

template <int WARPS, int MAXD, int K>
__global__ void __launch_bounds__(32 * WARPS) k_sweep_pm1w(const SweepLaunch L)
{
    extern __shared__ __align__(16) uint32_t smem_pm1w[];
    __shared__ int s_item;
    for (int iter = 0;; ++iter) {
        SweepJob job;
        int quad0, nq;
        if (!next_item(L, iter, &s_item, job, quad0, nq)) break;
        run_item_pm1w<WARPS, MAXD, K>(L, job, quad0, nq, smem_pm1w);
        __syncthreads();
    }
}

// K: spins in flight per lane (2 or 4).
void *select_w(int warps, int maxd, int K)
{
#define SPVAR_W_CASE(W, MD, KK) \
    if (warps == W && maxd == MD && K == KK) return reinterpret_cast<void *>(k_sweep_pm1w<W, MD, KK>);
    SPVAR_W_CASE(2, 6, 2) SPVAR_W_CASE(4, 6, 2) SPVAR_W_CASE(8, 6, 2) SPVAR_W_CASE(16, 6, 2)
    SPVAR_W_CASE(2, 8, 2) SPVAR_W_CASE(4, 8, 2) SPVAR_W_CASE(8, 8, 2) SPVAR_W_CASE(16, 8, 2)
    SPVAR_W_CASE(2, 6, 4) SPVAR_W_CASE(4, 6, 4) SPVAR_W_CASE(8, 6, 4) SPVAR_W_CASE(16, 6, 4)
    SPVAR_W_CASE(2, 8, 4) SPVAR_W_CASE(4, 8, 4) SPVAR_W_CASE(8, 8, 4) SPVAR_W_CASE(16, 8, 4)
#undef SPVAR_W_CASE
    return nullptr;
}

}  // namespace

bool pm1w_shape_ok(int warps, int maxd, int max_n, int K)
{
    return select_w(warps, maxd, K) && 2LL * max_n + 1 <= 0xFFFF;
}

size_t pm1w_smem_bytes(int max_n, int warps, int maxd) { return 4 * pm1w_words(max_n, warps, maxd); }

cudaError_t launch_sweep_pm1w(const SweepLaunch &L, int warps, int maxd, int K, int grid, size_t smem,
                              cudaStream_t st)
{
    void *k = select_w(warps, maxd, K);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<SweepLaunch *>(&L)};
    return cudaLaunchKernel(k, dim3(grid), dim3(32 * warps), args, smem, st);
}

int pm1w_max_active_blocks(int warps, int maxd, int K, size_t smem)
{
    void *k = select_w(warps, maxd, K);
    if (!k) return 0;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 32 * warps, smem);
    return nb;
}

}  // namespace spvar
