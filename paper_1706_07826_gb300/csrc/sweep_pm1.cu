// Register-resident simulated-annealing sweep for +-1 couplers (the sampler
// of Sec. III.A on the paper's +-J spin glasses and Chimera problems).
//
// Same dynamics, random words and result as the general sweep kernel, with
// the per-attempt instruction count cut down:
//  - every thread owns NSLOT fixed (spin, quad) items for the whole anneal;
//    their neighbour word offsets, SWAR constants and the parts of Philox
//    rounds 1-3 that do not depend on the sweep index stay in registers;
//  - shared memory holds each spin word twice, as is and with every replica
//    bit inverted, so a J < 0 neighbour is read from the inverted copy and the
//    local field of four replicas is one byte-wise sum of neighbour words;
//  - the flip-cost index of the four replicas is formed byte-wise (SWAR) and
//    looks up a shared row of the threshold table.
// Eligible when every |J| = 1, degree <= MAXD and dmax <= 254 (the biased
// index fits a byte).
#include "sweep_common.cuh"

namespace spvar {

namespace {

constexpr int kRowWords = 256;  // threshold row indexed by dE/2 + bias, bias <= 127
constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u, kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;

template <int MAXD>
struct SlotRegs {
    uint32_t own;      // byte offset of the slot's spin word in shared memory
    uint32_t nb[MAXD]; // byte offsets of the neighbours (inverted copy if J < 0, zero word if padding)
    uint32_t c0, c1;   // per byte: bias - deg + h, bias + deg - h
    uint32_t A, L0k, D, H3k, L3;  // Philox rounds 1-3 folded with the slot's fixed counter words
    int colour;        // colour class of the slot, -1 if the slot is empty
};

// Shared-memory word at a byte offset from the start of the dynamic window.
__device__ __forceinline__ uint32_t lds_b(const uint32_t *base, uint32_t byte_off)
{
    return *reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(base) + byte_off);
}
__device__ __forceinline__ void sts_b(uint32_t *base, uint32_t byte_off, uint32_t v)
{
    *reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(base) + byte_off) = v;
}

__device__ __forceinline__ void mulhilo(uint32_t m, uint32_t a, uint32_t &hi, uint32_t &lo)
{
    const uint64_t p = (uint64_t)m * a;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
}

// Counter (i, y, q, s): the sweep word y is the only input that changes
// between sweeps, so the products of round 1 and parts of rounds 2 and 3 are
// slot constants.
template <int MAXD>
__device__ __forceinline__ void philox_setup(SlotRegs<MAXD> &s, uint32_t i, uint32_t q, uint32_t start,
                                             uint32_t k0, uint32_t k1)
{
    uint32_t H0, L0, H1, L1, H2, L2, H3, L3;
    mulhilo(kM0, i, H0, L0);
    mulhilo(kM1, q, H1, L1);
    const uint32_t Z = H0 ^ start ^ k1;            // round-1 counter word 2
    mulhilo(kM1, Z, H2, L2);                        // round-2 product of word 2
    const uint32_t C1 = H2 ^ L1 ^ (k0 + kW0);       // round-2 counter word 0
    mulhilo(kM0, C1, H3, L3);                       // round-3 product of word 0
    s.A = H1 ^ k0;
    s.L0k = L0 ^ (k1 + kW1);
    s.D = L2 ^ (k0 + 2 * kW0);
    s.H3k = H3 ^ (k1 + 2 * kW1);
    s.L3 = L3;
}

// Round keys 3..9 of the item's seed.
struct RoundKeys {
    uint32_t k0[7], k1[7];
};

__device__ __forceinline__ RoundKeys round_keys(uint32_t k0, uint32_t k1)
{
    RoundKeys K;
#pragma unroll
    for (int r = 3; r < 10; ++r) {
        K.k0[r - 3] = k0 + (uint32_t)r * kW0;
        K.k1[r - 3] = k1 + (uint32_t)r * kW1;
    }
    return K;
}

template <int MAXD>
__device__ __forceinline__ uint4 philox_slot(const SlotRegs<MAXD> &s, uint32_t y, const RoundKeys &K)
{
    uint32_t h, l, h2, l2;
    mulhilo(kM0, s.A ^ y, h, l);          // round 2: word 0 product
    mulhilo(kM1, h ^ s.L0k, h2, l2);      // round 3: word 2 product
    uint4 c = make_uint4(h2 ^ s.D, l2, s.H3k ^ l, s.L3);
#pragma unroll
    for (int r = 3; r < 10; ++r) {
        uint32_t a, b, e, f;
        mulhilo(kM0, c.x, a, b);
        mulhilo(kM1, c.z, e, f);
        c = make_uint4(e ^ c.y ^ K.k0[r - 3], f, a ^ c.w ^ K.k1[r - 3], b);
    }
    return c;
}

template <int B, int NSLOT, int MAXD>
__device__ void run_item_pm1(const SweepLaunch &L, const SweepJob &job, int quad0, int nq, uint32_t *smem)
{
    const int tid = threadIdx.x;
    const DevProb *P = job.prob;
    const int n = P->n;
    const int ncol = P->ncol;
    const int cap_n = P->cap_n;
    const int bias = P->dmax >> 1;
    const uint32_t k0 = (uint32_t)job.seed, k1 = (uint32_t)(job.seed >> 32);
    const uint32_t phase_hi = job.phase << kSweepBits;
    const int T = L.T;
    const int S1 = nq * n;  // offset of the inverted copy

    uint32_t *sw = smem;                           // [S1] plain, [S1] inverted, [1] zero
    uint32_t *trow = smem + 2 * L.Q * L.max_n + 4; // 2 threshold rows
    int *e2 = reinterpret_cast<int *>(trow + 2 * kRowWords);
    __shared__ int s_cptr[kMaxColours + 1];

    for (int c = tid; c <= ncol; c += B) s_cptr[c] = P->cptr[c];
    init_spins(P, job, quad0, nq, sw, sw + S1);
    if (tid == 0) sw[2 * S1] = 0u;
    // first row of the thresholds: trow[bias + e] = thr[t0][2e], e = 1..bias
    const int t0 = job.t0;
    if (t0 < T)
        for (int e = tid + 1; e <= bias; e += B)
            trow[(t0 & 1) * kRowWords + bias + e] = L.thr[(size_t)t0 * L.thr_stride + 2 * e];
    __syncthreads();

    SlotRegs<MAXD> s[NSLOT];
    uint4 u[NSLOT];  // random words of each slot for the sweep about to run
    const RoundKeys K = round_keys(k0, k1);
    const int total = n * nq;
#pragma unroll
    for (int j = 0; j < NSLOT; ++j) {
        const int g = tid + j * B;
        s[j].colour = -1;
        s[j].own = 4u * (uint32_t)(2 * S1);
#pragma unroll
        for (int d = 0; d < MAXD; ++d) s[j].nb[d] = 4u * (uint32_t)(2 * S1);
        s[j].c0 = s[j].c1 = s[j].A = s[j].L0k = s[j].D = s[j].H3k = s[j].L3 = 0u;
        if (g < total) {
            int c = 0;
            while (s_cptr[c + 1] * nq <= g) ++c;
            const int nc = s_cptr[c + 1] - s_cptr[c];
            const int local = g - s_cptr[c] * nq;
            const int q = local / nc;
            const int p = s_cptr[c] + (local - q * nc);
            const uint32_t meta = P->meta[p];
            const int deg = (int)(meta & 0xFFFFu);
            const int h = (int)meta >> 16;
            s[j].own = 4u * (uint32_t)(q * n + p);
#pragma unroll
            for (int d = 0; d < MAXD; ++d) {
                if (d < deg) {
                    const uint32_t e = P->ell[(size_t)d * cap_n + p];
                    s[j].nb[d] = 4u * (uint32_t)(((e >> 31) ? S1 : 0) + q * n + (int)(e & 0xFFFFu));
                }
            }
            s[j].c0 = (uint32_t)(bias - deg + h) * 0x01010101u;
            s[j].c1 = (uint32_t)(bias + deg - h) * 0x01010101u;
            philox_setup(s[j], (uint32_t)P->idx_of_pos[p], (uint32_t)(quad0 + q), job.start, k0, k1);
            s[j].colour = c;
        }
        u[j] = philox_slot(s[j], phase_hi | (uint32_t)t0, K);  // first sweep
    }

    for (int t = t0; t < T; ++t) {
        const uint32_t *th = trow + (t & 1) * kRowWords;
        const uint32_t y = phase_hi | (uint32_t)t;
        for (int c = 0; c < ncol; ++c) {
            if (c == 0 && t + 1 < T) {
                uint32_t *nxt = trow + ((t + 1) & 1) * kRowWords;
                const uint32_t *src = L.thr + (size_t)(t + 1) * L.thr_stride;
                for (int e = tid + 1; e <= bias; e += B) nxt[bias + e] = src[2 * e];
            }
#pragma unroll
            for (int j = 0; j < NSLOT; ++j) {
                if (s[j].colour == c) {
                    // loads first; the next sweep's Philox block (independent of the spins)
                    // is computed while they are in flight
                    const uint32_t own = lds_b(sw, s[j].own);
                    uint32_t nbw[MAXD];
#pragma unroll
                    for (int d = 0; d < MAXD; ++d) nbw[d] = lds_b(sw, s[j].nb[d]);
                    const uint4 unext = philox_slot(s[j], y + 1u, K);
                    uint32_t x = 0;
#pragma unroll
                    for (int d = 0; d < MAXD; ++d) x += nbw[d];
                    // byte r: number of neighbours with b_j ^ [J_ij < 0] = 1; the
                    // flip-cost index dE/2 + bias is 2x + c0 if b_i = 0, c1 - 2x if b_i = 1
                    const uint32_t m = own * 0xFFu;
                    const uint32_t x2 = x + x;
                    const uint32_t idx4 = ((x2 + s[j].c0) & ~m) | ((s[j].c1 - x2) & m);
                    // byte r of `always` is 0x80 iff idx_r <= bias (dE <= 0): accepted without a draw
                    const uint32_t always = ((uint32_t)(bias + 0x80) * 0x01010101u - idx4) & 0x80808080u;
                    const uint32_t uu[4] = {u[j].x, u[j].y, u[j].z, u[j].w};
                    uint32_t flip = always >> 7;
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int ir = (int)((idx4 >> (8 * r)) & 0xFFu);
                        if (uu[r] < th[ir]) flip |= 1u << (8 * r);
                    }
                    const uint32_t nw = own ^ flip;
                    sts_b(sw, s[j].own, nw);
                    sts_b(sw, s[j].own + 4u * (uint32_t)S1, nw ^ 0x01010101u);
                    u[j] = unext;
                }
            }
            __syncthreads();
        }
    }
    finish_item<true>(P, job, quad0, nq, sw, e2);
}

template <int B, int NSLOT, int MAXD>
__global__ void __launch_bounds__(B) k_sweep_pm1(const SweepLaunch L)
{
    extern __shared__ __align__(16) uint32_t smem_pm1[];
    __shared__ int s_item;
    for (int iter = 0;; ++iter) {
        SweepJob job;
        int quad0, nq;
        if (!next_item(L, iter, &s_item, job, quad0, nq)) break;
        run_item_pm1<B, NSLOT, MAXD>(L, job, quad0, nq, smem_pm1);
        __syncthreads();
    }
}

template <int B, int NSLOT, int MAXD>
void *kernel_ptr()
{
    return reinterpret_cast<void *>(k_sweep_pm1<B, NSLOT, MAXD>);
}

void *select_kernel(int block, int nslot, int maxd)
{
#define SPVAR_PM1_CASE(BB, NS, MD) \
    if (block == BB && nslot == NS && maxd == MD) return kernel_ptr<BB, NS, MD>();
    SPVAR_PM1_CASE(128, 1, 6) SPVAR_PM1_CASE(128, 2, 6) SPVAR_PM1_CASE(128, 4, 6)
    SPVAR_PM1_CASE(256, 1, 6) SPVAR_PM1_CASE(256, 2, 6) SPVAR_PM1_CASE(256, 4, 6)
    SPVAR_PM1_CASE(512, 1, 6) SPVAR_PM1_CASE(512, 2, 6)
    SPVAR_PM1_CASE(128, 1, 8) SPVAR_PM1_CASE(128, 2, 8) SPVAR_PM1_CASE(128, 4, 8)
    SPVAR_PM1_CASE(256, 1, 8) SPVAR_PM1_CASE(256, 2, 8) SPVAR_PM1_CASE(256, 4, 8)
    SPVAR_PM1_CASE(512, 1, 8) SPVAR_PM1_CASE(512, 2, 8)
#undef SPVAR_PM1_CASE
    return nullptr;
}

}  // namespace

bool pm1_shape_ok(int block, int nslot, int maxd) { return select_kernel(block, nslot, maxd) != nullptr; }

size_t pm1_smem_bytes(int max_n, int Q)
{
    return 4 * (2 * (size_t)Q * max_n + 4 + 2 * (size_t)kRowWords + 4 * (size_t)Q);
}

cudaError_t launch_sweep_pm1(const SweepLaunch &L, int block, int nslot, int maxd, int grid, size_t smem,
                             cudaStream_t st)
{
    void *k = select_kernel(block, nslot, maxd);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<SweepLaunch *>(&L)};
    return cudaLaunchKernel(k, dim3(grid), dim3(block), args, smem, st);
}

int pm1_max_active_blocks(int block, int nslot, int maxd, size_t smem)
{
    void *k = select_kernel(block, nslot, maxd);
    if (!k) return 0;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem);
    return nb;
}

}  // namespace spvar
