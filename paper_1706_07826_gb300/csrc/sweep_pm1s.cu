// Streaming simulated-annealing sweep for +-1 couplers on large problems
// (the sampler of Sec. III.A; 3D spin glasses up to N = 8000 and beyond).
//
// Same dynamics, random words and result as the other sweep kernels.  Where
// the register-resident kernel keeps every item's constants in registers
// (and so holds at most ~1000 spins per CTA), this one stages per work item,
// in shared memory, the neighbour word offsets of every spin as 16-bit values
// with the inverted-copy offset of J < 0 neighbours already folded in (slots
// past a spin's degree point at a zero word).  Each thread then walks the
// items of a colour class two at a time: neighbour words are summed byte-wise
// (SWAR, four replicas per word), the flip-cost index is formed byte-wise and
// looked up in a shared threshold row, and the Philox block of each item is
// computed with hoisted round keys.
// One quad (four replicas) per work item.  Eligible when every |J| = 1,
// degree <= MAXD, dmax <= 254 and 2n + 1 < 65536.
#include "sweep_common.cuh"

namespace spvar {

namespace {

constexpr int kRowWordsS = 256;
using Keys10 = PhiloxKeys<0>;

// Philox4x32-10 of counter (i, y, quad, start) with the quad's products
// hoisted: L1k = lo(M1 quad) ^ key0 of round 2 (per CTA item), (HA, LA) = M0 (hi(M1 quad) ^ y ^ key0)
// (round 2, word 0: per sweep); zs = start ^ key1 of round 1.
__device__ __forceinline__ uint4 philox_quad(uint32_t i, uint32_t zs, uint32_t L1k, uint32_t HA, uint32_t LA,
                                             const Keys10 &K)
{
    uint32_t h0, l0, h1, l1;
    philox_mulhilo(kPhiloxM0, i, h0, l0);       // round 1, word 0
    philox_mulhilo(kPhiloxM1, h0 ^ zs, h1, l1);  // round 2, word 2
    return philox_rounds<2>(make_uint4(h1 ^ L1k, l1, HA ^ l0 ^ K.k1[1], LA), K);
}

template <int MAXD>
__device__ __forceinline__ uint32_t flip_item(const uint32_t *sw, const uint16_t *off, int n, int p,
                                              uint32_t own, uint32_t meta, int bias, uint4 u, const uint32_t *th)
{
    uint32_t x = 0;
#pragma unroll
    for (int d = 0; d < MAXD; ++d) x += sw[off[d * n + p]];
    const int deg = (int)(meta & 0xFFFFu);
    const int h = (int)meta >> 16;
    const uint32_t c0 = (uint32_t)(bias - deg + h) * 0x01010101u;
    const uint32_t c1 = (uint32_t)(bias + deg - h) * 0x01010101u;
    const uint32_t m = own * 0xFFu;
    const uint32_t x2 = x + x;
    const uint32_t idx4 = ((x2 + c0) & ~m) | ((c1 - x2) & m);
    const uint32_t always = ((uint32_t)(bias + 0x80) * 0x01010101u - idx4) & 0x80808080u;
    uint32_t flip = always >> 7;
    const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int ir = (int)((idx4 >> (8 * r)) & 0xFFu);
        if (uu[r] < th[ir]) flip |= 1u << (8 * r);
    }
    return flip;
}

template <int B, int MAXD>
__device__ void run_item_pm1s(const SweepLaunch &L, const SweepJob &job, int quad0, int nq, uint32_t *smem)
{
    const int tid = threadIdx.x;
    const DevProb *P = job.prob;
    const int n = P->n;
    const int ncol = P->ncol;
    const int cap_n = P->cap_n;
    const int bias = P->dmax >> 1;
    const uint32_t phase_hi = job.phase << kSweepBits;
    const int T = job_end(L, job);
    const int S1 = n;      // one quad per item: the inverted copy follows the plain one
    const int ZERO = 2 * n;

    // [0, 2n): spin words (plain, inverted); [2n]: zero word; then offsets, rows, e2
    const int swords = 2 * L.max_n + 2;
    uint32_t *sw = smem;
    uint16_t *off = reinterpret_cast<uint16_t *>(smem + swords);
    uint32_t *trow = smem + swords + (MAXD * L.max_n + 1) / 2;
    int *e2 = reinterpret_cast<int *>(trow + 2 * kRowWordsS);
    __shared__ int s_cptr[kMaxColours + 1];

    for (int c = tid; c <= ncol; c += B) s_cptr[c] = P->cptr[c];
    init_spins(P, job, quad0, nq, sw, sw + S1);
    if (tid == 0) sw[ZERO] = 0u;
    for (int x = tid; x < MAXD * n; x += B) {
        const int d = x / n, p = x - d * n;
        const int deg = (int)(P->meta[p] & 0xFFFFu);
        uint16_t o = (uint16_t)ZERO;
        if (d < deg) {
            const uint32_t e = P->ell[(size_t)d * cap_n + p];
            o = (uint16_t)(((e >> 31) ? S1 : 0) + (int)(e & 0xFFFFu));
        }
        off[x] = o;
    }
    const int t0 = job.t0;
    if (t0 < T)
        for (int e = tid + 1; e <= bias; e += B)
            trow[(t0 & 1) * kRowWordsS + bias + e] = L.thr[(size_t)t0 * L.thr_stride + 2 * e];
    __syncthreads();

    const Keys10 K = philox_keys<0>((uint32_t)job.seed, (uint32_t)(job.seed >> 32));

    // the quad's Philox products: round 1 word 2 per item, round 2 word 0 per sweep
    uint32_t H1, L1;
    philox_mulhilo(kPhiloxM1, (uint32_t)quad0, H1, L1);
    const uint32_t L1k = L1 ^ K.k0[1], zs = job.start ^ K.k1[0];
    for (int t = t0; t < T; ++t) {
        const uint32_t *th = trow + (t & 1) * kRowWordsS;
        const uint32_t y = phase_hi | (uint32_t)t;
        uint32_t HA, LA;
        philox_mulhilo(kPhiloxM0, H1 ^ y ^ K.k0[0], HA, LA);
        for (int c = 0; c < ncol; ++c) {
            if (c == 0 && t + 1 < T) {
                uint32_t *nxt = trow + ((t + 1) & 1) * kRowWordsS;
                const uint32_t *src = L.thr + (size_t)(t + 1) * L.thr_stride;
                for (int e = tid + 1; e <= bias; e += B) nxt[bias + e] = src[2 * e];
            }
            const int lo = s_cptr[c];
            const int hi = s_cptr[c + 1];
            // two spins per iteration: loads and Philox of both before either store
            for (int p1 = lo + tid; p1 < hi; p1 += 2 * B) {
                const bool has2 = p1 + B < hi;
                const int p2 = has2 ? p1 + B : p1;
                const uint32_t meta1 = __ldg(P->meta + p1), meta2 = __ldg(P->meta + p2);
                const uint32_t i1 = (uint32_t)__ldg(P->idx_of_pos + p1), i2 = (uint32_t)__ldg(P->idx_of_pos + p2);
                const uint4 u1 = philox_quad(i1, zs, L1k, HA, LA, K);
                const uint4 u2 = philox_quad(i2, zs, L1k, HA, LA, K);
                const uint32_t own1 = sw[p1], own2 = sw[p2];
                const uint32_t f1 = flip_item<MAXD>(sw, off, n, p1, own1, meta1, bias, u1, th);
                const uint32_t f2 = flip_item<MAXD>(sw, off, n, p2, own2, meta2, bias, u2, th);
                const uint32_t w1 = own1 ^ f1;
                sw[p1] = w1;
                sw[p1 + S1] = w1 ^ 0x01010101u;
                if (has2) {
                    const uint32_t w2 = own2 ^ f2;
                    sw[p2] = w2;
                    sw[p2 + S1] = w2 ^ 0x01010101u;
                }
            }
            __syncthreads();
        }
    }
    finish_item<true>(P, job, quad0, nq, sw, e2);
}

template <int B, int MAXD>
__global__ void __launch_bounds__(B) k_sweep_pm1s(const SweepLaunch L)
{
    extern __shared__ __align__(16) uint32_t smem_pm1s[];
    __shared__ int s_item;
    for (int iter = 0;; ++iter) {
        SweepJob job;
        int quad0, nq;
        if (!next_item(L, iter, &s_item, job, quad0, nq)) break;
        run_item_pm1s<B, MAXD>(L, job, quad0, nq, smem_pm1s);
        __syncthreads();
    }
}

void *select_s(int block, int maxd)
{
    if (maxd == 6) {
        if (block == 128) return reinterpret_cast<void *>(k_sweep_pm1s<128, 6>);
        if (block == 256) return reinterpret_cast<void *>(k_sweep_pm1s<256, 6>);
        if (block == 512) return reinterpret_cast<void *>(k_sweep_pm1s<512, 6>);
        if (block == 1024) return reinterpret_cast<void *>(k_sweep_pm1s<1024, 6>);
    } else if (maxd == 8) {
        if (block == 128) return reinterpret_cast<void *>(k_sweep_pm1s<128, 8>);
        if (block == 256) return reinterpret_cast<void *>(k_sweep_pm1s<256, 8>);
        if (block == 512) return reinterpret_cast<void *>(k_sweep_pm1s<512, 8>);
        if (block == 1024) return reinterpret_cast<void *>(k_sweep_pm1s<1024, 8>);
    }
    return nullptr;
}

}  // namespace

bool pm1s_shape_ok(int block, int maxd, int max_n, int Q)
{
    return select_s(block, maxd) != nullptr && Q == 1 && 2LL * max_n + 1 <= 0xFFFF;
}

size_t pm1s_smem_bytes(int max_n, int Q, int maxd)
{
    return 4 * ((size_t)(2 * max_n + 2) + ((size_t)maxd * max_n + 1) / 2 + 2 * kRowWordsS + 4 * (size_t)Q);
}

cudaError_t launch_sweep_pm1s(const SweepLaunch &L, int block, int maxd, int grid, size_t smem, cudaStream_t st)
{
    void *k = select_s(block, maxd);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<SweepLaunch *>(&L)};
    return cudaLaunchKernel(k, dim3(grid), dim3(block), args, smem, st);
}

int pm1s_max_active_blocks(int block, int maxd, size_t smem)
{
    void *k = select_s(block, maxd);
    if (!k) return 0;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem);
    return nb;
}

}  // namespace spvar
