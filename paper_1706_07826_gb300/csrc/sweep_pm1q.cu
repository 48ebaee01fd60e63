// Quad-group simulated-annealing sweep for +-1 couplers (the sampler of
// Sec. III.A): one work item is nq quads (4 nq replicas) of one start's
// problem, any n that fits shared memory.
//
// Same dynamics, random words and result as the other sweep kernels.  Shared
// memory holds only the item's spin words: per quad a plain copy and a copy
// with every replica bit inverted ([q][2][n + 1]; word n of each copy is zero,
// the target of missing neighbours).  A colour class is swept by units
// (spin k, quad group g): a thread loads its spin's neighbour word offsets
// (the inverted copy folded in for J < 0), flip-cost constant and the Philox
// products that depend only on the spin and the start once, then sweeps that
// spin in every quad of its group, two quads at a time; units left over for a
// last partial round of the block are split over more threads (class_split).
// The Philox products that depend only on the quad and the sweep come from a
// small per-CTA table refreshed once per sweep, so an item pays 16 wide
// multiplies.  The flip-cost
// index of the four replicas is formed byte-wise (SWAR), pre-scaled to the
// byte offset of a 64-bit carry entry (2^32 - thr, 0 where dE <= 0): u + entry
// carries into bit 32 exactly when the move is rejected.
// Eligible when every |J| = 1, degree <= MAXD and dmax <= 30.
#include "sweep_common.cuh"

namespace spvar {

namespace {

constexpr int kRowQ = 32;   // 64-bit entries per threshold row: index dE/2 + bias <= 30
constexpr int kQcap = 64;   // most quads per work item

__device__ __forceinline__ uint32_t madlo_p(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint32_t lds_p(const uint32_t *base, uint32_t byte_off)
{
    return *reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(base) + byte_off);
}
__device__ __forceinline__ void sts_p(uint32_t *base, uint32_t byte_off, uint32_t v)
{
    *reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(base) + byte_off) = v;
}

struct QuadSmem {
    unsigned long long row[2][kRowQ];  // carry rows of the current and the next sweep
    uint2 qk[kQcap];                   // per quad: lo(M1 q) ^ key0 of round 2, hi(M1 q) ^ key0 of round 1
    uint2 qs[2][kQcap];                // per quad and sweep parity: M0 (hi(M1 q) ^ y ^ key0) (round 2, word 0)
    int e2[4 * kQcap];
    int cptr[kMaxColours + 1];
    int4 split[kMaxColours];           // per colour class: G, full units, remainder units, their split
};

// How a colour class of nc spins is dealt over the block for nq quads.  Units
// (spin, group g of quads g, g + G, ...) fill full rounds of B threads; the
// units left for a last partial round are each split into G2 sub-units
// (every G2-th quad of the unit's group), so that round uses the whole block.
// G is the choice that minimises the rounds' length in quad pairs plus one
// pair's worth of set-up per two rounds (a unit loads its spin's offsets and
// products once).  Returns (G, full units, remainder units, G2).
__device__ __forceinline__ int4 class_split(int nc, int nq, int B)
{
    int best = 0x7FFFFFFF;
    int4 pick = make_int4(1, 0, 0, 1);
    for (int G = 1; G <= nq; ++G) {
        const int qpu = (nq + G - 1) / G;
        const int U = nc * G, R = U / B, Ur = U - R * B;
        int cost = R * (2 * ((qpu + 1) / 2) + 1), G2 = 1;
        if (Ur > 0) {
            G2 = max(1, min(qpu, B / Ur));
            const int q2 = (qpu + G2 - 1) / G2;
            cost += 2 * ((q2 + 1) / 2) + 1;
        }
        if (cost < best) {
            best = cost;
            pick = make_int4(G, R * B, Ur, G2);
        }
    }
    return pick;
}


// Counter (i, y, quad, start), rounds 3..10 (0-based 2..9) from the round-2
// output (H2 ^ L1k, L2, HA ^ L0k, LA).
__device__ __forceinline__ uint4 philox_tail(uint32_t cx, uint32_t cy, uint32_t cz, uint32_t cw,
                                             const PhiloxKeys<2> &K)
{
    return philox_rounds<2>(make_uint4(cx, cy, cz, cw), K);
}

template <int B, int MAXD>
__device__ void run_item_pm1q(const SweepLaunch &L, const SweepJob &job, int quad0, int nq, QuadSmem &sm,
                              uint32_t *sw)
{
    constexpr uint32_t M = 0x01010101u;
    const int tid = threadIdx.x;
    const DevProb *P = job.prob;
    const int n = P->n, ncol = P->ncol, cap_n = P->cap_n;
    const int bias = P->dmax >> 1;
    const int ns = n + 1;
    const uint32_t ns4 = 4u * (uint32_t)ns, q4 = 8u * (uint32_t)ns;  // bytes to the inverted copy / next quad
    const int T = job_end(L, job), t0 = job.t0;
    const uint32_t k0 = (uint32_t)job.seed, k1 = (uint32_t)(job.seed >> 32);
    const uint32_t phase_hi = job.phase << kSweepBits;
    const uint32_t k0w = k0 + kPhiloxW0, k1w = k1 + kPhiloxW1;
    // a 1 the compiler cannot fold, so the multiply-adds stay on the FMA pipe
    const uint32_t one = (uint32_t)(L.thr_stride > 0);

    for (int c = tid; c <= ncol; c += B) sm.cptr[c] = P->cptr[c];
    for (int c = tid; c < ncol; c += B) sm.split[c] = class_split(P->cptr[c + 1] - P->cptr[c], nq, B);
    for (int x = tid; x < nq * ns; x += B) {
        const int q = x / ns, p = x - q * ns;
        const uint32_t w = p < n ? start_word(P, job, quad0 + q, p) : 0u;
        sw[(size_t)q * 2 * ns + p] = w;
        sw[(size_t)q * 2 * ns + ns + p] = p < n ? (w ^ M) : 0u;
    }
    for (int q = tid; q < nq; q += B) {
        uint32_t H1, L1, HA, LA;
        philox_mulhilo(kPhiloxM1, (uint32_t)(quad0 + q), H1, L1);
        sm.qk[q] = make_uint2(L1 ^ k0w, H1 ^ k0);
        philox_mulhilo(kPhiloxM0, H1 ^ k0 ^ (phase_hi | (uint32_t)t0), HA, LA);
        sm.qs[t0 & 1][q] = make_uint2(HA, LA);
    }
    // threshold rows: entry i = 2^32 - thr[t][2 (i - bias)] for i > bias, 0 (always accept) otherwise
    for (int i = tid; i < 2 * kRowQ; i += B) {
        const int par = i / kRowQ, e = i % kRowQ - bias;
        unsigned long long v = 0;
        if (e > 0 && e <= bias && par == (t0 & 1) && t0 < T)
            v = (1ull << 32) - (unsigned long long)L.thr[(size_t)t0 * L.thr_stride + 2 * e];
        sm.row[par][i % kRowQ] = v;
    }
    __syncthreads();

    const PhiloxKeys<2> Kr = philox_keys<2>(k0, k1);
    const uint32_t k16 = (uint32_t)(16 * bias) * M;

    for (int t = t0; t < T; ++t) {
        const int par = t & 1;
        // next sweep's row and quad products (their buffers were last read in the previous sweep)
        if (t + 1 < T) {
            if (tid < bias) {
                const int e = tid + 1;
                sm.row[par ^ 1][bias + e] =
                    (1ull << 32) - (unsigned long long)L.thr[(size_t)(t + 1) * L.thr_stride + 2 * e];
            }
            for (int q = tid; q < nq; q += B) {
                uint32_t HA, LA;
                philox_mulhilo(kPhiloxM0, sm.qk[q].y ^ (phase_hi | (uint32_t)(t + 1)), HA, LA);
                sm.qs[par ^ 1][q] = make_uint2(HA, LA);
            }
        }
        const char *rowb = reinterpret_cast<const char *>(sm.row[par]);
        const uint2 *qsp = sm.qs[par];
        for (int c = 0; c < ncol; ++c) {
            const int lo = sm.cptr[c], nc = sm.cptr[c + 1] - lo;
            if (nc > 0) {
                // units (spin k, quad group g), k fastest; group g sweeps quads g, g + G, ...;
                // a remainder unit's sub-unit j sweeps every G2-th of them from the j-th
                const int4 sp = sm.split[c];
                const int G = sp.x, full = sp.y, Ur = sp.z, G2 = sp.w;
                for (int u = tid; u < full + Ur * G2; u += B) {
                    int uu = u, j = 0;
                    if (u >= full) {
                        const int v = u - full;
                        j = v / Ur;
                        uu = full + (v - j * Ur);
                    }
                    const int g = uu / nc, p = lo + (uu - g * nc);
                    const int qst = u < full ? G : G * G2;
                    const uint32_t meta = __ldg(P->meta + p);
                    const int deg = (int)(meta & 0xFFFFu);
                    uint32_t o4[MAXD];
#pragma unroll
                    for (int d = 0; d < MAXD; ++d) {
                        uint32_t o = (uint32_t)n;  // missing neighbour: the quad's zero word
                        if (d < deg) {
                            const uint32_t e = __ldg(P->ell + (size_t)d * cap_n + p);
                            o = ((e >> 31) ? (uint32_t)ns : 0u) + (e & 0xFFFFu);
                        }
                        o4[d] = 4u * o;
                    }
                    const uint32_t c0 = (uint32_t)(8 * (bias - deg + ((int)meta >> 16))) * M;
                    // Philox products of the spin and the start: rounds 1 (word 0) and 2 (word 2)
                    uint32_t H0, L0, H2, L2;
                    philox_mulhilo(kPhiloxM0, (uint32_t)__ldg(P->idx_of_pos + p), H0, L0);
                    philox_mulhilo(kPhiloxM1, H0 ^ job.start ^ k1, H2, L2);
                    const uint32_t L0k = L0 ^ k1w;
                    const uint32_t own4 = 4u * (uint32_t)p;
                    // quads g, g + G, ... two at a time (no item reads a word another writes)
                    for (int q = g + j * G; q < nq; q += 2 * qst) {
                        const bool two = q + qst < nq;
                        const int qq[2] = {q, two ? q + qst : q};
                        uint32_t own[2], x[2], oa[2];
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            const uint32_t base = (uint32_t)qq[k] * q4;
                            oa[k] = base + own4;
                            own[k] = lds_p(sw, oa[k]);
                            uint32_t s = 0;
#pragma unroll
                            for (int d = 0; d < MAXD; ++d) s += lds_p(sw, base + o4[d]);
                            x[k] = s;
                        }
                        uint32_t nw[2];
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            const uint2 qk = sm.qk[qq[k]], qs = qsp[qq[k]];
                            const uint4 r4 = philox_tail(H2 ^ qk.x, L2, qs.x ^ L0k, qs.y, Kr);
                            // 8 (dE/2 + bias) per byte: 16 x + 8 (bias - deg + h) for b_i = 0, its
                            // mirror 16 bias - that for b_i = 1
                            const uint32_t a = madlo_p(x[k], 16u * one, c0);
                            const uint32_t b = madlo_p(a, 0u - one, k16);
                            const uint32_t m = own[k] * 0xFFu;
                            const uint32_t idx8 = (a & ~m) | (b & m);
                            const uint32_t ur[4] = {r4.x, r4.y, r4.z, r4.w};
                            uint32_t rej = 0;
#pragma unroll
                            for (int r = 0; r < 4; ++r) {
                                const uint32_t off = __byte_perm(idx8, 0u, 0x4440u | (uint32_t)r);
                                const unsigned long long ent =
                                    *reinterpret_cast<const unsigned long long *>(rowb + off);
                                const uint32_t carry = (uint32_t)(((unsigned long long)ur[r] + ent) >> 32);
                                rej = r == 0 ? carry : madlo_p(carry, one << (8 * r), rej);
                            }
                            nw[k] = own[k] ^ rej ^ M;  // flip where not rejected
                        }
                        sts_p(sw, oa[0], nw[0]);
                        sts_p(sw, oa[0] + ns4, nw[0] ^ M);
                        if (two) {
                            sts_p(sw, oa[1], nw[1]);
                            sts_p(sw, oa[1] + ns4, nw[1] ^ M);
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    finish_item<true>(P, job, quad0, nq, sw, sm.e2, 2 * ns);
}

template <int B, int MAXD>
__global__ void __launch_bounds__(B, B == 512 ? (MAXD == 6 ? 2 : 1) : 1024 / B) k_sweep_pm1q(const SweepLaunch L)
{
    __shared__ QuadSmem sm;
    extern __shared__ __align__(16) uint32_t sw_pm1q[];
    __shared__ int s_item;
    for (int iter = 0;; ++iter) {
        SweepJob job;
        int quad0, nq;
        if (!next_item(L, iter, &s_item, job, quad0, nq)) break;
        run_item_pm1q<B, MAXD>(L, job, quad0, nq, sm, sw_pm1q);
        __syncthreads();
    }
}

void *select_q(int block, int maxd)
{
#define SPVAR_PM1Q_CASE(BB, MD) \
    if (block == BB && maxd == MD) return reinterpret_cast<void *>(k_sweep_pm1q<BB, MD>);
    SPVAR_PM1Q_CASE(128, 6) SPVAR_PM1Q_CASE(256, 6) SPVAR_PM1Q_CASE(512, 6)
    SPVAR_PM1Q_CASE(128, 8) SPVAR_PM1Q_CASE(256, 8) SPVAR_PM1Q_CASE(512, 8)
#undef SPVAR_PM1Q_CASE
    return nullptr;
}

}  // namespace

// Q quads of a problem of at most max_n spins per work item.
bool pm1q_shape_ok(int block, int maxd, int max_n, int Q)
{
    return select_q(block, maxd) != nullptr && Q >= 1 && Q <= kQcap && max_n < 0xFFFF;
}

size_t pm1q_smem_bytes(int max_n, int Q) { return 4 * 2 * (size_t)Q * ((size_t)max_n + 1); }

cudaError_t launch_sweep_pm1q(const SweepLaunch &L, int block, int maxd, int grid, size_t smem, cudaStream_t st)
{
    void *k = select_q(block, maxd);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<SweepLaunch *>(&L)};
    return cudaLaunchKernel(k, dim3(grid), dim3(block), args, smem, st);
}

int pm1q_max_active_blocks(int block, int maxd, size_t smem)
{
    void *k = select_q(block, maxd);
    if (!k) return 0;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem);
    return nb;
}

}  // namespace spvar
