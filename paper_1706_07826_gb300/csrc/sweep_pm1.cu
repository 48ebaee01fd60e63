// Register-resident simulated-annealing sweep for +-1 couplers (the sampler
// of Sec. III.A on the paper's +-J spin glasses and Chimera problems).
//
// Same dynamics, random words and result as the general sweep kernel, with
// the per-attempt instruction count cut down and moved off the integer ALU
// pipe (which issues at half the rate of the FMA pipe):
//  - every thread owns NSLOT fixed (spin, quad) items for the whole anneal;
//    slot j of every thread belongs to one colour class (a class fills
//    ceil(size * quads / B) whole slots), so the colour order is the slot
//    order and the only barriers are the ones between classes;
//  - each item keeps its neighbour word offsets, its flip-cost constant and
//    the parts of Philox rounds 1-3 that do not depend on the sweep index in
//    registers;
//  - shared memory holds each spin word twice, as is and with every replica
//    bit inverted, at a compile-time distance, so a J < 0 neighbour is read
//    from the inverted copy and the local field of four replicas is one
//    byte-wise sum of neighbour words;
//  - the flip-cost index of the four replicas is formed byte-wise (SWAR),
//    pre-scaled to the byte offset of a 64-bit threshold entry;
//  - acceptance is one 64-bit add per replica: the row holds 2^32 - thr (0
//    where dE <= 0), so u + entry carries into bit 32 exactly when the move
//    is rejected (u >= thr), and the four carries are the replicas' reject
//    bits (no compare, select or "always accept" mask).
// Eligible when every |J| = 1, degree <= MAXD and dmax <= 30 (so that the
// scaled index 8 (dE/2 + bias) fits a byte).
//
// SCALED variant, for couplers whose magnitude is one value J0_i per spin
// (weak-strong cluster problems: every |J| = 100): the byte-wise neighbour sum
// is the same, the local field is h + J0 (2x - deg), and the flip-cost index
// 16 (dE/2 + bias) of two replicas at a time is formed in 16-bit lanes; the
// two acceptance rows (2 bias + 1 entries each, rounded up to 16) are in
// dynamic shared memory with entry i at slot i ^ ((i >> 4) & 15): the indices
// a warp reads differ by multiples of the coupler magnitude (100 for the
// weak-strong problems), which in a plain layout put most of them on one or
// two banks.  Needs dmax <= 4094.  With SI (small integer couplers, every
// |J| <= 15: the reduced-degeneracy problems of Sec. III.C) the byte-wise sum
// is weighted, X = sum_j |J_ij| b'_j <= 120 per byte with the magnitudes packed
// four bits per neighbour in one register, and the local field is
// h + 2 X - sum_j |J_ij|.
#include "sweep_common.cuh"

namespace spvar {

namespace {

constexpr int kRowE = 32;  // 64-bit entries per threshold row: index dE/2 + bias <= 2 * 15

template <int MAXD>
struct SlotRegs {
    uint32_t own;       // byte offset of the item's spin word (plain copy)
    uint32_t nb[MAXD];  // byte offsets of the neighbours (inverted copy if J < 0, zero word if padding)
    uint32_t c0;        // per byte: 8 (bias - deg + h); SCALED: per 16-bit lane 16 (bias + h - J0 deg)
    uint32_t tj;        // SCALED: 32 J0 (SI: 32)
    uint32_t jp;        // SI: |J| of neighbour d in bits 4d .. 4d + 3
    uint32_t A, L0k, D, H3k, L3;  // Philox rounds 1-3 folded with the item's fixed counter words
};

__device__ __forceinline__ uint32_t lds_b(const uint32_t *base, uint32_t byte_off)
{
    return *reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(base) + byte_off);
}
__device__ __forceinline__ void sts_b(uint32_t *base, uint32_t byte_off, uint32_t v)
{
    *reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(base) + byte_off) = v;
}

// a * b + c on 32 bits.
__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// Counter (i, y, q, s): the sweep word y is the only input that changes
// between sweeps, so the products of round 1 and parts of rounds 2 and 3 are
// item constants.
template <int MAXD>
__device__ __forceinline__ void philox_setup(SlotRegs<MAXD> &s, uint32_t i, uint32_t q, uint32_t start,
                                             uint32_t k0, uint32_t k1)
{
    uint32_t H0, L0, H1, L1, H2, L2, H3, L3;
    philox_mulhilo(kPhiloxM0, i, H0, L0);
    philox_mulhilo(kPhiloxM1, q, H1, L1);
    const uint32_t Z = H0 ^ start ^ k1;            // round-1 counter word 2
    philox_mulhilo(kPhiloxM1, Z, H2, L2);                        // round-2 product of word 2
    const uint32_t C1 = H2 ^ L1 ^ (k0 + kPhiloxW0);       // round-2 counter word 0
    philox_mulhilo(kPhiloxM0, C1, H3, L3);                       // round-3 product of word 0
    s.A = H1 ^ k0;
    s.L0k = L0 ^ (k1 + kPhiloxW1);
    s.D = L2 ^ (k0 + 2 * kPhiloxW0);
    s.H3k = H3 ^ (k1 + 2 * kPhiloxW1);
    s.L3 = L3;
}

// Round keys 3..9 of the item's seed.
using RoundKeys = PhiloxKeys<3>;

// (h, l): the round-2 product of word 0, M0 (A ^ y).
template <int MAXD>
__device__ __forceinline__ uint4 philox_slot_hl(const SlotRegs<MAXD> &s, uint32_t h, uint32_t l, const RoundKeys &K)
{
    uint32_t h2, l2;
    philox_mulhilo(kPhiloxM1, h ^ s.L0k, h2, l2);      // round 3: word 2 product
    return philox_rounds<3>(make_uint4(h2 ^ s.D, l2, s.H3k ^ l, s.L3), K);
}

template <int MAXD>
__device__ __forceinline__ uint4 philox_slot(const SlotRegs<MAXD> &s, uint32_t y, const RoundKeys &K)
{
    uint32_t h, l;
    philox_mulhilo(kPhiloxM0, s.A ^ y, h, l);          // round 2: word 0 product
    return philox_slot_hl(s, h, l, K);
}

// Shared memory of one CTA: spin words (plain copy, a dummy word, inverted
// copy at a fixed distance, its dummy, a zero word) and two threshold rows.
template <int B, int NSLOT>
struct Pm1Smem {
    static constexpr int KW = B * NSLOT + 1;  // words per copy; word KW - 1 is the dummy
    uint32_t sw[2 * KW + 1];
    unsigned long long row[2][kRowE];
    int cptr[kMaxColours + 1];
    int late;  // the item's problem is small: its sweeps are short
};

// SCALED acceptance rows: row length (2 bias + 1 rounded up to 16 entries) and
// the slot of entry i, a bijection on every aligned block of 16 slots that
// spreads indices with the same low bits over the 16 bank pairs.
__device__ __forceinline__ int row_len(int bias) { return (2 * bias + 16) & ~15; }
__device__ __forceinline__ int row_slot(int i) { return i ^ ((i >> 4) & 15); }

// One sweep over the slots, reading threshold row PAR.  Every lane runs every
// slot (lanes without an item anneal the dummy word: no branch per slot); a
// barrier precedes slot j when it starts a new colour class (bit j of
// barmask) and closes the sweep.
// ONEQ: every item of the CTA is of one quad (word A of every slot is A0), so
// the round-2 product of word 0 is computed once per sweep, not per slot.
template <int B, int NSLOT, int MAXD, bool SCALED, bool SI, int PAR, bool ONEQ>
__device__ __forceinline__ void sweep_once(Pm1Smem<B, NSLOT> &sm, unsigned long long *drow,
                                           const SlotRegs<MAXD> (&s)[NSLOT], uint32_t y,
                                           const RoundKeys &K, uint32_t barmask, uint32_t one,
                                           uint32_t k16, const uint32_t *next_src, int bias, uint32_t A0)
{
    uint32_t hA = 0u, lA = 0u;
    if (ONEQ) philox_mulhilo(kPhiloxM0, A0 ^ y, hA, lA);
    constexpr uint32_t kInv = 4u * (uint32_t)Pm1Smem<B, NSLOT>::KW;  // byte distance to the inverted copy
    // next sweep's row (its buffer was last read in the previous sweep)
    if (SCALED) {
        if (next_src) {
            unsigned long long *nrow = drow + (PAR ^ 1) * row_len(bias);
            for (int e = (int)threadIdx.x + 1; e <= bias; e += B)
                nrow[row_slot(bias + e)] = (1ull << 32) - (unsigned long long)next_src[2 * e];
        }
    }
    // byte lanes: the next row's entry is loaded now; with at most two slots and a
    // small problem it is stored after the slots, so that a short sweep does not
    // wait for the load, otherwise at once (which keeps a register free for the
    // slots of a long sweep)
    const bool stage = !SCALED && next_src && (int)threadIdx.x < bias;
    const bool late = NSLOT <= 2 && sm.late;
    const uint32_t nthr = stage ? __ldg(next_src + 2 * ((int)threadIdx.x + 1)) : 0u;
    if (!late && stage) sm.row[PAR ^ 1][bias + (int)threadIdx.x + 1] = (1ull << 32) - (unsigned long long)nthr;
    const char *rowb = SCALED ? reinterpret_cast<const char *>(drow + PAR * row_len(bias))
                              : reinterpret_cast<const char *>(sm.row[PAR]);
#pragma unroll
    for (int j = 0; j < NSLOT; ++j) {
        if (barmask & (1u << j)) __syncthreads();
        {
            const uint32_t own = lds_b(sm.sw, s[j].own);
            uint32_t nbw[MAXD];
#pragma unroll
            for (int d = 0; d < MAXD; ++d) nbw[d] = lds_b(sm.sw, s[j].nb[d]);
            const uint4 u = ONEQ ? philox_slot_hl(s[j], hA, lA, K) : philox_slot(s[j], y, K);
            uint32_t x = 0;
#pragma unroll
            for (int d = 0; d < MAXD; ++d) x = SI ? mad_lo(nbw[d], (s[j].jp >> (4 * d)) & 15u, x) : x + nbw[d];
            // byte r of x: neighbours with b_j ^ [J_ij < 0] = 1
            uint32_t off[4];
            if (SCALED) {
                // replicas (0, 2) and (1, 3) in 16-bit lanes: 16 (dE/2 + bias) is
                // 16 (bias + h - J0 deg) + 32 J0 x for b_i = 0 and 32 bias minus that for b_i = 1
                const uint32_t xl = __byte_perm(x, 0u, 0x4240u), xh = __byte_perm(x, 0u, 0x4341u);
                const uint32_t ml = __byte_perm(own, 0u, 0x4240u) * 0xFFFFu;
                const uint32_t mh = __byte_perm(own, 0u, 0x4341u) * 0xFFFFu;
                const uint32_t al = mad_lo(xl, s[j].tj, s[j].c0), ah = mad_lo(xh, s[j].tj, s[j].c0);
                const uint32_t bl = mad_lo(al, 0u - one, k16), bh = mad_lo(ah, 0u - one, k16);
                const uint32_t kl = (al & ~ml) | (bl & ml), kh = (ah & ~mh) | (bh & mh);
                // byte offsets 8 row_slot(i) of both lanes: 16 i halved, bits 4..7 of i
                // xor-ed into bits 0..3 (16 i < 2^16, so no bit crosses a lane)
                const uint32_t ol = (kl >> 1) ^ ((kl >> 5) & 0x00780078u);
                const uint32_t oh = (kh >> 1) ^ ((kh >> 5) & 0x00780078u);
                off[0] = ol & 0xFFFFu;
                off[1] = oh & 0xFFFFu;
                off[2] = ol >> 16;
                off[3] = oh >> 16;
            } else {
                // the flip-cost index dE/2 + bias is 2x + bias - deg + h if b_i = 0 and its
                // mirror 2 bias - that if b_i = 1; all scaled by 8 (the byte offset of a
                // 64-bit row entry)
                const uint32_t a = mad_lo(x, 16u * one, s[j].c0);
                const uint32_t b = mad_lo(a, 0u - one, k16);
                const uint32_t m = own * 0xFFu;
                const uint32_t idx8 = (a & ~m) | (b & m);
#pragma unroll
                for (int r = 0; r < 4; ++r) off[r] = __byte_perm(idx8, 0u, 0x4440u | (uint32_t)r);
            }
            const uint32_t ur[4] = {u.x, u.y, u.z, u.w};
            uint32_t rej = 0;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const unsigned long long ent = *reinterpret_cast<const unsigned long long *>(rowb + off[r]);
                // carry of u + entry: a 64-bit add, on the integer pipe (the multiply
                // pipe is busy with Philox)
                const uint32_t carry = (uint32_t)(((unsigned long long)ur[r] + ent) >> 32);
                rej = r == 0 ? carry : mad_lo(carry, one << (8 * r), rej);
            }
            // flip where not rejected
            const uint32_t inv = own ^ rej;  // = new word with every replica bit inverted
            sts_b(sm.sw, s[j].own, inv ^ 0x01010101u);
            sts_b(sm.sw, s[j].own + kInv, inv);
        }
    }
    if (late && stage) sm.row[PAR ^ 1][bias + (int)threadIdx.x + 1] = (1ull << 32) - (unsigned long long)nthr;
    __syncthreads();
}

// Sweeps t0 .. T - 1, two per step (the rows alternate).
template <int B, int NSLOT, int MAXD, bool SCALED, bool SI, bool ONEQ>
__device__ __forceinline__ void sweeps(Pm1Smem<B, NSLOT> &sm, unsigned long long *drow, const SlotRegs<MAXD> (&s)[NSLOT],
                                       int t0, int T, uint32_t phase_hi, const RoundKeys &K, uint32_t barmask,
                                       uint32_t one, uint32_t k16, const uint32_t *thr, size_t ts, int bias, uint32_t A0)
{
    int t = t0;
    if (t < T && (t & 1)) {
        sweep_once<B, NSLOT, MAXD, SCALED, SI, 1, ONEQ>(sm, drow, s, phase_hi | (uint32_t)t, K, barmask, one, k16,
                                                    t + 1 < T ? thr + (size_t)(t + 1) * ts : nullptr, bias, A0);
        ++t;
    }
    for (; t + 1 < T; t += 2) {
        sweep_once<B, NSLOT, MAXD, SCALED, SI, 0, ONEQ>(sm, drow, s, phase_hi | (uint32_t)t, K, barmask, one, k16,
                                                    thr + (size_t)(t + 1) * ts, bias, A0);
        sweep_once<B, NSLOT, MAXD, SCALED, SI, 1, ONEQ>(sm, drow, s, phase_hi | (uint32_t)(t + 1), K, barmask, one,
                                                    k16, t + 2 < T ? thr + (size_t)(t + 2) * ts : nullptr, bias, A0);
    }
    if (t < T)
        sweep_once<B, NSLOT, MAXD, SCALED, SI, 0, ONEQ>(sm, drow, s, phase_hi | (uint32_t)t, K, barmask, one, k16,
                                                    nullptr, bias, A0);
}

template <int B, int NSLOT, int MAXD, bool SCALED, bool SI>
__device__ void run_item_pm1(const SweepLaunch &L, const SweepJob &job, int quad0, int nq, Pm1Smem<B, NSLOT> &sm,
                             unsigned long long *drow)
{
    constexpr int KW = Pm1Smem<B, NSLOT>::KW;
    const int tid = threadIdx.x;
    const DevProb *P = job.prob;
    const int n = P->n;
    const int ncol = P->ncol;
    const int cap_n = P->cap_n;
    const int bias = P->dmax >> 1;
    const uint32_t k0 = (uint32_t)job.seed, k1 = (uint32_t)(job.seed >> 32);
    const uint32_t phase_hi = job.phase << kSweepBits;
    const int T = job_end(L, job);
    const int t0 = job.t0;
    // a 1 the compiler cannot fold, so the multiply-adds stay on the FMA pipe
    const uint32_t one = (uint32_t)(L.thr_stride > 0);

    for (int c = tid; c <= ncol; c += B) sm.cptr[c] = P->cptr[c];
    if (tid == 0) sm.late = P->n <= 256;
    init_spins(P, job, quad0, nq, sm.sw, sm.sw + KW);
    if (tid == 0) {
        sm.sw[KW - 1] = 0u;
        sm.sw[2 * KW - 1] = 0u;
        sm.sw[2 * KW] = 0u;
    }
    // threshold rows: entry i = 2^32 - thr[t][2 (i - bias)] for i > bias, 0 (always accept) otherwise
    if (SCALED) {
        // row par holds entry i at par * row_len + row_slot(i)
        const int rl = row_len(bias);
        for (int x = tid; x < 2 * rl; x += B) {
            const int par = x >= rl, i = x - par * rl, e = i - bias;
            unsigned long long v = 0;
            if (e > 0 && i <= 2 * bias && par == (t0 & 1) && t0 < T)
                v = (1ull << 32) - (unsigned long long)L.thr[(size_t)t0 * L.thr_stride + 2 * e];
            drow[par * rl + row_slot(i)] = v;
        }
    } else {
        for (int i = tid; i < 2 * kRowE; i += B) {
            const int par = i / kRowE, e = i % kRowE - bias;
            unsigned long long v = 0;
            if (e > 0 && e <= bias && par == (t0 & 1) && t0 < T)
                v = (1ull << 32) - (unsigned long long)L.thr[(size_t)t0 * L.thr_stride + 2 * e];
            sm.row[par][i % kRowE] = v;
        }
    }
    __syncthreads();

    // colour-aligned slots
    SlotRegs<MAXD> s[NSLOT];
    uint32_t barmask = 0;
    const RoundKeys K = philox_keys<3>(k0, k1);
    const uint32_t dummy = 4u * (uint32_t)(KW - 1), zero = 4u * (uint32_t)(2 * KW);
#pragma unroll
    for (int j = 0; j < NSLOT; ++j) {
        s[j].own = dummy;
#pragma unroll
        for (int d = 0; d < MAXD; ++d) s[j].nb[d] = zero;
        s[j].c0 = SCALED ? (uint32_t)(16 * bias) * 0x00010001u : (uint32_t)(8 * bias) * 0x01010101u;
        s[j].tj = 0u;
        s[j].jp = 0u;
        s[j].A = s[j].L0k = s[j].D = s[j].H3k = s[j].L3 = 0u;
        // colour class of slot j
        int c = 0, jb = 0, items = 0;
        for (; c < ncol; ++c) {
            items = (sm.cptr[c + 1] - sm.cptr[c]) * nq;
            const int ns = (items + B - 1) / B;
            if (j < jb + ns) break;
            jb += ns;
        }
        if (c < ncol) {
            if (j == jb && j > 0) barmask |= 1u << j;
            const int local = (j - jb) * B + tid;
            if (local < items) {
                const int nc = sm.cptr[c + 1] - sm.cptr[c];
                const int q = local / nc;
                const int p = sm.cptr[c] + (local - q * nc);
                const uint32_t meta = P->meta[p];
                const int deg = (int)(meta & 0xFFFFu);
                const int h = (int)meta >> 16;
                s[j].own = 4u * (uint32_t)(q * n + p);
#pragma unroll
                for (int d = 0; d < MAXD; ++d) {
                    if (d < deg) {
                        const uint32_t e = P->ell[(size_t)d * cap_n + p];
                        s[j].nb[d] = 4u * (uint32_t)(((e >> 31) ? KW : 0) + q * n + (int)(e & 0xFFFFu));
                    }
                }
                if (SI) {
                    // small integer couplers: magnitudes packed four bits per neighbour
                    int sumj = 0;
                    for (int d = 0; d < deg && d < MAXD; ++d) {
                        const uint32_t a = (uint32_t)abs((int)P->ell[(size_t)d * cap_n + p] >> 16);
                        s[j].jp |= a << (4 * d);
                        sumj += (int)a;
                    }
                    s[j].c0 = (uint32_t)(16 * (bias + h - sumj)) * 0x00010001u;
                    s[j].tj = 32u;
                } else if (SCALED) {
                    // one coupler magnitude J0 per spin
                    const int J0 = deg > 0 ? abs((int)P->ell[p] >> 16) : 0;
                    s[j].c0 = (uint32_t)(16 * (bias + h - J0 * deg)) * 0x00010001u;
                    s[j].tj = (uint32_t)(32 * J0);
                } else {
                    s[j].c0 = (uint32_t)(8 * (bias - deg + h)) * 0x01010101u;
                }
                philox_setup(s[j], (uint32_t)P->idx_of_pos[p], (uint32_t)(quad0 + q), job.start, k0, k1);
            }
        }
    }
    const uint32_t k16 = SCALED ? (uint32_t)(32 * bias) * 0x00010001u : (uint32_t)(16 * bias) * 0x01010101u;
    const uint32_t *thr = L.thr;
    const size_t ts = (size_t)L.thr_stride;

    if (nq == 1) {
        uint32_t H1, L1;
        philox_mulhilo(kPhiloxM1, (uint32_t)quad0, H1, L1);
        sweeps<B, NSLOT, MAXD, SCALED, SI, true>(sm, drow, s, t0, T, phase_hi, K, barmask, one, k16, thr, ts, bias,
                                             H1 ^ k0);
    } else {
        sweeps<B, NSLOT, MAXD, SCALED, SI, false>(sm, drow, s, t0, T, phase_hi, K, barmask, one, k16, thr, ts, bias,
                                              0u);
    }
    // the inverted copy is dead now: its first 4 nq words hold the energy sums
    finish_item<!SCALED>(P, job, quad0, nq, sm.sw, reinterpret_cast<int *>(sm.sw + KW));  // general J for SCALED
}

// Resident CTAs per SM asked of the register allocator (0: no request).  The
// 128 x 4 byte-lane kernel for degree <= 6 uses 86 registers unasked, which
// leaves room for five 128-thread CTAs per SM; capped at 71 (seven CTAs, no
// spills) it runs 6 % faster on the Chimera C8 workload.  The 576-thread
// 16-bit-lane forms fit two CTAs per SM at 56 registers without spills (the
// degree-6 one-magnitude form takes 56 unasked; the others took 70 to 84).
// For the other shapes a cap either spilled or was not faster, and an
// explicit minimum of 1 makes the allocator take more registers than it does
// unasked.
template <int B, int NSLOT, int MAXD, bool SCALED>
constexpr int pm1_min_blocks()
{
    return (B == 128 && NSLOT == 4 && MAXD == 6 && !SCALED) ? 7 : (B == 576 && SCALED) ? 2 : 0;
}

template <int B, int NSLOT, int MAXD, bool SCALED, bool SI>
__global__ void __launch_bounds__(B, (pm1_min_blocks<B, NSLOT, MAXD, SCALED>())) k_sweep_pm1(const SweepLaunch L)
{
    __shared__ Pm1Smem<B, NSLOT> sm;
    extern __shared__ __align__(16) unsigned long long drow_pm1[];  // SCALED: the two acceptance rows
    __shared__ int s_item;
    for (int iter = 0;; ++iter) {
        SweepJob job;
        int quad0, nq;
        if (!next_item(L, iter, &s_item, job, quad0, nq)) break;
        run_item_pm1<B, NSLOT, MAXD, SCALED, SI>(L, job, quad0, nq, sm, drow_pm1);
        __syncthreads();
    }
}

template <int B, int NSLOT, int MAXD, bool SCALED, bool SI>
void *kernel_ptr()
{
    return reinterpret_cast<void *>(k_sweep_pm1<B, NSLOT, MAXD, SCALED, SI>);
}

void *select_kernel(int block, int nslot, int maxd, int mode)
{
#define SPVAR_PM1_CASE(BB, NS, MD) \
    if (mode == 0 && block == BB && nslot == NS && maxd == MD) return kernel_ptr<BB, NS, MD, false, false>();
#define SPVAR_UJ_CASE(BB, NS, MD) \
    if (mode == 1 && block == BB && nslot == NS && maxd == MD) return kernel_ptr<BB, NS, MD, true, false>();
#define SPVAR_SI_CASE(BB, NS, MD) \
    if (mode == 2 && block == BB && nslot == NS && maxd == MD) return kernel_ptr<BB, NS, MD, true, true>();
    SPVAR_PM1_CASE(128, 2, 6) SPVAR_PM1_CASE(128, 3, 6) SPVAR_PM1_CASE(128, 4, 6)
    SPVAR_PM1_CASE(256, 2, 6) SPVAR_PM1_CASE(256, 3, 6) SPVAR_PM1_CASE(256, 4, 6)
    SPVAR_PM1_CASE(512, 2, 6) SPVAR_PM1_CASE(1024, 2, 6)
    SPVAR_PM1_CASE(128, 2, 8) SPVAR_PM1_CASE(128, 3, 8) SPVAR_PM1_CASE(128, 4, 8)
    SPVAR_PM1_CASE(256, 2, 8) SPVAR_PM1_CASE(256, 3, 8) SPVAR_PM1_CASE(256, 4, 8)
    SPVAR_PM1_CASE(512, 2, 8) SPVAR_PM1_CASE(1024, 2, 8)
    // 576 threads: two colour classes of up to 576 spins (Chimera C12) fill one slot each
    SPVAR_UJ_CASE(256, 2, 6) SPVAR_UJ_CASE(256, 4, 6) SPVAR_UJ_CASE(512, 2, 6) SPVAR_UJ_CASE(576, 2, 6)
    SPVAR_UJ_CASE(1024, 2, 6)
    SPVAR_UJ_CASE(256, 2, 8) SPVAR_UJ_CASE(256, 4, 8) SPVAR_UJ_CASE(512, 2, 8) SPVAR_UJ_CASE(576, 2, 8)
    SPVAR_UJ_CASE(1024, 2, 8)
    SPVAR_SI_CASE(128, 4, 6) SPVAR_SI_CASE(256, 2, 6) SPVAR_SI_CASE(256, 4, 6) SPVAR_SI_CASE(512, 2, 6)
    SPVAR_SI_CASE(576, 2, 6) SPVAR_SI_CASE(1024, 2, 6)
    SPVAR_SI_CASE(128, 4, 8) SPVAR_SI_CASE(256, 2, 8) SPVAR_SI_CASE(256, 4, 8) SPVAR_SI_CASE(512, 2, 8)
    SPVAR_SI_CASE(576, 2, 8) SPVAR_SI_CASE(1024, 2, 8)
#undef SPVAR_PM1_CASE
#undef SPVAR_UJ_CASE
#undef SPVAR_SI_CASE
    return nullptr;
}

}  // namespace

bool pm1_shape_ok(int block, int nslot, int maxd, int mode) { return select_kernel(block, nslot, maxd, mode) != nullptr; }

// SCALED: two rows of 64-bit entries, each at most thr_stride (= dmax + 1 >= 2 bias + 1)
// rounded up to 16.
size_t pm1_smem_bytes(bool scaled, int thr_stride)
{
    return scaled ? 2 * 8 * (size_t)((thr_stride + 15) & ~15) : 0;
}

cudaError_t launch_sweep_pm1(const SweepLaunch &L, int block, int nslot, int maxd, int mode, int grid,
                             size_t smem, cudaStream_t st)
{
    const bool scaled = mode != 0;
    void *k = select_kernel(block, nslot, maxd, mode);
    if (!k) return cudaErrorInvalidValue;
    if (scaled) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    void *args[] = {const_cast<SweepLaunch *>(&L)};
    return cudaLaunchKernel(k, dim3(grid), dim3(block), args, scaled ? smem : 0, st);
}

int pm1_max_active_blocks(int block, int nslot, int maxd, int mode, size_t smem)
{
    const bool scaled = mode != 0;
    void *k = select_kernel(block, nslot, maxd, mode);
    if (!k) return 0;
    if (scaled) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, scaled ? smem : 0);
    return nb;
}

}  // namespace spvar
