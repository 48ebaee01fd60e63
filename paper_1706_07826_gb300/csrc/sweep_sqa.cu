// Simulated quantum annealing sweep: the second sampler for Alg. 1 ("obtain
// sample"), discrete-time path-integral Monte Carlo of the transverse-field
// Ising model (the SQA sampler of Sec. III).
//
// A run keeps P Trotter slices s^tau (tau = 0..P-1, periodic) of the
// problem.  Flipping s_i^tau changes the path-integral action by
//   dA = (2 beta / P) (k - bias) / scale + 4 Jp (a - 1),
// with k = dE/2 + bias (dE the classical flip cost inside slice tau) and a
// the number of its two slice neighbours s_i^(tau+-1) equal to s_i^tau
// (a = 1 for a single slice).  The host tabulates, per sweep, the 64-bit
// entry 2^32 - min(2^32, floor(2^32 exp(-dA))) for every (a, k); a move is
// accepted iff u + entry < 2^32 for the replica's uniform word u.
//
// One CTA anneals one quad (four independent runs, one byte lane each).  All
// P slices live in shared memory (and, for +-1 couplers, a copy with every
// replica bit inverted, so that J < 0 neighbours are read pre-negated and the
// local field of four replicas is one byte-wise sum).  A sweep visits the
// colour classes in order and, inside a class, the even slices and then the
// odd ones: no two spins updated together are coupled in space or in
// imaginary time, so the parallel sweep equals visiting them one at a time.
// The random word of spin i in slice tau uses the counter of the SA sweep
// with spin word i | tau << 16.  A run's sample is its lowest-energy slice.
#include "sweep_common.cuh"

namespace spvar {

namespace {

// Shared memory of one CTA, in 32-bit words: the two 64-bit acceptance rows
// (current and next sweep), spin words [P][n + 1] (word n of every slice is
// zero: the target of missing neighbours), for +-1 couplers their inverted
// copy [P][n + 1], per-spin meta and index, 16-bit neighbour offsets, per-slice
// energy sums and the chosen slices.
__host__ __device__ inline size_t sqa_words(int max_n, int P, int maxdeg, int W, bool pm1)
{
    const size_t slice = (size_t)max_n + 1;
    size_t w = 2 * 2 * 3 * (size_t)W;  // two rows of 3W 64-bit entries
    w += (size_t)P * slice * (pm1 ? 2 : 1);
    w += 2 * (size_t)max_n;
    if (pm1) w += ((size_t)(maxdeg <= 6 ? 6 : 8) * max_n + 1) / 2;  // the kernel's unrolled degree
    return w + 4 * (size_t)P + 4;
}


// Philox4x32-10 of counter (w0, y, quad, start) with the products that do not
// depend on w0 hoisted: (H1, L1) = M1 * quad (round 1, per CTA) and
// (HA, LA) = M0 * (H1 ^ y ^ k0) (round 2, per sweep).  Kr: keys of rounds 3..10 (0-based 2..9).
__device__ __forceinline__ uint4 philox_sqa(uint32_t w0, uint32_t start, uint32_t k1, uint32_t L1, uint32_t HA,
                                            uint32_t LA, uint32_t k0w, uint32_t k1w, const PhiloxKeys<2> &Kr)
{
    uint32_t h0, l0, hb, lb;
    philox_mulhilo(kPhiloxM0, w0, h0, l0);                       // round 1, word 0
    philox_mulhilo(kPhiloxM1, h0 ^ start ^ k1, hb, lb);          // round 2, word 2
    return philox_rounds<2>(make_uint4(hb ^ L1 ^ k0w, lb, HA ^ l0 ^ k1w, LA), Kr);
}

// a * b + c on 32 bits, on the FMA pipe.
__device__ __forceinline__ uint32_t madq(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t lds_q(const uint32_t *base, uint32_t byte_off)
{
    return *reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(base) + byte_off);
}
__device__ __forceinline__ void sts_q(uint32_t *base, uint32_t byte_off, uint32_t v)
{
    *reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(base) + byte_off) = v;
}

// Register-resident form, +-1 couplers: the thread's spin of one colour class
// (its word offsets, flip-cost constant and spin word of the counter held in
// registers) in slices PAR + 2 (g + G m), m = 0, 1, ...  Byte offsets:
// `own4` of the spin and `o4` of its neighbours inside a slice (the inverted
// copy folded in for J < 0; the slice's zero word for a missing neighbour),
// `ns4` per slice, `inv4` to the inverted copy.
struct SqaRegConsts {
    uint32_t ns4, inv4, wrap4, k2, W, start, k1, L1, HA, LA, k0w, k1w;
};

// U independent items (slices tau[u] of one parity, so none reads a word
// another writes): every load first, then the flip costs, the random words
// and the acceptance of all of them, then the stores.  `chain`: the items are
// consecutive slices of the thread's sequence (tau, tau + 2, ...), so the
// down neighbour of one is the up neighbour of the one before (`prev_up`,
// valid when `have`).  E32: acceptance entries are 32-bit (no entry of the
// table is 2^32, i.e. every flip has a nonzero acceptance probability).
// SI: small integer couplers (|J| <= 15; jp holds |J| of neighbour d in bits
// 4d .. 4d + 3): the byte-wise neighbour sum is weighted, X = sum |J| b', and
// the entry index a W + k is formed per replica (it may exceed a byte).
template <int PAR, int MAXD, int U, bool E32, bool SI>
__device__ __forceinline__ void sqa_reg_items(uint32_t *sw, const void *entv, int P, const int (&tau)[U],
                                              const uint32_t (&base)[U], const uint32_t (&iw)[U], uint32_t own4,
                                              const uint32_t (&o4)[MAXD], uint32_t c0, uint32_t jp,
                                              const SqaRegConsts &K, const PhiloxKeys<2> &Kr, bool chain, bool have, uint32_t &prev_up)
{
    constexpr uint32_t M = 0x01010101u;
    uint32_t oa[U], own[U], up[U], dn[U], x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        oa[u] = base[u] + own4;
        own[u] = lds_q(sw, oa[u]);
        // slice neighbours; only the first even slice (down) and the last odd one (up) wrap
        uint32_t ua = oa[u] + K.ns4, da = oa[u] - K.ns4;
        if (PAR == 0) {
            if (tau[u] == 0) da = oa[u] + K.wrap4;
        } else {
            if (tau[u] == P - 1) ua = oa[u] - K.wrap4;
        }
        up[u] = lds_q(sw, ua);
        if (chain && (u > 0 || have)) dn[u] = u > 0 ? up[u - 1] : prev_up;
        else dn[u] = lds_q(sw, da);
        x[u] = 0;
#pragma unroll
        for (int d = 0; d < MAXD; ++d) {
            const uint32_t w = lds_q(sw, base[u] + o4[d]);
            x[u] = SI ? madq(w, (jp >> (4 * d)) & 15u, x[u]) : x[u] + w;
        }
    }
    prev_up = up[U - 1];
    uint32_t nw[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint32_t a4 = (~(own[u] ^ up[u]) & M) + (~(own[u] ^ dn[u]) & M);
        // k = dE/2 + bias per byte: 2x + bias - deg + h for b_i = 0, its mirror 2 bias - that for b_i = 1
        const uint32_t a = x[u] + x[u] + c0;
        const uint32_t b = K.k2 - a;
        const uint32_t m = own[u] * 0xFFu;
        const uint32_t kk = (a & ~m) | (b & m);
        const uint32_t full = SI ? 0u : a4 * K.W + kk;  // entry a W + k per byte, <= 3W - 1 <= 255
        const uint4 r4 = philox_sqa(iw[u], K.start, K.k1, K.L1, K.HA, K.LA, K.k0w, K.k1w, Kr);
        const uint32_t ur[4] = {r4.x, r4.y, r4.z, r4.w};
        uint32_t rej = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            // u + entry carries into bit 32 exactly when the move is rejected
            const uint32_t sel = 0x4440u | (uint32_t)r;
            const uint32_t e = SI ? madq(__byte_perm(a4, 0u, sel), K.W, __byte_perm(kk, 0u, sel))
                                  : __byte_perm(full, 0u, sel);
            const unsigned long long v = E32 ? (unsigned long long)static_cast<const uint32_t *>(entv)[e]
                                             : static_cast<const unsigned long long *>(entv)[e];
            rej |= (uint32_t)(((unsigned long long)ur[r] + v) >> 32) << (8 * r);
        }
        nw[u] = own[u] ^ rej ^ M;  // flip where not rejected
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        sts_q(sw, oa[u], nw[u]);
        sts_q(sw, oa[u] + K.inv4, nw[u] ^ M);
    }
}

// One parity pass of one colour-class slot: slices two at a time.
template <int PAR, int MAXD, bool E32, bool SI>
__device__ __forceinline__ void sqa_reg_pass(uint32_t *sw, const void *ent, int g, int G, int P, uint32_t own4,
                                             const uint32_t (&o4)[MAXD], uint32_t c0, uint32_t jp, uint32_t ib,
                                             const SqaRegConsts &K, const PhiloxKeys<2> &Kr)
{
    if (g < 0) return;
    const int dt = 2 * G;
    const bool chain = G == 1;
    const uint32_t step = (uint32_t)dt * K.ns4, istep = (uint32_t)dt << 16;
    int tau = PAR + 2 * g;
    uint32_t base = (uint32_t)tau * K.ns4;
    uint32_t iw = ib | ((uint32_t)tau << 16);
    uint32_t prev_up = 0u;
    bool have = false;
    for (; tau + dt < P; tau += 2 * dt, base += 2 * step, iw += 2 * istep) {
        const int t2[2] = {tau, tau + dt};
        const uint32_t b2[2] = {base, base + step}, i2[2] = {iw, iw + istep};
        sqa_reg_items<PAR, MAXD, 2, E32, SI>(sw, ent, P, t2, b2, i2, own4, o4, c0, jp, K, Kr, chain, have,
                                             prev_up);
        have = true;
    }
    if (tau < P) {
        const int t1[1] = {tau};
        const uint32_t b1[1] = {base}, i1[1] = {iw};
        sqa_reg_items<PAR, MAXD, 1, E32, SI>(sw, ent, P, t1, b1, i1, own4, o4, c0, jp, K, Kr, chain, have,
                                             prev_up);
    }
}

template <bool PM1, int B, int MAXD, int NC, bool E32, bool SI>
__device__ void run_item_sqa(const SweepLaunch &L, const SweepJob &job, int quad, uint32_t *smem)
{
    const int tid = threadIdx.x;
    const DevProb *pr = job.prob;
    const int n = pr->n, ncol = pr->ncol, cap_n = pr->cap_n, maxdeg = pr->maxdeg;
    const int P = L.P, W = L.W, bias = (L.W - 1) / 2;
    const int T = L.T;
    const uint32_t k0 = (uint32_t)job.seed, k1 = (uint32_t)(job.seed >> 32);
    const uint32_t phase_hi = job.phase << kSweepBits;
    const int ns = n + 1;                 // words per slice
    const size_t Pn = (size_t)P * ns;

    unsigned long long *rows = reinterpret_cast<unsigned long long *>(smem);  // [2][3W]
    uint32_t *sw = smem + 2 * 2 * 3 * (size_t)W;                            // [P][n + 1] plain
    uint32_t *swi = sw + (PM1 ? Pn : 0);                                     // [P][n + 1] inverted
    uint32_t *meta_s = sw + (PM1 ? 2 * Pn : Pn);                             // [n]
    uint32_t *idx_s = meta_s + n;                                            // [n]
    uint16_t *off = reinterpret_cast<uint16_t *>(idx_s + n);                 // [MAXD][n] (+-1)
    int *e2 = reinterpret_cast<int *>(idx_s + n + (PM1 ? ((size_t)MAXD * n + 1) / 2 : 0));
    int *s_best = e2 + 4 * P;
    __shared__ int s_cptr[kMaxColours + 1];

    for (int c = tid; c <= ncol; c += B) s_cptr[c] = pr->cptr[c];
    for (int p = tid; p < n; p += B) {
        meta_s[p] = pr->meta[p];
        idx_s[p] = (uint32_t)pr->idx_of_pos[p];
    }
    // initial state: top bit of the word at the initial-state slot, per slice
    for (size_t x = tid; x < Pn; x += B) {
        const int tau = (int)(x / ns), p = (int)(x - (size_t)tau * ns);
        uint32_t w = 0u;
        if (p < n) {
            const uint32_t i = (uint32_t)pr->idx_of_pos[p] | ((uint32_t)tau << 16);
            const uint4 r = philox4x32_10(
                make_uint4(i, (job.phase << kSweepBits) | kInitSlot, (uint32_t)quad, job.start), k0, k1);
            w = (r.x >> 31) | ((r.y >> 31) << 8) | ((r.z >> 31) << 16) | ((r.w >> 31) << 24);
            if (PM1) swi[x] = w ^ 0x01010101u;
        } else if (PM1) {
            swi[x] = 0u;
        }
        sw[x] = w;
    }
    if (PM1) {
        for (int x = tid; x < MAXD * n; x += B) {
            const int d = x / n, p = x - d * n;
            uint16_t o = (uint16_t)n;  // missing neighbour: the slice's zero word
            if (d < maxdeg) {
                const uint32_t e = pr->ell[(size_t)d * cap_n + p];
                if (d < (int)(pr->meta[p] & 0xFFFFu)) o = (uint16_t)(((e >> 31) ? (int)Pn : 0) + (int)(e & 0xFFFFu));
            }
            off[x] = o;
        }
    }
    if (T > 0)
        for (int x = tid; x < 3 * W; x += B) rows[x] = L.ent[x];
    __syncthreads();

    // Philox parts fixed for this quad
    uint32_t H1, L1;
    philox_mulhilo(kPhiloxM1, (uint32_t)quad, H1, L1);
    const uint32_t k0w = k0 + kPhiloxW0, k1w = k1 + kPhiloxW1;
    const PhiloxKeys<2> Kr = philox_keys<2>(k0, k1);

    const int nt = (P > 1) ? P / 2 : 1;  // slices per parity
    // register form: +-1 couplers, two or more slices, at most NC colour classes of at most B spins
    bool reg = NC > 0 && PM1 && P > 1 && ncol <= NC;
    for (int c = 0; reg && c < ncol; ++c) reg = s_cptr[c + 1] - s_cptr[c] <= B;
    if constexpr (PM1 && NC > 0) {
      if (reg) {
        constexpr int NCR = NC;
        // class j: units (spin k, slice group g) = thread k + g nc, g < G = min(nt, B / nc)
        uint32_t own4[NCR], o4[NCR][MAXD], c0[NCR], ib[NCR], jp[NCR];
        int g[NCR], G[NCR];
#pragma unroll
        for (int j = 0; j < NCR; ++j) {
            g[j] = -1;
            G[j] = 1;
            own4[j] = c0[j] = ib[j] = jp[j] = 0u;
#pragma unroll
            for (int d = 0; d < MAXD; ++d) o4[j][d] = 0u;
            if (j < ncol) {
                const int lo = s_cptr[j], nc = s_cptr[j + 1] - lo;
                if (nc > 0) {
                    G[j] = min(nt, B / nc);
                    if (tid < nc * G[j]) {
                        const int gq = tid / nc, p = lo + (tid - gq * nc);
                        const uint32_t meta = meta_s[p];
                        g[j] = gq;
                        own4[j] = 4u * (uint32_t)p;
#pragma unroll
                        for (int d = 0; d < MAXD; ++d) o4[j][d] = 4u * (uint32_t)off[d * n + p];
                        // bias - sum_j |J_ij| + h per byte (every |J| = 1: bias - deg + h)
                        int sumj = (int)(meta & 0xFFFFu);
                        if (SI) {
                            sumj = 0;
                            for (int d = 0; d < (int)(meta & 0xFFFFu) && d < MAXD; ++d) {
                                const uint32_t aj = (uint32_t)abs((int)pr->ell[(size_t)d * cap_n + p] >> 16);
                                jp[j] |= aj << (4 * d);
                                sumj += (int)aj;
                            }
                        }
                        c0[j] = (uint32_t)(bias - sumj + ((int)meta >> 16)) * 0x01010101u;
                        ib[j] = idx_s[p];
                    }
                }
            }
        }
        SqaRegConsts K;
        K.ns4 = 4u * (uint32_t)ns;
        K.inv4 = 4u * (uint32_t)Pn;
        K.wrap4 = (uint32_t)(P - 1) * K.ns4;
        K.k2 = (uint32_t)(2 * bias) * 0x01010101u;
        K.W = (uint32_t)W;
        K.start = job.start;
        K.k1 = k1;
        K.L1 = L1;
        K.k0w = k0w;
        K.k1w = k1w;
        // E32: the rows as 32-bit entries (low words) in the same space
        uint32_t *rows32 = reinterpret_cast<uint32_t *>(rows);
        if (E32) {
            __syncthreads();  // every thread has read the 64-bit row 0
            for (int x = tid; x < 3 * W; x += B) rows32[x] = (uint32_t)L.ent[x];
            __syncthreads();
        }
        for (int t = 0; t < T; ++t) {
            const void *ent = E32 ? static_cast<const void *>(rows32 + (t & 1) * 3 * W)
                                  : static_cast<const void *>(rows + (t & 1) * 3 * W);
            if (t + 1 < T) {
                const unsigned long long *src = L.ent + (size_t)(t + 1) * 3 * W;
                if (E32)
                    for (int x = tid; x < 3 * W; x += B) rows32[((t + 1) & 1) * 3 * W + x] = (uint32_t)src[x];
                else
                    for (int x = tid; x < 3 * W; x += B) rows[((t + 1) & 1) * 3 * W + x] = src[x];
            }
            philox_mulhilo(kPhiloxM0, H1 ^ (phase_hi | (uint32_t)t) ^ k0, K.HA, K.LA);
#pragma unroll
            for (int j = 0; j < NCR; ++j) {
                if (j < ncol) {
                    sqa_reg_pass<0, MAXD, E32, SI>(sw, ent, g[j], G[j], P, own4[j], o4[j], c0[j], jp[j], ib[j], K, Kr);
                    __syncthreads();
                    sqa_reg_pass<1, MAXD, E32, SI>(sw, ent, g[j], G[j], P, own4[j], o4[j], c0[j], jp[j], ib[j], K, Kr);
                    __syncthreads();
                }
            }
        }
      }
    }
    if (!reg)
    for (int t = 0; t < T; ++t) {
        const unsigned long long *ent = rows + (t & 1) * 3 * W;
        if (t + 1 < T)
            for (int x = tid; x < 3 * W; x += B) rows[((t + 1) & 1) * 3 * W + x] = L.ent[(size_t)(t + 1) * 3 * W + x];
        const uint32_t y = phase_hi | (uint32_t)t;
        uint32_t HA, LA;  // round 2, word 0: fixed for this quad and sweep
        philox_mulhilo(kPhiloxM0, H1 ^ y ^ k0, HA, LA);
        for (int c = 0; c < ncol; ++c) {
            const int lo = s_cptr[c], nc = s_cptr[c + 1] - lo;
            if (nc == 0) continue;
            // items (slice pair index tq, position k), k fastest, walked without divisions
            const int dq = B / nc, dk = B - dq * nc;
            const int q0 = tid / nc, kk0 = tid - q0 * nc;
            for (int par = 0; par < (P > 1 ? 2 : 1); ++par) {
                int tq = q0, k = kk0;
                while (tq < nt) {
                    const int p = lo + k;
                    const int tau = par + 2 * tq;
                    const uint32_t *s = sw + (size_t)tau * ns;
                    const uint32_t own = s[p];
                    const uint32_t meta = meta_s[p];
                    const int deg = (int)(meta & 0xFFFFu);
                    const int h = (int)meta >> 16;
                    // a per byte: slice neighbours equal to the spin (1 for a single slice)
                    uint32_t a4 = 0x01010101u;
                    if (P > 1) {
                        const uint32_t up = sw[(size_t)(tau + 1 == P ? 0 : tau + 1) * ns + p];
                        const uint32_t dn = sw[(size_t)(tau == 0 ? P - 1 : tau - 1) * ns + p];
                        a4 = (~(own ^ up) & 0x01010101u) + (~(own ^ dn) & 0x01010101u);
                    }
                    int idx[4];
                    if (PM1 && !SI) {
                        // byte r of x: neighbours with b_j ^ [J_ij < 0] = 1; k = 2x + bias - deg + h
                        // for b_i = 0 and its mirror 2 bias - that for b_i = 1
                        uint32_t x = 0;
#pragma unroll
                        for (int d = 0; d < MAXD; ++d) x += s[off[d * n + p]];
                        const uint32_t m = own * 0xFFu;
                        const uint32_t c0 = (uint32_t)(bias - deg + h) * 0x01010101u;
                        const uint32_t c1 = (uint32_t)(bias + deg - h) * 0x01010101u;
                        const uint32_t k4 = ((x + x + c0) & ~m) | ((c1 - x - x) & m);
                        const uint32_t full = a4 * (uint32_t)W + k4;  // bytes <= 3W - 1 <= 255
#pragma unroll
                        for (int r = 0; r < 4; ++r) idx[r] = (int)__byte_perm(full, 0u, 0x4440u | (uint32_t)r);
                    } else {
                        int acc[4] = {0, 0, 0, 0}, sumJ = 0;
                        for (int d = 0; d < deg; ++d) {
                            const uint32_t e = __ldg(pr->ell + (size_t)d * cap_n + p);
                            const int Jv = (int)e >> 16;
                            const uint32_t w = s[e & 0xFFFFu];
                            sumJ += Jv;
#pragma unroll
                            for (int r = 0; r < 4; ++r) acc[r] += Jv * (int)((w >> (8 * r)) & 1u);
                        }
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            // f = h + sum_j J s_j; k = dE/2 + bias = bias - s f
                            const int f = h - sumJ + 2 * acc[r];
                            const int sg = 2 * (int)((own >> (8 * r)) & 1u) - 1;
                            idx[r] = (int)((a4 >> (8 * r)) & 0xFFu) * W + bias - sg * f;
                        }
                    }
                    const uint32_t i = idx_s[p] | ((uint32_t)tau << 16);
                    const uint4 u = philox_sqa(i, job.start, k1, L1, HA, LA, k0w, k1w, Kr);
                    const uint32_t ur[4] = {u.x, u.y, u.z, u.w};
                    uint32_t flip = 0;
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if ((((unsigned long long)ur[r] + ent[idx[r]]) >> 32) == 0ull) flip |= 1u << (8 * r);
                    const uint32_t nw = own ^ flip;
                    sw[(size_t)tau * ns + p] = nw;
                    if (PM1) swi[(size_t)tau * ns + p] = nw ^ 0x01010101u;
                    tq += dq;
                    k += dk;
                    if (k >= nc) { k -= nc; ++tq; }
                }
                __syncthreads();
            }
        }
    }

    // energies of every slice (2E summed per replica), then each run's lowest-energy slice
    for (int x = tid; x < 4 * P; x += B) e2[x] = 0;
    __syncthreads();
    for (size_t x = tid; x < (size_t)P * n; x += B) {
        const int tau = (int)(x / n), p = (int)(x - (size_t)tau * n);
        const uint32_t *s = sw + (size_t)tau * ns;
        int c2[4];
        energy2<PM1 && !SI>(s[p], meta_s[p], pr->ell, cap_n, p, s, c2);
#pragma unroll
        for (int r = 0; r < 4; ++r) atomicAdd(&e2[4 * tau + r], c2[r]);
    }
    __syncthreads();
    if (tid < 4) {
        int bt = 0;
        for (int tau = 1; tau < P; ++tau)
            if (e2[4 * tau + tid] < e2[4 * bt + tid]) bt = tau;
        s_best[tid] = bt;
        const int r = 4 * quad + tid;
        if (r < job.S) {
            job.energies[r] = (int64_t)(e2[4 * bt + tid] / 2) + pr->offset;
            if (L.slice_out) L.slice_out[r] = bt;
        }
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    const int Wn = (n + 31) >> 5;
    for (int w = warp; w < Wn; w += B / 32) {
        const int i = 32 * w + lane;
        const int pos = (i < n) ? pr->pos_of_idx[i] : 0;
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const uint32_t word = (i < n) ? sw[(size_t)s_best[rr] * ns + pos] : 0u;
            const uint32_t bits = __ballot_sync(0xFFFFFFFFu, (word >> (8 * rr)) & 1u);
            const int r = 4 * quad + rr;
            if (lane == 0 && r < job.S) job.spins[(size_t)r * job.W + w] = bits;
        }
    }
}

// NC > 0: register form for problems of at most NC colour classes of at most
// B spins (+-1 couplers, two or more slices); other items take the walk.
template <bool PM1, int B, int MAXD, int NC, bool E32, bool SI>
__global__ void __launch_bounds__(B, (NC > 0 && B == 256) ? 2 : 1) k_sweep_sqa(const SweepLaunch L)
{
    extern __shared__ __align__(16) uint32_t smem_sqa[];
    __shared__ int s_item;
    for (int iter = 0;; ++iter) {
        SweepJob job;
        int quad0, nq;
        if (!next_item(L, iter, &s_item, job, quad0, nq)) break;
        run_item_sqa<PM1, B, MAXD, NC, E32, SI>(L, job, quad0, smem_sqa);
        __syncthreads();
    }
}

// variant 0: general couplers (MAXD unused); 1: +-1 couplers, item walk; 2: +-1
// couplers, register form with ncls colour-class slots (2 or 4) and, with
// ent32, 32-bit acceptance entries; 3: the register form for small integer
// couplers (|J| <= 15; block 256).  +-1 and small integers: neighbour
// loop unrolled to MAXD (6 or 8).
void *select_sqa(int variant, int block, int maxdeg, int ncls, bool ent32)
{
#define SPVAR_SQA_CASE(PM, BB, MD, NCC, E, S) \
    if (block == BB) return reinterpret_cast<void *>(k_sweep_sqa<PM, BB, MD, NCC, E, S>);
#define SPVAR_SQA_REG(MD, NCC, E)                                                    \
    SPVAR_SQA_CASE(true, 256, MD, NCC, E, false) SPVAR_SQA_CASE(true, 512, MD, NCC, E, false) \
        SPVAR_SQA_CASE(true, 1024, MD, NCC, E, false)
#define SPVAR_SQA_SI(MD, NCC, E) SPVAR_SQA_CASE(true, 256, MD, NCC, E, true)
    const int md = maxdeg <= 6 ? 6 : maxdeg <= 8 ? 8 : 0;
    if (variant == 0) {
        SPVAR_SQA_CASE(false, 128, 0, 0, false, false) SPVAR_SQA_CASE(false, 256, 0, 0, false, false)
        SPVAR_SQA_CASE(false, 512, 0, 0, false, false)
    } else if (variant == 1 && md == 6) {
        SPVAR_SQA_CASE(true, 128, 6, 0, false, false) SPVAR_SQA_CASE(true, 256, 6, 0, false, false)
        SPVAR_SQA_CASE(true, 512, 6, 0, false, false)
    } else if (variant == 1 && md == 8) {
        SPVAR_SQA_CASE(true, 128, 8, 0, false, false) SPVAR_SQA_CASE(true, 256, 8, 0, false, false)
        SPVAR_SQA_CASE(true, 512, 8, 0, false, false)
    } else if (variant == 2) {
        if (md == 6 && ncls == 2 && !ent32) { SPVAR_SQA_REG(6, 2, false) }
        if (md == 6 && ncls == 2 && ent32) { SPVAR_SQA_REG(6, 2, true) }
        if (md == 6 && ncls == 4 && !ent32) { SPVAR_SQA_REG(6, 4, false) }
        if (md == 6 && ncls == 4 && ent32) { SPVAR_SQA_REG(6, 4, true) }
        if (md == 8 && ncls == 2 && !ent32) { SPVAR_SQA_REG(8, 2, false) }
        if (md == 8 && ncls == 2 && ent32) { SPVAR_SQA_REG(8, 2, true) }
        if (md == 8 && ncls == 4 && !ent32) { SPVAR_SQA_REG(8, 4, false) }
        if (md == 8 && ncls == 4 && ent32) { SPVAR_SQA_REG(8, 4, true) }
    } else if (variant == 3) {
        if (md == 6 && ncls == 2 && !ent32) { SPVAR_SQA_SI(6, 2, false) }
        if (md == 6 && ncls == 2 && ent32) { SPVAR_SQA_SI(6, 2, true) }
        if (md == 6 && ncls == 4 && !ent32) { SPVAR_SQA_SI(6, 4, false) }
        if (md == 6 && ncls == 4 && ent32) { SPVAR_SQA_SI(6, 4, true) }
        if (md == 8 && ncls == 2 && !ent32) { SPVAR_SQA_SI(8, 2, false) }
        if (md == 8 && ncls == 2 && ent32) { SPVAR_SQA_SI(8, 2, true) }
        if (md == 8 && ncls == 4 && !ent32) { SPVAR_SQA_SI(8, 4, false) }
        if (md == 8 && ncls == 4 && ent32) { SPVAR_SQA_SI(8, 4, true) }
    }
#undef SPVAR_SQA_SI
#undef SPVAR_SQA_REG
#undef SPVAR_SQA_CASE
    return nullptr;
}

}  // namespace

bool sqa_shape_ok(int variant, int block, int max_n, int max_deg, int P, int W, int ncls)
{
    if (!select_sqa(variant, block, max_deg, ncls, false) || P < 1 || (P > 1 && (P & 1)) || P > kSqaMaxSlices) return false;
    if (variant >= 2 && P < 2) return false;
    if ((long long)max_n >= (1 << 16) - 1) return false;
    if (variant != 0 && (long long)P * (max_n + 1) + max_n >= 0xFFFF) return false;
    // byte lanes: the entry index a W + k (+-1), or k alone (small integers)
    if ((variant == 1 || variant == 2) && 3LL * W - 1 > 255) return false;
    if (variant == 3 && W > 255) return false;
    return true;
}

size_t sqa_smem_bytes(int max_n, int P, int maxdeg, int W, bool pm1)
{
    return 4 * sqa_words(max_n, P, maxdeg, W, pm1);
}

cudaError_t launch_sweep_sqa(const SweepLaunch &L, int variant, int block, int ncls, bool ent32, int grid,
                             size_t smem, cudaStream_t st)
{
    void *k = select_sqa(variant, block, L.max_deg, ncls, ent32);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<SweepLaunch *>(&L)};
    return cudaLaunchKernel(k, dim3(grid), dim3(block), args, smem, st);
}

int sqa_max_active_blocks(int variant, int block, int max_deg, int ncls, bool ent32, size_t smem)
{
    void *k = select_sqa(variant, block, max_deg, ncls, ent32);
    if (!k) return 0;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem);
    return nb;
}

}  // namespace spvar
