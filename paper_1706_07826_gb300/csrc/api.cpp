// C ABI of the library: problem construction (Sec. I problem statement),
// annealing schedule, and the standalone sample / persistence / reduce calls
// of Alg. 1.  Host code only; kernels live in sweep.cu and persist.cu.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "spvar_internal.h"

using namespace spvar;

namespace {

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int device_smem_optin()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

int device_sms()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

// Colour classes of the sweep order.  Bipartite graphs: each connected
// component 2-coloured by the parity of its BFS distance from the component's
// lowest-index vertex.  Otherwise: first-fit greedy in increasing index.
int colour_classes(int n, const int32_t *rp, const int32_t *col, std::vector<int32_t> &c)
{
    c.assign(n, -1);
    std::vector<int32_t> queue;
    queue.reserve(n);
    for (int root = 0; root < n; ++root) {
        if (c[root] >= 0) continue;
        c[root] = 0;
        queue.clear();
        queue.push_back(root);
        for (size_t head = 0; head < queue.size(); ++head) {
            const int v = queue[head];
            for (int p = rp[v]; p < rp[v + 1]; ++p)
                if (c[col[p]] < 0) {
                    c[col[p]] = c[v] ^ 1;
                    queue.push_back(col[p]);
                }
        }
    }
    bool ok = true;
    int ncol = n > 0 ? 1 : 0;
    for (int v = 0; v < n && ok; ++v) {
        if (c[v] == 1) ncol = 2;
        for (int p = rp[v]; p < rp[v + 1]; ++p)
            if (c[col[p]] == c[v]) { ok = false; break; }
    }
    if (ok) return ncol;
    ncol = 0;
    std::vector<int32_t> mark(n + 1, -1);
    for (int v = 0; v < n; ++v) {
        for (int p = rp[v]; p < rp[v + 1]; ++p)
            if (col[p] < v) mark[c[col[p]]] = v;
        int k = 0;
        while (mark[k] == v) ++k;
        c[v] = k;
        ncol = std::max(ncol, k + 1);
    }
    return ncol;
}

}  // namespace

namespace spvar {

size_t prob_blob_bytes(int cap_n, int cap_nnz, int maxdeg)
{
    size_t b = align256(sizeof(DevProb));
    b += align256(4 * ((size_t)cap_n + 1));          // row_ptr
    b += 2 * align256(4 * (size_t)cap_nnz);          // col, val
    b += 2 * align256(4 * (size_t)cap_n);            // h, colour
    b += align256(4 * ((size_t)kMaxColours + 1));    // cptr
    b += 3 * align256(4 * (size_t)cap_n);            // idx_of_pos, pos_of_idx, meta
    b += align256(4 * (size_t)maxdeg * cap_n);       // ell
    return b;
}

void prob_carve(DevProb *hdr, void *blob, int cap_n, int cap_nnz, int maxdeg)
{
    char *p = static_cast<char *>(blob);
    size_t o = align256(sizeof(DevProb));
    auto take = [&](size_t bytes) {
        char *r = p + o;
        o += align256(bytes);
        return r;
    };
    hdr->cap_n = cap_n;
    hdr->cap_nnz = cap_nnz;
    hdr->maxdeg = maxdeg;
    hdr->row_ptr = (int32_t *)take(4 * ((size_t)cap_n + 1));
    hdr->col = (int32_t *)take(4 * (size_t)cap_nnz);
    hdr->val = (int32_t *)take(4 * (size_t)cap_nnz);
    hdr->h = (int32_t *)take(4 * (size_t)cap_n);
    hdr->colour = (int32_t *)take(4 * (size_t)cap_n);
    hdr->cptr = (int32_t *)take(4 * ((size_t)kMaxColours + 1));
    hdr->idx_of_pos = (int32_t *)take(4 * (size_t)cap_n);
    hdr->pos_of_idx = (int32_t *)take(4 * (size_t)cap_n);
    hdr->meta = (uint32_t *)take(4 * (size_t)cap_n);
    hdr->ell = (uint32_t *)take(4 * (size_t)maxdeg * cap_n);
}

int host_problem_build(int n, const int32_t *row_ptr, const int32_t *col, const int32_t *val, const int32_t *h,
                       int64_t offset, int energy_scale, HostProblem &hp)
{
    if (n < 0 || energy_scale < 1 || !row_ptr || (n > 0 && !h)) return SPVAR_EINVAL;
    if (n > SPVAR_MAX_N) return SPVAR_ELIMIT;
    if (row_ptr[0] != 0) return SPVAR_EINVAL;
    for (int i = 0; i < n; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) return SPVAR_EINVAL;
    const int nnz = row_ptr[n];
    if (nnz > 0 && (!col || !val)) return SPVAR_EINVAL;
    int maxdeg = 0;
    long long total = 0;
    long long maxrow = 0;
    for (int i = 0; i < n; ++i) {
        const int d = row_ptr[i + 1] - row_ptr[i];
        if (d > SPVAR_MAX_DEGREE) return SPVAR_ELIMIT;
        maxdeg = std::max(maxdeg, d);
        long long rowsum = std::llabs((long long)h[i]);
        total += 2 * std::llabs((long long)h[i]);
        for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            const int j = col[p];
            if (j < 0 || j >= n || j == i) return SPVAR_EINVAL;
            if (p > row_ptr[i] && col[p - 1] >= j) return SPVAR_EINVAL;
            if (val[p] == 0) return SPVAR_EINVAL;
            if (val[p] > 32767 || val[p] < -32767) return SPVAR_ELIMIT;
            // symmetric partner (j, i) with the same value
            const int32_t *b = col + row_ptr[j], *e = col + row_ptr[j + 1];
            const int32_t *f = std::lower_bound(b, e, i);
            if (f == e || *f != i || val[f - col] != val[p]) return SPVAR_EINVAL;
            rowsum += std::llabs((long long)val[p]);
            total += std::llabs((long long)val[p]);
        }
        maxrow = std::max(maxrow, rowsum);
        if (total >= (1ll << 31)) return SPVAR_EOVERFLOW;
    }
    if (maxrow > 32767) return SPVAR_ELIMIT;  // h' and dmax/2 must fit int16

    const int ncol = colour_classes(n, row_ptr, col, hp.colour);
    if (ncol > kMaxColours) return SPVAR_ELIMIT;
    hp.cap_n = std::max(n, 1);
    hp.cap_nnz = std::max(nnz, 1);
    hp.md = std::max(maxdeg, 1);
    DevProb &H = hp.hdr;
    std::memset(&H, 0, sizeof(H));
    H.n = n;
    H.nnz = nnz;
    H.ncol = ncol;
    H.maxdeg = hp.md;
    H.dmax = (int32_t)(2 * maxrow);
    H.offset = offset;
    H.scale = energy_scale;
    H.cap_n = hp.cap_n;
    H.cap_nnz = hp.cap_nnz;
    H.hzero = 1;
    H.pm1 = 1;
    for (int i = 0; i < n; ++i) if (h[i] != 0) H.hzero = 0;
    for (int p = 0; p < nnz; ++p) if (val[p] != 1 && val[p] != -1) H.pm1 = 0;
    H.ujs = 1;
    for (int i = 0; i < n && H.ujs; ++i)
        for (int p = row_ptr[i] + 1; p < row_ptr[i + 1]; ++p)
            if (std::abs(val[p]) != std::abs(val[row_ptr[i]])) { H.ujs = 0; break; }
    H.rho = -1;
    for (int i = 0, best = -1; i < n; ++i)
        if (row_ptr[i + 1] - row_ptr[i] > best) { best = row_ptr[i + 1] - row_ptr[i]; H.rho = i; }

    hp.row_ptr.assign(row_ptr, row_ptr + n + 1);
    hp.col.assign(col, col + nnz);
    hp.val.assign(val, val + nnz);
    hp.h.assign(h, h + n);
    // sweep layout: positions colour class by colour class, index ascending
    hp.cptr.assign(kMaxColours + 1, 0);
    hp.idx_of_pos.assign(hp.cap_n, 0);
    hp.pos_of_idx.assign(hp.cap_n, 0);
    hp.meta.assign(hp.cap_n, 0);
    hp.ell.assign((size_t)hp.md * hp.cap_n, 0);
    for (int i = 0; i < n; ++i) hp.cptr[hp.colour[i] + 1]++;
    for (int c = 0; c < ncol; ++c) hp.cptr[c + 1] += hp.cptr[c];
    for (int c = ncol + 1; c <= kMaxColours; ++c) hp.cptr[c] = hp.cptr[ncol];
    {
        std::vector<int32_t> fill(hp.cptr.begin(), hp.cptr.end());
        for (int i = 0; i < n; ++i) {
            const int pos = fill[hp.colour[i]]++;
            hp.idx_of_pos[pos] = i;
            hp.pos_of_idx[i] = pos;
        }
    }
    for (int i = 0; i < n; ++i) {
        const int pos = hp.pos_of_idx[i];
        const int deg = row_ptr[i + 1] - row_ptr[i];
        hp.meta[pos] = ((uint32_t)(h[i] & 0xFFFF) << 16) | (uint32_t)deg;
        for (int d = 0; d < deg; ++d) {
            const int p = row_ptr[i] + d;
            hp.ell[(size_t)d * hp.cap_n + pos] =
                ((uint32_t)hp.pos_of_idx[col[p]] & 0xFFFFu) | ((uint32_t)(val[p] & 0xFFFF) << 16);
        }
    }
    return SPVAR_OK;
}

int host_problem_upload(const HostProblem &hp, void *blob, cudaStream_t st, DevProb *hdr_out)
{
    DevProb H = hp.hdr;
    prob_carve(&H, blob, hp.cap_n, hp.cap_nnz, hp.md);
    const int n = H.n, nnz = H.nnz;
    *hdr_out = H;
    // the blob's image on the host (header with device pointers, then every array at
    // its offset), sent with one copy
    const size_t bytes = prob_blob_bytes(hp.cap_n, hp.cap_nnz, hp.md);
    std::vector<char> img(bytes, 0);
    char *const base = static_cast<char *>(blob);
    auto put = [&](const void *dst, const void *src, size_t nb) {
        if (nb) std::memcpy(img.data() + (static_cast<const char *>(dst) - base), src, nb);
    };
    put(blob, hdr_out, sizeof(DevProb));
    put(H.row_ptr, hp.row_ptr.data(), 4 * ((size_t)n + 1));
    put(H.col, hp.col.data(), 4 * (size_t)nnz);
    put(H.val, hp.val.data(), 4 * (size_t)nnz);
    put(H.h, hp.h.data(), 4 * (size_t)n);
    put(H.colour, hp.colour.data(), 4 * (size_t)n);
    put(H.cptr, hp.cptr.data(), 4 * hp.cptr.size());
    put(H.idx_of_pos, hp.idx_of_pos.data(), 4 * (size_t)n);
    put(H.pos_of_idx, hp.pos_of_idx.data(), 4 * (size_t)n);
    put(H.meta, hp.meta.data(), 4 * (size_t)n);
    put(H.ell, hp.ell.data(), 4 * hp.ell.size());
    // a copy from pageable memory returns once the source is staged, so img may go
    return cudaMemcpyAsync(blob, img.data(), bytes, cudaMemcpyHostToDevice, st) == cudaSuccess ? SPVAR_OK
                                                                                               : SPVAR_ECUDA;
}

}  // namespace spvar

extern "C" {

const char *spvar_strerror(int code)
{
    switch (code) {
    case SPVAR_OK: return "ok";
    case SPVAR_EINVAL: return "invalid argument or malformed problem";
    case SPVAR_EOVERFLOW: return "values overflow the 32-bit energy arithmetic";
    case SPVAR_ENOMEM: return "out of memory";
    case SPVAR_EBUDGET: return "request exceeds the device-memory budget";
    case SPVAR_ETIMEOUT: return "bounded device wait timed out";
    case SPVAR_ECUDA: return "CUDA runtime error";
    case SPVAR_ELIMIT: return "size beyond a library limit";
    default: return "unknown error";
    }
}

int spvar_device_count(int *count)
{
    if (!count) return SPVAR_EINVAL;
    int c = 0;
    if (cudaGetDeviceCount(&c) != cudaSuccess) c = 0;
    *count = c;
    return SPVAR_OK;
}

int spvar_csr_from_edges(int32_t n, int64_t m, const int32_t *ei, const int32_t *ej,
                         const int32_t *J, int32_t *row_ptr, int32_t *col, int32_t *val)
{
    if (n < 0 || m < 0 || !row_ptr || (m > 0 && (!ei || !ej || !J || !col || !val)))
        return SPVAR_EINVAL;
    if (2 * m > INT32_MAX) return SPVAR_ELIMIT;
    std::vector<int64_t> deg((size_t)n + 1, 0);
    for (int64_t e = 0; e < m; ++e) {
        if (ei[e] < 0 || ei[e] >= n || ej[e] < 0 || ej[e] >= n || ei[e] == ej[e]) return SPVAR_EINVAL;
        deg[ei[e]]++;
        deg[ej[e]]++;
    }
    row_ptr[0] = 0;
    for (int i = 0; i < n; ++i) row_ptr[i + 1] = row_ptr[i] + (int32_t)deg[i];
    // counting placement, then sort each row's (col, val) pairs
    std::vector<int32_t> fill(row_ptr, row_ptr + n);
    for (int64_t e = 0; e < m; ++e) {
        int32_t a = ei[e], b = ej[e];
        col[fill[a]] = b; val[fill[a]++] = J[e];
        col[fill[b]] = a; val[fill[b]++] = J[e];
    }
    std::vector<std::pair<int32_t, int32_t>> row;
    for (int i = 0; i < n; ++i) {
        row.clear();
        for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) row.emplace_back(col[p], val[p]);
        std::sort(row.begin(), row.end(),
                  [](const std::pair<int32_t, int32_t> &x, const std::pair<int32_t, int32_t> &y) {
                      return x.first < y.first;
                  });
        for (size_t q = 0; q < row.size(); ++q) {
            if (q > 0 && row[q].first == row[q - 1].first) return SPVAR_EINVAL;
            col[row_ptr[i] + q] = row[q].first;
            val[row_ptr[i] + q] = row[q].second;
        }
    }
    return SPVAR_OK;
}

int spvar_problem_create(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *val,
                         const int32_t *h, int64_t offset, int32_t energy_scale, void *stream,
                         spvar_problem **out)
{
    if (!out) return SPVAR_EINVAL;
    *out = nullptr;
    HostProblem hp;
    int rc = host_problem_build(n, row_ptr, col, val, h, offset, energy_scale, hp);
    if (rc != SPVAR_OK) return rc;
    Problem *P = new (std::nothrow) Problem();
    if (!P) return SPVAR_ENOMEM;
    cudaGetDevice(&P->device);
    P->blob_bytes = prob_blob_bytes(hp.cap_n, hp.cap_nnz, hp.md);
    if (cudaMalloc(&P->blob, P->blob_bytes) != cudaSuccess) {
        delete P;
        cudaGetLastError();
        return SPVAR_ENOMEM;
    }
    cudaStream_t st = as_stream(stream);
    rc = host_problem_upload(hp, P->blob, st, &P->hdr);
    if (rc == SPVAR_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = SPVAR_ECUDA;
    if (rc != SPVAR_OK) {
        cudaFree(P->blob);
        delete P;
        cudaGetLastError();
        return rc;
    }
    P->dev = static_cast<DevProb *>(P->blob);
    for (int c = 0; c < kMaxColours; ++c)
        P->csize[c] = c < hp.hdr.ncol ? hp.cptr[c + 1] - hp.cptr[c] : 0;
    for (size_t k = 0; k < hp.val.size(); ++k) P->jabs_max = std::max(P->jabs_max, std::abs(hp.val[k]));
    *out = reinterpret_cast<spvar_problem *>(P);
    return SPVAR_OK;
}

void spvar_problem_destroy(spvar_problem *p)
{
    if (!p) return;
    Problem *P = reinterpret_cast<Problem *>(p);
    cudaFree(P->blob);
    delete P;
}

int spvar_problem_get_info(const spvar_problem *p, spvar_problem_info *info)
{
    if (!p || !info) return SPVAR_EINVAL;
    const DevProb &H = reinterpret_cast<const Problem *>(p)->hdr;
    info->n = H.n;
    info->nnz = H.nnz;
    info->ncol = H.ncol;
    info->maxdeg = H.maxdeg;
    info->dmax = H.dmax;
    info->hzero = H.hzero;
    info->pm1 = H.pm1;
    info->energy_scale = H.scale;
    info->offset = H.offset;
    return SPVAR_OK;
}

int spvar_problem_download(const spvar_problem *p, int32_t *row_ptr, int32_t *col, int32_t *val,
                           int32_t *h, int32_t *colour, void *stream)
{
    if (!p) return SPVAR_EINVAL;
    const DevProb &H = reinterpret_cast<const Problem *>(p)->hdr;
    cudaStream_t st = as_stream(stream);
    auto dn = [&](void *dst, const void *src, size_t bytes) -> bool {
        return !dst || !bytes || cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st) == cudaSuccess;
    };
    bool ok = dn(row_ptr, H.row_ptr, 4 * ((size_t)H.n + 1)) && dn(col, H.col, 4 * (size_t)H.nnz) &&
              dn(val, H.val, 4 * (size_t)H.nnz) && dn(h, H.h, 4 * (size_t)H.n) &&
              dn(colour, H.colour, 4 * (size_t)H.n);
    if (ok) ok = cudaStreamSynchronize(st) == cudaSuccess;
    return ok ? SPVAR_OK : SPVAR_ECUDA;
}

int spvar_beta_geometric(int32_t T, double beta0, double beta1, double *beta)
{
    if (T < 1 || !beta || !(beta0 > 0.0) || !(beta1 > 0.0)) return SPVAR_EINVAL;
    for (int t = 0; t < T; ++t)
        beta[t] = (T == 1) ? beta0 : beta0 * std::pow(beta1 / beta0, (double)t / (double)(T - 1));
    return SPVAR_OK;
}

int spvar_thresholds(int32_t T, const double *beta, int32_t dmax, int32_t energy_scale,
                     uint32_t *thr)
{
    if (T < 0 || dmax < 0 || energy_scale < 1 || (T > 0 && (!beta || !thr))) return SPVAR_EINVAL;
    const size_t w = (size_t)dmax + 1;
    for (int t = 0; t < T; ++t) {
        if (!(beta[t] >= 0.0)) return SPVAR_EINVAL;
        for (int d = 0; d <= dmax; ++d) {
            const double x = std::floor(std::ldexp(std::exp(-beta[t] * (double)d / (double)energy_scale), 32));
            thr[(size_t)t * w + d] = (x >= 4294967295.0) ? 0xFFFFFFFFu : (uint32_t)x;
        }
    }
    return SPVAR_OK;
}

int spvar_sample(const spvar_problem *p, int32_t num_sweeps, const uint32_t *thr, int32_t thr_stride,
                 int32_t num_samples, uint64_t seed, uint32_t start, uint32_t phase, uint32_t *spins,
                 int64_t *energies, void *stream)
{
    return spvar_sample_range(p, 0, num_sweeps, thr, thr_stride, num_samples, seed, start, phase, nullptr, spins,
                              energies, stream);
}

int spvar_sample_range(const spvar_problem *p, int32_t sweep_begin, int32_t sweep_end, const uint32_t *thr,
                       int32_t thr_stride, int32_t num_samples, uint64_t seed, uint32_t start, uint32_t phase,
                       const uint32_t *init_spins, uint32_t *spins, int64_t *energies, void *stream)
{
    if (!p) return SPVAR_EINVAL;
    const Problem *P = reinterpret_cast<const Problem *>(p);
    const DevProb &H = P->hdr;
    const int32_t num_sweeps = sweep_end;
    if (sweep_begin < 0 || sweep_end < sweep_begin || num_samples < 0 || phase > SPVAR_MAX_PHASE)
        return SPVAR_EINVAL;
    if (sweep_begin > 0 && !init_spins) return SPVAR_EINVAL;
    if (init_spins && init_spins == spins) return SPVAR_EINVAL;  // rows are read while others are written
    if (num_sweeps > SPVAR_MAX_SWEEPS || num_samples > SPVAR_MAX_SAMPLES) return SPVAR_ELIMIT;
    if (num_samples == 0) return SPVAR_OK;
    if ((num_sweeps > 0 && !thr) || thr_stride < H.dmax + 1 || !energies || (H.n > 0 && !spins))
        return SPVAR_EINVAL;
    const int quads = ceil_div(num_samples, 4);
    const int sms = device_sms();
    const int Q = std::max(1, std::min(8, quads / (2 * sms)));
    const int optin = device_smem_optin();
    // shape: the register-resident +-1 kernel when it applies, else the general one
    SweepShape sh{0, (H.n >= 512) ? 256 : 128, Q, 1, 0, 0};
    if (pm1_kernel_eligible(H.pm1 != 0, H.dmax, H.maxdeg)) {
        const int md = H.maxdeg <= 6 ? 6 : 8;
        if (pm1r_kernel_eligible(H.pm1 != 0, H.dmax, H.maxdeg))
            for (int blk : {256, 512, 128}) {
                const int ns = pm1_nslot(P, Q, blk);
                if (ns > 0 && pm1_shape_ok(blk, ns, md, 0)) { sh = SweepShape{1, blk, Q, 0, ns, md}; break; }
            }
        // large problems: the streaming kernel (one quad per CTA)
        if (sh.kind == 0 && pm1s_shape_ok(512, md, H.n, 1) &&
            pm1s_smem_bytes(H.n, 1, md) <= (size_t)optin)
            sh = SweepShape{2, 512, 1, 0, 0, md};
    }
    const int mode16 = ujr_kernel_eligible(H.ujs != 0, H.dmax, H.maxdeg)          ? 1
                       : sir_kernel_eligible(P->jabs_max, H.dmax, H.maxdeg) ? 2
                                                                             : 0;
    if (sh.kind == 0 && mode16 != 0) {
        // one coupler magnitude per spin, or small integer couplers: the register
        // kernel's 16-bit-lane variants
        const int md = H.maxdeg <= 6 ? 6 : 8;
        for (int blk : {256, 512, 576, 1024}) {
            int ns = pm1_nslot(P, Q, blk);
            if (ns == 3) ns = 4;
            const SweepShape c{1, blk, Q, mode16, ns, md};
            if (ns > 0 && pm1_shape_ok(blk, ns, md, mode16) &&
                sweep_shape_smem(c, H.n, thr_stride, H.maxdeg) <= (size_t)optin) {
                sh = c;
                break;
            }
        }
    }
    if (sh.kind == 0 && sweep_shape_smem(sh, H.n, thr_stride, H.maxdeg) > (size_t)optin) sh.stage = 0;
    const size_t smem = sweep_shape_smem(sh, H.n, thr_stride, H.maxdeg);
    if (smem > (size_t)optin) return SPVAR_ELIMIT;

    SweepLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.single.prob = P->dev;
    L.single.spins = spins;
    L.single.energies = energies;
    L.single.seed = seed;
    L.single.S = num_samples;
    L.single.W = ceil_div(std::max(H.n, 0), 32);
    L.single.start = start;
    L.single.phase = phase;
    L.single.init = init_spins;
    L.single.t0 = sweep_begin;
    L.thr = thr;
    L.thr_stride = thr_stride;
    L.T = num_sweeps;
    L.Q = Q;
    L.stage_ell = sh.stage;
    L.max_n = H.n;
    L.max_deg = H.maxdeg;
    L.Q = sh.Q;
    const int grid = ceil_div(quads, sh.Q);
    SPVAR_CUDA_TRY(launch_sweep_shape(L, sh, H.pm1 != 0, grid, smem, as_stream(stream)));
    return SPVAR_OK;
}

int spvar_sqa_table(int32_t T, int32_t P, const double *beta, const double *gamma, int32_t dmax,
                    int32_t energy_scale, uint64_t *ent)
{
    if (T < 0 || P < 1 || (P > 1 && (P & 1)) || P > SPVAR_SQA_MAX_SLICES || dmax < 0 || energy_scale < 1 ||
        (T > 0 && (!beta || !gamma || !ent)))
        return SPVAR_EINVAL;
    const int32_t bias = dmax / 2, W = 2 * bias + 1;
    for (int32_t t = 0; t < T; ++t) {
        if (P > 1 && !(gamma[t] > 0.0)) return SPVAR_EINVAL;
        // coupling of neighbouring slices in this sweep (none for one slice)
        const double jp = (P > 1) ? -0.5 * std::log(std::tanh(beta[t] * gamma[t] / (double)P)) : 0.0;
        for (int32_t a = 0; a < 3; ++a)
            for (int32_t k = 0; k < W; ++k) {
                const double dA = (2.0 * beta[t] / (double)P) * (double)(k - bias) / (double)energy_scale +
                                  4.0 * jp * (double)(a - 1);
                const double x = std::floor(std::ldexp(std::exp(-dA), 32));
                const uint64_t thr = (x >= 4294967296.0) ? (1ull << 32) : (uint64_t)x;
                ent[((size_t)t * 3 + a) * W + k] = (1ull << 32) - thr;
            }
    }
    return SPVAR_OK;
}

int spvar_gamma_linear(int32_t T, double g0, double g1, double *gamma)
{
    if (T < 0 || (T > 0 && !gamma)) return SPVAR_EINVAL;
    for (int32_t t = 0; t < T; ++t) gamma[t] = (T == 1) ? g0 : g0 + (g1 - g0) * (double)t / (double)(T - 1);
    return SPVAR_OK;
}

int spvar_sqa_sample(const spvar_problem *p, int32_t num_sweeps, int32_t P, const uint64_t *ent, int32_t W,
                     int32_t num_samples, uint64_t seed, uint32_t start, uint32_t phase, uint32_t *spins,
                     int64_t *energies, int32_t *slice, void *stream)
{
    if (!p) return SPVAR_EINVAL;
    const Problem *Pr = reinterpret_cast<const Problem *>(p);
    const DevProb &H = Pr->hdr;
    if (num_sweeps < 0 || num_samples < 0 || phase > SPVAR_MAX_PHASE || P < 1 || (P > 1 && (P & 1)) ||
        P > SPVAR_SQA_MAX_SLICES || W < 1 || (W & 1) == 0 || W - 1 < H.dmax)
        return SPVAR_EINVAL;
    if (num_sweeps > SPVAR_MAX_SWEEPS || num_samples > SPVAR_MAX_SAMPLES) return SPVAR_ELIMIT;
    if (num_samples == 0) return SPVAR_OK;
    if ((num_sweeps > 0 && !ent) || !energies || (H.n > 0 && !spins)) return SPVAR_EINVAL;
    // +-1 couplers: the register form when every colour class fits a block of 512 (else 1024)
    // threads, else the item walk; general couplers: the general path
    int max_class = 0;
    for (int c = 0; c < H.ncol && c < kMaxColours; ++c) max_class = std::max(max_class, Pr->csize[c]);
    const int optin = device_smem_optin();
    int variant = 0, block = 256, ncls = 0;
    if (H.pm1 != 0) {
        for (int b : {512, 1024}) {
            ncls = sqa_reg_ncls(H.ncol, max_class, b, P);
            if (ncls > 0 && sqa_shape_ok(2, b, H.n, H.maxdeg, P, W, ncls) &&
                sqa_smem_bytes(H.n, P, H.maxdeg, W, true) <= (size_t)optin) {
                variant = 2;
                block = b;
                break;
            }
        }
        if (variant == 0 && sqa_shape_ok(1, 256, H.n, H.maxdeg, P, W)) variant = 1;
    } else if (sqa_si_eligible(Pr->jabs_max, H.dmax, H.maxdeg)) {
        // small integer couplers: their register form (256 threads) when every class fits
        ncls = sqa_reg_ncls(H.ncol, max_class, 256, P);
        if (ncls > 0 && sqa_shape_ok(3, 256, H.n, H.maxdeg, P, W, ncls) &&
            sqa_smem_bytes(H.n, P, H.maxdeg, W, true) <= (size_t)optin) {
            variant = 3;
            block = 256;
        }
    }
    if (variant < 2) ncls = 0;
    if (!sqa_shape_ok(variant, block, H.n, H.maxdeg, P, W, ncls)) return SPVAR_ELIMIT;
    const size_t smem = sqa_smem_bytes(H.n, P, H.maxdeg, W, variant != 0);
    if (smem > (size_t)optin) return SPVAR_ELIMIT;
    SweepLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.single.prob = Pr->dev;
    L.single.spins = spins;
    L.single.energies = energies;
    L.single.seed = seed;
    L.single.S = num_samples;
    L.single.W = ceil_div(std::max(H.n, 0), 32);
    L.single.start = start;
    L.single.phase = phase;
    L.T = num_sweeps;
    L.Q = 1;
    L.max_n = H.n;
    L.max_deg = H.maxdeg;
    L.ent = reinterpret_cast<const unsigned long long *>(ent);
    L.P = P;
    L.W = W;
    L.slice_out = slice;
    SPVAR_CUDA_TRY(launch_sweep_sqa(L, variant, block, ncls, false, ceil_div(num_samples, 4), smem, as_stream(stream)));
    return SPVAR_OK;
}

int spvar_pticm_sample(const spvar_problem *p, int32_t R, int32_t num_sweeps, const uint32_t *thr,
                       int32_t thr_stride, const uint32_t *xthr, int32_t dx, int32_t icm_from, int32_t keep_from,
                       int32_t K, int32_t flags, int32_t num_runs, uint64_t seed, uint32_t start0, uint32_t phase,
                       uint32_t *kept, int64_t *kept_e, int32_t *nkept, uint32_t *final_states, int64_t *final_e,
                       void *stream)
{
    if (!p) return SPVAR_EINVAL;
    const Problem *Pr = reinterpret_cast<const Problem *>(p);
    const DevProb &H = Pr->hdr;
    if (R < 1 || num_sweeps < 0 || icm_from < 0 || icm_from > R || keep_from < 0 || keep_from > R || K < 1 ||
        flags < 0 || flags > 3 || num_runs < 0 || phase > SPVAR_MAX_PHASE || thr_stride < H.dmax + 1 ||
        ((flags & 1) && R > 1 && (dx < 1 || !xthr)))
        return SPVAR_EINVAL;
    if (R > pticm_max_r() || K > SPVAR_PTICM_MAX_KEEP || num_sweeps > SPVAR_MAX_SWEEPS || H.n > pticm_max_n())
        return SPVAR_ELIMIT;
    if (num_runs == 0) return SPVAR_OK;
    if ((num_sweeps > 0 && !thr) || !final_e || !nkept || !kept_e || (H.n > 0 && (!final_states || !kept)))
        return SPVAR_EINVAL;
    const size_t smem = pticm_smem_bytes(H.n, R, H.dmax);
    if (smem > (size_t)device_smem_optin()) return SPVAR_ELIMIT;
    cudaStream_t st = as_stream(stream);
    const size_t ntr = 2 * (size_t)(R - keep_from);
    if (ntr > 0) SPVAR_CUDA_TRY(cudaMemsetAsync(nkept, 0, sizeof(int32_t) * ntr * (size_t)num_runs, st));
    SPVAR_CUDA_TRY(launch_pticm(Pr->dev, thr, thr_stride, xthr, dx, R, num_sweeps, icm_from, keep_from, K, flags, seed,
                                start0, phase, num_runs, smem, kept, kept_e, nkept, final_states, final_e, st));
    return SPVAR_OK;
}

int spvar_persistence(const spvar_problem *p, int32_t num_samples, const uint32_t *spins,
                      const int64_t *energies, double elite_threshold, int32_t fix_num,
                      int32_t fix_den, int32_t canon, int32_t *elite, int32_t *counts,
                      int8_t *fixed, int32_t *nfixed, int32_t *k_out, void *stream)
{
    if (!p) return SPVAR_EINVAL;
    const Problem *P = reinterpret_cast<const Problem *>(p);
    const DevProb &H = P->hdr;
    if (num_samples < 1 || !(elite_threshold > 0.0) || !(elite_threshold <= 1.0) || fix_num <= 0 ||
        fix_den <= 0 || fix_num > fix_den || canon < -1 || canon > 1)
        return SPVAR_EINVAL;
    if (num_samples > elite_max_samples()) return SPVAR_ELIMIT;
    if (!energies || !elite || !nfixed || (H.n > 0 && (!spins || !fixed))) return SPVAR_EINVAL;
    // k = ceil(elite * S), clamped to [1, S]
    const double x = std::ceil(elite_threshold * (double)num_samples);
    int k = (x >= (double)num_samples) ? num_samples : (int)x;
    k = std::max(1, std::min(k, num_samples));
    const int ce = (canon < 0) ? H.hzero : canon;
    cudaStream_t st = as_stream(stream);
    SPVAR_CUDA_TRY(launch_elite_single(energies, num_samples, k, elite, st));
    SPVAR_CUDA_TRY(launch_count_single(P->dev, H.n, spins, ceil_div(H.n, 32), elite, k, ce, fix_num,
                                       fix_den, counts, fixed, nfixed, st));
    if (k_out) *k_out = k;
    return SPVAR_OK;
}

int spvar_reduce(const spvar_problem *p, const int8_t *fixed, int32_t *old_of_new, void *stream,
                 spvar_problem **out)
{
    if (!p || !out) return SPVAR_EINVAL;
    *out = nullptr;
    const Problem *S = reinterpret_cast<const Problem *>(p);
    const DevProb &H = S->hdr;
    if (H.n > 0 && (!fixed || !old_of_new)) return SPVAR_EINVAL;
    Problem *D = new (std::nothrow) Problem();
    if (!D) return SPVAR_ENOMEM;
    D->device = S->device;
    D->blob_bytes = prob_blob_bytes(H.cap_n, H.cap_nnz, H.maxdeg);
    int32_t *scratch = nullptr;
    if (cudaMalloc(&D->blob, D->blob_bytes) != cudaSuccess) {
        delete D;
        cudaGetLastError();
        return SPVAR_ENOMEM;
    }
    if (cudaMalloc(&scratch, 8 * (size_t)H.cap_n) != cudaSuccess) {
        cudaFree(D->blob);
        delete D;
        cudaGetLastError();
        return SPVAR_ENOMEM;
    }
    std::memset(&D->hdr, 0, sizeof(DevProb));
    prob_carve(&D->hdr, D->blob, H.cap_n, H.cap_nnz, H.maxdeg);
    D->dev = static_cast<DevProb *>(D->blob);
    cudaStream_t st = as_stream(stream);
    bool ok = cudaMemcpyAsync(D->dev, &D->hdr, sizeof(DevProb), cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (ok) ok = launch_reduce_single(S->dev, D->dev, fixed, old_of_new, scratch, st) == cudaSuccess;
    DevProb back;
    if (ok) ok = cudaMemcpyAsync(&back, D->dev, sizeof(DevProb), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (ok) ok = cudaStreamSynchronize(st) == cudaSuccess;
    int32_t cptr[kMaxColours + 1] = {0};
    if (ok) ok = cudaMemcpy(cptr, back.cptr, sizeof(int32_t) * (back.ncol + 1), cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaFree(scratch);
    if (!ok) {
        cudaFree(D->blob);
        delete D;
        cudaGetLastError();
        return SPVAR_ECUDA;
    }
    D->hdr = back;
    D->jabs_max = S->jabs_max;  // the reduced couplers are a subset
    for (int c = 0; c < kMaxColours; ++c) D->csize[c] = c < back.ncol ? cptr[c + 1] - cptr[c] : 0;
    *out = reinterpret_cast<spvar_problem *>(D);
    return SPVAR_OK;
}

}  // extern "C"
