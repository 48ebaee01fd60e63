// Allocation-free fold/compact: spvar_reduce_noalloc.
//
// For callers that must not allocate device memory while they run -- for
// example code that executes inside a memory-pool budget that is already
// fully committed, or an embedding runtime that owns every allocation and
// forbids cudaMalloc/cudaFree (and allocating library routines) after
// start-up.  It computes the same reduced problem as spvar_reduce, but writes
// it as plain CSR arrays into buffers the caller provides, and keeps its
// working arrays in one statically sized device array of this file instead
// of allocating them.
//
// The static array exists once per device that loads the library and lives
// until the process exits.  Its device address is looked up with
// cudaGetSymbolAddress on the first call made on each device (with that
// device current); make that first call before any stream capture.  Every
// call shares the array: calls that can overlap on the GPU (different
// streams, or concurrent host threads) race on it and must be serialised by
// the caller.  Nothing in the array needs to start at zero: each call writes
// every entry it later reads.
#include <mutex>

#include "persist.cuh"

namespace spvar {
namespace {

// new index of every old spin, then the free-free row lengths: 2 x n ints
__device__ __align__(256) int32_t g_reduce_scratch[2 * SPVAR_NOALLOC_MAX_N];

std::mutex g_addr_mu;
int32_t *g_addr[64] = {nullptr};

int scratch_address(int32_t **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SPVAR_ECUDA;
    std::lock_guard<std::mutex> g(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_reduce_scratch) != cudaSuccess) {
            cudaGetLastError();
            return SPVAR_ECUDA;
        }
        g_addr[dev] = static_cast<int32_t *>(p);
    }
    *out = g_addr[dev];
    return SPVAR_OK;
}

// Fold the fixed spins into h and the offset and write the CSR of the free
// spins (renumbered in increasing old index) to the caller's arrays.  One
// 1024-thread CTA.
__global__ void __launch_bounds__(kBigBlock)
    k_reduce_csr(const DevProb *S, const int8_t *fixed, int32_t *row_ptr, int32_t *col, int32_t *val,
                 int32_t *h_out, int64_t *offset_out, int32_t *old_of_new, int32_t *n_out, int32_t *scratch)
{
    __shared__ int s_warp[32];
    __shared__ unsigned long long s_off;
    const int tid = threadIdx.x, B = blockDim.x;
    const int n = S->n;
    int32_t *new_of_old = scratch;
    int32_t *rowcnt = scratch + SPVAR_NOALLOC_MAX_N;
    if (tid == 0) s_off = 0ull;
    __syncthreads();

    int carry = 0;
    for (int base = 0; base < n; base += B) {
        const int i = base + tid;
        const int f = (i < n && fixed[i] == 0) ? 1 : 0;
        int tot;
        const int ex = block_scan_excl(f, s_warp, &tot);
        if (i < n) {
            new_of_old[i] = f ? carry + ex : -1;
            if (f) old_of_new[carry + ex] = i;
        }
        carry += tot;
    }
    const int m = carry;
    __syncthreads();

    long long off_part = 0;
    for (int i = tid; i < n; i += B) {
        const int vi = fixed[i];
        long long hf = S->h[i];
        int nfree = 0;
        for (int p = S->row_ptr[i]; p < S->row_ptr[i + 1]; ++p) {
            const int j = S->col[p];
            const int vj = fixed[j];
            if (vi) {
                if (vj && j > i) off_part += (long long)S->val[p] * vi * vj;
            } else {
                if (vj) hf += (long long)S->val[p] * vj;
                else ++nfree;
            }
        }
        if (vi) {
            off_part += (long long)S->h[i] * vi;
        } else {
            const int a = new_of_old[i];
            h_out[a] = (int32_t)hf;
            rowcnt[a] = nfree;
        }
    }
    atomicAdd(&s_off, (unsigned long long)off_part);
    __syncthreads();

    carry = 0;
    for (int base = 0; base < m; base += B) {
        const int a = base + tid;
        const int c = (a < m) ? rowcnt[a] : 0;
        int tot;
        const int ex = block_scan_excl(c, s_warp, &tot);
        if (a < m) row_ptr[a] = carry + ex;
        carry += tot;
    }
    if (tid == 0) row_ptr[m] = carry;
    __syncthreads();

    for (int a = tid; a < m; a += B) {
        const int i = old_of_new[a];
        int q = row_ptr[a];
        for (int p = S->row_ptr[i]; p < S->row_ptr[i + 1]; ++p) {
            const int j = S->col[p];
            if (fixed[j] == 0) {
                col[q] = new_of_old[j];
                val[q] = S->val[p];
                ++q;
            }
        }
    }
    if (tid == 0) {
        *n_out = m;
        *offset_out = S->offset + (long long)s_off;
    }
}

}  // namespace
}  // namespace spvar

using namespace spvar;

extern "C" int spvar_reduce_noalloc(const spvar_problem *p, const int8_t *fixed, int32_t *row_ptr,
                                    int32_t *col, int32_t *val, int32_t *h, int64_t *offset,
                                    int32_t *old_of_new, int32_t *n_out, void *stream)
{
    if (!p) return SPVAR_EINVAL;
    const Problem *S = reinterpret_cast<const Problem *>(p);
    const DevProb &H = S->hdr;
    if (H.n > SPVAR_NOALLOC_MAX_N) return SPVAR_ELIMIT;
    if (!row_ptr || !offset || !n_out || (H.n > 0 && (!fixed || !h || !old_of_new)) ||
        (H.nnz > 0 && (!col || !val)))
        return SPVAR_EINVAL;
    int32_t *scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc != SPVAR_OK) return rc;
    // launched through cudaLaunchKernel so that its own status is checked, not an
    // earlier error left pending on this thread by unrelated work
    const DevProb *src = S->dev;
    void *args[] = {(void *)&src, (void *)&fixed, (void *)&row_ptr, (void *)&col, (void *)&val, (void *)&h,
                    (void *)&offset, (void *)&old_of_new, (void *)&n_out, (void *)&scratch};
    const cudaError_t e = cudaLaunchKernel(reinterpret_cast<const void *>(k_reduce_csr), dim3(1), dim3(kBigBlock),
                                           args, 0, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SPVAR_OK : SPVAR_ECUDA;
}
