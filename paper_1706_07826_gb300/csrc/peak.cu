// Integer issue-rate probes: measured ceilings for the rooflines of the sweep
// kernels, whose time goes to 32-bit integer instructions (the Philox words,
// the byte-wise local fields, the carry-form acceptance) and not to memory.
//
// Each probe keeps kChains independent register chains per thread and runs
// kUnroll dependent steps of one instruction form per chain and iteration, on
// a grid of every CTA the SMs keep resident, so the rate is set by the issue
// ports and pipes, not by latency.  The forms:
//   0  three-input logic (lop3)                      integer ALU pipe
//   1  three-input add (a + b + c)                   integer ALU pipe
//   2  32-bit multiply-add, low half (mad.lo.u32)    FMA pipe
//   3  forms 0 and 2 on alternate chains             both pipes: the issue ceiling
//   4  32x32 -> 64-bit multiply (mul.wide.u32), its halves folded by one lop3
//                                                    FMA-heavy pipe + ALU
//   5  whole Philox4x32-10 blocks (20 wide multiplies, their folds and the
//      key schedule), one per chain group
// The count is of the probe's own operations (form 3: both kinds; form 4: the
// wide multiplies; form 5: Philox blocks), per thread, summed over the grid.
#include "philox.cuh"
#include "spvar_internal.h"

namespace spvar {
namespace {

__device__ uint32_t g_issue_sink;  // written only if a probe's result hits a value it never takes

constexpr int kChains = 16, kUnroll = 8, kThreads = 256;

__device__ __forceinline__ uint32_t lop3_x(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint32_t mad_x(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint32_t widefold_x(uint32_t a, uint32_t m, uint32_t c)
{
    uint64_t p;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(m));
    return lop3_x((uint32_t)p, (uint32_t)(p >> 32), c);
}

template <int FORM>
__global__ void __launch_bounds__(kThreads) k_issue(uint32_t s0, uint32_t s1, int iters)
{
    uint32_t a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = s0 * (threadIdx.x + 1u) + (uint32_t)c * kPhiloxW0 + blockIdx.x;
    if (FORM == 5) {
        // four chain groups of four counter words, one Philox block each per step
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int g = 0; g < kChains / 4; ++g) {
                const uint4 c = philox4x32_10(make_uint4(a[4 * g], a[4 * g + 1], a[4 * g + 2], a[4 * g + 3]), s1, s0);
                a[4 * g] = c.x;
                a[4 * g + 1] = c.y;
                a[4 * g + 2] = c.z;
                a[4 * g + 3] = c.w;
            }
        }
    } else {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int c = 0; c < kChains; ++c) {
                    const uint32_t b = a[(c + 5) % kChains];
                    if (FORM == 0) a[c] = lop3_x(a[c], b, s1);
                    if (FORM == 1) a[c] = a[c] + b + s1;
                    if (FORM == 2) a[c] = mad_x(a[c], s1, b);
                    if (FORM == 3) a[c] = (c & 1) ? mad_x(a[c], s1, b) : lop3_x(a[c], b, s1);
                    if (FORM == 4) a[c] = widefold_x(a[c], s1, b);
                }
            }
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc ^= a[c];
    if (acc == 0x7FFFFFFFu && s0 == 0u) g_issue_sink = acc;
}

const void *probe_kernel(int form)
{
    switch (form) {
    case 0: return reinterpret_cast<const void *>(k_issue<0>);
    case 1: return reinterpret_cast<const void *>(k_issue<1>);
    case 2: return reinterpret_cast<const void *>(k_issue<2>);
    case 3: return reinterpret_cast<const void *>(k_issue<3>);
    case 4: return reinterpret_cast<const void *>(k_issue<4>);
    case 5: return reinterpret_cast<const void *>(k_issue<5>);
    default: return nullptr;
    }
}

}  // namespace
}  // namespace spvar

using namespace spvar;

extern "C" int spvar_measure_issue_rate(int32_t form, int32_t iters, double *ops_per_s, double *ms, void *stream)
{
    if (!ops_per_s || iters < 1) return SPVAR_EINVAL;
    const void *k = probe_kernel(form);
    if (!k) return SPVAR_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0, occ = 0;
    SPVAR_CUDA_TRY(cudaGetDevice(&dev));
    SPVAR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SPVAR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kThreads, 0));
    const int grid = sms * std::max(occ, 1);
    uint32_t s0 = 0x2545F491u, s1 = 0x6C8E9CF5u;
    int warm = std::max(1, iters / 8);
    void *wargs[] = {(void *)&s0, (void *)&s1, (void *)&warm};
    void *args[] = {(void *)&s0, (void *)&s1, (void *)&iters};
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return SPVAR_ECUDA;
    }
    bool ok = cudaLaunchKernel(k, dim3(grid), dim3(kThreads), wargs, 0, st) == cudaSuccess &&
              cudaEventRecord(a, st) == cudaSuccess &&
              cudaLaunchKernel(k, dim3(grid), dim3(kThreads), args, 0, st) == cudaSuccess &&
              cudaEventRecord(b, st) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess;
    float t = 0.f;
    if (ok) ok = cudaEventElapsedTime(&t, a, b) == cudaSuccess;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (!ok || t <= 0.f) return SPVAR_ECUDA;
    const double per_iter = form == 5 ? (double)(kChains / 4) : (double)(kChains * kUnroll);
    *ops_per_s = (double)grid * kThreads * (double)iters * per_iter / (t * 1e-3);
    if (ms) *ms = t;
    return SPVAR_OK;
}
