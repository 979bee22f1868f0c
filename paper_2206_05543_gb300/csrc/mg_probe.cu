// mg_probe.cu -- measured issue rate of the FP64 pipe (diagnostics).
//
// The FP64 kernels of this library are bound by the FP64 pipe, not by HBM,
// so their roofline needs the pipe's rate on the part at hand. The nominal
// figure (2 FP64 operations per SM per clock) is what the vendor quotes;
// this probe measures what an instruction mix actually issues at: many
// independent dependency chains per thread, one wave of blocks on every SM;
// each SM's busy cycles run from the earliest start to the latest end of the
// blocks it ran (clock64, compared only within one SM).
//
// Kinds (thread-level operations, 8 independent chains per thread):
//   0  DFMA with every operand in a register (a = fma(a, x, y), x and y
//      loaded from memory so that no compiler stage sees their values);
//   1  DADD (a = a + y);
//   2  DMUL (a = a * x);
//   3  DFMA with one operand a kernel parameter (constant bank).
// The paper has no counterpart; mg_measure_fp64_rate in include/mg.h.
#include <cuda_runtime.h>

#include <vector>

#include "../../include/mg.h"
#include "mg_ctx.h"
#include "mg_internal.h"

namespace mg {
namespace {

constexpr int kProbeThreads = 512;
constexpr int kChains = 8;

__device__ __forceinline__ unsigned sm_id()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

// span[2 s], span[2 s + 1]: earliest start and latest end (SM clock of SM s)
// of the blocks that ran on SM s; the busy cycles of an SM are their difference
template <int KIND>
__global__ void __launch_bounds__(kProbeThreads)
fp64_rate_kernel(const double *__restrict__ xy, double kparam, int iters, double *__restrict__ sink,
                 unsigned long long *__restrict__ span, int max_sm)
{
    const double x = xy[0], y = xy[1];
    double a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = xy[2] + (double)(threadIdx.x * kChains + j);
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) {
            if (KIND == 0) a[j] = __fma_rn(a[j], x, y);
            if (KIND == 1) a[j] = __dadd_rn(a[j], y);
            if (KIND == 2) a[j] = __dmul_rn(a[j], x);
            if (KIND == 3) a[j] = __fma_rn(a[j], kparam, y);
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == 1234.5) sink[0] = s;  // keeps the chains live; never true for these inputs
    const unsigned sm = sm_id();
    if (threadIdx.x == 0 && (int)sm < max_sm) {
        atomicMin(&span[2 * sm], (unsigned long long)t0);
        atomicMax(&span[2 * sm + 1], (unsigned long long)t1);
    }
}

template <int KIND>
cudaError_t launch_rate(const double *xy, int blocks, int iters, double *sink, unsigned long long *span, int max_sm,
                        cudaStream_t s)
{
    fp64_rate_kernel<KIND><<<blocks, kProbeThreads, 0, s>>>(xy, 1.0, iters, sink, span, max_sm);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace
}  // namespace mg

extern "C" mg_status mg_measure_fp64_rate(int kind, double *ops_per_sm_clk, double *sm_mhz)
{
    if (kind < 0 || kind > 3 || !ops_per_sm_clk) return MG_EINVAL;
    using namespace mg;
    const int sms = num_sms();
    int per_sm = 0;
    cudaError_t e = cudaSuccess;
    switch (kind) {
    case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_rate_kernel<0>, kProbeThreads, 0); break;
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_rate_kernel<1>, kProbeThreads, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_rate_kernel<2>, kProbeThreads, 0); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_rate_kernel<3>, kProbeThreads, 0); break;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    if (per_sm < 1) per_sm = 1;
    const int blocks = sms * per_sm;  // exactly one wave
    const int iters = 4096;
    const int max_sm = 1024;  // %smid bound (152 on this part)
    double *buf = nullptr;
    const size_t span_bytes = 2 * (size_t)max_sm * sizeof(unsigned long long);
    e = cudaMalloc(&buf, 4 * sizeof(double) + span_bytes);
    if (e != cudaSuccess) return cuda_fail(e);
    unsigned long long *span = (unsigned long long *)(buf + 4);
    std::vector<unsigned long long> init(2 * max_sm), got(2 * max_sm);
    for (int i = 0; i < max_sm; ++i) {
        init[2 * i] = ~0ull;
        init[2 * i + 1] = 0;
    }
    const double host_xy[4] = {1.0, 1.0 / 1024.0, 0.5, 0.0};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    float ms = 0.f;
    cudaStream_t s = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreate(&ev0);
    if (!e) e = cudaEventCreate(&ev1);
    if (!e) e = cudaMemcpyAsync(buf, host_xy, sizeof host_xy, cudaMemcpyHostToDevice, s);
    for (int rep = 0; rep < 2 && !e; ++rep) {  // the first launch warms up
        e = cudaMemcpyAsync(span, init.data(), span_bytes, cudaMemcpyHostToDevice, s);
        if (!e) e = cudaEventRecord(ev0, s);
        if (!e) {
            switch (kind) {
            case 0: e = launch_rate<0>(buf, blocks, iters, buf + 3, span, max_sm, s); break;
            case 1: e = launch_rate<1>(buf, blocks, iters, buf + 3, span, max_sm, s); break;
            case 2: e = launch_rate<2>(buf, blocks, iters, buf + 3, span, max_sm, s); break;
            default: e = launch_rate<3>(buf, blocks, iters, buf + 3, span, max_sm, s); break;
            }
        }
        if (!e) e = cudaEventRecord(ev1, s);
    }
    if (!e) e = cudaMemcpyAsync(got.data(), span, span_bytes, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (!e) e = cudaEventElapsedTime(&ms, ev0, ev1);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (s) cudaStreamDestroy(s);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(e);
    // busy cycles summed over the SMs that ran blocks, and the longest one
    double busy = 0.0, longest = 0.0;
    for (int i = 0; i < max_sm; ++i)
        if (got[2 * i + 1] > got[2 * i]) {
            const double c = (double)(got[2 * i + 1] - got[2 * i]);
            busy += c;
            longest = c > longest ? c : longest;
        }
    if (busy <= 0.0) return MG_ECUDA;
    const double ops = (double)blocks * kProbeThreads * (double)iters * kChains;
    *ops_per_sm_clk = ops / busy;
    if (sm_mhz) *sm_mhz = ms > 0.f ? longest / (ms * 1e3) : 0.0;
    return MG_OK;
}
