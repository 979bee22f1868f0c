// mg_common.cuh -- shared device helpers of the sm_103a multigrid kernels.
//
// Rounding discipline. Every floating-point operation of the method is
// written with an explicit round-to-nearest intrinsic (__dadd_rn, __dmul_rn,
// __fma_rn and their float forms) so that the compiler cannot contract or
// reorder it. The operation order of each formula is fixed (it is written
// out next to each kernel) and is the same order in which the formulas of
// the paper are evaluated by an independent FP64 reference, so that FP64
// results agree to the last bit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mg {

__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// x * 2^k for a power-of-two scale, done on the exponent field with integer
// instructions when x and the result are normal numbers (then the product is
// exact, so the result equals __dmul_rn(x, 2^k) bit for bit); zeros,
// subnormals, infinities and NaNs take the FP64 multiply. On this part the
// FP64 pipe is the bottleneck while the integer pipe is idle.
template <int K>
__device__ __forceinline__ double scale2(double x)
{
    const long long bits = __double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7ff);
    if (e + K >= 1 && e + K <= 0x7fe && e != 0 && e != 0x7ff)
        return __longlong_as_double(bits + ((long long)K << 52));
    return __dmul_rn(x, K >= 0 ? (double)(1ll << (K >= 0 ? K : 0)) : 1.0 / (double)(1ll << (K < 0 ? -K : 0)));
}
template <int K>
__device__ __forceinline__ float scale2(float x)
{
    const int bits = __float_as_int(x);
    const int e = (bits >> 23) & 0xff;
    if (e + K >= 1 && e + K <= 0xfe && e != 0 && e != 0xff) return __int_as_float(bits + (K << 23));
    return __fmul_rn(x, K >= 0 ? (float)(1 << (K >= 0 ? K : 0)) : 1.0f / (float)(1 << (K < 0 ? -K : 0)));
}
// runtime exponent form (k = -2 log2 N for h^2 = 1/N^2)
__device__ __forceinline__ double scale2(double x, int k)
{
    const long long bits = __double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7ff);
    if (e + k >= 1 && e + k <= 0x7fe && e != 0 && e != 0x7ff) return __longlong_as_double(bits + ((long long)k << 52));
    return __dmul_rn(x, __longlong_as_double((long long)(1023 + k) << 52));  // 2^k, |k| < 1022
}
__device__ __forceinline__ float scale2(float x, int k)
{
    const int bits = __float_as_int(x);
    const int e = (bits >> 23) & 0xff;
    if (e + k >= 1 && e + k <= 0xfe && e != 0 && e != 0xff) return __int_as_float(bits + (k << 23));
    return __fmul_rn(x, __int_as_float((127 + k) << 23));  // 2^k, |k| < 126
}

// Sum of `v` over the block into *dst (fixed order: warp butterfly, then the
// warp sums in warp order by warp 0). Called by every thread of the block.
template <int NTHREADS>
__device__ __forceinline__ void block_sum_store(double v, double *dst)
{
    static_assert(NTHREADS % 32 == 0 && NTHREADS <= 1024, "block size");
    __shared__ double warp_sums[NTHREADS / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) warp_sums[w] = v;
    __syncthreads();
    if (w == 0) {
        double s = l < NTHREADS / 32 ? warp_sums[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (l == 0) *dst = s;
    }
}

// Exponent of h^2 = 1/(n+1)^2 for a level with n = 2^m - 1 points per axis.
__host__ __device__ inline int h2_exponent(int n)
{
    int m = 0;
    while ((1 << m) < n + 1) ++m;
    return -2 * m;
}

// Grid sizes of the marching kernels (host and device agree on them).
constexpr int kSweepThreads = 256;            // threads per sweep block (one column each)
constexpr int kSweepCols = kSweepThreads - 2; // output columns per sweep block
constexpr int kRestrictThreads = 256;         // one coarse column per thread
constexpr int kRestrictCols = kRestrictThreads - 1;
constexpr int kProlongThreads = 256;

}  // namespace mg
