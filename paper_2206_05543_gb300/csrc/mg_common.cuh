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

// Grid sizes of the marching kernels (host and device agree on them).
constexpr int kSweepThreads = 256;            // threads per sweep block (one column each)
constexpr int kSweepCols = kSweepThreads - 2; // output columns per sweep block
constexpr int kRestrictThreads = 256;         // one coarse column per thread
constexpr int kRestrictCols = kRestrictThreads - 1;
constexpr int kProlongThreads = 256;

}  // namespace mg
