// mg_common.cuh -- shared device helpers of the sm_103a multigrid kernels.
//
// Rounding discipline. Every floating-point operation of the method is
// written with an explicit round-to-nearest intrinsic (__fma_rn, __dmul_rn,
// __fadd_rn and the like) so that the compiler cannot contract or reorder
// it. The operation order of each formula is fixed (it is written
// out next to each kernel) and is the same order in which the formulas of
// the paper are evaluated by an independent FP64 reference, so that FP64
// results agree to the last bit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mg {

// FP64 addition issued as a fused multiply-add by 1.0: fma(a, 1, b) rounds
// exactly like a + b (the product a * 1 is exact and the sum is rounded
// once), and on this part a DFMA whose operands are all registers issues at
// 1.9 FP64 operations per clock per SM against 1.6 for DADD (chain
// microbenchmark; the 2D FP64 solve got 9 % faster). The 1.0 is read from
// global memory so that neither compiler stage can see its value and turn
// the FMA back into an addition; a 1.0 that is a literal, an immediate or a
// kernel parameter ends up as DADD or as a constant-bank operand, which
// issue at 1.6.
static __device__ double k_unit_one = 1.0;
__device__ __forceinline__ double radd(double a, double b) { return __fma_rn(a, __ldg(&k_unit_one), b); }
// A constant or kernel-parameter FMA operand (stencil weight, SPAI
// coefficient) copied into a register once per thread: v * 1 with the opaque
// 1.0, exact. A DFMA that takes one operand from the constant bank issued at
// 1.6 per clock per SM like DADD in a microbenchmark, with all operands in
// registers at 1.9. Used where it measured faster (the 3D FP64 sweep and
// restriction, 3D FP64 solve -2.6 %); the 2D kernels, whose register budget
// is tight, got slower with it.
__device__ __forceinline__ double in_reg(double v) { return __dmul_rn(v, __ldg(&k_unit_one)); }
__device__ __forceinline__ float in_reg(float v) { return v; }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// IEEE 754 binary64 -> binary32 conversion, round to nearest, ties to even,
// on the integer pipe: for results in the normal binary32 range the 23 kept
// fraction bits are the top of the 52, and the 29 dropped bits decide the
// rounding (above half: up; exactly half: up when the kept part is odd); a
// carry out of the fraction moves into the exponent, which is the correct
// result, including the overflow to infinity. Zeros and binary64 subnormals
// give the zero of their sign; results that would be binary32 subnormal,
// NaNs and infinities take the hardware conversion. Equal to
// __double2float_rn bit for bit; on this part the hardware conversion issues
// on the FP64 pipe, which the FP64 residual kernels saturate.
//
// The hardware conversions are kept out of line: inlined, the compiler
// executed the conversion of the rare branch on every call (one F2F per
// point in the executed-opcode counts of the FP64 residual), and an F2F
// occupies the FP64 pipe that these kernels saturate.
static __device__ __noinline__ float narrow_rn_hw(double x) { return __double2float_rn(x); }
static __device__ __noinline__ double widen_hw(float x) { return (double)x; }

__device__ __forceinline__ float narrow_rn(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned e = (hi >> 20) & 0x7ffu;  // biased binary64 exponent
    if (e - 897u > 253u) {  // binary32 exponent outside 1..254
        // zeros and binary64 subnormals (below 2^-1022, far under half the
        // smallest binary32 subnormal) round to zero of the same sign
        if (e == 0) return __uint_as_float(hi & 0x80000000u);
        return narrow_rn_hw(x);
    }
    const unsigned frac = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1fffffffu;
    unsigned r = (hi & 0x80000000u) | ((e - 896u) << 23) | frac;
    r += (rest > 0x10000000u || (rest == 0x10000000u && (frac & 1u))) ? 1u : 0u;
    return __uint_as_float(r);
}
// IEEE 754 binary32 -> binary64 conversion (exact) on the integer pipe:
// for normal inputs the exponent is rebiased (+896) and the 23 fraction bits
// move to the top of the 52, zeros keep their sign; subnormals, infinities
// and NaNs take the hardware conversion (out of line, see above), which on
// this part issues on the FP64 pipe.
__device__ __forceinline__ double widen(float x)
{
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xffu;
    if (e - 1u > 253u) {
        if ((b & 0x7fffffffu) == 0) return __longlong_as_double((long long)((unsigned long long)b << 32));  // +-0
        return widen_hw(x);
    }
    return __longlong_as_double((long long)(((unsigned long long)(b & 0x80000000u) << 32) |
                                            ((unsigned long long)(e + 896u) << 52) |
                                            ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// value of an InT result stored as OutT (conversions round to nearest even)
template <typename OutT, typename InT>
__device__ __forceinline__ OutT to_out(InT x)
{
    if constexpr (sizeof(OutT) < sizeof(InT))
        return narrow_rn(x);
    else if constexpr (sizeof(OutT) > sizeof(InT))
        return widen(x);
    else
        return x;
}

// ---------------------------------------------------------------------------
// Sum of squares of FP64 values without FP64 arithmetic per term. The kernels
// that form an FP64 residual also return its squared 2-norm, and one DFMA
// per point for it was a thirteenth (sweep) to a sixth (refinement residual)
// of the work of a pipe that bounds them. Each normal r = (h + l) 2^(ex-1023)
// is split by integer operations into h = 1.f[51..29] (exact in FP32) and
// l = f[28..6] 2^-46 (exact in FP32; the last six fraction bits are dropped,
// 2^-46 of r); r^2 2^-2(ex-1023) = h^2 + 2hl (+ l^2, below 2^-45, dropped) is
// the FP32 pair (p, q) = (h h, fma(2h, l, fma(h, h, -p))). It is added to a
// float-float accumulator that carries its own power-of-two exponent (that of
// the largest term so far), so no magnitude under- or overflows. The caller
// flushes it (widened exactly, scaled on the exponent field, added to an FP64
// total) at a loop boundary of its own, at most every 32 terms, which keeps a
// counter out of the registers. Relative error of a thread's sum: about
// 2^-44 per term plus 2^-47 per addition (all terms are positive). Zeros and
// binary64 subnormals, whose squares are zero in FP64 as well, add nothing;
// an infinity or a NaN makes the sum NaN. The FP32 operations are written as
// intrinsics so that no contraction changes the two-sum.
// ---------------------------------------------------------------------------
constexpr int kSqNoExp = -8192;

struct SqSum {
    double total = 0.0;        // flushed part
    float hi = 0.f, lo = 0.f;  // pending part (hi + lo) 2^e
    int e = kSqNoExp;
};

__device__ __forceinline__ float sq_pow2f(int k)  // 2^k for -126 <= k <= 0
{
    return __int_as_float((k + 127) << 23);
}

// 2^k as a binary64 for -1022 <= k <= 1023
__device__ __forceinline__ double sq_pow2d(int k) { return __longlong_as_double((long long)(k + 1023) << 52); }

// v 2^k for a positive normal v: on the exponent field (exact) while the
// result is normal; below that by two hardware multiplies, rounding into the
// subnormal range as an FP64 square there would; infinity above
__device__ __forceinline__ double sq_ldexp(double v, int k)
{
    const long long b = __double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff) + k;
    if (e >= 0x7ff) return __longlong_as_double(0x7ff0000000000000LL);
    if (e <= 0) {
        const int k1 = k / 2;  // k >= -2044 (a square's exponent): both factors are normal
        return __dmul_rn(__dmul_rn(v, sq_pow2d(max(k1, -1022))), sq_pow2d(max(k - k1, -1022)));
    }
    return __longlong_as_double((b & ~(0x7ffLL << 52)) | ((long long)e << 52));
}

__device__ __forceinline__ void sq_flush(SqSum &a)
{
    if (a.hi > 0.f) a.total = __dadd_rn(a.total, sq_ldexp(__dadd_rn(widen(a.hi), widen(a.lo)), a.e));
    a.hi = 0.f;
    a.lo = 0.f;
    a.e = kSqNoExp;
}

__device__ __forceinline__ void sq_add(SqSum &a, double r)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(r);
    const int ex = (int)(bits >> 52) & 0x7ff;
    if (ex == 0) return;  // zero or subnormal
    if (ex == 0x7ff) {    // infinity or NaN
        a.total = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    const float h = __int_as_float(0x3f800000 | (int)((bits >> 29) & 0x7fffffu));
    const float m = __fsub_rn(__int_as_float(0x4b000000 | (int)((bits >> 6) & 0x7fffffu)), 8388608.f);
    const float l = __fmul_rn(m, 0x1p-46f);
    const float p = __fmul_rn(h, h);
    float tq = __fmaf_rn(__fadd_rn(h, h), l, __fmaf_rn(h, h, -p));
    float tp = p;
    const int et = 2 * (ex - 1023);
    if (et > a.e) {  // the accumulator moves to the new exponent
        const float sc = sq_pow2f(max(a.e - et, -126));
        a.hi = __fmul_rn(a.hi, sc);
        a.lo = __fmul_rn(a.lo, sc);
        a.e = et;
    } else {
        const float sc = sq_pow2f(max(et - a.e, -126));
        tp = __fmul_rn(tp, sc);
        tq = __fmul_rn(tq, sc);
    }
    // (hi, lo) += (tp, tq): two-sum of the heads, tails added, renormalised
    const float sh = __fadd_rn(a.hi, tp);
    const float bv = __fsub_rn(sh, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(sh, bv)), __fsub_rn(tp, bv));
    const float tl = __fadd_rn(__fadd_rn(err, a.lo), tq);
    a.hi = __fadd_rn(sh, tl);
    a.lo = __fsub_rn(tl, __fsub_rn(a.hi, sh));
}
__device__ __forceinline__ void sq_add(SqSum &a, float r) { sq_add(a, widen(r)); }

__device__ __forceinline__ double sq_value(SqSum &a)
{
    sq_flush(a);
    return a.total;
}

// The same interface with one FP64 FMA per term, for kernels whose register
// budget the accumulator above would overrun (they spill with it)
struct Fp64Sum {
    double total = 0.0;
};
__device__ __forceinline__ void sq_add(Fp64Sum &a, double r) { a.total = fma(r, r, a.total); }
__device__ __forceinline__ void sq_add(Fp64Sum &a, float r) { sq_add(a, widen(r)); }
__device__ __forceinline__ void sq_flush(Fp64Sum &) {}
__device__ __forceinline__ double sq_value(Fp64Sum &a) { return a.total; }

// fetch the 128-byte line at p into L2 (no register result, no fault on a
// valid address); callers pass addresses inside their arrays
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// x * 2^k for a power-of-two scale, done on the exponent field with integer
// instructions when x and the result are normal numbers (then the product is
// exact, so the result equals __dmul_rn(x, 2^k) bit for bit); zeros,
// subnormals, infinities and NaNs take the FP64 multiply. On this part the
// FP64 pipe is the bottleneck while the integer pipe is idle.
// scale2_ool keeps the multiply out of line for the reason given at
// narrow_rn: inlined, it was executed on every call in the 2D prolongation
// (0.43 DMUL per DFMA in the executed-opcode counts) and restriction (2D
// FP64 solve 56.8 -> 55.3 ms); the 3D FP64 kernels measured slower with it
// (209.4 -> 217.2 ms) and keep the inline form.
template <int K>
__device__ __forceinline__ double scale2(double x)
{
    const long long bits = __double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7ff);
    if (e + K >= 1 && e + K <= 0x7fe && e != 0 && e != 0x7ff)
        return __longlong_as_double(bits + ((long long)K << 52));
    return __dmul_rn(x, K >= 0 ? (double)(1ll << (K >= 0 ? K : 0)) : 1.0 / (double)(1ll << (K < 0 ? -K : 0)));
}
static __device__ __noinline__ double scale2_hw(double x, double s) { return __dmul_rn(x, s); }
template <int K>
__device__ __forceinline__ double scale2_ool(double x)
{
    const long long bits = __double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7ff);
    if (e + K >= 1 && e + K <= 0x7fe && e != 0 && e != 0x7ff)
        return __longlong_as_double(bits + ((long long)K << 52));
    return scale2_hw(x, K >= 0 ? (double)(1ll << (K >= 0 ? K : 0)) : 1.0 / (double)(1ll << (K < 0 ? -K : 0)));
}
// FP32: a plain multiply by the power of two (one FP32 instruction; the FP32
// pipes are not the limit of any FP32 kernel here). It rounds exactly like
// the exponent-field form wherever that form applies (the product is exact)
// and is that form's own fallback elsewhere, so the result is the same.
template <int K>
__device__ __forceinline__ float scale2(float x)
{
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
__device__ __forceinline__ double scale2_ool(double x, int k)
{
    const long long bits = __double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7ff);
    if (e + k >= 1 && e + k <= 0x7fe && e != 0 && e != 0x7ff) return __longlong_as_double(bits + ((long long)k << 52));
    return scale2_hw(x, __longlong_as_double((long long)(1023 + k) << 52));  // 2^k, |k| < 1022
}
__device__ __forceinline__ float scale2(float x, int k)
{
    return __fmul_rn(x, __int_as_float((127 + k) << 23));  // 2^k, |k| < 126
}
// FP32: the fallback multiply is on the FP32 pipe, inline is fine
template <int K>
__device__ __forceinline__ float scale2_ool(float x) { return scale2<K>(x); }
__device__ __forceinline__ float scale2_ool(float x, int k) { return scale2(x, k); }

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
constexpr int kRestrictThreads = 128;         // one coarse column per thread
constexpr int kRestrictCols = kRestrictThreads - 1;
constexpr int kProlongThreads = 256;

}  // namespace mg
