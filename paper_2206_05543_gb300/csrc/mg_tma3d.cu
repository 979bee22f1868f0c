// mg_tma3d.cu -- 3D FP32 SPAI sweep with TMA-staged planes (padded layout).
//
// A z-marching 3D sweep in which every thread loads its own u and b values
// keeps too few bytes in flight to cover HBM latency. Here one thread issues
// tensor-memory-accelerator copies (cp.async.bulk.tensor, completion counted
// by mbarriers) of whole u and b tiles (halo included) into rings of shared
// memory slots kAhead planes ahead of the computation, so the copy engine
// keeps HBM busy while the block computes. Out-of-range rows and planes of a
// box are filled with zeros by the hardware: the Dirichlet ghost value.
//
// Per plane zz a block
//   A. forms the scaled residual of plane zz (u planes zz-1..zz+1, b plane zz)
//      and stores it in a two-plane shared ring,
//   B. synchronises (u plane zz-1 and b plane zz are dead from here on),
//   C. refills those two slots with copies of planes kAhead+1 further on,
//   D. applies the SPAI stencil to the residual of plane zz-1 and writes it,
//   E. waits for the planes the next step reads, and synchronises.
// Every wait is bounded by a clock limit; on expiry the block sets an error
// word (the host reports MG_ETIMEOUT), waits, again bounded, for its copies
// still in flight (best effort: a drain that also expires sets a second bit),
// and returns.
//
// Formula and rounding order: those of the compact 3D sweep (Sec. 3.2,
// u' = u + c0 r + c1 (sum of the six face neighbours of r)), so results are
// bit-identical to it.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <mutex>

#include "mg_common.cuh"
#include "mg_internal.h"

namespace mg {

namespace {

constexpr int kTX = 32;                   // threads along x, 4 columns each
constexpr int kTCols = 4 * kTX;           // 128 output columns
constexpr int kTTY = 14;                  // output rows
constexpr int kTRows = kTTY + 2;          // residual rows (16)
constexpr int kTThreads = kTX * kTRows;   // 512 consumer threads (+ one helper warp)
constexpr int kTW = kTCols + 8;           // tile width: 4 extra columns each side (136)
constexpr int kURows = kTRows + 2;        // u rows (18)
constexpr int kAhead = 2;                 // planes of prefetch beyond the next step
constexpr int kUSlots = 3 + kAhead, kBSlots = 1 + kAhead;
constexpr int kUBoxBytes = kURows * kTW * 4, kBBoxBytes = kTRows * kTW * 4;
constexpr int kUSlotBytes = (kUBoxBytes + 127) / 128 * 128;
constexpr int kBSlotBytes = (kBBoxBytes + 127) / 128 * 128;
constexpr int kRSlotBytes = kBSlotBytes;  // residual plane: kTRows x kTW
constexpr int kSmemBytes = kUSlots * kUSlotBytes + kBSlots * kBSlotBytes + 2 * kRSlotBytes + 128;
constexpr int kAccBytes = kTRows * kTCols * 4;  // ACC64 staging: one 128-float row per consumer warp
constexpr long long kWaitCycles = 1LL << 31;  // about one second

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ float4 ld4s(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float &f4(float4 &v, int k) { return (&v.x)[k]; }
__device__ __forceinline__ float cf4(const float4 &v, int k) { return (&v.x)[k]; }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// false when the phase did not complete within kWaitCycles
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity)
{
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// The tensor maps view a padded level array (see pitch3) as a pitch x (n+2) x
// (n+2) box starting at element (-4, -1, -1): element (x, y, z) has tensor
// coordinates (x + 4, y + 1, z + 1). A u tile of block (x0, y0) covers
// columns x0-4 .. x0+131 and rows y0-2 .. y0+15; a b tile rows y0-1 .. y0+14.
//
// Warps 0..15 (consumers) own residual row ty = warp, four columns per lane.
// Warp 16 (helper) computes the 32 residuals of the two halo columns
// (lane & 15 = row, lane >> 4 = side), and its lane 0 drives the copies.
//
// ACC64 (the last post-sweep of a refinement cycle): instead of storing the
// FP32 result, add it to the caller's FP64 solution (compact n^3 array),
// whose values are loaded at the start of the step that updates them.
constexpr int kF64Lead = 2;  // planes between the L2 prefetch and the load of an FP64 row (2 and 4 alike)
template <bool ZERO_U, bool ACC64 = false>
__global__ void __launch_bounds__(kTThreads + 32, 2)
sweep3d_tma_kernel(const __grid_constant__ CUtensorMap tu, const __grid_constant__ CUtensorMap tb,
                   float *__restrict__ out, Pitch3 g, int Z, float c0, float c1, int *__restrict__ err,
                   double *__restrict__ u64, int inject)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // 128-byte alignment by indexing (not by integer casts), so that the
    // compiler still sees shared-memory pointers
    unsigned char *base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    float *const su = (float *)base;
    float *const sb = (float *)(base + kUSlots * kUSlotBytes);
    float *const sr = (float *)(base + kUSlots * kUSlotBytes + kBSlots * kBSlotBytes);
    __shared__ __align__(8) unsigned long long bars[kUSlots + kBSlots];
    __shared__ int s_fail;
    constexpr int kUF = kUSlotBytes / 4, kBF = kBSlotBytes / 4, kRF = kRSlotBytes / 4;

    const int n = g.n, t = threadIdx.x;
    const bool helper = t >= kTThreads;
    const int x0 = blockIdx.x * kTCols, y0 = blockIdx.y * kTTY;
    const int z0 = blockIdx.z * Z, z1 = min(z0 + Z, n);
    // consumer: row ty, columns x..x+3; helper: row ty, halo column x
    const int lane = t & 31;
    const int ty = helper ? (lane & 15) : t / kTX;
    const int tx = helper ? 0 : t % kTX;
    const int yr = y0 - 1 + ty;
    const bool yin = yr >= 0 && yr < n;
    const int x = helper ? ((lane >> 4) ? x0 + kTCols : x0 - 1) : x0 + 4 * tx;
    const int col = helper ? ((lane >> 4) ? kTCols + 4 : 3) : 4 + 4 * tx;  // tile column of x
    const int ib = ty * kTW + col;        // in a b / residual tile
    const int iu = (ty + 1) * kTW + col;  // in a u tile
    unsigned xmask = 0;                   // bit k: column x + k is an interior point of row yr
    for (int k = 0; k < (helper ? 1 : 4); ++k)
        if (yin && x + k >= 0 && x + k < n) xmask |= 1u << k;
    const bool own_row = !helper && ty >= 1 && ty <= kTTY && yin;
    const bool producer = helper && lane == 0;

    // ring offsets (floats) of u planes zz-1, zz, zz+1 and of b plane zz;
    // plane p sits in slot (p - first) % slots, its k-th fill has parity k & 1
    const int ufirst = z0 - 2, bfirst = z0 - 1, ulast = z1 + 1, blast = z1;
    int om = 0, oc = kUF, op = 2 * kUF, ob = 0;
    auto ubar = [&](int p) { return smem_u32(&bars[(p - ufirst) % kUSlots]); };
    auto bbar = [&](int p) { return smem_u32(&bars[kUSlots + (p - bfirst) % kBSlots]); };
    auto upar = [&](int p) { return (unsigned)(((p - ufirst) / kUSlots) & 1); };
    auto bpar = [&](int p) { return (unsigned)(((p - bfirst) / kBSlots) & 1); };
    // producer state: planes issued and planes whose copy has landed
    int u_issued = ufirst - 1, u_done = ufirst - 1, b_issued = bfirst - 1, b_done = bfirst - 1;
    // inject (test hook): the first copy's barrier expects 16 bytes that never come
    auto issue_u = [&](int p) {
        mbar_expect(ubar(p), kUBoxBytes + (p == ufirst ? inject : 0));
        tma_load_3d(smem_u32(su + ((p - ufirst) % kUSlots) * kUF), &tu, x0, y0 - 1, p + 1, ubar(p));
        u_issued = p;
    };
    auto issue_b = [&](int p) {
        mbar_expect(bbar(p), kBBoxBytes + (ZERO_U && p == bfirst ? inject : 0));
        tma_load_3d(smem_u32(sb + ((p - bfirst) % kBSlots) * kBF), &tb, x0, y0, p + 1, bbar(p));
        b_issued = p;
    };
    auto wait_u = [&](int p) {
        if (!mbar_wait(ubar(p), upar(p))) return false;
        u_done = p;
        return true;
    };
    auto wait_b = [&](int p) {
        if (!mbar_wait(bbar(p), bpar(p))) return false;
        b_done = p;
        return true;
    };

    if (producer) {
        for (int i = 0; i < kUSlots + kBSlots; ++i) mbar_init(smem_u32(&bars[i]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        bool ok = true;
        if (!ZERO_U)
            for (int p = ufirst; p <= min(z0 + kAhead, ulast); ++p) issue_u(p);
        for (int p = bfirst; p <= min(z0 - 1 + kAhead, blast); ++p) issue_b(p);
        if (!ZERO_U)
            for (int p = ufirst; ok && p <= z0; ++p) ok = wait_u(p);
        ok = ok && wait_b(bfirst);
        s_fail = ok ? 0 : 1;
    }
    __syncthreads();

    long di = g.off + (long)(z0 - 2) * g.plane + (long)yr * g.pitch + x;  // (x, yr, zz-1) at step zz
    float4 rm = make_float4(0.f, 0.f, 0.f, 0.f), rc = rm;
    // ACC64: each consumer warp stages its 128 results (behind the residual
    // ring) and lane l updates the FP64 columns x0 + l + 32 k, so that every
    // FP64 access of the warp covers 256 contiguous bytes
    float *const sacc = sr + 2 * kRF + (helper ? 0 : ty) * kTCols;
    for (int zz = z0 - 1; zz <= z1 && !s_fail; ++zz) {
        double u64v[4] = {0.0, 0.0, 0.0, 0.0};
        if (ACC64 && zz > z0 && own_row) {
            const double *ur = u64 + ((long)(zz - 1) * n + yr) * n + x0 + lane;
            for (int k = 0; k < 4; ++k)
                if (x0 + lane + 32 * k < n) u64v[k] = ur[32 * k];
            // the row of plane zz - 1 + kF64Lead into L2 (lanes 0..7: one
            // 128-byte line each of the warp's 1 KB), for the load above later
            const int zp = zz - 1 + kF64Lead;
            if (lane < 8 && zp < z1)
                prefetch_l2(u64 + ((long)zp * n + yr) * n + min(x0 + 16 * lane, n - 1));
        }
        // A. scaled residual of plane zz (zero outside the interior)
        const unsigned m = (zz >= 0 && zz < n) ? xmask : 0u;
        const float *bp = sb + ob;
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f), um4 = r;
        if (helper) {
            float rh;
            if (!ZERO_U) {
                const float *uc = su + oc + iu;
                rh = radd(rfma(-6.f, uc[0], bp[ib]),
                          radd(radd(radd(uc[-1], uc[1]), radd(uc[-kTW], uc[kTW])), radd(su[om + iu], su[op + iu])));
            } else {
                rh = bp[ib];
            }
            sr[(zz & 1) * kRF + ib] = (m & 1u) ? rh : 0.f;
        } else {
            if (!ZERO_U) {
                const float *uc = su + oc + iu;
                const float4 b4 = ld4s(bp + ib), c4 = ld4s(uc);
                const float4 s4 = ld4s(uc - kTW), n4 = ld4s(uc + kTW), u4 = ld4s(su + op + iu);
                um4 = ld4s(su + om + iu);
                const float w[6] = {uc[-1], c4.x, c4.y, c4.z, c4.w, uc[4]};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float ss = radd(radd(radd(w[k], w[k + 2]), radd(cf4(s4, k), cf4(n4, k))),
                                          radd(cf4(um4, k), cf4(u4, k)));
                    f4(r, k) = radd(rfma(-6.f, w[k + 1], cf4(b4, k)), ss);
                }
            } else {
                r = ld4s(bp + ib);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (!((m >> k) & 1u)) f4(r, k) = 0.f;
            *reinterpret_cast<float4 *>(sr + (zz & 1) * kRF + ib) = r;
        }
        // B.
        __syncthreads();
        // C. refill the slots of u plane zz-1 and b plane zz
        if (producer) {
            if (!ZERO_U && zz + 2 + kAhead <= ulast) issue_u(zz + 2 + kAhead);
            if (zz + 1 + kAhead <= blast) issue_b(zz + 1 + kAhead);
        }
        // D. SPAI update of plane zz-1
        if (zz > z0 && own_row) {
            const float *p = sr + ((zz - 1) & 1) * kRF + ib;
            const float4 pc = ld4s(p), ps = ld4s(p - kTW), pn = ld4s(p + kTW);
            const float w[6] = {p[-1], pc.x, pc.y, pc.z, pc.w, p[4]};
            float4 o;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float E = radd(radd(radd(w[k], w[k + 2]), radd(cf4(ps, k), cf4(pn, k))),
                                     radd(cf4(rm, k), cf4(r, k)));
                const float b0 = ZERO_U ? rmul(c0, cf4(rc, k)) : rfma(c0, cf4(rc, k), cf4(um4, k));
                f4(o, k) = rfma(c1, E, b0);
            }
            if (ACC64) {
                *reinterpret_cast<float4 *>(sacc + 4 * lane) = o;
                __syncwarp();
                double *ur = u64 + ((long)(zz - 1) * n + yr) * n + x0 + lane;
                for (int k = 0; k < 4; ++k)
                    if (x0 + lane + 32 * k < n) ur[32 * k] = __dadd_rn(u64v[k], widen(sacc[lane + 32 * k]));
                __syncwarp();
            } else {
                float *dst = out + di;
                if (x + 3 < n) {
                    *reinterpret_cast<float4 *>(dst) = o;
                } else {
                    for (int k = 0; k < 4; ++k)
                        if (x + k < n) dst[k] = f4(o, k);
                }
            }
        }
        rm = rc;
        rc = r;
        di += g.plane;
        om = oc;
        oc = op;
        op = op + kUF == kUSlots * kUF ? 0 : op + kUF;
        ob = ob + kBF == kBSlots * kBF ? 0 : ob + kBF;
        // E. planes of the next step
        if (producer && zz < z1) {
            bool ok = ZERO_U || wait_u(zz + 2);
            ok = ok && wait_b(zz + 1);
            if (!ok) s_fail = 1;
        }
        __syncthreads();
    }
    if (producer && s_fail) {
        atomicOr(err, 1);
        // shared memory should not be released while a copy may still land in
        // it: wait for the copies in flight, each wait again bounded. This is
        // best effort: if a drain wait expires too, bit 1 of the error word
        // tells the host that a copy may land after the block has ended.
        bool drained = true;
        for (int p = u_done + 1; drained && p <= u_issued; ++p) drained = mbar_wait(ubar(p), upar(p));
        for (int p = b_done + 1; drained && p <= b_issued; ++p) drained = mbar_wait(bbar(p), bpar(p));
        if (!drained) atomicOr(err, 2);
    }
}

// ---------------------------------------------------------------------------
// Residual + full weighting on TMA-staged planes (formula and order as
// resrestrict3d_kernel), as a warp pipeline without block barriers. A block
// owns 32 x 16 coarse columns. Consumer warp w (of 8) owns coarse rows
// jc0 + 2w, jc0 + 2w + 1 and lane l the coarse column ic = ic0 + l; per
// fine plane f the warp walks its 5 fine rows y = 2 (jc0 + 2w) + r with a
// rolling window of u rows in registers: lane l forms the residuals at fine
// columns 2ic + 1 and 2ic + 2, takes the one at 2ic from lane l - 1 by a
// shuffle (lane 0 computes it), does the x pass, the y pass every second row
// and the z pass every second plane, all in registers. The helper warp's lane
// 0 fills rings of u planes (72 x 35 boxes from fine column 2 ic0 - 4, row
// 2 jc0 - 1) and b planes (72 x 33 from row 2 jc0), one plane ahead of
// the consumers' next step, through "full" mbarriers
// (expect_tx); each consumer warp releases a slot through an "empty"
// mbarrier (one arrival per warp) once it has read it. Every wait is bounded.
// ---------------------------------------------------------------------------
constexpr int kRX = 32;                  // coarse columns per block (one per lane)
constexpr int kRWarps = 8;               // consumer warps
constexpr int kRRows = 2;                // coarse rows per consumer warp
constexpr int kRY = kRWarps * kRRows;    // 16 coarse rows per block
constexpr int kRW = 72;                  // box width: fine columns 2 ic0 - 4 .. 2 ic0 + 67
constexpr int kRUR = 2 * kRY + 3;        // 35 u rows: fine rows 2 jc0 - 1 .. 2 jc0 + 33
constexpr int kRBR = 2 * kRY + 1;        // 33 b rows: fine rows 2 jc0 .. 2 jc0 + 32
constexpr int kRThreads = 32 * (kRWarps + 1);
// one plane of prefetch (smaller rings: three blocks per SM; measured faster)
constexpr int kRUSlots = 4, kRBSlots = 2;
constexpr int kRUBox = kRUR * kRW * 4, kRBBox = kRBR * kRW * 4;
constexpr int kRUSlotBytes = (kRUBox + 127) / 128 * 128, kRBSlotBytes = (kRBBox + 127) / 128 * 128;
constexpr int kRSmemBytes = kRUSlots * kRUSlotBytes + kRBSlots * kRBSlotBytes + 128;

__device__ __forceinline__ void mbar_arrive(unsigned bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ float2 ld2s(const float *p) { return *reinterpret_cast<const float2 *>(p); }

__global__ void __launch_bounds__(kRThreads)
resrestrict3d_tma_kernel(const __grid_constant__ CUtensorMap tu, const __grid_constant__ CUtensorMap tb,
                         float *__restrict__ bc, Pitch3 g, Pitch3 gc, int Zc, int *__restrict__ err, int inject)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    float *const su = (float *)base;
    float *const sb = (float *)(base + kRUSlots * kRUSlotBytes);
    // full[0 .. kRUSlots + kRBSlots), then empty[same]
    __shared__ __align__(8) unsigned long long bars[2 * (kRUSlots + kRBSlots)];
    __shared__ volatile int s_fail;
    constexpr int kUF = kRUSlotBytes / 4, kBF = kRBSlotBytes / 4, kNB = kRUSlots + kRBSlots;

    const int n = g.n, nc = gc.n, t = threadIdx.x, warp = t / 32, lane = t % 32;
    const int ic0 = blockIdx.x * kRX, jc0 = blockIdx.y * kRY;
    const int fx0 = 2 * ic0, fy0 = 2 * jc0;
    const int kc0 = blockIdx.z * Zc, kc1 = min(kc0 + Zc, nc);
    const int f0 = 2 * kc0, f1 = 2 * kc1;
    const int ufirst = f0 - 1, bfirst = f0, blast = f1;  // u planes f0 - 1 .. f1 + 1
    auto uslot = [&](int p) { return (p - ufirst) % kRUSlots; };
    auto bslot = [&](int p) { return (p - bfirst) % kRBSlots; };
    auto upar = [&](int p) { return (unsigned)(((p - ufirst) / kRUSlots) & 1); };
    auto bpar = [&](int p) { return (unsigned)(((p - bfirst) / kRBSlots) & 1); };
    auto full_u = [&](int p) { return smem_u32(&bars[uslot(p)]); };
    auto full_b = [&](int p) { return smem_u32(&bars[kRUSlots + bslot(p)]); };
    auto empty_u = [&](int p) { return smem_u32(&bars[kNB + uslot(p)]); };
    auto empty_b = [&](int p) { return smem_u32(&bars[kNB + kRUSlots + bslot(p)]); };

    if (t == 0) {
        for (int i = 0; i < kNB; ++i) {
            mbar_init(smem_u32(&bars[i]), 1);
            mbar_init(smem_u32(&bars[kNB + i]), kRWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    __syncthreads();  // the only block barrier: barriers initialised

    if (warp == kRWarps) {
        // ---------------- producer (one thread) ----------------
        if (lane != 0) return;
        int u_last = ufirst - 1, b_last = bfirst - 1;  // last plane issued
        bool ok = true;
        // a slot is refilled once every consumer warp has released its previous plane
        auto issue_u = [&](int p) {
            if (p - kRUSlots >= ufirst && !mbar_wait(empty_u(p), upar(p - kRUSlots))) return false;
            mbar_expect(full_u(p), kRUBox + (p == ufirst ? inject : 0));
            tma_load_3d(smem_u32(su + uslot(p) * kUF), &tu, fx0, fy0, p + 1, full_u(p));
            u_last = p;
            return true;
        };
        auto issue_b = [&](int p) {
            if (p - kRBSlots >= bfirst && !mbar_wait(empty_b(p), bpar(p - kRBSlots))) return false;
            mbar_expect(full_b(p), kRBBox);
            tma_load_3d(smem_u32(sb + bslot(p) * kBF), &tb, fx0, fy0 + 1, p + 1, full_b(p));
            b_last = p;
            return true;
        };
        ok = issue_u(ufirst) && issue_u(ufirst + 1);
        for (int q = bfirst; ok && q <= blast; ++q) {
            ok = issue_u(q + 1) && issue_b(q);  // consumer step q reads u(q - 1 .. q + 1), b(q)
            if (s_fail) ok = false;
        }
        if (!ok) {
            s_fail = 1;
            atomicOr(err, 1);
        }
        // before the block ends every issued copy should have landed; each
        // wait is bounded, and bit 1 of the error word records a drain that
        // gave up (a copy may then land after the block has ended)
        bool drained = true;
        for (int p = max(ufirst, u_last - kRUSlots + 1); drained && p <= u_last; ++p)
            drained = mbar_wait(full_u(p), upar(p));
        for (int p = max(bfirst, b_last - kRBSlots + 1); drained && p <= b_last; ++p)
            drained = mbar_wait(full_b(p), bpar(p));
        if (!drained) atomicOr(err, 3);
        return;
    }

    // ---------------- consumers ----------------
    const int l = lane;
    const int ic = ic0 + l;
    const int cu = 2 * l + 4;       // box column of fine 2 ic
    const int X0 = fx0 + 2 * l;     // fine 2 ic
    const int ry0 = 2 * kRRows * warp;  // first fine row of this warp relative to fy0
    float t2a[kRRows], t2b[kRRows];
#pragma unroll
    for (int m = 0; m < kRRows; ++m) t2a[m] = t2b[m] = 0.f;
    bool ok = true;
    auto wait_full = [&](unsigned bar, unsigned par) {
        if (!mbar_wait(bar, par)) {
            s_fail = 1;
            atomicOr(err, 1);
            return false;
        }
        return true;
    };
    ok = wait_full(full_u(ufirst), upar(ufirst)) && wait_full(full_u(ufirst + 1), upar(ufirst + 1));
    for (int f = f0; ok && f <= f1; ++f) {
        ok = wait_full(full_u(f + 1), upar(f + 1)) && wait_full(full_b(f), bpar(f));
        if (!ok || s_fail) break;
        const float *um = su + uslot(f - 1) * kUF, *uc = su + uslot(f) * kUF, *up = su + uslot(f + 1) * kUF;
        const float *bp = sb + bslot(f) * kBF;
        // rolling rows (box row = fine row - (fy0 - 1)): columns 2ic .. 2ic + 3
        float2 pA = ld2s(uc + (ry0) * kRW + cu), pB = ld2s(uc + (ry0) * kRW + cu + 2);          // y - 1
        float2 cA = ld2s(uc + (ry0 + 1) * kRW + cu), cB = ld2s(uc + (ry0 + 1) * kRW + cu + 2);  // y
        float tq1 = 0.f, tq2 = 0.f;  // x passes of rows y - 1, y - 2
#pragma unroll
        for (int r = 0; r <= 2 * kRRows; ++r) {
            const int row = ry0 + 1 + r;  // box row of fine row y
            const float2 nA = ld2s(uc + (row + 1) * kRW + cu), nB = ld2s(uc + (row + 1) * kRW + cu + 2);
            const int y = fy0 + ry0 + r;
            const bool yin = y < n;
            const float *zm = um + row * kRW + cu, *zp = up + row * kRW + cu;
            const float *bb = bp + (row - 1) * kRW + cu;
            // fine 2ic + 1 (box column cu + 1) and 2ic + 2 (cu + 2)
            const float s1 = radd(radd(radd(cA.x, cB.x), radd(pA.y, nA.y)), radd(zm[1], zp[1]));
            float r1 = radd(rfma(-6.f, cA.y, bb[1]), s1);
            const float s2 = radd(radd(radd(cA.y, cB.y), radd(pB.x, nB.x)), radd(zm[2], zp[2]));
            float r2 = radd(rfma(-6.f, cB.x, bb[2]), s2);
            if (!(yin && X0 + 1 < n)) r1 = 0.f;
            if (!(yin && X0 + 2 < n)) r2 = 0.f;
            float r0 = __shfl_up_sync(0xffffffffu, r2, 1);
            if (l == 0) {  // fine 2 ic0 (box column 4)
                const float w = uc[row * kRW + cu - 1];
                const float s0 = radd(radd(radd(w, cA.y), radd(pA.x, nA.x)), radd(zm[0], zp[0]));
                r0 = radd(rfma(-6.f, cA.x, bb[0]), s0);
                if (!(yin && X0 < n)) r0 = 0.f;
            }
            const float tx = rfma(2.f, r1, radd(r0, r2));
            if (r >= 2 && (r & 1) == 0) {  // coarse row m = r / 2 - 1 of this warp
                const int m = r / 2 - 1;
                const float t2 = rfma(2.f, tq1, radd(tq2, tx));
                const int jc = jc0 + kRRows * warp + m;
                if (f >= f0 + 2 && (f & 1) == 0 && ic < nc && jc < nc) {
                    const int kc = f / 2 - 1;
                    bc[gc.off + (long)kc * gc.plane + (long)jc * gc.pitch + ic] =
                        scale2<-4>(rfma(2.f, t2b[m], radd(t2a[m], t2)));
                }
                t2a[m] = t2b[m];
                t2b[m] = t2;
            }
            tq2 = tq1;
            tq1 = tx;
            pA = cA;
            pB = cB;
            cA = nA;
            cB = nB;
        }
        __syncwarp();
        if (l == 0) {  // this warp is done with u(f - 1) and b(f)
            mbar_arrive(empty_u(f - 1));
            mbar_arrive(empty_b(f));
        }
    }
    if (!ok) {
        s_fail = 1;
        atomicOr(err, 1);
    }
}

// launches still armed by mg_test_arm_wait_expiry
std::atomic<int> g_armed{0};

bool take_armed()
{
    int a = g_armed.load();
    while (a > 0)
        if (g_armed.compare_exchange_weak(a, a - 1)) return true;
    return false;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// tensor map over a padded 3D level array, box width x rows x 1
bool make_map(CUtensorMap *map, const float *base, const Pitch3 &g, int width, int rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn || ((uintptr_t)base & 15)) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.pitch, (cuuint64_t)(g.n + 2), (cuuint64_t)(g.n + 2)};
    const cuuint64_t strides[2] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.plane * 4};
    const cuuint32_t box[3] = {(cuuint32_t)width, (cuuint32_t)rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// z-chunks per tile column for a launch of `tiles` tile columns on `slots`
// resident blocks: the fewest chunks that fill the last wave to >= 95 %
// (each chunk boundary re-reads a plane or two; a partly filled last wave
// leaves SMs idle), else the best fill up to 8x the one-wave count
static int fill_chunks(int tiles, int slots, int max_chunks)
{
    const int base = std::max(1, slots / std::max(1, tiles));
    int best = std::min(base, max_chunks);
    double best_fill = 0.0;
    for (int c = 1; c <= std::min(max_chunks, 8 * base); ++c) {
        const double waves = (double)tiles * c / slots;
        const double fill = waves / std::ceil(waves);
        if (fill >= 0.95 && c >= base) return c;
        if (fill > best_fill + 1e-9) {
            best_fill = fill;
            best = c;
        }
    }
    return best;
}

static cudaError_t sweep3d_tma_any(const float *u, const float *b, float *out, double *u64, int n, const double *c,
                                   int *err, cudaStream_t s)
{
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        attr_err = cudaFuncSetAttribute(sweep3d_tma_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kSmemBytes);
        if (attr_err == cudaSuccess)
            attr_err = cudaFuncSetAttribute(sweep3d_tma_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            kSmemBytes);
        if (attr_err == cudaSuccess)
            attr_err = cudaFuncSetAttribute(sweep3d_tma_kernel<false, true>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes + kAccBytes);
    });
    if (attr_err != cudaSuccess) return attr_err;
    if (!err || (u64 && !u)) return cudaErrorInvalidValue;
    const Pitch3 g = pitch3(n);
    CUtensorMap tu, tb;
    if (!make_map(&tb, b, g, kTW, kTRows)) return cudaErrorInvalidValue;
    if (u) {
        if (!make_map(&tu, u, g, kTW, kURows)) return cudaErrorInvalidValue;
    } else {
        tu = tb;
    }
    const int bx = (n + kTCols - 1) / kTCols, by = (n + kTTY - 1) / kTTY;
    // two blocks per SM; chunks of at least four planes, the last wave filled
    const int chunks = fill_chunks(bx * by, 2 * num_sms(), std::max(1, n / 4));
    const int Z = (n + chunks - 1) / chunks;
    const dim3 grid(bx, by, (n + Z - 1) / Z);
    const float c0 = (float)c[0], c1 = (float)c[1];
    const int inject = take_armed() ? 16 : 0;
    if (u64)
        sweep3d_tma_kernel<false, true><<<grid, kTThreads + 32, kSmemBytes + kAccBytes, s>>>(tu, tb, nullptr, g, Z, c0,
                                                                                             c1, err, u64, inject);
    else if (u)
        sweep3d_tma_kernel<false><<<grid, kTThreads + 32, kSmemBytes, s>>>(tu, tb, out, g, Z, c0, c1, err, nullptr,
                                                                           inject);
    else
        sweep3d_tma_kernel<true><<<grid, kTThreads + 32, kSmemBytes, s>>>(tu, tb, out, g, Z, c0, c1, err, nullptr,
                                                                          inject);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_sweep3d_tma(const float *u, const float *b, float *out, int n, const double *c, int *err,
                               cudaStream_t s)
{
    return sweep3d_tma_any(u, b, out, nullptr, n, c, err, s);
}

cudaError_t launch_sweep3d_tma_acc64(const float *u, const float *b, double *u64, int n, const double *c, int *err,
                                     cudaStream_t s)
{
    return sweep3d_tma_any(u, b, nullptr, u64, n, c, err, s);
}

cudaError_t launch_resrestrict3d_tma(const float *u, const float *b, float *bc, int n, int *err, cudaStream_t s)
{
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    static int resident = 1;
    std::call_once(attr_once, [] {
        attr_err = cudaFuncSetAttribute(resrestrict3d_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        kRSmemBytes);
        if (attr_err == cudaSuccess)
            attr_err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, resrestrict3d_tma_kernel, kRThreads,
                                                                     kRSmemBytes);
        if (resident < 1) resident = 1;
    });
    if (attr_err != cudaSuccess) return attr_err;
    if (!err) return cudaErrorInvalidValue;
    const Pitch3 g = pitch3(n), gc = pitch3((n - 1) / 2);
    const int nc = gc.n;
    CUtensorMap tu, tb;
    if (!make_map(&tu, u, g, kRW, kRUR) || !make_map(&tb, b, g, kRW, kRBR)) return cudaErrorInvalidValue;
    const int bx = (nc + kRX - 1) / kRX, by = (nc + kRY - 1) / kRY;
    // z-chunks of coarse planes (at least two), the last wave filled
    const int chunks = fill_chunks(bx * by, resident * num_sms(), std::max(1, nc / 2));
    const int Zc = (nc + chunks - 1) / chunks;
    const int inject = take_armed() ? 16 : 0;
    resrestrict3d_tma_kernel<<<dim3(bx, by, (nc + Zc - 1) / Zc), kRThreads, kRSmemBytes, s>>>(tu, tb, bc, g, gc, Zc,
                                                                                            err, inject);
    count_launch(1);
    return cudaGetLastError();
}


}  // namespace mg

extern "C" int mg_test_arm_wait_expiry(int launches)
{
    return mg::g_armed.exchange(launches > 0 ? launches : 0);
}
