// mg_fused2d.cu -- temporally blocked FP32 2D kernels for V(1,1) cycles on
// the padded level layout (the FP32 levels of the refinement solves).
//
// An unfused V(1,1) visit of a level moves, per fine point, 8 bytes for the
// pre-sweep from zero (b in, u out), 8.25 for residual + full weighting
// (u, b in, coarse b out), 8.25 for interpolation + correction (u, coarse e
// in, u out) and 12 for the post-sweep (u, b in, u out): 36.5 bytes. Two
// passes do the same work:
//   A. sweep + residual + full weighting: b (and u unless the sweep starts
//      from zero) in; the smoothed u and the coarse right-hand side out;
//   B. interpolation + correction + sweep: u, coarse e and b in; the
//      smoothed u out (or, on the finest refinement level, added to the FP64
//      solution),
// 9 + 13 = 22 bytes per fine point from zero. Every value is formed by the
// same formula in the same operation order as in the unfused kernels
// (mg_pl2d.cu, mg_kernels2d.cu), so the results are identical bit for bit.
//
// Layout of the work: a warp owns a tile of 32 lanes x 4 fine columns and
// marches down a chunk of rows; lane l holds its 4 columns of every
// intermediate row in registers, and the horizontal neighbours come from
// the adjacent lanes by shuffles. Lanes 0 and 31 are halo lanes: they
// compute like the others (their outer columns are wrong, for lack of a
// neighbour) but store nothing; lanes 1..30 own 120 fine columns (60
// coarse columns), so adjacent tiles overlap by two lanes. Global loads are
// issued two row steps ahead of their use. No block barrier and no shared
// memory are needed except for the FP64 epilogue.
//
// Pipeline per row step (A, from zero; newest row q):
//   r0(q)  = bh(q)                              (zero outside the interior)
//   hp(q)  = r0_W + r0_E                        (x pair, shuffles at the lane edges)
//   u1(q-1) = fma(c2, hp(q-2) + hp(q), fma(c1, hp(q-1) + (r0(q-2) + r0(q)), c0 r0(q-1)))
//   r1(q-2) = fma(-4, u1, bh) + ((u1_W + u1_E) + (u1(q-3) + u1(q-1)))
//   x pass and, every second row, y pass of the full weighting of r1.
// With a non-zero start r0 itself is the residual of u0, one row earlier.
#include "mg_common.cuh"
#include "mg_internal.h"

namespace mg {

namespace {

constexpr int kFC = 4;                 // fine columns per lane
constexpr int kFOut = 30 * kFC;        // fine columns a warp stores (lanes 1..30)
constexpr int kFWarps = 4;             // warps per block: adjacent tiles, same rows
constexpr int kFThreads = 32 * kFWarps;

struct Row8 {
    float v[kFC];
};

__device__ __forceinline__ Row8 zero8()
{
    Row8 r;
#pragma unroll
    for (int k = 0; k < kFC; ++k) r.v[k] = 0.f;
    return r;
}

// A float4 at columns x .. x + 3 of a row of a padded level lies inside the
// row's slot (columns -4 .. pitch - 5) when -4 <= x and x + 3 <= pitch - 5.
__device__ __forceinline__ bool in_slot(const Pitch2 &g, int x) { return x >= -4 && x + 3 <= g.pitch - 5; }

// Global rows reach the lanes through per-warp rings in shared memory filled
// by asynchronous copies (cp.async), kFDepth row steps ahead of their use:
// the bytes in flight no longer cost registers. Lane l copies and later
// reads only its own entries, so completion needs no barrier, only
// cp.async.wait_group in the lane itself. A ring has kFSlots > kFDepth slots,
// so the slot refilled at a step was read two steps earlier.
constexpr int kFDepth = 6;
constexpr int kFSlots = 8;  // power of two
static_assert(kFSlots > kFDepth + 1, "a refilled slot must have been read at least two steps earlier");

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
// copy `bytes` (16 or 8) from src to shared dst; !valid: fill zeros, read nothing
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most kFDepth - 1 of this lane's copy groups are still pending
__device__ __forceinline__ void cp_wait_depth() { asm volatile("cp.async.wait_group %0;" ::"n"(kFDepth - 1) : "memory"); }

// One float4 per lane and row of a padded level, issued row after row:
// ring[slot][lane]. The element offset of the next row advances by the
// pitch; only rows in [-1, n] with the lane's float4 inside the row's slot
// are read, other rows arrive as zeros.
struct Ring4 {
    float4 *s;
    const float *base;
    long off;       // element offset of row y, column x
    long pitch;
    int y, n;       // next row to issue; rows [-1, n] hold data
    bool col_ok;    // the lane's float4 lies inside the row's slot
    __device__ __forceinline__ void init(float4 *ring, const float *b, const Pitch2 &g, int x, int y_first)
    {
        s = ring;
        base = b;
        pitch = g.pitch;
        n = g.n;
        y = y_first;
        off = g.off + (long)y_first * g.pitch + x;
        col_ok = in_slot(g, x);
    }
    __device__ __forceinline__ void issue(int lane)
    {
        const bool ok = col_ok && y >= -1 && y <= n;
        cp_async16(&s[(y & (kFSlots - 1)) * 32 + lane], ok ? base + off : base, ok);
        off += pitch;
        ++y;
    }
    __device__ __forceinline__ Row8 read(int row, int lane) const
    {
        const float4 a = s[(row & (kFSlots - 1)) * 32 + lane];
        Row8 r;
        r.v[0] = a.x, r.v[1] = a.y, r.v[2] = a.z, r.v[3] = a.w;
        return r;
    }
};

// x pair sums v_W + v_E of the lane's 8 columns (neighbours across lanes by shuffles)
__device__ __forceinline__ Row8 xpair(const Row8 &v)
{
    const float left = __shfl_up_sync(0xffffffffu, v.v[kFC - 1], 1);
    const float right = __shfl_down_sync(0xffffffffu, v.v[0], 1);
    Row8 h;
#pragma unroll
    for (int k = 0; k < kFC; ++k) h.v[k] = radd(k == 0 ? left : v.v[k - 1], k == kFC - 1 ? right : v.v[k + 1]);
    return h;
}

// scaled 5-point residual of row j: fma(-4, u, bh) + ((u_W + u_E) + (u_S + u_N)),
// zero outside the interior (cols: bit k set when column x + k is interior)
__device__ __forceinline__ Row8 residual8(const Row8 &us, const Row8 &uc, const Row8 &un, const Row8 &bh, unsigned cols,
                                          bool jin)
{
    const Row8 h = xpair(uc);
    Row8 r;
#pragma unroll
    for (int k = 0; k < kFC; ++k) {
        const float v = radd(rfma(-4.f, uc.v[k], bh.v[k]), radd(h.v[k], radd(us.v[k], un.v[k])));
        r.v[k] = jin && ((cols >> k) & 1u) ? v : 0.f;
    }
    return r;
}

// SPAI update of row j from the residual rows j-1, j, j+1 and their x pairs:
// E = hp(j) + (r(j-1) + r(j+1)), C = hp(j-1) + hp(j+1),
// out = fma(c2, C, fma(c1, E, fma(c0, r, u)))    (from zero: c0 r)
template <bool ZERO_U>
__device__ __forceinline__ Row8 spai8(const Row8 &rs, const Row8 &rc, const Row8 &rn, const Row8 &hs, const Row8 &hc,
                                      const Row8 &hn, const Row8 &u, float c0, float c1, float c2)
{
    Row8 o;
#pragma unroll
    for (int k = 0; k < kFC; ++k) {
        const float E = radd(hc.v[k], radd(rs.v[k], rn.v[k]));
        const float C = radd(hs.v[k], hn.v[k]);
        const float base = ZERO_U ? rmul(c0, rc.v[k]) : rfma(c0, rc.v[k], u.v[k]);
        o.v[k] = rfma(c2, C, rfma(c1, E, base));
    }
    return o;
}

__device__ __forceinline__ Row8 mask8(Row8 v, unsigned cols, bool jin)
{
#pragma unroll
    for (int k = 0; k < kFC; ++k)
        if (!(jin && ((cols >> k) & 1u))) v.v[k] = 0.f;
    return v;
}

// bit k: column x + k is an interior column (0 <= x + k < n)
__device__ __forceinline__ unsigned col_bits(int x, int n)
{
    unsigned m = 0;
#pragma unroll
    for (int k = 0; k < kFC; ++k)
        if (x + k >= 0 && x + k < n) m |= 1u << k;
    return m;
}

__device__ __forceinline__ void store8(float *base, const Pitch2 &g, int x, int j, const Row8 &v)
{
    float *p = base + g.off + (long)j * g.pitch + x;
    if (x + kFC - 1 < g.n) {
        *reinterpret_cast<float4 *>(p) = make_float4(v.v[0], v.v[1], v.v[2], v.v[3]);
    } else {
#pragma unroll
        for (int k = 0; k < kFC; ++k)
            if (x + k < g.n) p[k] = v.v[k];
    }
}

// ---------------------------------------------------------------------------
// A. sweep + residual + full weighting. Block (bx, by): warp w of the block
// owns tile t = bx * kFWarps + w (lane l: fine columns x = 120 t - 4 + 4 l)
// and coarse rows [by Hc, by Hc + Hc). Writes u1 at fine rows [2 jc0, 2 jc1)
// (the last chunk also row n - 1) and the coarse rows [jc0, jc1).
// Rings: bh row R and, from a non-zero start, u0 row R + 1 at step R.
// ---------------------------------------------------------------------------
// One warp's part of block (bx, by); `ring`: the warp's shared-memory rings
// (one ring from zero, two otherwise).
template <bool ZERO_U>
__device__ __forceinline__ void sweep_restrict2d_tile(const float *__restrict__ u0, const float *__restrict__ bh,
                                                      float *__restrict__ u1out, float *__restrict__ bc, Pitch2 g,
                                                      Pitch2 gc, int Hc, float c0, float c1, float c2, int bx, int by,
                                                      float4 *ring)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tile = bx * kFWarps + w;
    const int n = g.n, nc = gc.n;
    const int x = kFOut * tile - kFC + kFC * lane;
    if (kFOut * tile >= n) return;  // the whole warp leaves together
    const bool owner = lane >= 1 && lane <= 30;
    const unsigned cols = col_bits(x, n);
    const int jc0 = by * Hc, jc1 = min(jc0 + Hc, nc);
    // fine rows of u1 this chunk stores
    const int w0 = 2 * jc0, w1 = jc1 == nc ? n : 2 * jc1;
    // the newest residual row r0 is row R; u1 row R - 1; r1 row R - 2
    const int Rfirst = 2 * jc0 - 2, Rlast = 2 * jc1 + 2;
    // rings: bh row R and (non-zero start) u0 row R + 1 at step R; the
    // prologue issues steps Rfirst .. Rfirst + kFDepth - 1 (one group per step)
    Ring4 rb, ru;
    rb.init(ring, bh, g, x, Rfirst);
    if (!ZERO_U) ru.init(rb.s + kFSlots * 32, u0, g, x, Rfirst - 1);
    for (int k = 0; k < kFDepth; ++k) {
        rb.issue(lane);
        if (!ZERO_U) {
            if (k == 0) {  // u0 rows Rfirst - 1, Rfirst
                ru.issue(lane);
                ru.issue(lane);
            }
            ru.issue(lane);
        }
        cp_commit();
    }
    Row8 r0s = zero8(), r0c = zero8(), hs = zero8(), hc = zero8();
    Row8 u1s = zero8(), u1c = zero8();  // u1 rows R-3, R-2
    Row8 bq1 = zero8(), bq2 = zero8();  // bh rows R-1, R-2
    // non-zero start: u0 rows R-1, R (the residual r0(R) also needs R+1)
    Row8 ua = zero8(), ub = zero8(), ucur = zero8();  // ucur: u0 row R-1, the sweep's base
    constexpr int kCC = kFC / 2;  // coarse columns per lane
    float t1[kCC], t2[kCC];       // x passes of r1 rows f-1, f-2
#pragma unroll
    for (int k = 0; k < kCC; ++k) t1[k] = t2[k] = 0.f;
    for (int R = Rfirst; R <= Rlast; ++R) {
        cp_wait_depth();  // the copies of step R have landed
        const Row8 bR = rb.read(R, lane);
        Row8 r0;
        if (ZERO_U) {
            r0 = bR;  // the ghost ring of bh is zero
        } else {
            if (R == Rfirst) {
                ua = ru.read(R - 1, lane);
                ub = ru.read(R, lane);
            }
            const Row8 uc = ru.read(R + 1, lane);
            r0 = residual8(ua, ub, uc, bR, cols, R >= 0 && R < n);
            ucur = ua;  // u0 row R - 1
            ua = ub;
            ub = uc;
        }
        // the copies of step R + kFDepth
        rb.issue(lane);
        if (!ZERO_U) ru.issue(lane);
        cp_commit();
        const Row8 hn = xpair(r0);
        // u1 row R - 1 (masked to the interior: the residual below reads it as the boundary value)
        const Row8 u1n = mask8(spai8<ZERO_U>(r0s, r0c, r0, hs, hc, hn, ucur, c0, c1, c2), cols, R - 1 >= 0 && R - 1 < n);
        if (owner && R - 1 >= w0 && R - 1 < w1 && x < n) store8(u1out, g, x, R - 1, u1n);
        // r1 row R - 2 from u1 rows R-3 .. R-1 and bh(R-2)
        const Row8 r1 = residual8(u1s, u1c, u1n, bq2, cols, R - 2 >= 0 && R - 2 < n);
        // full weighting: x pass of r1 row f = R - 2 at fine columns 2 ic, 2 ic + 1, 2 ic + 2
        const int f = R - 2;
        const float rnext = __shfl_down_sync(0xffffffffu, r1.v[0], 1);
        float tx[kCC];
#pragma unroll
        for (int k = 0; k < kCC; ++k)
            tx[k] = rfma(2.f, r1.v[2 * k + 1], radd(r1.v[2 * k], k == kCC - 1 ? rnext : r1.v[2 * k + 2]));
        if (f >= 2 * jc0 + 2 && (f & 1) == 0) {
            const int jc = f / 2 - 1;
            const int ic = x / 2;
            if (owner && jc < jc1 && ic < nc) {
                float v[kCC];
#pragma unroll
                for (int k = 0; k < kCC; ++k) v[k] = scale2<-2>(rfma(2.f, t1[k], radd(t2[k], tx[k])));
                float *p = bc + gc.off + (long)jc * gc.pitch + ic;
                if (ic + kCC - 1 < nc) {
                    *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
                } else {
#pragma unroll
                    for (int k = 0; k < kCC; ++k)
                        if (ic + k < nc) p[k] = v[k];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kCC; ++k) {
            t2[k] = t1[k];
            t1[k] = tx[k];
        }
        r0s = r0c;
        r0c = r0;
        hs = hc;
        hc = hn;
        u1s = u1c;
        u1c = u1n;
        bq2 = bq1;
        bq1 = bR;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");  // no copy may land after the warp has left
}

// ---------------------------------------------------------------------------
// B. interpolation + correction + sweep. Block (bx, by): warp tiles as in A,
// fine output rows [by H, by H + H). u2 = u1 + P e; r = bh - A u2 (scaled);
// out = u2 + W r, stored (ACC64: added to the compact FP64 array u64).
// Rings at step Q: u1 row Q, bh row Q - 1 and the coarse e rows as they are
// first needed; (ACC64) the FP64 values of output row Q - 2 come by plain
// loads issued one step earlier.
// ---------------------------------------------------------------------------
// x pass of the coarse row held in e2 (the lane's coarse columns k0 = x / 2,
// k0 + 1) for its fine columns x .. x + 3: fine 2k: 0.5 (e[k-1] + e[k]);
// fine 2k + 1: e[k]
__device__ __forceinline__ Row8 interp_x8(float2 e2)
{
    const float c[2] = {e2.x, e2.y};
    const float left = __shfl_up_sync(0xffffffffu, c[1], 1);
    Row8 v;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        v.v[2 * k] = scale2<-1>(radd(k == 0 ? left : c[k - 1], c[k]));
        v.v[2 * k + 1] = c[k];
    }
    return v;
}

constexpr int kF64Lead = 2;  // steps between the L2 prefetch and the load of an FP64 row (2, 4, 8: 2 fastest)

// float4s of shared memory per warp of pass B: u1 and bh rings (float4),
// the e ring (float2) and, ACC64, the staging row of the FP64 epilogue
constexpr int kRing4 = kFSlots * 32;
__host__ __device__ constexpr int warp_f4_b(bool acc64) { return 2 * kRing4 + kRing4 / 2 + (acc64 ? 32 : 0); }

// One warp's part of block (bx, by); `base`: the warp's shared memory.
template <bool ACC64>
__device__ __forceinline__ void prolong_sweep2d_tile(const float *__restrict__ u1, const float *__restrict__ e,
                                                     const float *__restrict__ bh, float *__restrict__ out,
                                                     double *__restrict__ u64, Pitch2 g, Pitch2 gc, int H, float c0,
                                                     float c1, float c2, int bx, int by, float4 *base)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tile = bx * kFWarps + w;
    const int n = g.n;
    const int x = kFOut * tile - kFC + kFC * lane;
    if (kFOut * tile >= n) return;
    float2 *re = reinterpret_cast<float2 *>(base + 2 * kRing4);  // [slot][lane]
    float *sacc = reinterpret_cast<float *>(base + 2 * kRing4 + kRing4 / 2);
    const bool owner = lane >= 1 && lane <= 30;
    const int k0 = x / 2;
    const int xw = kFOut * tile - kFC;  // column of lane 0's first value
    const int y0 = by * H, y1 = min(y0 + H, n);
    // the newest corrected row u2 is row Q; residual row Q - 1; output row Q - 2
    const int Qfirst = y0 - 2, Qlast = y1 + 1;
    // coarse row m (0-based) sits at fine row 2m + 1; fine row Q needs the
    // coarse rows mQ = floor((Q - 1) / 2) and mQ + 1
    const unsigned cols = col_bits(x, n);
    // FP64 columns of this lane in the epilogue: xw + lane + 32 q, q < kFC,
    // valid when inside the grid and produced by an owner lane
    unsigned cols64 = 0;
#pragma unroll
    for (int q = 0; q < kFC; ++q) {
        const int col = xw + lane + 32 * q, src = (lane + 32 * q) / kFC;
        if (src >= 1 && src <= 30 && col >= 0 && col < n) cols64 |= 1u << q;
    }
    // rings: u1 row F and bh row F - 1 for fine row F, e rows as first needed
    Ring4 ru, rb;
    ru.init(base, u1, g, x, Qfirst);
    rb.init(base + kRing4, bh, g, x, Qfirst - 1);
    const bool e_col_ok = k0 >= -4 && k0 + 1 <= gc.pitch - 5;  // a float2 inside the coarse row's slot
    long e_off = gc.off + (long)(((Qfirst - 1) >> 1) - 1) * gc.pitch + k0;
    int m_issued = ((Qfirst - 1) >> 1) - 1;
    // ACC64: the FP64 values of output row j are loaded (plain loads into
    // registers) one step before the step that updates them
    auto load64 = [&](int j, double *dst) {
        const bool jok = j >= y0 && j < y1;
        const double *src = u64 + (long)j * n + xw + lane;
#pragma unroll
        for (int q = 0; q < kFC; ++q) dst[q] = jok && ((cols64 >> q) & 1u) ? src[32 * q] : 0.0;
    };
    auto issue_step = [&](int F) {  // the copies for fine row F
        ru.issue(lane);
        rb.issue(lane);
        const int mneed = ((F - 1) >> 1) + 1;
        while (m_issued < mneed) {
            ++m_issued;
            e_off += gc.pitch;
            const bool ok = e_col_ok && m_issued >= -1 && m_issued <= gc.n;
            cp_async8(&re[(m_issued & (kFSlots - 1)) * 32 + lane], ok ? e + e_off : e, ok);
        }
        cp_commit();
    };
    for (int k = 0; k < kFDepth; ++k) issue_step(Qfirst + k);
    double a64n[kFC];
    if (ACC64) load64(Qfirst - 2, a64n);
    int mcur = 0;
    Row8 vprev = zero8(), vcur = zero8();
    Row8 u2s = zero8(), u2c = zero8();                            // u2 rows Q-2, Q-1
    Row8 rs = zero8(), rc = zero8(), hs = zero8(), hc = zero8();  // residual rows Q-3, Q-2 and x pairs
    for (int Q = Qfirst; Q <= Qlast; ++Q) {
        cp_wait_depth();  // the copies of step Q have landed
        Row8 u2 = ru.read(Q, lane);
        const Row8 bQ = rb.read(Q - 1, lane);
        const int mQ = (Q - 1) >> 1;
        if (Q == Qfirst) {
            mcur = mQ + 1;
            vprev = interp_x8(re[(mQ & (kFSlots - 1)) * 32 + lane]);
            vcur = interp_x8(re[(mcur & (kFSlots - 1)) * 32 + lane]);
        }
        while (mcur < mQ + 1) {
            vprev = vcur;
            ++mcur;
            vcur = interp_x8(re[(mcur & (kFSlots - 1)) * 32 + lane]);
        }
        double a64[kFC];  // row Q - 2, loaded at the previous step
        if (ACC64) {
#pragma unroll
            for (int q = 0; q < kFC; ++q) a64[q] = a64n[q];
            load64(Q - 1, a64n);
            // the FP64 row kF64Lead steps on into L2: the one-step register
            // load above then waits for L2 instead of DRAM (lanes 0..7 touch
            // one 128-byte line each of the warp's 960 bytes)
            const int jp = Q - 1 + kF64Lead;
            if (lane < 8 && jp >= y0 && jp < y1) {
                const int col = min(max(xw + 16 * lane, 0), n - 1);
                prefetch_l2(u64 + (long)jp * n + col);
            }
        }
        issue_step(Q + kFDepth);
        // here vcur = x pass of coarse row mQ + 1, vprev = of mQ
        if (Q & 1) {  // Q = 2 mQ + 1
#pragma unroll
            for (int k = 0; k < kFC; ++k) u2.v[k] = radd(u2.v[k], vprev.v[k]);
        } else {      // Q = 2 (mQ + 1): 0.5 (v_{mQ} + v_{mQ+1})
#pragma unroll
            for (int k = 0; k < kFC; ++k) u2.v[k] = radd(u2.v[k], scale2<-1>(radd(vprev.v[k], vcur.v[k])));
        }
        u2 = mask8(u2, cols, Q >= 0 && Q < n);
        // residual of row Q - 1 and its x pairs
        const Row8 r = residual8(u2s, u2c, u2, bQ, cols, Q - 1 >= 0 && Q - 1 < n);
        const Row8 hn = xpair(r);
        // sweep of row Q - 2
        const int j = Q - 2;
        if (j >= y0) {
            const Row8 o = spai8<false>(rs, rc, r, hs, hc, hn, u2s, c0, c1, c2);
            if (ACC64) {
                // stage the warp's 32 kFC FP32 results; lane l then updates the
                // FP64 columns xw + l + 32 q (q < kFC), 256 contiguous bytes per access
#pragma unroll
                for (int k = 0; k < kFC; ++k) sacc[kFC * lane + k] = o.v[k];
                __syncwarp();
                double *dst = u64 + (long)j * n + xw + lane;
#pragma unroll
                for (int q = 0; q < kFC; ++q)
                    if ((cols64 >> q) & 1u) dst[32 * q] = radd(a64[q], widen(sacc[lane + 32 * q]));
                __syncwarp();
            } else if (owner && x < n) {
                store8(out, g, x, j, o);
            }
        }
        rs = rc;
        rc = r;
        hs = hc;
        hc = hn;
        u2s = u2c;
        u2c = u2;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");  // no copy may land after the warp has left
}

template <bool ZERO_U>
__global__ void __launch_bounds__(kFThreads)
sweep_restrict2d_kernel(const float *__restrict__ u0, const float *__restrict__ bh, float *__restrict__ u1out,
                        float *__restrict__ bc, Pitch2 g, Pitch2 gc, int Hc, float c0, float c1, float c2)
{
    extern __shared__ __align__(16) float4 fsm[];
    const int w = threadIdx.x >> 5;
    sweep_restrict2d_tile<ZERO_U>(u0, bh, u1out, bc, g, gc, Hc, c0, c1, c2, blockIdx.x, blockIdx.y,
                                  fsm + (ZERO_U ? 1 : 2) * w * kFSlots * 32);
}

template <bool ACC64>
__global__ void __launch_bounds__(kFThreads)
prolong_sweep2d_kernel(const float *__restrict__ u1, const float *__restrict__ e, const float *__restrict__ bh,
                       float *__restrict__ out, double *__restrict__ u64, Pitch2 g, Pitch2 gc, int H, float c0,
                       float c1, float c2)
{
    extern __shared__ __align__(16) float4 fsm[];
    const int w = threadIdx.x >> 5;
    prolong_sweep2d_tile<ACC64>(u1, e, bh, out, u64, g, gc, H, c0, c1, c2, blockIdx.x, blockIdx.y,
                                fsm + w * warp_f4_b(ACC64));
}

// Batched forms: persistent loops over the (problem, block) items of every
// problem with a level of size n, skipping inactive problems. Pass A takes
// each item's start (u == nullptr: from zero) per item; every warp keeps two
// rings, so that warps of a block that are at different items never share one.
__global__ void __launch_bounds__(kFThreads)
sweep_restrict2d_batched(const FItem *__restrict__ tab, int nprob, const int *__restrict__ active, Pitch2 g,
                         Pitch2 gc, int Hc, int bx, int by, float c0, float c1, float c2)
{
    extern __shared__ __align__(16) float4 fsm[];
    float4 *ring = fsm + 2 * (threadIdx.x >> 5) * kFSlots * 32;
    const int per = bx * by, total = nprob * per;
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int j = it / per, r = it - j * per;
        const FItem f = tab[j];
        if (!active[f.problem]) continue;
        if (f.u)
            sweep_restrict2d_tile<false>(f.u, f.b, f.out, f.out2, g, gc, Hc, c0, c1, c2, r % bx, r / bx, ring);
        else
            sweep_restrict2d_tile<true>(nullptr, f.b, f.out, f.out2, g, gc, Hc, c0, c1, c2, r % bx, r / bx, ring);
    }
}

__global__ void __launch_bounds__(kFThreads)
prolong_sweep2d_batched(const FItem *__restrict__ tab, int nprob, const int *__restrict__ active, Pitch2 g, Pitch2 gc,
                        int H, int bx, int by, float c0, float c1, float c2)
{
    extern __shared__ __align__(16) float4 fsm[];
    float4 *base = fsm + (threadIdx.x >> 5) * warp_f4_b(false);
    const int per = bx * by, total = nprob * per;
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int j = it / per, r = it - j * per;
        const FItem f = tab[j];
        if (!active[f.problem]) continue;
        prolong_sweep2d_tile<false>(f.u, f.e, f.b, f.out, nullptr, g, gc, H, c0, c1, c2, r % bx, r / bx, base);
    }
}

}  // namespace

// tiles of kFOut fine columns, kFWarps per block
static int fused_tiles(int n) { return (n + kFOut - 1) / kFOut; }

static size_t smem_a(bool zero_u) { return (size_t)kFWarps * (zero_u ? 1 : 2) * kFSlots * 32 * sizeof(float4); }
static size_t smem_b(bool acc64) { return (size_t)kFWarps * warp_f4_b(acc64) * sizeof(float4); }

cudaError_t launch_sweep_restrict2d_pl(const float *u0, const float *bh, float *u1, float *bc, int n, const double *c,
                                       cudaStream_t s)
{
    const Pitch2 g = pitch2(n), gc = pitch2((n - 1) / 2);
    const int nc = gc.n;
    const int bx = (fused_tiles(n) + kFWarps - 1) / kFWarps;
    const int Hc = chunk_rows(bx, nc, 8 * num_sms(), 8, 64);
    const dim3 grid(bx, (nc + Hc - 1) / Hc);
    const float c0 = (float)c[0], c1 = (float)c[1], c2 = (float)c[2];
    if (u0)
        sweep_restrict2d_kernel<false><<<grid, kFThreads, smem_a(false), s>>>(u0, bh, u1, bc, g, gc, Hc, c0, c1, c2);
    else
        sweep_restrict2d_kernel<true><<<grid, kFThreads, smem_a(true), s>>>(u0, bh, u1, bc, g, gc, Hc, c0, c1, c2);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_prolong_sweep2d_pl(const float *u1, const float *e, const float *bh, float *out, double *u64, int n,
                                      const double *c, cudaStream_t s)
{
    static cudaError_t attr = cudaErrorNotReady;
    if (attr == cudaErrorNotReady) {
        attr = cudaFuncSetAttribute(prolong_sweep2d_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem_b(true));
        if (attr == cudaSuccess)
            attr = cudaFuncSetAttribute(prolong_sweep2d_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem_b(false));
    }
    if (attr != cudaSuccess) return attr;
    const Pitch2 g = pitch2(n), gc = pitch2((n - 1) / 2);
    const int bx = (fused_tiles(n) + kFWarps - 1) / kFWarps;
    const int H = chunk_rows(bx, n, 8 * num_sms(), 16, 128);
    const dim3 grid(bx, (n + H - 1) / H);
    const float c0 = (float)c[0], c1 = (float)c[1], c2 = (float)c[2];
    if (u64)
        prolong_sweep2d_kernel<true><<<grid, kFThreads, smem_b(true), s>>>(u1, e, bh, out, u64, g, gc, H, c0, c1, c2);
    else
        prolong_sweep2d_kernel<false><<<grid, kFThreads, smem_b(false), s>>>(u1, e, bh, out, u64, g, gc, H, c0, c1,
                                                                             c2);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace mg

namespace mg {

static int fused_persistent_grid(const void *fn, size_t smem, long items)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kFThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return (int)std::max<long>(1, std::min<long>(items, (long)per_sm * num_sms()));
}

int fused_blocks_x(int n) { return (fused_tiles(n) + kFWarps - 1) / kFWarps; }

cudaError_t launch_sweep_restrict2d_pl_batched(const FItem *tab, int nprob, const int *active, int n, int Hc,
                                               const double *c, cudaStream_t s)
{
    const Pitch2 g = pitch2(n), gc = pitch2((n - 1) / 2);
    const int bx = fused_blocks_x(n), by = (gc.n + Hc - 1) / Hc;
    const size_t smem = smem_a(false);
    const int grid = fused_persistent_grid((const void *)sweep_restrict2d_batched, smem, (long)nprob * bx * by);
    sweep_restrict2d_batched<<<grid, kFThreads, smem, s>>>(tab, nprob, active, g, gc, Hc, bx, by, (float)c[0],
                                                           (float)c[1], (float)c[2]);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_prolong_sweep2d_pl_batched(const FItem *tab, int nprob, const int *active, int n, int H,
                                              const double *c, cudaStream_t s)
{
    const Pitch2 g = pitch2(n), gc = pitch2((n - 1) / 2);
    const int bx = fused_blocks_x(n), by = (n + H - 1) / H;
    const size_t smem = smem_b(false);
    const int grid = fused_persistent_grid((const void *)prolong_sweep2d_batched, smem, (long)nprob * bx * by);
    prolong_sweep2d_batched<<<grid, kFThreads, smem, s>>>(tab, nprob, active, g, gc, H, bx, by, (float)c[0],
                                                          (float)c[1], (float)c[2]);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace mg
