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
// Layout of the work: a warp owns a tile of 32 lanes x 8 fine columns and
// marches down a chunk of rows; lane l holds its 8 columns of every
// intermediate row in registers, and the horizontal neighbours come from
// the adjacent lanes by shuffles. Lanes 0 and 31 are halo lanes: they
// compute like the others (their outer columns are wrong, for lack of a
// neighbour) but store nothing; lanes 1..30 own 240 fine columns (120
// coarse columns), so adjacent tiles overlap by two lanes. No block barrier
// and no shared memory are needed except for the FP64 epilogue.
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

constexpr int kFC = 8;                 // fine columns per lane
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

// 8 floats of row y at column x (x % 8 == 0) of a padded level; rows outside
// [-1, n] and float4s outside the row's slot read as zero (inside the slot,
// the ghost ring and the padding are zero in memory)
__device__ __forceinline__ Row8 load8(const float *base, const Pitch2 &g, int x, int y)
{
    Row8 r = zero8();
    if (y < -1 || y > g.n) return r;
    const float *p = base + g.off + (long)y * g.pitch + x;
    if (in_slot(g, x)) {
        const float4 a = *reinterpret_cast<const float4 *>(p);
        r.v[0] = a.x, r.v[1] = a.y, r.v[2] = a.z, r.v[3] = a.w;
    }
    if (in_slot(g, x + 4)) {
        const float4 b = *reinterpret_cast<const float4 *>(p + 4);
        r.v[4] = b.x, r.v[5] = b.y, r.v[6] = b.z, r.v[7] = b.w;
    }
    return r;
}

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
// zero outside the interior
__device__ __forceinline__ Row8 residual8(const Row8 &us, const Row8 &uc, const Row8 &un, const Row8 &bh, int x, int j,
                                          int n)
{
    const Row8 h = xpair(uc);
    Row8 r;
    const bool jin = j >= 0 && j < n;
#pragma unroll
    for (int k = 0; k < kFC; ++k) {
        const float v = radd(rfma(-4.f, uc.v[k], bh.v[k]), radd(h.v[k], radd(us.v[k], un.v[k])));
        r.v[k] = jin && x + k >= 0 && x + k < n ? v : 0.f;
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

__device__ __forceinline__ Row8 mask8(Row8 v, int x, int j, int n)
{
    const bool jin = j >= 0 && j < n;
#pragma unroll
    for (int k = 0; k < kFC; ++k)
        if (!(jin && x + k >= 0 && x + k < n)) v.v[k] = 0.f;
    return v;
}

__device__ __forceinline__ void store8(float *base, const Pitch2 &g, int x, int j, const Row8 &v)
{
    float *p = base + g.off + (long)j * g.pitch + x;
    if (x + 7 < g.n) {
        *reinterpret_cast<float4 *>(p) = make_float4(v.v[0], v.v[1], v.v[2], v.v[3]);
        *reinterpret_cast<float4 *>(p + 4) = make_float4(v.v[4], v.v[5], v.v[6], v.v[7]);
    } else {
#pragma unroll
        for (int k = 0; k < kFC; ++k)
            if (x + k < g.n) p[k] = v.v[k];
    }
}

// ---------------------------------------------------------------------------
// A. sweep + residual + full weighting. Block (bx, by): warp w of the block
// owns tile t = bx * kFWarps + w (lane l: fine columns x = 240 t - 8 + 8 l)
// and coarse rows [by Hc, by Hc + Hc). Writes u1 at fine rows [2 jc0, 2 jc1)
// (the last chunk also row n - 1) and the coarse rows [jc0, jc1).
// ---------------------------------------------------------------------------
template <bool ZERO_U>
__global__ void __launch_bounds__(kFThreads)
sweep_restrict2d_kernel(const float *__restrict__ u0, const float *__restrict__ bh, float *__restrict__ u1out,
                        float *__restrict__ bc, Pitch2 g, Pitch2 gc, int Hc, float c0, float c1, float c2)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tile = blockIdx.x * kFWarps + w;
    const int n = g.n, nc = gc.n;
    const int x = kFOut * tile - kFC + kFC * lane;
    if (kFOut * tile >= n) return;  // the whole warp leaves together
    const bool owner = lane >= 1 && lane <= 30;
    const int jc0 = blockIdx.y * Hc, jc1 = min(jc0 + Hc, nc);
    // fine rows of u1 this chunk stores
    const int w0 = 2 * jc0, w1 = jc1 == nc ? n : 2 * jc1;
    // the newest residual row r0 is row R; u1 row R - 1; r1 row R - 2
    const int Rfirst = 2 * jc0 - 2, Rlast = 2 * jc1 + 2;
    Row8 r0s = zero8(), r0c = zero8(), hs = zero8(), hc = zero8();
    Row8 u1s = zero8(), u1c = zero8();  // u1 rows R-3, R-2
    Row8 bq1 = zero8(), bq2 = zero8();  // bh rows R-1, R-2
    // non-zero start: u0 rows R-1, R (the residual r0(R) also needs R+1)
    Row8 ua = zero8(), ub = zero8(), ucur = zero8();  // ucur: u0 row R-1, the sweep's base
    // loads are issued one row step ahead of their use
    Row8 bnext = load8(bh, g, x, Rfirst), unext = zero8();
    if (!ZERO_U) {
        ua = load8(u0, g, x, Rfirst - 1);
        ub = load8(u0, g, x, Rfirst);
        unext = load8(u0, g, x, Rfirst + 1);
    }
    float t1[4] = {0.f, 0.f, 0.f, 0.f}, t2[4] = {0.f, 0.f, 0.f, 0.f};  // x passes of r1 rows f-1, f-2
    for (int R = Rfirst; R <= Rlast; ++R) {
        const Row8 bR = bnext;
        bnext = load8(bh, g, x, R + 1);
        Row8 r0;
        if (ZERO_U) {
            r0 = bR;  // the ghost ring of bh is zero
        } else {
            const Row8 uc = unext;
            unext = load8(u0, g, x, R + 2);
            r0 = residual8(ua, ub, uc, bR, x, R, n);
            ucur = ua;  // u0 row R - 1
            ua = ub;
            ub = uc;
        }
        const Row8 hn = xpair(r0);
        // u1 row R - 1 (masked to the interior: the residual below reads it as the boundary value)
        const Row8 u1n = mask8(spai8<ZERO_U>(r0s, r0c, r0, hs, hc, hn, ucur, c0, c1, c2), x, R - 1, n);
        if (owner && R - 1 >= w0 && R - 1 < w1 && x < n) store8(u1out, g, x, R - 1, u1n);
        // r1 row R - 2 from u1 rows R-3 .. R-1 and bh(R-2)
        const Row8 r1 = residual8(u1s, u1c, u1n, bq2, x, R - 2, n);
        // full weighting: x pass of r1 row f = R - 2 at fine columns 2 ic, 2 ic + 1, 2 ic + 2
        const int f = R - 2;
        const float r8 = __shfl_down_sync(0xffffffffu, r1.v[0], 1);
        float tx[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) tx[k] = rfma(2.f, r1.v[2 * k + 1], radd(r1.v[2 * k], k == 3 ? r8 : r1.v[2 * k + 2]));
        if (f >= 2 * jc0 + 2 && (f & 1) == 0) {
            const int jc = f / 2 - 1;
            const int ic = x / 2;
            if (owner && jc < jc1 && ic < nc) {
                float v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) v[k] = scale2<-2>(rfma(2.f, t1[k], radd(t2[k], tx[k])));
                float *p = bc + gc.off + (long)jc * gc.pitch + ic;
                if (ic + 3 < nc) {
                    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (ic + k < nc) p[k] = v[k];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
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
}

// ---------------------------------------------------------------------------
// B. interpolation + correction + sweep. Block (bx, by): warp tiles as in A,
// fine output rows [by H, by H + H). u2 = u1 + P e; r = bh - A u2 (scaled);
// out = u2 + W r, stored (ACC64: added to the compact FP64 array u64).
// ---------------------------------------------------------------------------
// x pass of coarse row m for the lane's fine columns x .. x + 7 (coarse
// k0 = x / 2 .. k0 + 3): fine 2k: 0.5 (e[k-1] + e[k]); fine 2k + 1: e[k]
__device__ __forceinline__ Row8 interp_x8(const float *e, const Pitch2 &gc, int k0, int m)
{
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    if (m >= -1 && m <= gc.n && in_slot(gc, k0)) {
        const float4 a = *reinterpret_cast<const float4 *>(e + gc.off + (long)m * gc.pitch + k0);
        c[0] = a.x, c[1] = a.y, c[2] = a.z, c[3] = a.w;
    }
    const float left = __shfl_up_sync(0xffffffffu, c[3], 1);
    Row8 v;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v.v[2 * k] = scale2<-1>(radd(k == 0 ? left : c[k - 1], c[k]));
        v.v[2 * k + 1] = c[k];
    }
    return v;
}

template <bool ACC64>
__global__ void __launch_bounds__(kFThreads)
prolong_sweep2d_kernel(const float *__restrict__ u1, const float *__restrict__ e, const float *__restrict__ bh,
                       float *__restrict__ out, double *__restrict__ u64, Pitch2 g, Pitch2 gc, int H, float c0,
                       float c1, float c2)
{
    __shared__ __align__(16) float sacc[kFWarps][32 * kFC];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tile = blockIdx.x * kFWarps + w;
    const int n = g.n;
    const int x = kFOut * tile - kFC + kFC * lane;
    if (kFOut * tile >= n) return;
    const bool owner = lane >= 1 && lane <= 30;
    const int k0 = x / 2;
    const int xw = kFOut * tile - kFC;  // column of lane 0's first value
    const int y0 = blockIdx.y * H, y1 = min(y0 + H, n);
    // the newest corrected row u2 is row Q; residual row Q - 1; output row Q - 2
    const int Qfirst = y0 - 2, Qlast = y1 + 1;
    // x passes v_m of the coarse rows: fine row 2m + 1 takes v_m, fine row 2m
    // takes 0.5 (v_{m-1} + v_m); vprev = v_{mQ}, vcur = v_{mQ + 1} with
    // mQ = floor((Q - 1) / 2)
    int mcur = (Qfirst - 1) >> 1;
    Row8 vprev = interp_x8(e, gc, k0, mcur - 1), vcur = interp_x8(e, gc, k0, mcur);
    Row8 u2s = zero8(), u2c = zero8();                            // u2 rows Q-2, Q-1
    Row8 rs = zero8(), rc = zero8(), hs = zero8(), hc = zero8();  // residual rows Q-3, Q-2 and x pairs
    Row8 unext = load8(u1, g, x, Qfirst), bnext = load8(bh, g, x, Qfirst - 1);
    double a64[kFC];  // ACC64: the FP64 values of output row Q - 2, loaded one step ahead
#pragma unroll
    for (int q = 0; q < kFC; ++q) a64[q] = 0.0;
    auto load64 = [&](int j, double *dst) {
#pragma unroll
        for (int q = 0; q < kFC; ++q) {
            const int col = xw + lane + 32 * q;
            const int src = (lane + 32 * q) / kFC;
            dst[q] = (j >= y0 && j < y1 && src >= 1 && src <= 30 && col >= 0 && col < n) ? u64[(long)j * n + col] : 0.0;
        }
    };
    if (ACC64) load64(Qfirst - 2, a64);
    for (int Q = Qfirst; Q <= Qlast; ++Q) {
        // fine row Q (0-based) = 2m + 1 sits on coarse m; Q = 2m lies between m - 1 and m
        Row8 u2 = unext;
        unext = load8(u1, g, x, Q + 1);
        const Row8 bq = bnext;
        bnext = load8(bh, g, x, Q);
        double a64n[kFC];
        if (ACC64) load64(Q - 1, a64n);
        const int mQ = (Q - 1) >> 1;
        while (mcur < mQ + 1) {
            vprev = vcur;
            ++mcur;
            vcur = interp_x8(e, gc, k0, mcur);
        }
        if (Q & 1) {  // Q = 2 mQ + 1
#pragma unroll
            for (int k = 0; k < kFC; ++k) u2.v[k] = radd(u2.v[k], vprev.v[k]);
        } else {      // Q = 2 (mQ + 1): 0.5 (v_{mQ} + v_{mQ+1})
#pragma unroll
            for (int k = 0; k < kFC; ++k) u2.v[k] = radd(u2.v[k], scale2<-1>(radd(vprev.v[k], vcur.v[k])));
        }
        u2 = mask8(u2, x, Q, n);
        // residual of row Q - 1 and its x pairs
        const Row8 r = residual8(u2s, u2c, u2, bq, x, Q - 1, n);
        const Row8 hn = xpair(r);
        // sweep of row Q - 2
        const int j = Q - 2;
        if (j >= y0) {
            const Row8 o = spai8<false>(rs, rc, r, hs, hc, hn, u2s, c0, c1, c2);
            if (ACC64) {
                // stage the warp's 256 FP32 results; lane l then updates the
                // FP64 columns xw + l + 32 q (q < 8), 256 contiguous bytes per access
#pragma unroll
                for (int k = 0; k < kFC; ++k) sacc[w][kFC * lane + k] = o.v[k];
                __syncwarp();
#pragma unroll
                for (int q = 0; q < kFC; ++q) {
                    const int col = xw + lane + 32 * q;
                    const int src = (lane + 32 * q) / kFC;
                    if (src >= 1 && src <= 30 && col >= 0 && col < n)
                        u64[(long)j * n + col] = __dadd_rn(a64[q], widen(sacc[w][lane + 32 * q]));
                }
                __syncwarp();
            } else if (owner && x < n) {
                store8(out, g, x, j, o);
            }
        }
        if (ACC64) {
#pragma unroll
            for (int q = 0; q < kFC; ++q) a64[q] = a64n[q];
        }
        rs = rc;
        rc = r;
        hs = hc;
        hc = hn;
        u2s = u2c;
        u2c = u2;
    }
}

}  // namespace

// tiles of 240 fine columns, kFWarps per block
static int fused_tiles(int n) { return (n + kFOut - 1) / kFOut; }

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
        sweep_restrict2d_kernel<false><<<grid, kFThreads, 0, s>>>(u0, bh, u1, bc, g, gc, Hc, c0, c1, c2);
    else
        sweep_restrict2d_kernel<true><<<grid, kFThreads, 0, s>>>(u0, bh, u1, bc, g, gc, Hc, c0, c1, c2);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_prolong_sweep2d_pl(const float *u1, const float *e, const float *bh, float *out, double *u64, int n,
                                      const double *c, cudaStream_t s)
{
    const Pitch2 g = pitch2(n), gc = pitch2((n - 1) / 2);
    const int bx = (fused_tiles(n) + kFWarps - 1) / kFWarps;
    const int H = chunk_rows(bx, n, 8 * num_sms(), 16, 128);
    const dim3 grid(bx, (n + H - 1) / H);
    const float c0 = (float)c[0], c1 = (float)c[1], c2 = (float)c[2];
    if (u64)
        prolong_sweep2d_kernel<true><<<grid, kFThreads, 0, s>>>(u1, e, bh, out, u64, g, gc, H, c0, c1, c2);
    else
        prolong_sweep2d_kernel<false><<<grid, kFThreads, 0, s>>>(u1, e, bh, out, u64, g, gc, H, c0, c1, c2);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace mg
