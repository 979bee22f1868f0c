// mg_kernels2d.cu -- 2D kernels: SPAI sweep, residual + full weighting,
// bilinear interpolation + correction (He, Liu, Wang, arXiv:2206.05543,
// Sec. 2 Eq. (2.1), Sec. 3.1, Sec. 4).
//
// Design. All three kernels march along y: a block owns a strip of columns
// (one column per thread) and a chunk of rows, and keeps a rolling window of
// rows in registers; the horizontal neighbours come through a double-buffered
// shared-memory row. Every residual and every interpolated value is computed
// once per point (plus a two-row halo per chunk and a one-column halo per
// strip), which matters because FP64 on this part is ALU-bound: the stencil
// work, not the bytes, sets the time.
//
// Scaled form (per level, spacing h): bh = h^2 b, rh = h^2 (b - A u) and the
// sweep weights c_j = omega m_j / h^2 are h-free. On the finest level b is
// the caller's unscaled array and bh = h^2 b is formed in the kernel (exact:
// h is a power of two).
#include "mg_common.cuh"
#include "mg_internal.h"

namespace mg {

// ---------------------------------------------------------------------------
// SPAI sweep.  Canonical evaluation at each interior point p:
//   s  = (u_W + u_E) + (u_S + u_N)
//   rh = fma(-4, u_p, bh_p) + s             (rh := 0 outside the interior)
//   E  = (rh_W + rh_E) + (rh_S + rh_N)
//   C  = (rh_SW + rh_SE) + (rh_NW + rh_NE)
//   u' = fma(c2, C, fma(c1, E, fma(c0, rh_p, u_p)))
// The pairs are shared between points: hp(q) = rh(q - x) + rh(q + x) gives
// E = hp(p) + (rh_S + rh_N) and C = hp(p - y) + hp(p + y).
// Block: K adjacent columns per thread (K independent FP64 chains; K = 2,
// measured fastest against 1 and 4): 256 / K threads cover the 256 columns
// X0 .. X0 + 255 of a strip, X0 = 254 bx - 1; columns 1 .. 254 of the strip
// are written, 0 and 255 supply halo residuals. Rows [y0, y0 + H). One
// barrier per row: at step j the u row j + 1 goes to the other half of the
// double buffer next to the residual row j, and every global load is issued
// one step before its use. Warps whose columns all lie at x >= n skip the
// FP64 arithmetic and only store the zeros their neighbours read.
// ZERO_U: the input is u = 0 (first sweep on a coarse level): rh = bh.
// NORM: accumulate the squared residual of the input over owned points.
// ---------------------------------------------------------------------------
template <typename T, bool ZERO_U, bool UNSCALED_B, bool NORM, int K>
__device__ __forceinline__ void sweep2d_tile(const T *__restrict__ u, const T *__restrict__ b, T *__restrict__ out,
                                              int n, int H, T c0, T c1, T c2, int hk, int tbx, int tby,
                                              double *__restrict__ partial)
{
    constexpr int NT = kSweepThreads / K;
    __shared__ T su[2][kSweepThreads + 2];
    __shared__ T sr[2][kSweepThreads + 2];
    const int t = threadIdx.x;
    const int X0 = tbx * kSweepCols - 1;
    const int xc0 = X0 + K * t;
    const int y0 = tby * H, y1 = min(y0 + H, n);
    const bool lt = t == 0, rt = t == NT - 1;
    const bool wact = X0 + K * (t & ~31) < n;  // the warp has a column inside the grid
    const size_t ld = (size_t)n;
    auto get = [&](const T *a, int yy, int xx) -> T {
        return (yy >= 0 && yy < n && xx >= 0 && xx < n) ? a[(size_t)yy * ld + xx] : T(0);
    };
    bool in[K], own[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int x = xc0 + k, c = K * t + k;
        in[k] = x >= 0 && x < n;
        own[k] = in[k] && c >= 1 && c <= kSweepCols;
    }
    T up[K], uc[K], un[K], unn[K], bcur[K], r1[K], r2[K], p1[K], p2[K];
    T hn = T(0), hnn = T(0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        up[k] = uc[k] = un[k] = unn[k] = T(0);
        r1[k] = r2[k] = p1[k] = p2[k] = T(0);
    }
    if (!ZERO_U) {
        const int b0 = (y0 - 1) & 1;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            up[k] = get(u, y0 - 2, xc0 + k);
            uc[k] = get(u, y0 - 1, xc0 + k);
            un[k] = get(u, y0, xc0 + k);
            su[b0][K * t + k + 1] = uc[k];
        }
        if (lt) su[b0][0] = get(u, y0 - 1, xc0 - 1);
        if (rt) su[b0][kSweepThreads + 1] = get(u, y0 - 1, xc0 + K);
        if (lt) hn = get(u, y0, xc0 - 1);
        if (rt) hn = get(u, y0, xc0 + K);
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < K; ++k) bcur[k] = get(b, y0 - 1, xc0 + k);
    SqSum acc;
    for (int j = y0 - 1; j <= y1; ++j) {
        const int buf = j & 1;
        T f[K], r[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            f[k] = bcur[k];
            bcur[k] = get(b, j + 1, xc0 + k);
            if (UNSCALED_B) f[k] = scale2(f[k], hk);
            r[k] = T(0);
        }
        if (!ZERO_U) {
#pragma unroll
            for (int k = 0; k < K; ++k) unn[k] = get(u, j + 2, xc0 + k);
            if (lt) hnn = get(u, j + 2, xc0 - 1);
            if (rt) hnn = get(u, j + 2, xc0 + K);
            if (wact) {
                const T wl = su[buf][K * t], wr = su[buf][K * t + K + 1];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const T W = k == 0 ? wl : uc[k - 1], E = k == K - 1 ? wr : uc[k + 1];
                    r[k] = radd(rfma(T(-4), uc[k], f[k]), radd(radd(W, E), radd(up[k], un[k])));
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) su[1 - buf][K * t + k + 1] = un[k];
            if (lt) su[1 - buf][0] = hn;
            if (rt) su[1 - buf][kSweepThreads + 1] = hn;
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) r[k] = f[k];
        }
        const bool jin = j >= 0 && j < n;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (!(in[k] && jin)) r[k] = T(0);
            if (NORM && own[k] && j >= y0 && j < y1) sq_add(acc, r[k]);
            sr[buf][K * t + k + 1] = r[k];
        }
        if (NORM && (j & 15) == 15) sq_flush(acc);  // at most 32 terms pending
        __syncthreads();
        T p[K];
        {
            const T rl = sr[buf][K * t], rr = sr[buf][K * t + K + 1];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const T W = k == 0 ? rl : r[k - 1], E = k == K - 1 ? rr : r[k + 1];
                const int c = K * t + k;
                p[k] = (c >= 1 && c <= kSweepCols && wact) ? radd(W, E) : T(0);
            }
        }
        if (j - 1 >= y0) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (!own[k]) continue;
                const T E = radd(p1[k], radd(r2[k], r[k]));
                const T C = radd(p2[k], p[k]);
                const T base = ZERO_U ? rmul(c0, r1[k]) : rfma(c0, r1[k], up[k]);
                out[(size_t)(j - 1) * ld + xc0 + k] = rfma(c2, C, rfma(c1, E, base));
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            r2[k] = r1[k];
            r1[k] = r[k];
            p2[k] = p1[k];
            p1[k] = p[k];
            if (!ZERO_U) {
                up[k] = uc[k];
                uc[k] = un[k];
                un[k] = unn[k];
            }
        }
        hn = hnn;
    }
    if (NORM) block_sum_store<NT>(sq_value(acc), partial);
}

// 128 threads, two columns each; the occupancy bound (10 blocks per SM)
// keeps the register count at 48, measured fastest for the FP64 form
template <typename T, bool ZERO_U, bool UNSCALED_B, bool NORM>
__global__ void __launch_bounds__(kSweepThreads / 2, 10)
sweep2d_kernel(const T *__restrict__ u, const T *__restrict__ b, T *__restrict__ out, int n, int H,
               T c0, T c1, T c2, int hk, double *__restrict__ partials)
{
    sweep2d_tile<T, ZERO_U, UNSCALED_B, NORM, 2>(u, b, out, n, H, c0, c1, c2, hk, blockIdx.x, blockIdx.y,
                                              NORM ? &partials[blockIdx.y * gridDim.x + blockIdx.x] : nullptr);
}

// ---------------------------------------------------------------------------
// Residual + full-weighting restriction. For coarse point (ic, jc) (0-based)
// with fine centre (2ic+1, 2jc+1):
//   along x, per fine row f:  t_f = (rh(2ic) + rh(2ic+2)) + 2 rh(2ic+1)
//   along y:                  v   = (t_{2jc} + t_{2jc+2}) + 2 t_{2jc+1}
//   bh_c = 0.25 v   (= 4 R rh with R = (1,2,1)/4 per axis, H^2/h^2 = 4)
// with rh evaluated as in the sweep. Block: kRestrictThreads (128) threads,
// thread t owns fine columns 2ic, 2ic+1 with ic = kRestrictCols*bx + t;
// threads 0 .. kRestrictCols-1 write.
// ---------------------------------------------------------------------------
template <typename T, bool UNSCALED_B>
__device__ __forceinline__ void resrestrict2d_tile(const T *__restrict__ u, const T *__restrict__ b,
                                                   T *__restrict__ bc, int n, int Hc, int hk, int tbx, int tby)
{
    __shared__ T su[2][2 * kRestrictThreads + 2];
    __shared__ T sr[2][kRestrictThreads + 1];
    const int nc = (n - 1) / 2;
    const int t = threadIdx.x;
    const int ic = tbx * kRestrictCols + t;
    const int fx = 2 * ic;  // this thread's fine columns: fx, fx + 1
    const int jc0 = tby * Hc;
    const int jc1 = min(jc0 + Hc, nc);
    const size_t ld = (size_t)n;
    auto get = [&](const T *a, int yy, int xx) -> T {
        return (yy >= 0 && yy < n && xx >= 0 && xx < n) ? a[(size_t)yy * ld + xx] : T(0);
    };
    const bool in0 = fx < n, in1 = fx + 1 < n;

    const int f0 = 2 * jc0, f1 = 2 * jc1;  // fine rows f0 .. f1 feed coarse rows jc0 .. jc1-1
    // one barrier per fine row: the u row f + 1 goes to the other half of the
    // double buffer at step f; global loads are issued one step before use
    const bool lt = t == 0, rt = t == kRestrictThreads - 1;
    T ua_prev = get(u, f0 - 1, fx), ub_prev = get(u, f0 - 1, fx + 1);
    T ua = get(u, f0, fx), ub = get(u, f0, fx + 1);
    T ua_next = get(u, f0 + 1, fx), ub_next = get(u, f0 + 1, fx + 1);
    T h_next = lt ? get(u, f0 + 1, fx - 1) : rt ? get(u, f0 + 1, fx + 2) : T(0);
    su[f0 & 1][2 * t + 1] = ua;
    su[f0 & 1][2 * t + 2] = ub;
    if (lt) su[f0 & 1][0] = get(u, f0, fx - 1);
    if (rt) su[f0 & 1][2 * kRestrictThreads + 1] = get(u, f0, fx + 2);
    T ba_next = get(b, f0, fx), bb_next = get(b, f0, fx + 1);
    __syncthreads();
    T t1 = T(0), t2 = T(0);  // x-pass of fine rows f-1, f-2
    for (int f = f0; f <= f1; ++f) {
        const int buf = f & 1;
        T ba = ba_next, bb = bb_next;
        ba_next = get(b, f + 1, fx);
        bb_next = get(b, f + 1, fx + 1);
        const T ua_nn = get(u, f + 2, fx), ub_nn = get(u, f + 2, fx + 1);
        const T h_nn = lt ? get(u, f + 2, fx - 1) : rt ? get(u, f + 2, fx + 2) : T(0);
        if (UNSCALED_B) {
            ba = scale2_ool(ba, hk);
            bb = scale2_ool(bb, hk);
        }
        const T sa = radd(radd(su[buf][2 * t], su[buf][2 * t + 2]), radd(ua_prev, ua_next));
        const T sb = radd(radd(su[buf][2 * t + 1], su[buf][2 * t + 3]), radd(ub_prev, ub_next));
        T ra = radd(rfma(T(-4), ua, ba), sa);
        T rb = radd(rfma(T(-4), ub, bb), sb);
        if (!in0 || f >= n) ra = T(0);
        if (!in1 || f >= n) rb = T(0);
        sr[buf][t] = ra;
        if (rt) sr[buf][kRestrictThreads] = T(0);  // never read by a writer
        su[1 - buf][2 * t + 1] = ua_next;
        su[1 - buf][2 * t + 2] = ub_next;
        if (lt) su[1 - buf][0] = h_next;
        if (rt) su[1 - buf][2 * kRestrictThreads + 1] = h_next;
        __syncthreads();
        const T tx = rfma(T(2), rb, radd(ra, sr[buf][t + 1]));
        if (f >= f0 + 2 && (f & 1) == 0 && t < kRestrictCols && ic < nc) {
            const int jc = f / 2 - 1;
            const T v = rfma(T(2), t1, radd(t2, tx));
            bc[(size_t)jc * nc + ic] = scale2_ool<-2>(v);  // 0.25 v
        }
        t2 = t1;
        t1 = tx;
        ua_prev = ua;
        ub_prev = ub;
        ua = ua_next;
        ub = ub_next;
        ua_next = ua_nn;
        ub_next = ub_nn;
        h_next = h_nn;
    }
}

// 128-thread blocks, at most 10 per SM (measured fastest for the FP64 form
// against 256-thread blocks at 4 to 8 per SM and 128-thread blocks at 8, 12)
template <typename T, bool UNSCALED_B>
__global__ void __launch_bounds__(kRestrictThreads, 10)
resrestrict2d_kernel(const T *__restrict__ u, const T *__restrict__ b, T *__restrict__ bc, int n,
                     int Hc, int hk)
{
    resrestrict2d_tile<T, UNSCALED_B>(u, b, bc, n, Hc, hk, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Bilinear interpolation + correction u += P e. Thread k owns fine columns
// 2k (between coarse k-1 and k) and 2k+1 (on coarse k); per coarse row m:
//   along x: ex(2k) = 0.5 (e[m][k-1] + e[m][k]),  ex(2k+1) = e[m][k]
//   along y: fine row 2m+1 gets ex_m, fine row 2m gets 0.5 (ex_{m-1} + ex_m)
//   u = u + value            (e is zero outside the coarse interior)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void prolong2d_tile(const T *__restrict__ e, T *__restrict__ u, int n, int Hc, int tbx,
                                               int tby)
{
    const int nc = (n - 1) / 2;
    const int k = tbx * kProlongThreads + threadIdx.x;
    if (k > nc) return;
    const int m0 = tby * Hc;
    const int m1 = min(m0 + Hc, nc + 1);
    const size_t ldc = (size_t)nc, ld = (size_t)n;
    auto ge = [&](int mm, int kk) -> T {
        return (mm >= 0 && mm < nc && kk >= 0 && kk < nc) ? e[(size_t)mm * ldc + kk] : T(0);
    };
    auto xpass = [&](int mm, T &odd, T &on) {
        on = ge(mm, k);
        odd = scale2_ool<-1>(radd(ge(mm, k - 1), on));  // 0.5 (a + b)
    };
    T pa, pb;  // x-pass of coarse row m-1: columns 2k, 2k+1
    xpass(m0 - 1, pa, pb);
    const int fa = 2 * k, fb = 2 * k + 1;
    const bool inb = fb < n;
    // software pipeline: step m + 1's coarse values and u values are loaded
    // before step m is written (this thread owns columns fa, fb, the block its
    // fine rows 2 m0 .. 2 m1 - 1)
    auto ld_rows = [&](int m, T &ea, T &eb, T &oa, T &ob) {
        const T *re = u + (size_t)(2 * m) * ld;
        ea = re[fa];
        eb = inb ? re[fb] : T(0);
        oa = ob = T(0);
        if (m < nc) {
            const T *ro = re + ld;
            oa = ro[fa];
            ob = inb ? ro[fb] : T(0);
        }
    };
    T ca, cb, ea, eb, oa, ob;
    xpass(m0, ca, cb);
    ld_rows(m0, ea, eb, oa, ob);
    for (int m = m0; m < m1; ++m) {
        T na = T(0), nb = T(0), nea = T(0), neb = T(0), noa = T(0), nob = T(0);
        if (m + 1 < m1) {
            xpass(m + 1, na, nb);
            ld_rows(m + 1, nea, neb, noa, nob);
        }
        {   // fine row 2m
            T *row = u + (size_t)(2 * m) * ld;
            row[fa] = radd(ea, scale2_ool<-1>(radd(pa, ca)));
            if (inb) row[fb] = radd(eb, scale2_ool<-1>(radd(pb, cb)));
        }
        if (m < nc) {  // fine row 2m+1
            T *row = u + (size_t)(2 * m + 1) * ld;
            row[fa] = radd(oa, ca);
            if (inb) row[fb] = radd(ob, cb);
        }
        pa = ca;
        pb = cb;
        ca = na;
        cb = nb;
        ea = nea;
        eb = neb;
        oa = noa;
        ob = nob;
    }
}

template <typename T>
__global__ void __launch_bounds__(kProlongThreads)
prolong2d_kernel(const T *__restrict__ e, T *__restrict__ u, int n, int Hc)
{
    prolong2d_tile<T>(e, u, n, Hc, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// FP64 residual for iterative refinement: rh = fma(-4, u, h^2 b) + s exactly
// as in the sweep, written as OutT (the cycle's precision) together with one
// partial sum of rh^2 per block. Same layout as the sweep: 128 threads, two
// adjacent columns each (columns 1 .. 254 of the strip are written), one
// barrier per row, loads one step ahead. Acc: the squared-norm accumulator
// (SqSum off the FP64 pipe; Fp64Sum where registers are short).
// ---------------------------------------------------------------------------
template <typename InT, typename OutT, typename Acc = SqSum>
__device__ __forceinline__ void residual2d_tile(const InT *__restrict__ u, const InT *__restrict__ b,
                                                OutT *__restrict__ rh_out, int n, int H, int hk, bool unscaled,
                                                int tbx, int tby, double *__restrict__ partial, long opitch = 0,
                                                long ooff = 0)
{
    constexpr int NT = kSweepThreads / 2;
    __shared__ InT su[2][kSweepThreads + 2];  // [c + 1]: column X0 + c, c in -1 .. 256
    const int t = threadIdx.x;
    const int X0 = tbx * kSweepCols - 1;
    const int xa = X0 + 2 * t, xb = xa + 1;
    const int y0 = tby * H;
    const int y1 = min(y0 + H, n);
    const bool owna = t >= 1 && xa < n, ownb = t <= NT - 2 && xb < n;
    const bool lt = t == 0, rt = t == NT - 1;
    const bool wact = X0 + 2 * (t & ~31) < n;  // as in the sweep: all-outside warps skip the FP64 work
    const size_t ld = (size_t)n;
    auto get = [&](const InT *a, int yy, int xx) -> InT {
        return (yy >= 0 && yy < n && xx >= 0 && xx < n) ? a[(size_t)yy * ld + xx] : InT(0);
    };
    InT ap = get(u, y0 - 1, xa), bp = get(u, y0 - 1, xb);
    InT ac = get(u, y0, xa), bc = get(u, y0, xb);
    InT an = get(u, y0 + 1, xa), bn = get(u, y0 + 1, xb);
    InT hn = lt ? get(u, y0 + 1, xa - 1) : rt ? get(u, y0 + 1, xb + 1) : InT(0);
    su[y0 & 1][2 * t + 1] = ac;
    su[y0 & 1][2 * t + 2] = bc;
    if (lt) su[y0 & 1][0] = get(u, y0, xa - 1);
    if (rt) su[y0 & 1][kSweepThreads + 1] = get(u, y0, xb + 1);
    InT fa_next = get(b, y0, xa), fb_next = get(b, y0, xb);
    __syncthreads();
    Acc acc;
    for (int j = y0; j < y1; ++j) {
        const int buf = j & 1;
        InT fa = fa_next, fb = fb_next;
        fa_next = get(b, j + 1, xa);
        fb_next = get(b, j + 1, xb);
        const InT ann = get(u, j + 2, xa), bnn = get(u, j + 2, xb);
        const InT hnn = lt ? get(u, j + 2, xa - 1) : rt ? get(u, j + 2, xb + 1) : InT(0);
        if (unscaled) {
            fa = scale2(fa, hk);
            fb = scale2(fb, hk);
        }
        InT ra = InT(0), rb = InT(0);
        if (wact) {
            ra = radd(rfma(InT(-4), ac, fa), radd(radd(su[buf][2 * t], bc), radd(ap, an)));
            rb = radd(rfma(InT(-4), bc, fb), radd(radd(ac, su[buf][2 * t + 3]), radd(bp, bn)));
        }
        if (owna) {
            sq_add(acc, ra);
            if (rh_out) rh_out[opitch ? ooff + j * opitch + xa : (long)j * ld + xa] = to_out<OutT>(ra);
        }
        if (ownb) {
            sq_add(acc, rb);
            if (rh_out) rh_out[opitch ? ooff + j * opitch + xb : (long)j * ld + xb] = to_out<OutT>(rb);
        }
        if ((j & 15) == 15) sq_flush(acc);  // at most 32 terms pending
        su[1 - buf][2 * t + 1] = an;
        su[1 - buf][2 * t + 2] = bn;
        if (lt) su[1 - buf][0] = hn;
        if (rt) su[1 - buf][kSweepThreads + 1] = hn;
        __syncthreads();
        ap = ac;
        ac = an;
        an = ann;
        bp = bc;
        bc = bn;
        bn = bnn;
        hn = hnn;
    }
    if (partial) block_sum_store<NT>(sq_value(acc), partial);
}

// at most 12 blocks per SM (measured fastest for the FP64 form); UNSC and
// PAD (padded output layout) are compile-time so that the inlined tile
// carries neither choice in registers
template <typename InT, typename OutT, bool UNSC, bool PAD>
__global__ void __launch_bounds__(kSweepThreads / 2, 12)
residual2d_kernel(const InT *__restrict__ u, const InT *__restrict__ b, OutT *__restrict__ rh_out,
                  int n, int H, int hk, double *__restrict__ partials, long opitch, long ooff)
{
    residual2d_tile<InT, OutT>(u, b, rh_out, n, H, hk, UNSC, blockIdx.x, blockIdx.y,
                               partials ? &partials[blockIdx.y * gridDim.x + blockIdx.x] : nullptr,
                               PAD ? opitch : 0, PAD ? ooff : 0);
}

// ---------------------------------------------------------------------------
// Batched FP64 residual (the refinement step of mg_batched.cu): one launch
// covers the same-size finest level of many problems. The launch is
// persistent: gridDim.x blocks loop over (problem, tile) items; items of
// problems whose flag in `active` is 0 are skipped.
// ---------------------------------------------------------------------------
// FP64 residual of the caller's arrays, written as OutT, with one partial sum
// per tile at the item's partial offset.
template <typename OutT>
__global__ void __launch_bounds__(kSweepThreads / 2, 12)
residual2d_batched(const BRes<OutT> *__restrict__ tab, int nprob, const int *__restrict__ active, int n, int H,
                   int bx, int by, int hk, long opitch, long ooff)
{
    const int per = bx * by, total = nprob * per;
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int j = it / per, r = it - j * per;
        const BRes<OutT> e = tab[j];
        if (active[e.problem])
            residual2d_tile<double, OutT, Fp64Sum>(e.u, e.b, e.out, n, H, hk, true, r % bx, r / bx, e.partials + r,
                                                   opitch, ooff);
        __syncthreads();
    }
}

// All sizes in one launch: the item's group is found by a scan over the few
// groups' first items (descending n: the large items are handed out first).
__global__ void __launch_bounds__(kSweepThreads / 2, 12)
residual2d_batched_all(const BResGroup *__restrict__ groups, int ngroups, int total, const int *__restrict__ active)
{
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        int gi = 0;
        while (gi + 1 < ngroups && it >= groups[gi + 1].item0) ++gi;
        const BResGroup G = groups[gi];
        const int local = it - G.item0, per = G.bx * G.by;
        const int j = local / per, r = local - j * per;
        const BRes<float> e = G.tab[j];
        if (active[e.problem])
            residual2d_tile<double, float, Fp64Sum>(e.u, e.b, e.out, G.n, G.H, G.hk, true, r % G.bx, r / G.bx,
                                                    e.partials + r, G.pitch, G.off);
        __syncthreads();
    }
}

// The same items for a solve from u = 0: the residual of every tile is h^2 b
// itself (the residual kernel's value for u = 0: fma(-4, 0, h^2 b) plus a
// zero neighbour sum, which turns -0 into +0), rounded to FP32 once, with
// the tile's squared-norm partial; no FP64 arithmetic per point.
__global__ void __launch_bounds__(kSweepThreads / 2)
residual2d_batched_zero(const BResGroup *__restrict__ groups, int ngroups, int total)
{
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        int gi = 0;
        while (gi + 1 < ngroups && it >= groups[gi + 1].item0) ++gi;
        const BResGroup G = groups[gi];
        const int local = it - G.item0, per = G.bx * G.by;
        const int j = local / per, r = local - j * per;
        const BRes<float> e = G.tab[j];
        const int tbx = r % G.bx, tby = r / G.bx, n = G.n;
        const int x0 = tbx * kSweepCols, x1 = min(x0 + kSweepCols, n);
        const int y0 = tby * G.H, y1 = min(y0 + G.H, n);
        SqSum acc;
        int cnt = 0;
        for (int y = y0; y < y1; ++y) {
            for (int x = x0 + (int)threadIdx.x; x < x1; x += blockDim.x) {
                double v = scale2(e.b[(long)y * n + x], G.hk);
                if ((__double_as_longlong(v) << 1) == 0) v = 0.0;  // -0 -> +0
                sq_add(acc, v);
                e.out[G.off + (long)y * G.pitch + x] = narrow_rn(v);
            }
            if (++cnt == 16) {  // at most 32 terms pending
                sq_flush(acc);
                cnt = 0;
            }
        }
        block_sum_store<kSweepThreads / 2>(sq_value(acc), e.partials + r);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

constexpr int kBatchedResidualRows = 32;

// Row chunks sized for about one wave of resident blocks (10 per SM, the
// occupancy bound of the sweep and the restriction); fewer, taller chunks
// save prologue rows but measured slower (8 or fewer per SM), more did not help
Grid2 sweep2d_grid(int n)
{
    Grid2 g;
    g.bx = (n + kSweepCols - 1) / kSweepCols;
    g.H = chunk_rows(g.bx, n, 10 * num_sms(), 2, 64);
    g.by = (n + g.H - 1) / g.H;
    return g;
}

template <typename T>
cudaError_t launch_sweep2d(const T *u, const T *b, bool unscaled, T *out, int n, const double *c,
                           double *partials, cudaStream_t s)
{
    const Grid2 g = sweep2d_grid(n);
    const dim3 grid(g.bx, g.by);
    const int hk = h2_exponent(n);
    const T c0 = T(c[0]), c1 = T(c[1]), c2 = T(c[2]);
#define MG_SWEEP(ZU, UB, NRM) \
    sweep2d_kernel<T, ZU, UB, NRM><<<grid, kSweepThreads / 2, 0, s>>>(u, b, out, n, g.H, c0, c1, c2, hk, partials)
    const bool z = u == nullptr, nrm = partials != nullptr;
    if (z) {
        if (unscaled) {
            if (nrm) MG_SWEEP(true, true, true); else MG_SWEEP(true, true, false);
        } else {
            if (nrm) MG_SWEEP(true, false, true); else MG_SWEEP(true, false, false);
        }
    } else {
        if (unscaled) {
            if (nrm) MG_SWEEP(false, true, true); else MG_SWEEP(false, true, false);
        } else {
            if (nrm) MG_SWEEP(false, false, true); else MG_SWEEP(false, false, false);
        }
    }
#undef MG_SWEEP
    count_launch(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_resrestrict2d(const T *u, const T *b, bool unscaled, T *bc, int n, cudaStream_t s)
{
    const int nc = (n - 1) / 2;
    const int bx = (nc + kRestrictCols - 1) / kRestrictCols;
    const int Hc = chunk_rows(bx, nc, 10 * num_sms(), 1, 32);
    const dim3 grid(bx, (nc + Hc - 1) / Hc);
    const int hk = h2_exponent(n);
    if (unscaled)
        resrestrict2d_kernel<T, true><<<grid, kRestrictThreads, 0, s>>>(u, b, bc, n, Hc, hk);
    else
        resrestrict2d_kernel<T, false><<<grid, kRestrictThreads, 0, s>>>(u, b, bc, n, Hc, hk);
    count_launch(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong2d(const T *e, T *u, int n, cudaStream_t s)
{
    const int nc = (n - 1) / 2;
    const int bx = (nc + 1 + kProlongThreads - 1) / kProlongThreads;
    const int Hc = chunk_rows(bx, nc + 1, 8 * num_sms(), 1, 32);
    const dim3 grid(bx, (nc + 1 + Hc - 1) / Hc);
    prolong2d_kernel<T><<<grid, kProlongThreads, 0, s>>>(e, u, n, Hc);
    count_launch(1);
    return cudaGetLastError();
}

template <typename InT, typename OutT>
cudaError_t launch_residual2d(const InT *u, const InT *b, bool unscaled, OutT *rh, int n, double *partials,
                              cudaStream_t s, long out_pitch, long out_off)
{
    const Grid2 g = sweep2d_grid(n);
    const dim3 grid(g.bx, g.by);
    const int hk = h2_exponent(n);
    const bool pad = out_pitch != 0;
    if (unscaled && pad)
        residual2d_kernel<InT, OutT, true, true><<<grid, kSweepThreads / 2, 0, s>>>(u, b, rh, n, g.H, hk, partials,
                                                                                  out_pitch, out_off);
    else if (unscaled)
        residual2d_kernel<InT, OutT, true, false><<<grid, kSweepThreads / 2, 0, s>>>(u, b, rh, n, g.H, hk, partials,
                                                                                   out_pitch, out_off);
    else if (pad)
        residual2d_kernel<InT, OutT, false, true><<<grid, kSweepThreads / 2, 0, s>>>(u, b, rh, n, g.H, hk, partials,
                                                                                   out_pitch, out_off);
    else
        residual2d_kernel<InT, OutT, false, false><<<grid, kSweepThreads / 2, 0, s>>>(u, b, rh, n, g.H, hk, partials,
                                                                                    out_pitch, out_off);
    count_launch(1);
    return cudaGetLastError();
}
template cudaError_t launch_residual2d<double, double>(const double *, const double *, bool, double *, int,
                                                       double *, cudaStream_t, long, long);
template cudaError_t launch_residual2d<double, float>(const double *, const double *, bool, float *, int,
                                                      double *, cudaStream_t, long, long);
template cudaError_t launch_residual2d<float, float>(const float *, const float *, bool, float *, int,
                                                     double *, cudaStream_t, long, long);


// ---- batched launchers ------------------------------------------------------
static int persistent_grid(const void *fn, int threads, long items)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
    return (int)std::max<long>(1, std::min<long>(items, (long)per_sm * num_sms()));
}

// The batch supplies the parallelism, so the batched residual marches tall
// row chunks (a chunk's prologue costs three rows and a barrier)
static Grid2 residual2d_batched_grid(int n)
{
    Grid2 g;
    g.bx = (n + kSweepCols - 1) / kSweepCols;
    g.H = n < kBatchedResidualRows ? n : kBatchedResidualRows;
    g.by = (n + g.H - 1) / g.H;
    return g;
}

int residual2d_batched_tiles(int n)
{
    const Grid2 g = residual2d_batched_grid(n);
    return g.bx * g.by;
}

int residual2d_batched_group(BResGroup &g, int nprob)
{
    const Grid2 q = residual2d_batched_grid(g.n);
    g.H = q.H;
    g.bx = q.bx;
    g.by = q.by;
    g.hk = h2_exponent(g.n);
    return nprob * q.bx * q.by;
}

cudaError_t launch_residual2d_batched_zero(const BResGroup *groups, int ngroups, int items, cudaStream_t s)
{
    const int grid = persistent_grid((const void *)residual2d_batched_zero, kSweepThreads / 2, items);
    residual2d_batched_zero<<<grid, kSweepThreads / 2, 0, s>>>(groups, ngroups, items);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_residual2d_batched_all(const BResGroup *groups, int ngroups, int items, const int *active,
                                          cudaStream_t s)
{
    const int grid = persistent_grid((const void *)residual2d_batched_all, kSweepThreads / 2, items);
    residual2d_batched_all<<<grid, kSweepThreads / 2, 0, s>>>(groups, ngroups, items, active);
    count_launch(1);
    return cudaGetLastError();
}

template <typename OutT>
cudaError_t launch_residual2d_batched(const BRes<OutT> *tab, int nprob, const int *active, int n, cudaStream_t s,
                                      long opitch, long ooff)
{
    const Grid2 g = residual2d_batched_grid(n);
    const long items = (long)nprob * g.bx * g.by;
    const int grid = persistent_grid((const void *)residual2d_batched<OutT>, kSweepThreads / 2, items);
    residual2d_batched<OutT><<<grid, kSweepThreads / 2, 0, s>>>(tab, nprob, active, n, g.H, g.bx, g.by, h2_exponent(n),
                                                            opitch, ooff);
    count_launch(1);
    return cudaGetLastError();
}

template cudaError_t launch_residual2d_batched<float>(const BRes<float> *, int, const int *, int, cudaStream_t, long,
                                                      long);
template cudaError_t launch_residual2d_batched<double>(const BRes<double> *, int, const int *, int, cudaStream_t, long,
                                                       long);

#define MG_INST(T)                                                                                   \
    template cudaError_t launch_sweep2d<T>(const T *, const T *, bool, T *, int, const double *,     \
                                           double *, cudaStream_t);                                  \
    template cudaError_t launch_resrestrict2d<T>(const T *, const T *, bool, T *, int, cudaStream_t); \
    template cudaError_t launch_prolong2d<T>(const T *, T *, int, cudaStream_t);
MG_INST(double)
MG_INST(float)
#undef MG_INST

}  // namespace mg
