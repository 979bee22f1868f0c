// mg_pl2d.cu -- FP32 2D kernels on the padded level layout (internal levels
// of the FP32 cycles: refinement and batched solves).
//
// FP32 stencil work is bound by HBM bandwidth, not arithmetic, so these
// kernels are built for bytes: every level is stored with a zero ghost ring
// and padded, 16-byte-aligned rows (Pitch2 below), so a thread moves four
// consecutive columns with one float4 load/store and no per-element bounds
// checks (ghost cells read as zero; only the residual is forced to zero
// outside the interior). The formulas and their operation order are those of
// the compact kernels in mg_kernels2d.cu (same results bit for bit).
#include "mg_common.cuh"
#include "mg_internal.h"

namespace mg {

constexpr int kPLThreads = 128;             // threads per block
constexpr int kPLCols = 4 * kPLThreads;     // columns per strip (sweep, residual)

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float &c4(float4 &v, int k) { return (&v.x)[k]; }
__device__ __forceinline__ float cc4(const float4 &v, int k) { return (&v.x)[k]; }

// store the valid columns of a float4 at interior column x (x % 4 == 0)
__device__ __forceinline__ void st4_valid(float *p, float4 v, int x, int n)
{
    if (x + 3 < n) {
        st4(p, v);
    } else {
        for (int k = 0; k < 4; ++k)
            if (x + k < n) p[k] = cc4(v, k);
    }
}

// ---------------------------------------------------------------------------
// SPAI sweep (formula as sweep2d_kernel). Block: 128 threads x 4 columns =
// 512-column strip, marching over rows [y0, y0 + H). Shared rows hold the
// strip plus 4 columns on each side; the residual at the two halo columns is
// computed by the edge threads from rolling scalars.
// ---------------------------------------------------------------------------
template <bool ZERO_U, bool NORM, bool ACC64 = false>
__device__ __forceinline__ void sweep2d_pl_tile(const float *__restrict__ u, const float *__restrict__ b,
                                                float *__restrict__ out, Pitch2 g, int H, float c0, float c1, float c2,
                                                int tbx, int tby, double *__restrict__ partial,
                                                double *__restrict__ u64 = nullptr)
{
    __shared__ __align__(16) float su[2][kPLCols + 8];
    __shared__ __align__(16) float sr[2][kPLCols + 8];
    const int n = g.n, t = threadIdx.x;
    const int xb = tbx * kPLCols, x = xb + 4 * t;
    const int y0 = tby * H, y1 = min(y0 + H, n);
    const float *U = u + g.off, *Bp = b + g.off;  // element (x, y) at [y * pitch + x], x, y in [-1, n]
    float *O = out + g.off;
    const long P = g.pitch;
    auto rowok = [&](int j) { return j >= -1 && j <= n; };
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    auto row4 = [&](const float *a, int j, int xx) { return rowok(j) ? ld4(a + j * P + xx) : z4; };
    auto row1 = [&](const float *a, int j, int xx) { return rowok(j) ? a[j * P + xx] : 0.f; };

    float4 up = z4, uc = z4, un = z4, bn = z4;
    float4 r1 = z4, r2 = z4, h1 = z4, h2 = z4;
    // halo columns: thread 0 owns xb - 1, thread 127 owns xb + kPLCols
    const bool lt = t == 0, rt = t == kPLThreads - 1;
    const int xh = lt ? xb - 1 : xb + kPLCols;
    float hp_ = 0.f, hc = 0.f, hn = 0.f, hb = 0.f;
    if (!ZERO_U) {
        up = row4(U, y0 - 2, x);
        uc = row4(U, y0 - 1, x);
        if (lt || rt) {
            hp_ = row1(U, y0 - 2, xh);
            hc = row1(U, y0 - 1, xh);
        }
    }
    bn = row4(Bp, y0 - 1, x);
    if (lt || rt) hb = row1(Bp, y0 - 1, xh);
    SqSum acc;
    // refinement epilogue: each warp stages its 128 FP32 results in shared
    // memory and lane l updates the FP64 columns xw + l + 32 k (k < 4), so
    // every FP64 access of the warp covers 256 contiguous bytes; the FP64
    // row j is loaded at step j and updated at step j + 1
    __shared__ __align__(16) float sacc[kPLThreads / 32][4 * 32];
    const int lane = t & 31, wrp = t >> 5;
    const int xw = xb + 128 * wrp;
    double u64c[4] = {0.0, 0.0, 0.0, 0.0}, u64n[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = y0 - 1; j <= y1; ++j) {
        const int buf = j & 1;
        const float4 bc = bn;
        const float hbc = hb;
        if (ACC64 && j >= y0 && j < y1) {
            const double *ur = u64 + (long)j * n + xw + lane;
            for (int k = 0; k < 4; ++k)
                if (xw + lane + 32 * k < n) u64n[k] = ur[32 * k];
        }
        bn = row4(Bp, j + 1, x);  // prefetch
        if (lt || rt) hb = row1(Bp, j + 1, xh);
        float4 r;
        float rh = 0.f;
        const bool jin = j >= 0 && j < n;
        if (!ZERO_U) {
            un = row4(U, j + 1, x);
            if (lt || rt) hn = row1(U, j + 1, xh);
            st4(&su[buf][4 + 4 * t], uc);
            if (lt) st4(&su[buf][0], row4(U, j, xb - 4));
            if (rt) st4(&su[buf][kPLCols + 4], row4(U, j, xb + kPLCols));
            __syncthreads();
            const float *s = &su[buf][4 + 4 * t];
            for (int k = 0; k < 4; ++k) {
                const float ss = radd(radd(s[k - 1], s[k + 1]), radd(c4(up, k), c4(un, k)));
                c4(r, k) = radd(rfma(-4.f, c4(uc, k), cc4(bc, k)), ss);
            }
            if (lt || rt) {
                const float *sh = lt ? &su[buf][3] : &su[buf][kPLCols + 4];
                const float ss = radd(radd(sh[-1], sh[1]), radd(hp_, hn));
                rh = radd(rfma(-4.f, hc, hbc), ss);
            }
        } else {
            r = bc;
            rh = hbc;
        }
        for (int k = 0; k < 4; ++k)
            if (!(jin && x + k < n)) c4(r, k) = 0.f;
        if ((lt || rt) && !(jin && xh >= 0 && xh < n)) rh = 0.f;
        if (NORM && j >= y0 && j < y1)
            for (int k = 0; k < 4; ++k) sq_add(acc, c4(r, k));
        if (NORM && (j & 7) == 7) sq_flush(acc);  // at most 32 terms pending
        st4(&sr[buf][4 + 4 * t], r);
        if (lt) sr[buf][3] = rh;
        if (rt) sr[buf][kPLCols + 4] = rh;
        __syncthreads();
        float4 hp;
        {
            const float *s = &sr[buf][4 + 4 * t];
            for (int k = 0; k < 4; ++k) c4(hp, k) = radd(s[k - 1], s[k + 1]);
        }
        if (j - 1 >= y0) {
            float4 o;
            for (int k = 0; k < 4; ++k) {
                const float E = radd(c4(h1, k), radd(c4(r2, k), c4(r, k)));
                const float C = radd(c4(h2, k), c4(hp, k));
                const float base = ZERO_U ? rmul(c0, c4(r1, k)) : rfma(c0, c4(r1, k), c4(up, k));
                c4(o, k) = rfma(c2, C, rfma(c1, E, base));
            }
            if (ACC64) {
                // the correction goes straight into the caller's FP64
                // solution (compact rows of n doubles)
                st4(&sacc[wrp][4 * lane], o);
                __syncwarp();
                double *ur = u64 + (long)(j - 1) * n + xw + lane;
                for (int k = 0; k < 4; ++k)
                    if (xw + lane + 32 * k < n) ur[32 * k] = __dadd_rn(u64c[k], widen(sacc[wrp][lane + 32 * k]));
                __syncwarp();
            } else if (x < n) {
                st4_valid(O + (long)(j - 1) * P + x, o, x, n);
            }
        }
        r2 = r1;
        r1 = r;
        h2 = h1;
        h1 = hp;
        if (!ZERO_U) {
            up = uc;
            uc = un;
            hp_ = hc;
            hc = hn;
        }
        if (ACC64)
            for (int k = 0; k < 4; ++k) u64c[k] = u64n[k];
    }
    if (NORM) block_sum_store<kPLThreads>(sq_value(acc), partial);
}

template <bool ZERO_U, bool NORM>
__global__ void __launch_bounds__(kPLThreads)
sweep2d_pl_kernel(const float *__restrict__ u, const float *__restrict__ b, float *__restrict__ out, Pitch2 g, int H,
                  float c0, float c1, float c2, double *__restrict__ partials)
{
    sweep2d_pl_tile<ZERO_U, NORM>(u, b, out, g, H, c0, c1, c2, blockIdx.x, blockIdx.y,
                                  NORM ? &partials[blockIdx.y * gridDim.x + blockIdx.x] : nullptr);
}

// the last post-sweep of a refinement cycle: u64 += (u + W rh) computed in FP32
__global__ void __launch_bounds__(kPLThreads)
sweep2d_pl_acc64_kernel(const float *__restrict__ u, const float *__restrict__ b, double *__restrict__ u64, Pitch2 g,
                        int H, float c0, float c1, float c2)
{
    sweep2d_pl_tile<false, false, true>(u, b, nullptr, g, H, c0, c1, c2, blockIdx.x, blockIdx.y, nullptr, u64);
}

// ---------------------------------------------------------------------------
// Residual + full weighting (formula as resrestrict2d_kernel). Thread t owns
// coarse columns 4t .. 4t+3 of the block's 512-column coarse strip, i.e. the
// fine columns 2 ic .. 2 ic + 7 (two float4), marching over fine rows.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void resrestrict2d_pl_tile(const float *__restrict__ u, const float *__restrict__ b,
                                                      float *__restrict__ bc, Pitch2 g, Pitch2 gc, int Hc, int tbx,
                                                      int tby)
{
    // fine strip: columns [2 icb, 2 icb + 2*kPLCols) plus one column each side
    __shared__ __align__(16) float su[2][2 * kPLCols + 8];
    __shared__ __align__(16) float sr[2][2 * kPLCols + 8];
    const int n = g.n, nc = gc.n, t = threadIdx.x;
    const int icb = tbx * kPLCols, ic = icb + 4 * t;
    const int fxb = 2 * icb, fx = 2 * ic;  // fine column of this thread's first value
    const int jc0 = tby * Hc, jc1 = min(jc0 + Hc, nc);
    const float *U = u + g.off, *Bp = b + g.off;
    float *Oc = bc + gc.off;
    const long P = g.pitch, Pc = gc.pitch;
    auto rowok = [&](int j) { return j >= -1 && j <= n; };
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // a float4 starting at column xx <= n stays inside the padded row
    auto row4 = [&](const float *a, int j, int xx) { return rowok(j) && xx <= n ? ld4(a + j * P + xx) : z4; };
    const int f0 = 2 * jc0, f1 = 2 * jc1;
    // rolling fine rows (8 columns per thread: two float4)
    float4 pa = row4(U, f0 - 1, fx), pb = row4(U, f0 - 1, fx + 4);
    float4 ca = row4(U, f0, fx), cb = row4(U, f0, fx + 4);
    float4 t1 = z4, t2 = z4;  // x-pass of fine rows f-1, f-2 (4 coarse columns)
    for (int f = f0; f <= f1; ++f) {
        const int buf = f & 1;
        const float4 na = row4(U, f + 1, fx), nb = row4(U, f + 1, fx + 4);
        const float4 ba = row4(Bp, f, fx), bb = row4(Bp, f, fx + 4);
        // horizontal neighbours: within a thread from registers, across
        // threads of a warp by shuffles, across warps through shared memory
        // (only the warp-edge values are stored)
        const int lane = t & 31;
        if (lane == 0) su[buf][4 + 8 * t] = ca.x;
        if (lane == 31) su[buf][11 + 8 * t] = cb.w;
        if (t == 0) su[buf][3] = row4(U, f, fxb - 4).w;
        if (t == kPLThreads - 1) su[buf][2 * kPLCols + 4] = row4(U, f, fxb + 2 * kPLCols).x;
        __syncthreads();
        float r[8];
        {
            float uw = __shfl_up_sync(0xffffffffu, cb.w, 1), ue = __shfl_down_sync(0xffffffffu, ca.x, 1);
            if (lane == 0) uw = su[buf][3 + 8 * t];
            if (lane == 31) ue = su[buf][12 + 8 * t];
            const float uc8[8] = {ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
            for (int k = 0; k < 8; ++k) {
                const float uu = k < 4 ? cc4(pa, k) : cc4(pb, k - 4);
                const float ud = k < 4 ? cc4(na, k) : cc4(nb, k - 4);
                const float bk = k < 4 ? cc4(ba, k) : cc4(bb, k - 4);
                const float W = k == 0 ? uw : uc8[k - 1], E = k == 7 ? ue : uc8[k + 1];
                const float ss = radd(radd(W, E), radd(uu, ud));
                r[k] = radd(rfma(-4.f, uc8[k], bk), ss);
                if (!(fx + k < n && f < n)) r[k] = 0.f;
            }
        }
        // the right neighbour fine column 2 ic + 8 comes from the next thread
        if (lane == 0) sr[buf][4 + 8 * t] = r[0];
        if (t == kPLThreads - 1) {
            // fine column fxb + 2*kPLCols: residual recomputed from global memory
            const int xr = fxb + 2 * kPLCols;
            float rr = 0.f;
            if (xr < n && f < n) {
                const float ss = radd(radd(U[(long)f * P + xr - 1], U[(long)f * P + xr + 1]),
                                      radd(U[(long)(f - 1) * P + xr], U[(long)(f + 1) * P + xr]));
                rr = radd(rfma(-4.f, U[(long)f * P + xr], Bp[(long)f * P + xr]), ss);
            }
            sr[buf][2 * kPLCols + 4] = rr;
        }
        __syncthreads();
        float4 tx;
        {
            float r8 = __shfl_down_sync(0xffffffffu, r[0], 1);
            if (lane == 31) r8 = sr[buf][12 + 8 * t];
            for (int k = 0; k < 4; ++k) c4(tx, k) = rfma(2.f, r[2 * k + 1], radd(r[2 * k], k == 3 ? r8 : r[2 * k + 2]));
        }
        if (f >= f0 + 2 && (f & 1) == 0 && ic < nc) {
            const int jc = f / 2 - 1;
            float4 v;
            for (int k = 0; k < 4; ++k) c4(v, k) = scale2<-2>(rfma(2.f, c4(t1, k), radd(c4(t2, k), c4(tx, k))));
            st4_valid(Oc + (long)jc * Pc + ic, v, ic, nc);
        }
        t2 = t1;
        t1 = tx;
        pa = ca;
        pb = cb;
        ca = na;
        cb = nb;
    }
}

__global__ void __launch_bounds__(kPLThreads)
resrestrict2d_pl_kernel(const float *__restrict__ u, const float *__restrict__ b, float *__restrict__ bc, Pitch2 g,
                        Pitch2 gc, int Hc)
{
    resrestrict2d_pl_tile(u, b, bc, g, gc, Hc, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Interpolation + correction (formula as prolong2d_kernel). Thread t owns
// coarse columns k = 4t .. 4t+3 of a 512-column coarse strip, i.e. fine
// columns 2k, 2k+1 (8 values), marching over coarse rows m.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void prolong2d_pl_tile(const float *__restrict__ e, float *__restrict__ u, Pitch2 g,
                                                  Pitch2 gc, int Hc, int tbx, int tby)
{
    const int n = g.n, nc = gc.n;
    const int kb = tbx * kPLCols + 4 * threadIdx.x;  // first coarse column of this thread
    if (kb > nc) return;
    const int m0 = tby * Hc, m1 = min(m0 + Hc, nc + 1);
    const float *E = e + gc.off;
    float *Uf = u + g.off;
    const long P = g.pitch, Pc = gc.pitch;
    // x-pass of coarse row m: fine columns 2k (0.5 (e[k-1] + e[k])) and 2k+1 (e[k])
    auto xpass = [&](int m, float *v) {
        // coarse rows -1 and nc are the zero ghost rows
        const float4 c = ld4(E + (long)m * Pc + kb);
        const float left = E[(long)m * Pc + kb - 1];
        for (int k = 0; k < 4; ++k) {
            const float ek = cc4(c, k), ekm = k ? cc4(c, k - 1) : left;
            v[2 * k] = scale2<-1>(radd(ekm, ek));
            v[2 * k + 1] = ek;
        }
    };
    float pv[8], cv[8];
    xpass(m0 - 1, pv);
    const int fx = 2 * kb;
    for (int m = m0; m < m1; ++m) {
        xpass(m, cv);
        {   // fine row 2m: 0.5 (previous + current)
            float *row = Uf + (long)(2 * m) * P + fx;
            float4 a = ld4(row), bq = ld4(row + 4);
            for (int k = 0; k < 4; ++k) {
                c4(a, k) = radd(c4(a, k), scale2<-1>(radd(pv[k], cv[k])));
                c4(bq, k) = radd(c4(bq, k), scale2<-1>(radd(pv[k + 4], cv[k + 4])));
            }
            st4_valid(row, a, fx, n);
            if (fx + 4 < n) st4_valid(row + 4, bq, fx + 4, n);
        }
        if (m < nc) {  // fine row 2m+1
            float *row = Uf + (long)(2 * m + 1) * P + fx;
            float4 a = ld4(row), bq = ld4(row + 4);
            for (int k = 0; k < 4; ++k) {
                c4(a, k) = radd(c4(a, k), cv[k]);
                c4(bq, k) = radd(c4(bq, k), cv[k + 4]);
            }
            st4_valid(row, a, fx, n);
            if (fx + 4 < n) st4_valid(row + 4, bq, fx + 4, n);
        }
        for (int k = 0; k < 8; ++k) pv[k] = cv[k];
    }
}

__global__ void __launch_bounds__(kPLThreads)
prolong2d_pl_kernel(const float *__restrict__ e, float *__restrict__ u, Pitch2 g, Pitch2 gc, int Hc)
{
    prolong2d_pl_tile(e, u, g, gc, Hc, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Batched forms (persistent loops over (problem, tile) items; see
// mg_kernels2d.cu). All problems of one launch share the level size n.
// ---------------------------------------------------------------------------
// MODE 0: every item from its u; 1: every item from zero; 2: per item (u == nullptr: from zero)
template <int MODE>
__global__ void __launch_bounds__(kPLThreads)
sweep2d_pl_batched(const BItem<float> *__restrict__ tab, int nprob, const int *__restrict__ active, Pitch2 g, int H,
                   int bx, int by, float c0, float c1, float c2)
{
    const int per = bx * by, total = nprob * per;
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int j = it / per, r = it - j * per;
        const BItem<float> e = tab[j];
        if (active[e.problem]) {
            if (MODE == 1 || (MODE == 2 && !e.u))
                sweep2d_pl_tile<true, false>(e.u, e.b, e.out, g, H, c0, c1, c2, r % bx, r / bx, nullptr);
            else
                sweep2d_pl_tile<false, false>(e.u, e.b, e.out, g, H, c0, c1, c2, r % bx, r / bx, nullptr);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kPLThreads)
resrestrict2d_pl_batched(const BItem<float> *__restrict__ tab, int nprob, const int *__restrict__ active, Pitch2 g,
                         Pitch2 gc, int Hc, int bx, int by)
{
    const int per = bx * by, total = nprob * per;
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int j = it / per, r = it - j * per;
        const BItem<float> e = tab[j];
        if (active[e.problem]) resrestrict2d_pl_tile(e.u, e.b, e.out, g, gc, Hc, r % bx, r / bx);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kPLThreads)
prolong2d_pl_batched(const BItem<float> *__restrict__ tab, int nprob, const int *__restrict__ active, Pitch2 g,
                     Pitch2 gc, int Hc, int bx, int by)
{
    const int per = bx * by, total = nprob * per;
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int j = it / per, r = it - j * per;
        const BItem<float> e = tab[j];
        if (active[e.problem]) prolong2d_pl_tile(e.u, e.out, g, gc, Hc, r % bx, r / bx);
    }
}

// ---------------------------------------------------------------------------
// layout conversion (compact <-> padded), used by the single-level entry points
// ---------------------------------------------------------------------------
__global__ void pack2d_kernel(const float *__restrict__ in, float *__restrict__ out, Pitch2 g)
{
    const int n = g.n;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < (long)n * n; i += (long)gridDim.x * blockDim.x)
        out[g.off + (i / n) * g.pitch + i % n] = in[i];
}
__global__ void unpack2d_kernel(const float *__restrict__ in, float *__restrict__ out, Pitch2 g)
{
    const int n = g.n;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < (long)n * n; i += (long)gridDim.x * blockDim.x)
        out[i] = in[g.off + (i / n) * g.pitch + i % n];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
Pitch2 pitch2(int n)
{
    Pitch2 g;
    g.n = n;
    const int strips = (n + kPLCols - 1) / kPLCols;
    // every column a strip (plus its 4-column halos) touches stays inside the row
    g.pitch = ((strips * kPLCols + 8 + 31) / 32) * 32;
    g.rows = n + 2;
    g.off = g.pitch + 4;  // element (0, 0): one ghost row, then 4 columns (16-byte aligned)
    return g;
}

size_t pitch2_floats(int n)
{
    const Pitch2 g = pitch2(n);
    return (size_t)g.rows * g.pitch + 8;  // + tail slack for the right halo of the last row
}

int sweep2d_pl_blocks(int n, int H) { return ((n + kPLCols - 1) / kPLCols) * ((n + H - 1) / H); }

int sweep2d_pl_H(int n)
{
    const int bx = (n + kPLCols - 1) / kPLCols;
    return chunk_rows(bx, n, 8 * num_sms(), 2, 64);
}

cudaError_t launch_sweep2d_pl(const float *u, const float *b, float *out, int n, const double *c, double *partials,
                              cudaStream_t s)
{
    const Pitch2 g = pitch2(n);
    const int H = sweep2d_pl_H(n);
    const dim3 grid((n + kPLCols - 1) / kPLCols, (n + H - 1) / H);
    const float c0 = (float)c[0], c1 = (float)c[1], c2 = (float)c[2];
    if (u == nullptr) {
        if (partials) sweep2d_pl_kernel<true, true><<<grid, kPLThreads, 0, s>>>(u, b, out, g, H, c0, c1, c2, partials);
        else sweep2d_pl_kernel<true, false><<<grid, kPLThreads, 0, s>>>(u, b, out, g, H, c0, c1, c2, partials);
    } else {
        if (partials) sweep2d_pl_kernel<false, true><<<grid, kPLThreads, 0, s>>>(u, b, out, g, H, c0, c1, c2, partials);
        else sweep2d_pl_kernel<false, false><<<grid, kPLThreads, 0, s>>>(u, b, out, g, H, c0, c1, c2, partials);
    }
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_sweep2d_pl_acc64(const float *u, const float *b, double *u64, int n, const double *c, cudaStream_t s)
{
    const Pitch2 g = pitch2(n);
    const int H = sweep2d_pl_H(n);
    const dim3 grid((n + kPLCols - 1) / kPLCols, (n + H - 1) / H);
    sweep2d_pl_acc64_kernel<<<grid, kPLThreads, 0, s>>>(u, b, u64, g, H, (float)c[0], (float)c[1], (float)c[2]);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_resrestrict2d_pl(const float *u, const float *b, float *bc, int n, cudaStream_t s)
{
    const Pitch2 g = pitch2(n), gc = pitch2((n - 1) / 2);
    const int nc = gc.n;
    const int bx = (nc + kPLCols - 1) / kPLCols;
    const int Hc = chunk_rows(bx, nc, 8 * num_sms(), 1, 32);
    resrestrict2d_pl_kernel<<<dim3(bx, (nc + Hc - 1) / Hc), kPLThreads, 0, s>>>(u, b, bc, g, gc, Hc);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_prolong2d_pl(const float *e, float *u, int n, cudaStream_t s)
{
    const Pitch2 g = pitch2(n), gc = pitch2((n - 1) / 2);
    const int nc = gc.n;
    const int bx = (nc + 1 + kPLCols - 1) / kPLCols;
    const int Hc = chunk_rows(bx, nc + 1, 8 * num_sms(), 1, 32);
    prolong2d_pl_kernel<<<dim3(bx, (nc + 1 + Hc - 1) / Hc), kPLThreads, 0, s>>>(e, u, g, gc, Hc);
    count_launch(1);
    return cudaGetLastError();
}

static int pl_persistent_grid(const void *fn, long items)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPLThreads, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
    return (int)std::max<long>(1, std::min<long>(items, (long)per_sm * num_sms()));
}

cudaError_t launch_sweep2d_pl_batched(const BItem<float> *tab, int nprob, const int *active, int n, int H, int mode,
                                      const double *c, cudaStream_t s)
{
    const Pitch2 g = pitch2(n);
    const int bx = (n + kPLCols - 1) / kPLCols, by = (n + H - 1) / H;
    const long items = (long)nprob * bx * by;
    const float c0 = (float)c[0], c1 = (float)c[1], c2 = (float)c[2];
    if (mode == 1)
        sweep2d_pl_batched<1><<<pl_persistent_grid((const void *)sweep2d_pl_batched<1>, items), kPLThreads, 0, s>>>(
            tab, nprob, active, g, H, bx, by, c0, c1, c2);
    else if (mode == 2)
        sweep2d_pl_batched<2><<<pl_persistent_grid((const void *)sweep2d_pl_batched<2>, items), kPLThreads, 0, s>>>(
            tab, nprob, active, g, H, bx, by, c0, c1, c2);
    else
        sweep2d_pl_batched<0><<<pl_persistent_grid((const void *)sweep2d_pl_batched<0>, items), kPLThreads, 0, s>>>(
            tab, nprob, active, g, H, bx, by, c0, c1, c2);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_resrestrict2d_pl_batched(const BItem<float> *tab, int nprob, const int *active, int n, int Hc,
                                            cudaStream_t s)
{
    const Pitch2 g = pitch2(n), gc = pitch2((n - 1) / 2);
    const int bx = (gc.n + kPLCols - 1) / kPLCols, by = (gc.n + Hc - 1) / Hc;
    const long items = (long)nprob * bx * by;
    resrestrict2d_pl_batched<<<pl_persistent_grid((const void *)resrestrict2d_pl_batched, items), kPLThreads, 0, s>>>(
        tab, nprob, active, g, gc, Hc, bx, by);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_prolong2d_pl_batched(const BItem<float> *tab, int nprob, const int *active, int n, int Hc,
                                        cudaStream_t s)
{
    const Pitch2 g = pitch2(n), gc = pitch2((n - 1) / 2);
    const int bx = (gc.n + 1 + kPLCols - 1) / kPLCols, by = (gc.n + 1 + Hc - 1) / Hc;
    const long items = (long)nprob * bx * by;
    prolong2d_pl_batched<<<pl_persistent_grid((const void *)prolong2d_pl_batched, items), kPLThreads, 0, s>>>(
        tab, nprob, active, g, gc, Hc, bx, by);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_pack2d(const float *in, float *out, int n, bool to_padded, cudaStream_t s)
{
    const Pitch2 g = pitch2(n);
    const int blocks = (int)std::min<long>(((long)n * n + 255) / 256, 8L * num_sms());
    if (to_padded) pack2d_kernel<<<blocks, 256, 0, s>>>(in, out, g);
    else unpack2d_kernel<<<blocks, 256, 0, s>>>(in, out, g);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace mg
