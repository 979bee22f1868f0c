// mg_adjoint.cu -- reverse-mode derivative of K multigrid cycles on the GPU.
//
// Forward map (Sec. 4 cycle in the scaled form): u_K = K V(nu1, nu2) cycles
// from u_0 = 0 for right-hand side b and omega-folded weights c. Given
// g = dL/du_K this computes dL/db and dL/dc_j by applying, in reverse
// order, the transpose of each operator of the cycles:
//   sweep    u' = u + W rh, rh = bh - Ah u  ->  t = W g',  g = g' - Ah t,
//            gbh += t,  gc_j += <N_j g', rh>          (W, Ah, N_j symmetric)
//   restrict bh_c = 4 R (bh - Ah u)         ->  t = (4/2^d) P g_c,
//            gbh += t,  g = g - Ah t                 (4 R^T = (4/2^d) P)
//   correct  u' = u + P e                   ->  g_e = P^T g' = 2^d R g'
//   solve    e = A0^{-1} bh                 ->  g_bh = A0^{-1} g_e
//   load     bh_0 = h^2 b                   ->  g_b = h^2 g_bh_0
//
// Checkpoints: only the cycle inputs u_1 .. u_{K-1} (finest level) are kept
// from a first forward pass; before cycle k is reversed, it is replayed from
// its input, keeping for every level the inputs of its sweeps and its
// right-hand side (one cycle's worth), so the workspace grows with the
// number of levels, not with K (the sweeps are computed twice).
//
// The transposed sweep is one marching kernel (t = W g on the tile and a
// one-point halo, then g' = g - Ah t, gbh += t and the per-block partials of
// <g, rh>, <N_1 g, rh>, <N_2 g, rh>, in the same pass; g' goes to a second
// buffer, since neighbouring tiles read g). The coefficient partials of all
// reverse sweeps are reduced once, in a fixed order, at the end. The whole
// evaluation (forward, replays, reverse, reduction) is recorded into one
// CUDA graph, replayed while the caller's arrays stay the same.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>

#include "../../include/mg.h"
#include "mg_common.cuh"
#include "mg_ctx.h"
#include "mg_internal.h"

namespace mg {

template <typename T>
__device__ __forceinline__ T ld(const T *a, int n, int x, int y, int z)
{
    if (x < 0 || x >= n || y < 0 || y >= n || z < 0 || z >= n) return T(0);
    return a[((size_t)z * n + y) * n + x];
}

// ---------------------------------------------------------------------------
// fused transposed sweep, 3D (7-point M and A). Block: 32 x 8 output columns
// marching over the planes [z0, z1); per step q: (A) g plane q on the tile
// plus a 2-point halo and u plane q on the tile plus a 1-point halo into
// shared rings; (B) t = W g of plane q - 1 on the tile plus a 1-point halo,
// and the partials of plane q - 1 at the tile; (C) g' and gbh of plane q - 2
// at the tile. Formulas (zero outside the interior):
//   E  = ((g_W + g_E) + (g_S + g_N)) + (g_D + g_U)
//   t  = fma(c1, E, c0 g)
//   rh = fma(-6, u, bh) + (((u_W + u_E) + (u_S + u_N)) + (u_D + u_U))   (u = 0: bh)
//   g' = fma(-6, t, g) + (((t_W + t_E) + (t_S + t_N)) + (t_D + t_U)),  gbh += t
//   partials: sum g rh, sum E rh (FP64)
// ---------------------------------------------------------------------------
constexpr int kAX = 32, kAY = 8, kAThreads = kAX * kAY;
constexpr int kAGX = kAX + 4, kAGY = kAY + 4;  // g region (2-point halo)
constexpr int kATX = kAX + 2, kATY = kAY + 2;  // t and u region (1-point halo)

template <typename T, bool ZERO_U, bool UNSCALED>
__global__ void __launch_bounds__(kAThreads)
adj_sweep3d_kernel(const T *__restrict__ g, T *__restrict__ gout, const T *__restrict__ u, const T *__restrict__ b,
                   T *__restrict__ gbh, int n, int Z, T c0, T c1, int hk, double *__restrict__ partials)
{
    __shared__ T sg[4][kAGX * kAGY];
    __shared__ T st[3][kATX * kATY];
    __shared__ T su[ZERO_U ? 1 : 3][kATX * kATY];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kAX, y0 = blockIdx.y * kAY;
    const int z0 = blockIdx.z * Z, z1 = min(z0 + Z, n);
    const int ox = tid % kAX, oy = tid / kAX;  // the thread's output column
    const int X = x0 + ox, Y = y0 + oy;
    const bool own = X < n && Y < n;
    const int it = (oy + 1) * kATX + (ox + 1);  // its index in the t / u region
    const int ig = (oy + 2) * kAGX + (ox + 2);  // in the g region
    const size_t plane = (size_t)n * n;
    double a0 = 0.0, a1 = 0.0;
    // the plane loads of step q are issued at step q - 1 (registers), so that
    // their latency overlaps the work of a step: thread tid owns the region
    // points tid and tid + 256 (when inside the region)
    constexpr int kGN = (kAGX * kAGY + kAThreads - 1) / kAThreads, kUN = (kATX * kATY + kAThreads - 1) / kAThreads;
    T gq[kGN], uq[kUN];
    auto load_plane = [&](int q) {
        const bool qin = q >= 0 && q < n;
#pragma unroll
        for (int k = 0; k < kGN; ++k) {
            const int i = tid + k * kAThreads;
            const int gx = x0 - 2 + i % kAGX, gy = y0 - 2 + i / kAGX;
            gq[k] = i < kAGX * kAGY && qin && gx >= 0 && gx < n && gy >= 0 && gy < n ? g[q * plane + (size_t)gy * n + gx]
                                                                                   : T(0);
        }
        if (!ZERO_U) {
#pragma unroll
            for (int k = 0; k < kUN; ++k) {
                const int i = tid + k * kAThreads;
                const int ux = x0 - 1 + i % kATX, uy = y0 - 1 + i / kATX;
                uq[k] = i < kATX * kATY && qin && ux >= 0 && ux < n && uy >= 0 && uy < n
                            ? u[q * plane + (size_t)uy * n + ux]
                            : T(0);
            }
        }
    };
    load_plane(z0 - 2);
    for (int q = z0 - 2; q <= z1 + 1; ++q) {
        // A. g plane q (2-point halo), u plane q (1-point halo), then the loads of plane q + 1
#pragma unroll
        for (int k = 0; k < kGN; ++k)
            if (tid + k * kAThreads < kAGX * kAGY) sg[q & 3][tid + k * kAThreads] = gq[k];
        if (!ZERO_U) {
#pragma unroll
            for (int k = 0; k < kUN; ++k)
                if (tid + k * kAThreads < kATX * kATY) su[(q + 3) % 3][tid + k * kAThreads] = uq[k];
        }
        if (q < z1 + 1) load_plane(q + 1);
        __syncthreads();
        // B. t of plane p = q - 1 on the 1-point halo region
        const int p = q - 1;
        if (p >= z0 - 1) {
            const bool pin = p >= 0 && p < n;
            const T *gm = sg[(p + 3) & 3], *gc = sg[p & 3], *gp = sg[(p + 1) & 3];
            for (int k = 0; k < 2; ++k) {
                // the thread's own column first, then the 84 halo points
                int tx, ty;
                if (k == 0) {
                    tx = ox + 1;
                    ty = oy + 1;
                } else {
                    if (tid >= 2 * kATX + 2 * kAY) break;
                    const int h = tid;
                    if (h < kATX) { tx = h; ty = 0; }
                    else if (h < 2 * kATX) { tx = h - kATX; ty = kATY - 1; }
                    else if (h < 2 * kATX + kAY) { tx = 0; ty = h - 2 * kATX + 1; }
                    else { tx = kATX - 1; ty = h - 2 * kATX - kAY + 1; }
                }
                const int j = (ty + 1) * kAGX + (tx + 1);
                const T E = radd(radd(radd(gc[j - 1], gc[j + 1]), radd(gc[j - kAGX], gc[j + kAGX])), radd(gm[j], gp[j]));
                const T tv = rfma(c1, E, rmul(c0, gc[j]));
                const int Xt = x0 - 1 + tx, Yt = y0 - 1 + ty;
                st[(p + 3) % 3][ty * kATX + tx] = pin && Xt >= 0 && Xt < n && Yt >= 0 && Yt < n ? tv : T(0);
                if (k == 0 && own && p >= z0 && p < z1) {
                    T bb = b[p * plane + (size_t)Y * n + X];
                    if (UNSCALED) bb = scale2(bb, hk);
                    T rh = bb;
                    if (!ZERO_U) {
                        const T *uc = su[(p + 3) % 3];
                        const T s = radd(radd(radd(uc[it - 1], uc[it + 1]), radd(uc[it - kATX], uc[it + kATX])),
                                         radd(su[(p + 2) % 3][it], su[(p + 4) % 3][it]));
                        rh = radd(rfma(T(-6), uc[it], bb), s);
                    }
                    a0 = fma((double)gc[j], (double)rh, a0);
                    a1 = fma((double)E, (double)rh, a1);
                }
            }
        }
        __syncthreads();
        // C. g' and gbh of plane r = q - 2 at the tile
        const int r = q - 2;
        if (own && r >= z0 && r < z1) {
            const T *tc = st[(r + 3) % 3];
            const T tv = tc[it];
            const T s = radd(radd(radd(tc[it - 1], tc[it + 1]), radd(tc[it - kATX], tc[it + kATX])),
                             radd(st[(r + 2) % 3][it], st[(r + 4) % 3][it]));
            const size_t o = r * plane + (size_t)Y * n + X;
            gout[o] = radd(rfma(T(-6), tv, sg[r & 3][ig]), s);
            gbh[o] = radd(gbh[o], tv);
        }
    }
    const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    block_sum_store<kAThreads>(a0, &partials[3 * bid]);
    __syncthreads();
    block_sum_store<kAThreads>(a1, &partials[3 * bid + 1]);
    if (tid == 0) partials[3 * bid + 2] = 0.0;
}

// ---------------------------------------------------------------------------
// fused transposed sweep, 2D (9-point M, 5-point A): 256 output columns
// marching over rows [y0, y1); the same three phases per row step:
//   E  = (g_W + g_E) + (g_S + g_N),  C = (g_SW + g_SE) + (g_NW + g_NE)
//   t  = fma(c2, C, fma(c1, E, c0 g))
//   rh = fma(-4, u, bh) + ((u_W + u_E) + (u_S + u_N))          (u = 0: bh)
//   g' = fma(-4, t, g) + ((t_W + t_E) + (t_S + t_N)),  gbh += t
//   partials: sum g rh, sum E rh, sum C rh (FP64)
// ---------------------------------------------------------------------------
constexpr int kA2X = 256;
constexpr int kA2G = kA2X + 4, kA2T = kA2X + 2;

template <typename T, bool ZERO_U, bool UNSCALED>
__global__ void __launch_bounds__(kA2X)
adj_sweep2d_kernel(const T *__restrict__ g, T *__restrict__ gout, const T *__restrict__ u, const T *__restrict__ b,
                   T *__restrict__ gbh, int n, int H, T c0, T c1, T c2, int hk, double *__restrict__ partials)
{
    __shared__ T sg[4][kA2G];
    __shared__ T st[3][kA2T];
    __shared__ T su[ZERO_U ? 1 : 3][kA2T];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kA2X;
    const int y0 = blockIdx.y * H, y1 = min(y0 + H, n);
    const int X = x0 + tid;
    const bool own = X < n;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    // the row loads of step q are issued at step q - 1 (registers)
    T gq[2], uq[2];
    auto load_row = [&](int q) {
        const bool qin = q >= 0 && q < n;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int i = tid + k * kA2X;
            const int gx = x0 - 2 + i, ux = x0 - 1 + i;
            gq[k] = i < kA2G && qin && gx >= 0 && gx < n ? g[(size_t)q * n + gx] : T(0);
            if (!ZERO_U) uq[k] = i < kA2T && qin && ux >= 0 && ux < n ? u[(size_t)q * n + ux] : T(0);
        }
    };
    load_row(y0 - 2);
    for (int q = y0 - 2; q <= y1 + 1; ++q) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int i = tid + k * kA2X;
            if (i < kA2G) sg[q & 3][i] = gq[k];
            if (!ZERO_U && i < kA2T) su[(q + 3) % 3][i] = uq[k];
        }
        if (q < y1 + 1) load_row(q + 1);
        __syncthreads();
        const int p = q - 1;
        if (p >= y0 - 1) {
            const bool pin = p >= 0 && p < n;
            const T *gm = sg[(p + 3) & 3], *gc = sg[p & 3], *gp = sg[(p + 1) & 3];
            for (int k = 0; k < 2; ++k) {
                int tx;
                if (k == 0) tx = tid + 1;
                else if (tid < 2) tx = tid == 0 ? 0 : kA2T - 1;
                else break;
                const int j = tx + 1;
                const T E = radd(radd(gc[j - 1], gc[j + 1]), radd(gm[j], gp[j]));
                const T C = radd(radd(gm[j - 1], gm[j + 1]), radd(gp[j - 1], gp[j + 1]));
                const T tv = rfma(c2, C, rfma(c1, E, rmul(c0, gc[j])));
                const int Xt = x0 - 1 + tx;
                st[(p + 3) % 3][tx] = pin && Xt >= 0 && Xt < n ? tv : T(0);
                if (k == 0 && own && p >= y0 && p < y1) {
                    T bb = b[(size_t)p * n + X];
                    if (UNSCALED) bb = scale2(bb, hk);
                    T rh = bb;
                    if (!ZERO_U) {
                        const T *uc = su[(p + 3) % 3];
                        const T s = radd(radd(uc[tx - 1], uc[tx + 1]), radd(su[(p + 2) % 3][tx], su[(p + 4) % 3][tx]));
                        rh = radd(rfma(T(-4), uc[tx], bb), s);
                    }
                    a0 = fma((double)gc[j], (double)rh, a0);
                    a1 = fma((double)E, (double)rh, a1);
                    a2 = fma((double)C, (double)rh, a2);
                }
            }
        }
        __syncthreads();
        const int r = q - 2;
        if (own && r >= y0 && r < y1) {
            const T *tc = st[(r + 3) % 3];
            const int it = tid + 1;
            const T tv = tc[it];
            const T s = radd(radd(tc[it - 1], tc[it + 1]), radd(st[(r + 2) % 3][it], st[(r + 4) % 3][it]));
            const size_t o = (size_t)r * n + X;
            gout[o] = radd(rfma(T(-4), tv, sg[r & 3][it + 1]), s);
            gbh[o] = radd(gbh[o], tv);
        }
    }
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    block_sum_store<kA2X>(a0, &partials[3 * bid]);
    __syncthreads();
    block_sum_store<kA2X>(a1, &partials[3 * bid + 1]);
    __syncthreads();
    block_sum_store<kA2X>(a2, &partials[3 * bid + 2]);
}

// g = g - Ah t (= fma(-2d, t, g) + neighbour sum of t);  gbh += t
template <typename T, int D>
__global__ void __launch_bounds__(256)
adj_stage2(T *__restrict__ g, const T *__restrict__ t, T *__restrict__ gbh, int n)
{
    const size_t np = D == 2 ? (size_t)n * n : (size_t)n * n * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < np; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % n), y = (int)((i / n) % n), z = D == 2 ? 0 : (int)(i / ((size_t)n * n));
        T s;
        if (D == 2)
            s = radd(radd(ld(t, n, x - 1, y, 0), ld(t, n, x + 1, y, 0)), radd(ld(t, n, x, y - 1, 0), ld(t, n, x, y + 1, 0)));
        else
            s = radd(radd(radd(ld(t, n, x - 1, y, z), ld(t, n, x + 1, y, z)), radd(ld(t, n, x, y - 1, z), ld(t, n, x, y + 1, z))),
                     radd(ld(t, n, x, y, z - 1), ld(t, n, x, y, z + 1)));
        const T ti = t[i];
        g[i] = radd(rfma(T(-2 * D), ti, g[i]), s);
        gbh[i] = radd(gbh[i], ti);
    }
}

// out = scale * (full weighting along x, y (, z) of the fine field f), i.e.
// scale * 16 R f (2D) or scale * 64 R f (3D) in units of the (1,2,1) sums.
template <typename T, int D>
__global__ void __launch_bounds__(256)
adj_fw(const T *__restrict__ f, T *__restrict__ out, int n, T scale)
{
    const int nc = (n - 1) / 2;
    const size_t npc = D == 2 ? (size_t)nc * nc : (size_t)nc * nc * nc;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < npc; i += (size_t)gridDim.x * blockDim.x) {
        const int ic = (int)(i % nc), jc = (int)((i / nc) % nc), kc = D == 2 ? 0 : (int)(i / ((size_t)nc * nc));
        auto tx = [&](int fy, int fz) {
            const T *row = f + ((size_t)fz * n + fy) * n;
            return rfma(T(2), row[2 * ic + 1], radd(row[2 * ic], row[2 * ic + 2]));
        };
        T v;
        if (D == 2) {
            v = rfma(T(2), tx(2 * jc + 1, 0), radd(tx(2 * jc, 0), tx(2 * jc + 2, 0)));
        } else {
            T tz[3];
            for (int k = 0; k < 3; ++k) {
                const int fz = 2 * kc + k;
                tz[k] = rfma(T(2), tx(2 * jc + 1, fz), radd(tx(2 * jc, fz), tx(2 * jc + 2, fz)));
            }
            v = rfma(T(2), tz[1], radd(tz[0], tz[2]));
        }
        out[i] = rmul(scale, v);
    }
}

// out = scale * P e (linear interpolation of the coarse field e)
template <typename T>
__device__ __forceinline__ T ip_x(const T *e, int nc, int fx, int jc, int kc)
{
    if (fx & 1) return ld(e, nc, fx >> 1, jc, kc);
    const int k = fx >> 1;
    return rmul(T(0.5), radd(ld(e, nc, k - 1, jc, kc), ld(e, nc, k, jc, kc)));
}
template <typename T>
__device__ __forceinline__ T ip_xy(const T *e, int nc, int fx, int fy, int kc)
{
    if (fy & 1) return ip_x(e, nc, fx, fy >> 1, kc);
    const int m = fy >> 1;
    return rmul(T(0.5), radd(ip_x(e, nc, fx, m - 1, kc), ip_x(e, nc, fx, m, kc)));
}
template <typename T, int D>
__global__ void __launch_bounds__(256)
adj_interp(const T *__restrict__ e, T *__restrict__ out, int n, T scale)
{
    const int nc = (n - 1) / 2;
    const size_t np = D == 2 ? (size_t)n * n : (size_t)n * n * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < np; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % n), y = (int)((i / n) % n), z = D == 2 ? 0 : (int)(i / ((size_t)n * n));
        T v;
        if (D == 2) {
            v = ip_xy(e, nc, x, y, 0);
        } else if (z & 1) {
            v = ip_xy(e, nc, x, y, z >> 1);
        } else {
            const int q = z >> 1;
            v = rmul(T(0.5), radd(ip_xy(e, nc, x, y, q - 1), ip_xy(e, nc, x, y, q)));
        }
        out[i] = rmul(scale, v);
    }
}

// acc[j] = sum over all nblocks block partials partials[3 b + j], in a fixed
// order: thread t sums the blocks t, t + 256, ..., then a fixed warp tree
__global__ void __launch_bounds__(256) adj_reduce(const double *__restrict__ partials, long nblocks,
                                                  double *__restrict__ acc)
{
    __shared__ double tot;
    for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (long b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[3 * b + j];
        block_sum_store<256>(s, &tot);
        __syncthreads();
        if (threadIdx.x == 0) acc[j] = tot;
        __syncthreads();
    }
}

template <typename T>
__global__ void adj_scale(const T *__restrict__ in, T *__restrict__ out, size_t np, T s)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < np; i += (size_t)gridDim.x * blockDim.x)
        out[i] = rmul(s, in[i]);
}

static int grid_for(size_t np)
{
    return (int)std::max<size_t>(1, std::min<size_t>((np + 255) / 256, (size_t)num_sms() * 8));
}

static size_t npts(int d, int n) { return d == 2 ? (size_t)n * n : (size_t)n * n * n; }

// launch shape of the fused transposed sweep on a level with n points per axis
struct AdjGrid {
    dim3 grid;
    int Z;  // planes (3D) or rows (2D) per block
};
static AdjGrid adj_grid(int d, int n)
{
    AdjGrid a;
    if (d == 3) {
        const int bx = (n + kAX - 1) / kAX, by = (n + kAY - 1) / kAY;
        a.Z = chunk_rows(bx * by, n, 4 * num_sms(), 4, 64);
        a.grid = dim3(bx, by, (n + a.Z - 1) / a.Z);
    } else {
        const int bx = (n + kA2X - 1) / kA2X;
        a.Z = chunk_rows(bx, n, 4 * num_sms(), 8, 128);
        a.grid = dim3(bx, (n + a.Z - 1) / a.Z, 1);
    }
    return a;
}
static long adj_blocks(int d, int n)
{
    const AdjGrid a = adj_grid(d, n);
    return (long)a.grid.x * a.grid.y * a.grid.z;
}

void free_adjoint(mg_ctx *c)
{
    if (!c->adj) return;
    if (c->adj->graph) cudaGraphExecDestroy(c->adj->graph);
    for (void *p : c->adj->owned) cudaFree(p);
    if (c->adj->h_acc) cudaFreeHost(c->adj->h_acc);
    delete c->adj;
    c->adj = nullptr;
}

namespace {

template <typename T>
struct Adjoint {
    mg_ctx *c;
    AdjointWork *w;
    const T *b;  // caller's unscaled finest right-hand side
    long pofs = 0;  // next free block slot of the coefficient partials
    int cur[32] = {0};  // which of the two gradient buffers G[2l], G[2l+1] is current
    cudaError_t err = cudaSuccess;

    bool ok(cudaError_t e)
    {
        if (e != cudaSuccess && err == cudaSuccess) err = e;
        return err == cudaSuccess;
    }
    int n(int l) const { return c->n[l]; }
    const T *bh(int l) const { return l == 0 ? b : (const T *)w->bh[l]; }
    T *slot(int l, int s) const { return (T *)w->sw[l][s]; }
    T *G(int l) const { return (T *)w->G[2 * l + cur[l]]; }
    T *G2(int l) const { return (T *)w->G[2 * l + 1 - cur[l]]; }

    void solve_coarsest(const T *rhs, T *x)
    {
        TailArgs a;
        memset(&a, 0, sizeof a);
        a.d = c->d;
        a.lu = c->lu;
        a.lv[0] = tail_level(x, nullptr, (void *)rhs, nullptr, 3);
        a.ops[0].kind = TAIL_SOLVE;
        a.nops = 1;
        ok(launch_tail<T>(a, c->s));
    }

    cudaError_t op_sweep_any(const T *u, const T *rhs, bool unsc, T *out, int nn)
    {
        return c->d == 2 ? launch_sweep2d<T>(u, rhs, unsc, out, nn, c->c, nullptr, c->s)
                         : launch_sweep3d<T>(u, rhs, unsc, out, nn, c->c, nullptr, c->s);
    }

    // ---- forward: visit of level l with input `in` (nullptr = zero); the
    // sweep outputs go to the level's slots, the output is the last slot ----
    T *fwd_visit(int l, const T *in)
    {
        const int nn = n(l);
        if (nn == 3) {
            T *x = slot(l, 0);
            solve_coarsest(bh(l), x);
            return x;
        }
        const bool unsc = l == 0;
        const T *cur_u = in;
        for (int s = 0; s < c->nu1; ++s) {
            T *out = slot(l, s);
            if (!ok(op_sweep_any(cur_u, bh(l), unsc, out, nn))) return nullptr;
            cur_u = out;
        }
        T *ua = slot(l, c->nu1 - 1);
        if (!ok(c->d == 2 ? launch_resrestrict2d<T>(ua, bh(l), unsc, (T *)w->bh[l + 1], nn, c->s)
                          : launch_resrestrict3d<T>(ua, bh(l), unsc, (T *)w->bh[l + 1], nn, c->s)))
            return nullptr;
        const T *e = fwd_visit(l + 1, nullptr);
        if (!e) return nullptr;
        // the correction is applied in place: the transposes need the inputs
        // of the sweeps, and the last pre-sweep's output is not one of them
        if (!ok(c->d == 2 ? launch_prolong2d<T>(e, ua, nn, c->s) : launch_prolong3d<T>(e, ua, nn, c->s)))
            return nullptr;
        cur_u = ua;
        for (int s = 0; s < c->nu2; ++s) {
            T *out = slot(l, c->nu1 + s);
            if (!ok(op_sweep_any(cur_u, bh(l), unsc, out, nn))) return nullptr;
            cur_u = out;
        }
        return (T *)cur_u;
    }

    // input of sweep s (pre-sweeps 0 .. nu1-1, then post-sweeps) of the
    // visit of level l (nullptr: zero); the first post-sweep's input is the
    // corrected field, which replaced the last pre-sweep's output
    const T *sweep_in(int l, int s, const T *in) const { return s == 0 ? in : slot(l, s - 1); }

    // ---- reverse -----------------------------------------------------------
    void adj_sweep(int l, const T *u_in)
    {
        const int nn = n(l);
        const AdjGrid a = adj_grid(c->d, nn);
        const int hk = h2_exponent(nn);
        const bool unsc = l == 0;
        double *part = w->partials + 3 * pofs;
        pofs += (long)a.grid.x * a.grid.y * a.grid.z;
        const T *gin = G(l);
        T *gout = G2(l), *gbh = (T *)w->GB[l];
        const T *bb = bh(l);
        const T c0 = T(c->c[0]), c1 = T(c->c[1]), c2 = T(c->c[2]);
#define MG_ADJ3(ZU, UN)                                                                                               \
    adj_sweep3d_kernel<T, ZU, UN><<<a.grid, kAThreads, 0, c->s>>>(gin, gout, u_in, bb, gbh, nn, a.Z, c0, c1, hk, part)
#define MG_ADJ2(ZU, UN)                                                                                               \
    adj_sweep2d_kernel<T, ZU, UN><<<a.grid, kA2X, 0, c->s>>>(gin, gout, u_in, bb, gbh, nn, a.Z, c0, c1, c2, hk, part)
        if (c->d == 3) {
            if (u_in) { if (unsc) MG_ADJ3(false, true); else MG_ADJ3(false, false); }
            else { if (unsc) MG_ADJ3(true, true); else MG_ADJ3(true, false); }
        } else {
            if (u_in) { if (unsc) MG_ADJ2(false, true); else MG_ADJ2(false, false); }
            else { if (unsc) MG_ADJ2(true, true); else MG_ADJ2(true, false); }
        }
#undef MG_ADJ3
#undef MG_ADJ2
        count_launch(1);
        ok(cudaGetLastError());
        cur[l] = 1 - cur[l];
    }

    // on entry G(l) = gradient w.r.t. the visit's output; on exit G(l) =
    // gradient w.r.t. its input and GB[l] has received the gradient w.r.t.
    // its right-hand side
    void rev_visit(int l, const T *in)
    {
        const int nn = n(l);
        const size_t np = npts(c->d, nn);
        if (nn == 3) {
            solve_coarsest(G(l), (T *)w->GB[l]);
            ok(cudaMemsetAsync(G(l), 0, np * sizeof(T), c->s));
            return;
        }
        for (int s = c->nu2 - 1; s >= 0; --s) adj_sweep(l, sweep_in(l, c->nu1 + s, in));
        // interpolation + correction: the child's output gradient is P^T g
        const int ncoarse = (nn - 1) / 2;
        const size_t npc = npts(c->d, ncoarse);
        const int gridc = grid_for(npc);
        if (c->d == 2)
            adj_fw<T, 2><<<gridc, 256, 0, c->s>>>(G(l), G(l + 1), nn, T(0.25));
        else
            adj_fw<T, 3><<<gridc, 256, 0, c->s>>>(G(l), G(l + 1), nn, T(0.125));
        count_launch(1);
        ok(cudaMemsetAsync(w->GB[l + 1], 0, npc * sizeof(T), c->s));
        rev_visit(l + 1, nullptr);
        // restriction: t = (4/2^d) P g_bh_child; g -= Ah t; gbh += t
        const int grid = grid_for(np);
        if (c->d == 2)
            adj_interp<T, 2><<<grid, 256, 0, c->s>>>((const T *)w->GB[l + 1], (T *)w->T[l], nn, T(1.0));
        else
            adj_interp<T, 3><<<grid, 256, 0, c->s>>>((const T *)w->GB[l + 1], (T *)w->T[l], nn, T(0.5));
        if (c->d == 2)
            adj_stage2<T, 2><<<grid, 256, 0, c->s>>>(G(l), (const T *)w->T[l], (T *)w->GB[l], nn);
        else
            adj_stage2<T, 3><<<grid, 256, 0, c->s>>>(G(l), (const T *)w->T[l], (T *)w->GB[l], nn);
        count_launch(2);
        ok(cudaGetLastError());
        for (int s = c->nu1 - 1; s >= 0; --s) adj_sweep(l, sweep_in(l, s, in));
    }

    // the whole evaluation for dL/du_K = g_uK: forward to the checkpoints,
    // then per cycle (last first) a replay and the reverse
    cudaError_t record_all(int K, const T *g_uK, T *g_b)
    {
        const size_t np0 = npts(c->d, c->n[0]);
        const size_t bytes0 = np0 * sizeof(T);
        // forward: u_1 .. u_{K-1}
        const T *u = nullptr;
        for (int k = 0; k + 1 < K; ++k) {
            const T *out = fwd_visit(0, u);
            if (!out) return err;
            if (!ok(cudaMemcpyAsync(w->ck[k + 1], out, bytes0, cudaMemcpyDeviceToDevice, c->s))) return err;
            u = (const T *)w->ck[k + 1];
        }
        for (int l = 0; l < c->L; ++l) cur[l] = 0;
        if (!ok(cudaMemcpyAsync(G(0), g_uK, bytes0, cudaMemcpyDeviceToDevice, c->s)) ||
            !ok(cudaMemsetAsync(w->GB[0], 0, bytes0, c->s)))
            return err;
        for (int k = K - 1; k >= 0; --k) {
            const T *in = k == 0 ? nullptr : (const T *)w->ck[k];
            if (!fwd_visit(0, in)) return err;  // replay: the sweep inputs of cycle k
            rev_visit(0, in);
            if (err) return err;
        }
        adj_reduce<<<1, 256, 0, c->s>>>(w->partials, pofs, w->acc);
        const T h2 = T(1.0 / ((double)c->N * c->N));
        adj_scale<T><<<grid_for(np0), 256, 0, c->s>>>((const T *)w->GB[0], g_b, np0, h2);
        count_launch(2);
        if (!ok(cudaGetLastError())) return err;
        ok(cudaMemcpyAsync(w->h_acc, w->acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
        return err;
    }
};

}  // namespace
}  // namespace mg

using namespace mg;

// blocks of coefficient partials written by the reverse of K cycles
static long adj_partial_blocks(const mg_ctx *c, int K)
{
    long per_cycle = 0;
    for (int l = 0; l < c->L; ++l)
        if (c->n[l] > 3) per_cycle += (long)(c->nu1 + c->nu2) * adj_blocks(c->d, c->n[l]);
    return per_cycle * K;
}

// device bytes of the adjoint workspace for K cycles (see AdjointWork)
static unsigned long long adj_bytes(const mg_ctx *c, int K)
{
    const size_t es = c->esize;
    unsigned long long total = (unsigned long long)(K - 1) * npts(c->d, c->n[0]) * es;
    const int slots = c->nu1 + c->nu2;
    for (int l = 0; l < c->L; ++l) {
        const unsigned long long f = (unsigned long long)npts(c->d, c->n[l]) * es;
        total += f * ((c->n[l] == 3 ? 1 : slots) + (l >= 1 ? 1 : 0) + 4);
    }
    const long nb = adj_partial_blocks(c, K);
    total += (unsigned long long)3 * (nb > 0 ? nb : 1) * sizeof(double) + 3 * sizeof(double);
    return total;
}

static mg_status adj_alloc(mg_ctx *c, int K)
{
    if (c->adj && c->adj->K == K) return MG_OK;
    free_adjoint(c);
    AdjointWork *w = new (std::nothrow) AdjointWork;
    if (!w) return MG_ENOMEM;
    c->adj = w;
    w->K = K;
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        w->owned.push_back(p);
        w->bytes += bytes;
        return p;
    };
    const size_t es = c->esize;
    const size_t bytes0 = npts(c->d, c->n[0]) * es;
    w->ck.assign(K, nullptr);
    for (int k = 1; k < K; ++k)
        if (!(w->ck[k] = alloc(bytes0))) return MG_ENOMEM;
    // per level: the sweep outputs of one visit (nu1 + nu2 fields; the
    // coarsest: its solution), the right-hand side (level >= 1), two
    // gradient buffers, the gradient of the right-hand side and a scratch
    // field
    const int slots = c->nu1 + c->nu2;
    w->sw.assign(c->L, {});
    w->bh.assign(c->L, nullptr);
    w->G.assign(2 * c->L, nullptr);
    w->GB.assign(c->L, nullptr);
    w->T.assign(c->L, nullptr);
    for (int l = 0; l < c->L; ++l) {
        const size_t bytes = npts(c->d, c->n[l]) * es;
        const int ns = c->n[l] == 3 ? 1 : slots;
        for (int s = 0; s < ns; ++s) {
            void *p = alloc(bytes);
            if (!p) return MG_ENOMEM;
            w->sw[l].push_back(p);
        }
        if (l >= 1 && !(w->bh[l] = alloc(bytes))) return MG_ENOMEM;
        if (!(w->G[2 * l] = alloc(bytes)) || !(w->G[2 * l + 1] = alloc(bytes)) || !(w->GB[l] = alloc(bytes)) ||
            !(w->T[l] = alloc(bytes)))
            return MG_ENOMEM;
    }
    const long nb = adj_partial_blocks(c, K);
    w->npartials = (size_t)3 * (nb > 0 ? nb : 1);
    if (!(w->partials = (double *)alloc(w->npartials * sizeof(double)))) return MG_ENOMEM;
    if (!(w->acc = (double *)alloc(3 * sizeof(double)))) return MG_ENOMEM;
    if (cudaMallocHost((void **)&w->h_acc, 3 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        w->h_acc = nullptr;
        return MG_ENOMEM;
    }
    return MG_OK;
}

template <typename T>
static mg_status run_adjoint(mg_ctx *c, int K, const T *b, const T *g_uK, T *g_b, double *g_c)
{
    AdjointWork *w = c->adj;
    if (!w->graph || w->cap_b != b || w->cap_g != g_uK || w->cap_gb != g_b) {
        if (w->graph) cudaGraphExecDestroy(w->graph);
        w->graph = nullptr;
        Adjoint<T> A{c, w, b};
        mg_status st =
            capture_graph(c, &w->graph, &w->nodes, [&]() -> cudaError_t { return A.record_all(K, g_uK, g_b); });
        if (st != MG_OK) return st;
        w->cap_b = b;
        w->cap_g = g_uK;
        w->cap_gb = g_b;
    }
    cudaError_t e = cudaGraphLaunch(w->graph, c->s);
    if (!e) count_launch(w->nodes);
    if (!e) e = cudaStreamSynchronize(c->s);
    if (e) return cuda_fail(e);
    for (int j = 0; j < c->ncoef; ++j) g_c[j] = w->h_acc[j];
    return MG_OK;
}

extern "C" mg_status mg_vcycles_adjoint(mg_ctx *ctx, int K, const void *b, const void *grad_uK, void *grad_b_out,
                                        double *grad_coeffs_out)
{
    if (!ctx || K < 1 || !b || !grad_uK || !grad_b_out || !grad_coeffs_out || ctx->batch ||
        ctx->gamma != 1 || ctx->nu1 < 1 || ctx->prec == MG_FP32_IR || ctx->L < 2 || ctx->L > 32 ||
        (ctx->d == 3 && ctx->ncoef > 2))  // the adjoint covers the 7-point M in 3D
        return MG_EINVAL;
    if (cudaSetDevice(ctx->dev) != cudaSuccess) return cuda_fail(cudaGetLastError());
    if (cudaEventRecord(ctx->ev_in, ctx->user) != cudaSuccess || cudaStreamWaitEvent(ctx->s, ctx->ev_in, 0) != cudaSuccess)
        return cuda_fail(cudaGetLastError());
    mg_status st = adj_alloc(ctx, K);
    if (st == MG_OK)
        st = ctx->prec == MG_FP64 ? run_adjoint<double>(ctx, K, (const double *)b, (const double *)grad_uK,
                                                        (double *)grad_b_out, grad_coeffs_out)
                                  : run_adjoint<float>(ctx, K, (const float *)b, (const float *)grad_uK,
                                                       (float *)grad_b_out, grad_coeffs_out);
    // order the caller's stream after the work queued here, on every exit
    const bool ordered = cudaEventRecord(ctx->ev_out, ctx->s) == cudaSuccess &&
                         cudaStreamWaitEvent(ctx->user, ctx->ev_out, 0) == cudaSuccess;
    if (st != MG_OK) return st;
    return ordered ? MG_OK : cuda_fail(cudaGetLastError());
}

extern "C" mg_status mg_adjoint_workspace_bytes(mg_ctx *ctx, int K, unsigned long long *bytes_out)
{
    if (!ctx || K < 1 || !bytes_out || ctx->batch) return MG_EINVAL;
    *bytes_out = adj_bytes(ctx, K);
    return MG_OK;
}
