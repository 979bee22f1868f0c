// mg_adjoint.cu -- reverse-mode derivative of K multigrid cycles on the GPU.
//
// Forward map (Sec. 4 cycle in the scaled form): u_K = K V(nu1, nu2) cycles
// from u_0 = 0 for right-hand side b and omega-folded weights c. Given
// g = dL/du_K this computes dL/db and dL/dc_j by replaying the forward once
// with every sweep input kept (one field per sweep of every level visit plus
// the visit's restricted right-hand side) and applying, in reverse order,
// the transpose of each operator:
//   sweep    u' = u + W rh, rh = bh - Ah u  ->  t = W g',  g = g' - Ah t,
//            gbh += t,  gc_j += <N_j g', rh>          (W, Ah, N_j symmetric)
//   restrict bh_c = 4 R (bh - Ah u)         ->  t = (4/2^d) P g_c,
//            gbh += t,  g = g - Ah t                 (4 R^T = (4/2^d) P)
//   correct  u' = u + P e                   ->  g_e = P^T g' = 2^d R g'
//   solve    e = A0^{-1} bh                 ->  g_bh = A0^{-1} g_e
//   load     bh_0 = h^2 b                   ->  g_b = h^2 g_bh_0
// Note g - Ah t = fma(-2d, t, g) + (neighbour sum of t): the residual kernel
// with u := t, bh := g. Coefficient gradients are accumulated in FP64 with a
// fixed-order reduction after every adjoint sweep.
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

// t = W g at every point; per block: sum g rh, sum (N_1 g) rh, sum (N_2 g) rh
// with rh = bh - Ah u_in (u_in == nullptr: zero).
template <typename T, int D>
__global__ void __launch_bounds__(256)
adj_sweep_stage1(const T *__restrict__ g, const T *__restrict__ u, const T *__restrict__ b, bool unscaled,
                 T *__restrict__ t, int n, T c0, T c1, T c2, int hk, double *__restrict__ partials)
{
    const size_t np = D == 2 ? (size_t)n * n : (size_t)n * n * n;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < np; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % n), y = (int)((i / n) % n), z = D == 2 ? 0 : (int)(i / ((size_t)n * n));
        const T gp = g[i];
        T E, C = T(0), s = T(0);
        if (D == 2) {
            E = radd(radd(ld(g, n, x - 1, y, 0), ld(g, n, x + 1, y, 0)), radd(ld(g, n, x, y - 1, 0), ld(g, n, x, y + 1, 0)));
            C = radd(radd(ld(g, n, x - 1, y - 1, 0), ld(g, n, x + 1, y - 1, 0)),
                     radd(ld(g, n, x - 1, y + 1, 0), ld(g, n, x + 1, y + 1, 0)));
            if (u)
                s = radd(radd(ld(u, n, x - 1, y, 0), ld(u, n, x + 1, y, 0)), radd(ld(u, n, x, y - 1, 0), ld(u, n, x, y + 1, 0)));
            t[i] = rfma(c2, C, rfma(c1, E, rmul(c0, gp)));
        } else {
            E = radd(radd(radd(ld(g, n, x - 1, y, z), ld(g, n, x + 1, y, z)), radd(ld(g, n, x, y - 1, z), ld(g, n, x, y + 1, z))),
                     radd(ld(g, n, x, y, z - 1), ld(g, n, x, y, z + 1)));
            if (u)
                s = radd(radd(radd(ld(u, n, x - 1, y, z), ld(u, n, x + 1, y, z)), radd(ld(u, n, x, y - 1, z), ld(u, n, x, y + 1, z))),
                         radd(ld(u, n, x, y, z - 1), ld(u, n, x, y, z + 1)));
            t[i] = rfma(c1, E, rmul(c0, gp));
        }
        T bb = b[i];
        if (unscaled) bb = scale2(bb, hk);
        const T rh = u ? radd(rfma(T(-2 * D), u[i], bb), s) : bb;
        a0 = fma((double)gp, (double)rh, a0);
        a1 = fma((double)E, (double)rh, a1);
        a2 = fma((double)C, (double)rh, a2);
    }
    __shared__ double red[3][256 / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[0][w] = a0;
        red[1][w] = a1;
        red[2][w] = a2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int k = 0; k < 256 / 32; ++k) s += red[threadIdx.x][k];
        partials[3 * blockIdx.x + threadIdx.x] = s;
    }
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

// acc[j] += sum over blocks of partials[3 b + j]: thread t sums the blocks
// t, t + 256, ... in that order, then a fixed shuffle/warp tree (the same
// order every run, independent of timing)
__global__ void __launch_bounds__(256) adj_accumulate(const double *__restrict__ partials, int nblocks,
                                                      double *__restrict__ acc)
{
    __shared__ double tot;
    for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[3 * b + j];
        block_sum_store<256>(s, &tot);
        __syncthreads();
        if (threadIdx.x == 0) acc[j] += tot;
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

void free_adjoint(mg_ctx *c)
{
    if (!c->adj) return;
    for (void *p : c->adj->owned) cudaFree(p);
    delete c->adj;
    c->adj = nullptr;
}

namespace {

template <typename T>
struct Adjoint {
    mg_ctx *c;
    AdjointWork *w;
    const T *b;  // caller's unscaled finest right-hand side
    cudaError_t err = cudaSuccess;

    bool ok(cudaError_t e)
    {
        if (e != cudaSuccess && err == cudaSuccess) err = e;
        return err == cudaSuccess;
    }
    int n(int l) const { return c->n[l]; }
    const T *bh(int k, int l) const { return l == 0 ? b : (const T *)w->bh[k][l]; }
    T *slot(int k, int l, int s) const { return (T *)w->work[k][l][s]; }

    // ---- forward replay with checkpoints ---------------------------------
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

    // visit of level l in cycle k with input `in` (nullptr = zero); the output
    // is left in the visit's last slot
    T *fwd_visit(int k, int l, const T *in)
    {
        const int nn = n(l);
        if (nn == 3) {
            T *x = slot(k, l, 0);
            solve_coarsest(bh(k, l), x);
            return x;
        }
        const bool unsc = l == 0;
        const T *cur = in;
        for (int s = 0; s < c->nu1; ++s) {
            T *out = slot(k, l, s);
            if (!ok(op_sweep_any(cur, bh(k, l), unsc, out, nn))) return nullptr;
            cur = out;
        }
        T *ua = slot(k, l, c->nu1 - 1);
        if (!ok(c->d == 2 ? launch_resrestrict2d<T>(ua, bh(k, l), unsc, (T *)w->bh[k][l + 1], nn, c->s)
                          : launch_resrestrict3d<T>(ua, bh(k, l), unsc, (T *)w->bh[k][l + 1], nn, c->s)))
            return nullptr;
        const T *e = fwd_visit(k, l + 1, nullptr);
        if (!e) return nullptr;
        if (!ok(c->d == 2 ? launch_prolong2d<T>(e, ua, nn, c->s) : launch_prolong3d<T>(e, ua, nn, c->s)))
            return nullptr;
        cur = ua;
        for (int s = 0; s < c->nu2; ++s) {
            T *out = slot(k, l, c->nu1 + s);
            if (!ok(op_sweep_any(cur, bh(k, l), unsc, out, nn))) return nullptr;
            cur = out;
        }
        return (T *)cur;
    }

    cudaError_t op_sweep_any(const T *u, const T *rhs, bool unsc, T *out, int nn)
    {
        return c->d == 2 ? launch_sweep2d<T>(u, rhs, unsc, out, nn, c->c, nullptr, c->s)
                         : launch_sweep3d<T>(u, rhs, unsc, out, nn, c->c, nullptr, c->s);
    }

    // ---- reverse ---------------------------------------------------------
    void adj_sweep(int k, int l, const T *u_in)
    {
        const int nn = n(l);
        const size_t np = npts(c->d, nn);
        const int grid = grid_for(np);
        const int hk = h2_exponent(nn);
        T *G = (T *)w->G[l], *Tt = (T *)w->T[l], *GB = (T *)w->GB[l];
        if (c->d == 2)
            adj_sweep_stage1<T, 2><<<grid, 256, 0, c->s>>>(G, u_in, bh(k, l), l == 0, Tt, nn, T(c->c[0]),
                                                           T(c->c[1]), T(c->c[2]), hk, w->partials);
        else
            adj_sweep_stage1<T, 3><<<grid, 256, 0, c->s>>>(G, u_in, bh(k, l), l == 0, Tt, nn, T(c->c[0]),
                                                           T(c->c[1]), T(0), hk, w->partials);
        adj_accumulate<<<1, 256, 0, c->s>>>(w->partials, grid, w->acc);
        if (c->d == 2)
            adj_stage2<T, 2><<<grid, 256, 0, c->s>>>(G, Tt, GB, nn);
        else
            adj_stage2<T, 3><<<grid, 256, 0, c->s>>>(G, Tt, GB, nn);
        count_launch(3);
        ok(cudaGetLastError());
    }

    // on entry w->G[l] = gradient w.r.t. the visit's output; on exit
    // w->G[l] = gradient w.r.t. its input and w->GB[l] has received the
    // gradient w.r.t. its right-hand side
    void rev_visit(int k, int l, const T *in)
    {
        const int nn = n(l);
        const size_t np = npts(c->d, nn);
        if (nn == 3) {
            solve_coarsest((const T *)w->G[l], (T *)w->GB[l]);
            ok(cudaMemsetAsync(w->G[l], 0, np * sizeof(T), c->s));
            return;
        }
        for (int s = c->nu2 - 1; s >= 0; --s) adj_sweep(k, l, slot(k, l, c->nu1 - 1 + s));
        // interpolation + correction: the child's output gradient is P^T g
        const int ncoarse = (nn - 1) / 2;
        const size_t npc = npts(c->d, ncoarse);
        const int gridc = grid_for(npc);
        if (c->d == 2)
            adj_fw<T, 2><<<gridc, 256, 0, c->s>>>((const T *)w->G[l], (T *)w->G[l + 1], nn, T(0.25));
        else
            adj_fw<T, 3><<<gridc, 256, 0, c->s>>>((const T *)w->G[l], (T *)w->G[l + 1], nn, T(0.125));
        count_launch(1);
        ok(cudaMemsetAsync(w->GB[l + 1], 0, npc * sizeof(T), c->s));
        rev_visit(k, l + 1, nullptr);
        // restriction: t = (4/2^d) P g_bh_child; g -= Ah t; gbh += t
        const int grid = grid_for(np);
        if (c->d == 2)
            adj_interp<T, 2><<<grid, 256, 0, c->s>>>((const T *)w->GB[l + 1], (T *)w->T[l], nn, T(1.0));
        else
            adj_interp<T, 3><<<grid, 256, 0, c->s>>>((const T *)w->GB[l + 1], (T *)w->T[l], nn, T(0.5));
        if (c->d == 2)
            adj_stage2<T, 2><<<grid, 256, 0, c->s>>>((T *)w->G[l], (const T *)w->T[l], (T *)w->GB[l], nn);
        else
            adj_stage2<T, 3><<<grid, 256, 0, c->s>>>((T *)w->G[l], (const T *)w->T[l], (T *)w->GB[l], nn);
        count_launch(2);
        ok(cudaGetLastError());
        for (int s = c->nu1 - 1; s >= 0; --s) adj_sweep(k, l, s == 0 ? in : slot(k, l, s - 1));
    }
};

}  // namespace
}  // namespace mg

using namespace mg;

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
        return p;
    };
    const size_t es = c->esize;
    const int slots = c->nu1 + c->nu2;
    w->work.assign(K, std::vector<std::vector<void *>>(c->L));
    w->bh.assign(K, std::vector<void *>(c->L, nullptr));
    for (int k = 0; k < K; ++k)
        for (int l = 0; l < c->L; ++l) {
            const size_t bytes = npts(c->d, c->n[l]) * es;
            const int ns = c->n[l] == 3 ? 1 : slots;
            for (int s = 0; s < ns; ++s) {
                void *p = alloc(bytes);
                if (!p) return MG_ENOMEM;
                w->work[k][l].push_back(p);
            }
            if (l >= 1 && !(w->bh[k][l] = alloc(bytes))) return MG_ENOMEM;
        }
    w->G.assign(c->L, nullptr);
    w->GB.assign(c->L, nullptr);
    w->T.assign(c->L, nullptr);
    for (int l = 0; l < c->L; ++l) {
        const size_t bytes = npts(c->d, c->n[l]) * es;
        if (!(w->G[l] = alloc(bytes)) || !(w->GB[l] = alloc(bytes)) || !(w->T[l] = alloc(bytes))) return MG_ENOMEM;
    }
    w->npartials = grid_for(npts(c->d, c->n[0]));
    if (!(w->partials = (double *)alloc((size_t)3 * w->npartials * sizeof(double)))) return MG_ENOMEM;
    if (!(w->acc = (double *)alloc(3 * sizeof(double)))) return MG_ENOMEM;
    return MG_OK;
}

template <typename T>
static mg_status run_adjoint(mg_ctx *c, int K, const T *b, const T *g_uK, T *g_b, double *g_c)
{
    AdjointWork *w = c->adj;
    Adjoint<T> A{c, w, b};
    // forward replay
    const T *u = nullptr;
    for (int k = 0; k < K; ++k) {
        u = A.fwd_visit(k, 0, u);
        if (!u) return cuda_fail(A.err);
    }
    // reverse
    const size_t np0 = npts(c->d, c->n[0]);
    if (cudaMemcpyAsync(w->G[0], g_uK, np0 * sizeof(T), cudaMemcpyDeviceToDevice, c->s) != cudaSuccess ||
        cudaMemsetAsync(w->GB[0], 0, np0 * sizeof(T), c->s) != cudaSuccess ||
        cudaMemsetAsync(w->acc, 0, 3 * sizeof(double), c->s) != cudaSuccess)
        return cuda_fail(cudaGetLastError());
    for (int k = K - 1; k >= 0; --k) {
        const T *in = k == 0 ? nullptr : A.slot(k - 1, 0, c->nu1 + c->nu2 - 1);
        A.rev_visit(k, 0, in);
        if (A.err != cudaSuccess) return cuda_fail(A.err);
    }
    const T h2 = T(1.0 / ((double)c->N * c->N));
    adj_scale<T><<<grid_for(np0), 256, 0, c->s>>>((const T *)w->GB[0], g_b, np0, h2);
    count_launch(1);
    double acc[3];
    cudaError_t e = cudaGetLastError();
    if (!e) e = cudaMemcpyAsync(acc, w->acc, sizeof acc, cudaMemcpyDeviceToHost, c->s);
    if (!e) e = cudaStreamSynchronize(c->s);
    if (e) return cuda_fail(e);
    for (int j = 0; j < c->ncoef; ++j) g_c[j] = acc[j];
    return MG_OK;
}

extern "C" mg_status mg_vcycles_adjoint(mg_ctx *ctx, int K, const void *b, const void *grad_uK, void *grad_b_out,
                                        double *grad_coeffs_out)
{
    if (!ctx || K < 1 || !b || !grad_uK || !grad_b_out || !grad_coeffs_out || ctx->batch ||
        ctx->gamma != 1 || ctx->nu1 < 1 || ctx->prec == MG_FP32_IR || ctx->L < 2 ||
        (ctx->d == 3 && ctx->ncoef > 2))  // the adjoint covers the 7-point M in 3D
        return MG_EINVAL;
    if (cudaSetDevice(ctx->dev) != cudaSuccess) return cuda_fail(cudaGetLastError());
    if (cudaEventRecord(ctx->ev_in, ctx->user) != cudaSuccess || cudaStreamWaitEvent(ctx->s, ctx->ev_in, 0) != cudaSuccess)
        return cuda_fail(cudaGetLastError());
    mg_status st = adj_alloc(ctx, K);
    if (st != MG_OK) return st;
    st = ctx->prec == MG_FP64
             ? run_adjoint<double>(ctx, K, (const double *)b, (const double *)grad_uK, (double *)grad_b_out, grad_coeffs_out)
             : run_adjoint<float>(ctx, K, (const float *)b, (const float *)grad_uK, (float *)grad_b_out, grad_coeffs_out);
    if (st != MG_OK) return st;
    if (cudaEventRecord(ctx->ev_out, ctx->s) != cudaSuccess || cudaStreamWaitEvent(ctx->user, ctx->ev_out, 0) != cudaSuccess)
        return cuda_fail(cudaGetLastError());
    return MG_OK;
}
