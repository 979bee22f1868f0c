// mg_tail.cu -- the coarse tail of the cycle in one thread block, and the
// coarsest-grid solve (He, Liu, Wang, arXiv:2206.05543, Sec. 4).
//
// The last levels of the hierarchy (a few hundred points) are far too small
// to fill the GPU; one launch per operator per level would be pure launch
// latency. One block therefore runs the whole tail of a cycle: the host
// writes the cycle's operations on these levels (zero, sweep, residual +
// restriction, exact solve, interpolation + correction, V or W order) into
// the kernel's argument block, and the block executes them in order with a
// block barrier between operations. Level arrays stay in global memory
// (resident in L1/L2 at these sizes).
//
// Formulas and their rounding order are identical to the marching kernels
// (see mg_kernels2d.cu / mg_kernels3d.cu); the coarsest solve uses the LU
// factors of h0^2 A_h0 computed once on the host by Gaussian elimination
// without pivoting in the natural order (unknowns x fastest):
//   forward:  y_i = y_i - l_ik y_k          for k = 0 .. i-1
//   backward: s = y_i - u_ij x_j (j = i+1 .. m-1, increasing); x_i = s / u_ii
// with every product rounded before the subtraction.
#include "mg_common.cuh"
#include "mg_internal.h"

namespace mg {

struct Lay {
    int n, pitch;
    long plane, off;
};
__device__ __forceinline__ long lidx(const Lay &L, int x, int y, int z)
{
    return L.off + z * L.plane + (long)y * L.pitch + x;
}

template <typename T>
__device__ __forceinline__ T at(const T *a, const Lay &L, int x, int y, int z)
{
    if (x < 0 || x >= L.n || y < 0 || y >= L.n || z < 0 || z >= L.n) return T(0);
    return a[lidx(L, x, y, z)];
}

template <typename T>
__device__ T residual_at(int d, const T *u, const T *bh, const Lay &L, int x, int y, int z)
{
    const long p = lidx(L, x, y, z);
    if (d == 2) {
        const T s = radd(radd(at(u, L, x - 1, y, 0), at(u, L, x + 1, y, 0)),
                         radd(at(u, L, x, y - 1, 0), at(u, L, x, y + 1, 0)));
        return radd(rfma(T(-4), u[p], bh[p]), s);
    }
    const T s = radd(radd(radd(at(u, L, x - 1, y, z), at(u, L, x + 1, y, z)),
                          radd(at(u, L, x, y - 1, z), at(u, L, x, y + 1, z))),
                     radd(at(u, L, x, y, z - 1), at(u, L, x, y, z + 1)));
    return radd(rfma(T(-6), u[p], bh[p]), s);
}

// in-plane sums of the 27-point sweep (see mg_kernels3d.cu): x pair, the 4
// edge neighbours and the 4 corner neighbours of (x, y) in plane z
template <typename T>
__device__ __forceinline__ T hp_at(const T *rh, const Lay &L, int x, int y, int z)
{
    return radd(at(rh, L, x - 1, y, z), at(rh, L, x + 1, y, z));
}
template <typename T>
__device__ __forceinline__ T p1_at(const T *rh, const Lay &L, int x, int y, int z)
{
    return radd(hp_at(rh, L, x, y, z), radd(at(rh, L, x, y - 1, z), at(rh, L, x, y + 1, z)));
}
template <typename T>
__device__ __forceinline__ T p2_at(const T *rh, const Lay &L, int x, int y, int z)
{
    return radd(hp_at(rh, L, x, y - 1, z), hp_at(rh, L, x, y + 1, z));
}

template <typename T>
__device__ T sweep_at(int d, const T *rh, const T *u, const Lay &L, int x, int y, int z, T c0, T c1, T c2, T c3)
{
    const long p = lidx(L, x, y, z);
    if (d == 2) {
        const T E = radd(radd(at(rh, L, x - 1, y, 0), at(rh, L, x + 1, y, 0)),
                         radd(at(rh, L, x, y - 1, 0), at(rh, L, x, y + 1, 0)));
        const T C = radd(radd(at(rh, L, x - 1, y - 1, 0), at(rh, L, x + 1, y - 1, 0)),
                         radd(at(rh, L, x - 1, y + 1, 0), at(rh, L, x + 1, y + 1, 0)));
        return rfma(c2, C, rfma(c1, E, rfma(c0, rh[p], u[p])));
    }
    if (c2 != T(0) || c3 != T(0)) {  // 27-point M
        const T F = radd(p1_at(rh, L, x, y, z), radd(at(rh, L, x, y, z - 1), at(rh, L, x, y, z + 1)));
        const T E = radd(p2_at(rh, L, x, y, z), radd(p1_at(rh, L, x, y, z - 1), p1_at(rh, L, x, y, z + 1)));
        const T C = radd(p2_at(rh, L, x, y, z - 1), p2_at(rh, L, x, y, z + 1));
        return rfma(c3, C, rfma(c2, E, rfma(c1, F, rfma(c0, rh[p], u[p]))));
    }
    const T E = radd(radd(radd(at(rh, L, x - 1, y, z), at(rh, L, x + 1, y, z)),
                          radd(at(rh, L, x, y - 1, z), at(rh, L, x, y + 1, z))),
                     radd(at(rh, L, x, y, z - 1), at(rh, L, x, y, z + 1)));
    return rfma(c1, E, rfma(c0, rh[p], u[p]));
}

// full weighting along x of fine row (fy, fz) around fine column 2ic+1
template <typename T>
__device__ __forceinline__ T fw_x(const T *rh, const Lay &L, int ic, int fy, int fz)
{
    const T *row = rh + lidx(L, 0, fy, fz);
    return rfma(T(2), row[2 * ic + 1], radd(row[2 * ic], row[2 * ic + 2]));
}

template <typename T>
__device__ T restrict_at(int d, const T *rh, const Lay &L, int ic, int jc, int kc)
{
    if (d == 2) {
        const T t0 = fw_x(rh, L, ic, 2 * jc, 0), t1 = fw_x(rh, L, ic, 2 * jc + 1, 0),
                t2 = fw_x(rh, L, ic, 2 * jc + 2, 0);
        return scale2<-2>(rfma(T(2), t1, radd(t0, t2)));  // 0.25 v
    }
    T tz[3];
    for (int k = 0; k < 3; ++k) {
        const int fz = 2 * kc + k;
        const T t0 = fw_x(rh, L, ic, 2 * jc, fz), t1 = fw_x(rh, L, ic, 2 * jc + 1, fz),
                t2 = fw_x(rh, L, ic, 2 * jc + 2, fz);
        tz[k] = rfma(T(2), t1, radd(t0, t2));
    }
    return scale2<-4>(rfma(T(2), tz[1], radd(tz[0], tz[2])));  // 0.0625 v
}

// linear interpolation of the coarse array e at fine 0-based coordinates:
// along x, then y, then z.
template <typename T>
__device__ T interp_x(const T *e, const Lay &Lc, int fx, int jc, int kc)
{
    // fine 0-based fx = 2k+1 sits on coarse k; fx = 2k lies between k-1 and k
    if (fx & 1) return at(e, Lc, fx >> 1, jc, kc);
    const int k = fx >> 1;
    return scale2<-1>(radd(at(e, Lc, k - 1, jc, kc), at(e, Lc, k, jc, kc)));
}

template <typename T>
__device__ T interp_xy(const T *e, const Lay &Lc, int fx, int fy, int kc)
{
    if (fy & 1) return interp_x(e, Lc, fx, fy >> 1, kc);
    const int m = fy >> 1;
    return scale2<-1>(radd(interp_x(e, Lc, fx, m - 1, kc), interp_x(e, Lc, fx, m, kc)));
}

template <typename T>
__device__ T interp_at(int d, const T *e, const Lay &Lc, int fx, int fy, int fz)
{
    if (d == 2) return interp_xy(e, Lc, fx, fy, 0);
    if (fz & 1) return interp_xy(e, Lc, fx, fy, fz >> 1);
    const int q = fz >> 1;
    return scale2<-1>(radd(interp_xy(e, Lc, fx, fy, q - 1), interp_xy(e, Lc, fx, fy, q)));
}

// Coarsest solve x = B bh with B the exact inverse of h0^2 A_h0 (formed on
// the host by coarse_inverse): thread i < m forms x_i = sum_j B_ij bh_j in
// increasing j, each product rounded before the addition. The m dot
// products run in parallel (a triangular solve on this part is a long
// dependent FP64 chain).
template <typename T>
__device__ void coarse_apply(int d, const double *__restrict__ inv, const T *bh, T *x, const Lay &L)
{
    const int m = d == 2 ? 9 : 27;
    const int i = threadIdx.x;
    if (i < m) {
        double s = 0.0;
        for (int j = 0; j < m; ++j)
            s = __dadd_rn(s, __dmul_rn(__ldg(&inv[i * m + j]), (double)bh[lidx(L, j % 3, (j / 3) % 3, j / 9)]));
        x[lidx(L, i % 3, (i / 3) % 3, i / 9)] = (T)s;
    }
}

template <typename T>
__device__ void run_tail(const TailLevel *lv, const TailOp *ops, int nops, int d, T c0, T c1, T c2, T c3,
                         const double *lu)
{
    for (int o = 0; o < nops; ++o) {
        const int kind = ops[o].kind, l = ops[o].level;
        const TailLevel &TL = lv[l];
        const Lay L{TL.n, TL.pitch, TL.plane, TL.off};
        const int n = TL.n;
        const int np = d == 2 ? n * n : n * n * n;
        T *u = (T *)TL.u, *tmp = (T *)TL.tmp, *bh = (T *)TL.bh, *rh = (T *)TL.rh;
        auto coords = [&](int i, int nn, int &x, int &y, int &z) {
            x = i % nn;
            y = (i / nn) % nn;
            z = d == 2 ? 0 : i / (nn * nn);
        };
        if (kind == TAIL_ZERO) {
            for (int i = threadIdx.x; i < np; i += blockDim.x) {
                int x, y, z;
                coords(i, n, x, y, z);
                u[lidx(L, x, y, z)] = T(0);
            }
        } else if (kind == TAIL_SWEEP || kind == TAIL_RESTRICT) {
            for (int i = threadIdx.x; i < np; i += blockDim.x) {
                int x, y, z;
                coords(i, n, x, y, z);
                rh[lidx(L, x, y, z)] = residual_at(d, u, bh, L, x, y, z);
            }
            __syncthreads();
            if (kind == TAIL_SWEEP) {
                for (int i = threadIdx.x; i < np; i += blockDim.x) {
                    int x, y, z;
                    coords(i, n, x, y, z);
                    tmp[lidx(L, x, y, z)] = sweep_at(d, rh, u, L, x, y, z, c0, c1, c2, c3);
                }
                __syncthreads();
                for (int i = threadIdx.x; i < np; i += blockDim.x) {
                    int x, y, z;
                    coords(i, n, x, y, z);
                    u[lidx(L, x, y, z)] = tmp[lidx(L, x, y, z)];
                }
            } else {
                const TailLevel &C = lv[l + 1];
                const Lay Lc{C.n, C.pitch, C.plane, C.off};
                const int nc = C.n, npc = d == 2 ? nc * nc : nc * nc * nc;
                T *bc = (T *)C.bh;
                for (int i = threadIdx.x; i < npc; i += blockDim.x) {
                    int x, y, z;
                    coords(i, nc, x, y, z);
                    bc[lidx(Lc, x, y, z)] = restrict_at(d, rh, L, x, y, z);
                }
            }
        } else if (kind == TAIL_SOLVE) {
            coarse_apply<T>(d, lu, bh, u, L);
        } else if (kind == TAIL_PROLONG) {
            const TailLevel &C = lv[l + 1];
            const Lay Lc{C.n, C.pitch, C.plane, C.off};
            const T *e = (const T *)C.u;
            for (int i = threadIdx.x; i < np; i += blockDim.x) {
                int x, y, z;
                coords(i, n, x, y, z);
                const long p = lidx(L, x, y, z);
                u[p] = radd(u[p], interp_at(d, e, Lc, x, y, z));
            }
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(kTailThreads) tail_kernel(TailArgs a)
{
    run_tail<T>(a.lv, a.ops, a.nops, a.d, T(a.c[0]), T(a.c[1]), T(a.c[2]), T(a.c[3]), a.lu);
}

// one block per problem: the tail of problem blockIdx.x (skipped when inactive)
template <typename T>
__global__ void __launch_bounds__(kTailThreads)
tail_batched(const TailLevel *__restrict__ lv, const TailOp *__restrict__ ops, const int *__restrict__ op_off,
             const int *__restrict__ op_cnt, const int *__restrict__ active, int d, double c0, double c1, double c2,
             const double *__restrict__ lu)
{
    const int p = blockIdx.x;
    if (!active[p]) return;
    run_tail<T>(lv + (size_t)p * kMaxTailLevels, ops + op_off[p], op_cnt[p], d, T(c0), T(c1), T(c2), T(0), lu);
}

template <typename T>
cudaError_t launch_tail_batched(const TailLevel *lv, const TailOp *ops, const int *op_off, const int *op_cnt,
                                const int *active, int count, int d, const double *c, const double *lu, cudaStream_t s)
{
    tail_batched<T><<<count, kTailThreads, 0, s>>>(lv, ops, op_off, op_cnt, active, d, c[0], c[1], c[2], lu);
    count_launch(1);
    return cudaGetLastError();
}
template cudaError_t launch_tail_batched<float>(const TailLevel *, const TailOp *, const int *, const int *,
                                                const int *, int, int, const double *, const double *, cudaStream_t);
template cudaError_t launch_tail_batched<double>(const TailLevel *, const TailOp *, const int *, const int *,
                                                 const int *, int, int, const double *, const double *, cudaStream_t);

template <typename T>
cudaError_t launch_tail(const TailArgs &a, cudaStream_t s)
{
    tail_kernel<T><<<1, kTailThreads, 0, s>>>(a);
    count_launch(1);
    return cudaGetLastError();
}

template cudaError_t launch_tail<double>(const TailArgs &, cudaStream_t);
template cudaError_t launch_tail<float>(const TailArgs &, cudaStream_t);

// LU factors of the scaled coarsest operator h0^2 A_h0 (3^d unknowns, natural
// order), written into lu (m*m, row-major): strict lower part = multipliers,
// upper part incl. diagonal = U. Host code, compiled without contraction.
void coarse_inverse(int d, double *inv)
{
    // Gaussian elimination without pivoting on h0^2 A_h0 (natural order),
    // products rounded before each subtraction; column j of the inverse is
    // the forward substitution (y_i -= l_ik y_k, k increasing) and back
    // substitution (s -= u_ij x_j, j increasing; x_i = s / u_ii) of e_j.
    const int n = 3, m = d == 2 ? 9 : 27;
    double lu[27 * 27];
    for (int i = 0; i < m; ++i) {
        const int xi = i % n, yi = (i / n) % n, zi = i / (n * n);
        for (int j = 0; j < m; ++j) {
            const int xj = j % n, yj = (j / n) % n, zj = j / (n * n);
            const int dist = abs(xi - xj) + abs(yi - yj) + abs(zi - zj);
            lu[i * m + j] = i == j ? 2.0 * d : (dist == 1 ? -1.0 : 0.0);
        }
    }
    for (int k = 0; k < m; ++k)
        for (int i = k + 1; i < m; ++i) {
            const double l = lu[i * m + k] / lu[k * m + k];
            for (int j = k + 1; j < m; ++j) lu[i * m + j] = lu[i * m + j] - l * lu[k * m + j];
            lu[i * m + k] = l;
        }
    for (int c = 0; c < m; ++c) {
        double y[27], x[27];
        for (int i = 0; i < m; ++i) y[i] = i == c ? 1.0 : 0.0;
        for (int i = 0; i < m; ++i)
            for (int k = 0; k < i; ++k) y[i] = y[i] - lu[i * m + k] * y[k];
        for (int i = m - 1; i >= 0; --i) {
            double s = y[i];
            for (int j = i + 1; j < m; ++j) s = s - lu[i * m + j] * x[j];
            x[i] = s / lu[i * m + i];
        }
        for (int i = 0; i < m; ++i) inv[i * m + c] = x[i];
    }
}

}  // namespace mg
