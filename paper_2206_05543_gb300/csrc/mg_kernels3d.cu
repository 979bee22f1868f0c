// mg_kernels3d.cu -- 3D kernels: SPAI sweep (7-point A, 7-point M), residual
// + full weighting, trilinear interpolation + correction, FP64 residual
// (He, Liu, Wang, arXiv:2206.05543, Sec. 2 Eq. (2.1), Sec. 3.2, Sec. 4).
//
// Design. Every kernel marches along z over a chunk of planes while a block
// owns a tile in (x, y); values along z live in registers, in-plane
// neighbours come through double-buffered shared-memory planes. Formulas and
// their rounding order are written next to each kernel and match the 2D
// kernels' conventions (scaled right-hand sides, h-free weights).
#include "mg_common.cuh"
#include "mg_internal.h"

namespace mg {

// SPAI sweeps (7- and 27-point M): output tiles of kT3 x kT3 points
constexpr int kT3 = 32;                  // output tile edge
constexpr int kT3R = kT3 + 2;            // residual tile edge (tile + one-point ring)
constexpr int kT3U = kT3 + 4;            // u plane edge (residual tile + one-point ring)
constexpr int kT3Ring = 4 * (kT3 + 1);   // residual ring points (132)
constexpr int kT3Ring2 = 4 * (kT3 + 3);  // outer u ring points (140)
constexpr int kS3Threads = 256;
constexpr int kS3Pts = kT3 * kT3 / kS3Threads;  // tile points per thread (4)
constexpr int kT3Rows = kS3Threads / kT3;
static_assert(kT3Ring <= kS3Threads && kT3Ring2 <= kS3Threads, "one ring point per thread");
static_assert(kT3Rows * kS3Pts == kT3, "four rows per thread");

template <typename T>
__device__ __forceinline__ T get3(const T *a, int n, int x, int y, int z)
{
    return (x >= 0 && x < n && y >= 0 && y < n && z >= 0 && z < n) ? a[((size_t)z * n + y) * n + x] : T(0);
}

// ---------------------------------------------------------------------------
// SPAI sweep, canonical evaluation at interior point p:
//   s  = ((u_W + u_E) + (u_S + u_N)) + (u_D + u_U)
//   rh = fma(-6, u_p, bh_p) + s          (rh := 0 outside the interior)
//   E  = ((rh_W + rh_E) + (rh_S + rh_N)) + (rh_D + rh_U)
//   u' = fma(c1, E, fma(c0, rh_p, u_p))
// (W/E = x-1/x+1, S/N = y-1/y+1, D/U = z-1/z+1). A block owns a 32x32 output
// tile; it forms rh on the tile and on the one-point ring around it (34x34),
// the u planes it reads cover one more ring (36x36). Thread t = 32 w + lane
// holds the tile points (lane, w + 8k), k < 4, with their z-windows of u and
// b in registers; the 132 residual-ring points belong one each to threads
// t < 132 (with their own z-windows), the 140 points of the outer u ring
// one each to the last 140 threads (the current plane only). Residual planes
// go through a ring of three shared planes, so the update of plane zz - 1
// takes rh(zz - 2) and rh(zz - 1) from shared memory and rh(zz) from the
// register it was just formed in. One barrier per plane: at step zz the u
// plane zz + 1 goes to the other half of the double buffer next to residual
// plane zz, and every global load is issued one step before its use. With
// 32-wide outputs an n = 2^k - 1 level needs no tile that is almost empty,
// and every warp of the update has all its lanes busy.
// ---------------------------------------------------------------------------
// point q of the ring at distance d (1 or 2) around the kT3 x kT3 tile,
// tile-relative; the four sides have kT3 + 2d - 1 points each
__device__ __forceinline__ void tile_ring_point(int q, int d, int &ri, int &rj)
{
    const int len = kT3 + 2 * d - 1, side = q / len, p = q - side * len;
    if (side == 0) { ri = p - d; rj = -d; }
    else if (side == 1) { ri = kT3 - 1 + d; rj = p - d; }
    else if (side == 2) { ri = p - d + 1; rj = kT3 - 1 + d; }
    else { ri = -d; rj = p - d + 1; }
}

// One segment: output planes [z0, z1) of tile (tx, ty). Starts and ends with
// the shared buffers free (the last step of the march ends in a barrier).
template <typename T, bool ZERO_U, bool UNSCALED_B, bool NORM>
__device__ __forceinline__ void sweep3d_segment(T (&su)[2][kT3U * kT3U], T (&sr)[3][kT3R * kT3R],
                                                const T *__restrict__ u, const T *__restrict__ b,
                                                T *__restrict__ out, int n, int tx, int ty, int z0, int z1,
                                                T c0, T c1, int hk, SqSum &acc)
{
    const int t = threadIdx.x, lane = t % kT3, w = t / kT3;
    const int ox0 = tx * kT3, oy0 = ty * kT3;
    const int px = ox0 + lane;
    const size_t plane = (size_t)n * n;
    const T m6 = in_reg(T(-6));
    c0 = in_reg(c0);
    c1 = in_reg(c1);

    bool own[kS3Pts];
    T u_prev[kS3Pts], u_cur[kS3Pts], u_next[kS3Pts], b_next[kS3Pts];
#pragma unroll
    for (int k = 0; k < kS3Pts; ++k) {
        const int py = oy0 + w + kT3Rows * k;
        own[k] = px < n && py < n;
        u_prev[k] = ZERO_U ? T(0) : get3(u, n, px, py, z0 - 2);
        u_cur[k] = ZERO_U ? T(0) : get3(u, n, px, py, z0 - 1);
        u_next[k] = ZERO_U ? T(0) : get3(u, n, px, py, z0);
        b_next[k] = get3(b, n, px, py, z0 - 1);
    }
    // residual ring point of threads t < kT3Ring
    const bool rr = t < kT3Ring;
    int ri = 0, rj = 0;
    tile_ring_point(rr ? t : 0, 1, ri, rj);
    const int rx = ox0 + ri, ry = oy0 + rj;
    const bool r_in = rr && rx >= 0 && rx < n && ry >= 0 && ry < n;
    T ru_prev = T(0), ru_cur = T(0), ru_next = T(0), rb_next = T(0);
    if (rr) {
        if (!ZERO_U) {
            ru_prev = get3(u, n, rx, ry, z0 - 2);
            ru_cur = get3(u, n, rx, ry, z0 - 1);
            ru_next = get3(u, n, rx, ry, z0);
        }
        rb_next = get3(b, n, rx, ry, z0 - 1);
    }
    // outer u ring point of the last kT3Ring2 threads
    const bool ro = !ZERO_U && t >= kS3Threads - kT3Ring2;
    int oi = 0, oj = 0;
    tile_ring_point(ro ? t - (kS3Threads - kT3Ring2) : 0, 2, oi, oj);
    T o_next = T(0);
    if (!ZERO_U) {
        const int zb = (z0 - 1) & 1;
#pragma unroll
        for (int k = 0; k < kS3Pts; ++k) su[zb][(w + kT3Rows * k + 2) * kT3U + lane + 2] = u_cur[k];
        if (rr) su[zb][(rj + 2) * kT3U + ri + 2] = ru_cur;
        if (ro) {
            su[zb][(oj + 2) * kT3U + oi + 2] = get3(u, n, ox0 + oi, oy0 + oj, z0 - 1);
            o_next = get3(u, n, ox0 + oi, oy0 + oj, z0);
        }
        __syncthreads();
    }

    // residual slots: s0 holds plane zz, s1 plane zz - 1, s2 plane zz - 2
    int s0 = 0, s1 = 2, s2 = 1;
    for (int zz = z0 - 1; zz <= z1; ++zz) {  // residual plane zz, output plane zz - 1
        const int buf = zz & 1;
        const bool zin = zz >= 0 && zz < n;
        T r_new[kS3Pts], u_nn[kS3Pts];
        T ru_nn = T(0), o_nn = T(0);
        if (!ZERO_U) {
#pragma unroll
            for (int k = 0; k < kS3Pts; ++k) u_nn[k] = get3(u, n, px, oy0 + w + kT3Rows * k, zz + 2);
            if (rr) ru_nn = get3(u, n, rx, ry, zz + 2);
            if (ro) o_nn = get3(u, n, ox0 + oi, oy0 + oj, zz + 2);
        }
#pragma unroll
        for (int k = 0; k < kS3Pts; ++k) {
            const int j = w + kT3Rows * k;
            T bb = b_next[k];
            b_next[k] = get3(b, n, px, oy0 + j, zz + 1);
            if (UNSCALED_B) bb = scale2(bb, hk);  // h^2 b, exact
            T r;
            if (!ZERO_U) {
                const T *row = &su[buf][(j + 2) * kT3U + lane + 2];
                const T s = radd(radd(radd(row[-1], row[1]), radd(row[-kT3U], row[kT3U])),
                                 radd(u_prev[k], u_next[k]));
                r = radd(rfma(m6, u_cur[k], bb), s);
                su[1 - buf][(j + 2) * kT3U + lane + 2] = u_next[k];
            } else {
                r = bb;
            }
            if (!(own[k] && zin)) r = T(0);
            if (NORM && own[k] && zz >= z0 && zz < z1) sq_add(acc, r);
            r_new[k] = r;
            sr[s0][(j + 1) * kT3R + lane + 1] = r;
        }
        if (NORM && (zz & 7) == 7) sq_flush(acc);  // at most 32 terms pending
        if (rr) {
            T bb = rb_next;
            rb_next = get3(b, n, rx, ry, zz + 1);
            if (UNSCALED_B) bb = scale2(bb, hk);
            T r;
            if (!ZERO_U) {
                const T *row = &su[buf][(rj + 2) * kT3U + ri + 2];
                const T s = radd(radd(radd(row[-1], row[1]), radd(row[-kT3U], row[kT3U])), radd(ru_prev, ru_next));
                r = radd(rfma(m6, ru_cur, bb), s);
                su[1 - buf][(rj + 2) * kT3U + ri + 2] = ru_next;
            } else {
                r = bb;
            }
            if (!(r_in && zin)) r = T(0);
            sr[s0][(rj + 1) * kT3R + ri + 1] = r;
        }
        if (ro) su[1 - buf][(oj + 2) * kT3U + oi + 2] = o_next;
        if (zz - 1 >= z0) {
#pragma unroll
            for (int k = 0; k < kS3Pts; ++k) {
                if (!own[k]) continue;
                const int j = w + kT3Rows * k, c = (j + 1) * kT3R + lane + 1;
                const T *row = &sr[s1][c];
                const T E = radd(radd(radd(row[-1], row[1]), radd(row[-kT3R], row[kT3R])), radd(sr[s2][c], r_new[k]));
                const T base = ZERO_U ? rmul(c0, row[0]) : rfma(c0, row[0], u_prev[k]);
                out[(size_t)(zz - 1) * plane + (size_t)(oy0 + j) * n + px] = rfma(c1, E, base);
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kS3Pts; ++k) {
            if (!ZERO_U) {
                u_prev[k] = u_cur[k];
                u_cur[k] = u_next[k];
                u_next[k] = u_nn[k];
            }
        }
        ru_prev = ru_cur;
        ru_cur = ru_next;
        ru_next = ru_nn;
        o_next = o_nn;
        const int sn = s2;
        s2 = s1;
        s1 = s0;
        s0 = sn;
    }
}

// Persistent and balanced: the (tile, plane) items, tile-major, are cut into
// gridDim.x equal runs of `per` consecutive items, one per block; a run is
// one or more z-segments of consecutive tiles. Every block does the same
// work, so the launch has no partly filled last wave (with 2 blocks per SM a
// tile-by-z-chunk grid left up to half of a wave idle). One squared partial
// sum per block. Resident blocks per SM: FP64 2 (no register cap that forces
// spills; measured fastest against 1, 3 and 4), FP32 3 (4 spills).
template <typename T, bool ZERO_U, bool UNSCALED_B, bool NORM>
__global__ void __launch_bounds__(kS3Threads, sweep3d_blocks_per_sm((int)sizeof(T)))
sweep3d_kernel(const T *__restrict__ u, const T *__restrict__ b, T *__restrict__ out, int n, int bx, long total,
               long per, T c0, T c1, int hk, double *__restrict__ partials)
{
    __shared__ T su[2][kT3U * kT3U];
    __shared__ T sr[3][kT3R * kT3R];
    SqSum acc;
    const long w0 = (long)blockIdx.x * per, w1 = w0 + per < total ? w0 + per : total;
    for (long w = w0; w < w1;) {
        const int tile = (int)(w / n), z0 = (int)(w - (long)tile * n);
        const int z1 = (int)(z0 + (w1 - w) < (long)n ? z0 + (w1 - w) : (long)n);
        sweep3d_segment<T, ZERO_U, UNSCALED_B, NORM>(su, sr, u, b, out, n, tile % bx, tile / bx, z0, z1, c0, c1,
                                                     hk, acc);
        w += z1 - z0;
    }
    if (NORM) block_sum_store<kS3Threads>(sq_value(acc), &partials[blockIdx.x]);
}

// ---------------------------------------------------------------------------
// 27-point SPAI sweep: a symmetric M with one weight per class of offsets,
// c0 the centre, c1 the 6 faces, c2 the 12 edges, c3 the 8 corners (the
// wider 3D stencils of Sec. 3.2's closing remark). Canonical evaluation at
// interior point p (rh as in the 7-point sweep, zero outside the interior):
//   per plane:  hp = rh_W + rh_E,  P1 = hp + (rh_S + rh_N),
//               P2 = hp(y - 1) + hp(y + 1)
//   F  = P1(z) + (rh(z - 1) + rh(z + 1))          (faces)
//   E  = P2(z) + (P1(z - 1) + P1(z + 1))          (edges)
//   C  = P2(z - 1) + P2(z + 1)                    (corners)
//   u' = fma(c3, C, fma(c2, E, fma(c1, F, fma(c0, rh_p, u_p))))
// With c2 = c3 = 0 the face sum F is the 7-point sweep's E; the library uses
// this kernel only when c2 or c3 is non-zero.
// The tiles are those of the 7-point sweep: a block owns a 32x32 output
// tile, forms rh on it and on the one-point ring around it (threads
// t < 132, one ring point each) and reads u planes of 36x36. Thread t owns
// column i = t % 32 of the output tile and the four consecutive rows
// 4 (t / 32) .. + 3: its x-pair sums hp of rows j - 1 .. j + 4 serve P1 and
// P2 of all four rows. Per output point (rh, P1, P2) of planes z - 1 and z
// stay in registers, plane z + 1's are formed at the step; the residual plane
// goes through shared memory once (double-buffered, one barrier per plane).
// ---------------------------------------------------------------------------
template <typename T, bool ZERO_U, bool UNSCALED_B, bool NORM>
__device__ __forceinline__ void sweep27_segment(T (&su)[2][kT3U * kT3U], T (&sr)[2][kT3R * kT3R],
                                                const T *__restrict__ u, const T *__restrict__ b,
                                                T *__restrict__ out, int n, int tx, int ty, int z0, int z1,
                                                T c0, T c1, T c2, T c3, int hk, SqSum &acc)
{
    const int t = threadIdx.x;
    const int i = t % kT3, j0 = kS3Pts * (t / kT3);
    const int ox0 = tx * kT3, oy0 = ty * kT3;
    const int px = ox0 + i;
    const size_t plane = (size_t)n * n;
    const T m6 = in_reg(T(-6));
    c0 = in_reg(c0);
    c1 = in_reg(c1);
    c2 = in_reg(c2);
    c3 = in_reg(c3);

    bool own[kS3Pts];
    T u_prev[kS3Pts], u_cur[kS3Pts], u_next[kS3Pts], b_next[kS3Pts];
    T r_m[kS3Pts], r_c[kS3Pts], p1_m[kS3Pts], p1_c[kS3Pts], p2_m[kS3Pts], p2_c[kS3Pts];
#pragma unroll
    for (int k = 0; k < kS3Pts; ++k) {
        const int py = oy0 + j0 + k;
        own[k] = px < n && py < n;
        u_prev[k] = ZERO_U ? T(0) : get3(u, n, px, py, z0 - 2);
        u_cur[k] = ZERO_U ? T(0) : get3(u, n, px, py, z0 - 1);
        u_next[k] = ZERO_U ? T(0) : get3(u, n, px, py, z0);
        b_next[k] = get3(b, n, px, py, z0 - 1);
        r_m[k] = r_c[k] = p1_m[k] = p1_c[k] = p2_m[k] = p2_c[k] = T(0);
    }
    // residual ring point of threads t < kT3Ring
    const bool rr = t < kT3Ring;
    int ri = 0, rj = 0;
    tile_ring_point(rr ? t : 0, 1, ri, rj);
    const int rx = ox0 + ri, ry = oy0 + rj;
    const bool r_in = rr && rx >= 0 && rx < n && ry >= 0 && ry < n;
    T ru_prev = T(0), ru_cur = T(0), ru_next = T(0), rb_next = T(0);
    if (rr) {
        if (!ZERO_U) {
            ru_prev = get3(u, n, rx, ry, z0 - 2);
            ru_cur = get3(u, n, rx, ry, z0 - 1);
            ru_next = get3(u, n, rx, ry, z0);
        }
        rb_next = get3(b, n, rx, ry, z0 - 1);
    }
    // outer u ring point of the last kT3Ring2 threads
    const bool ro = !ZERO_U && t >= kS3Threads - kT3Ring2;
    int oi = 0, oj = 0;
    tile_ring_point(ro ? t - (kS3Threads - kT3Ring2) : 0, 2, oi, oj);
    T o_next = T(0);
    if (!ZERO_U) {
        const int zb = (z0 - 1) & 1;
#pragma unroll
        for (int k = 0; k < kS3Pts; ++k) su[zb][(j0 + k + 2) * kT3U + i + 2] = u_cur[k];
        if (rr) su[zb][(rj + 2) * kT3U + ri + 2] = ru_cur;
        if (ro) {
            su[zb][(oj + 2) * kT3U + oi + 2] = get3(u, n, ox0 + oi, oy0 + oj, z0 - 1);
            o_next = get3(u, n, ox0 + oi, oy0 + oj, z0);
        }
        __syncthreads();
    }

    for (int zz = z0 - 1; zz <= z1; ++zz) {  // residual plane zz, output plane zz - 1
        const int buf = zz & 1;
        const bool zin = zz >= 0 && zz < n;
        T r_n[kS3Pts], u_nn[kS3Pts];
        T ru_nn = T(0), o_nn = T(0);
        if (!ZERO_U) {
#pragma unroll
            for (int k = 0; k < kS3Pts; ++k) u_nn[k] = get3(u, n, px, oy0 + j0 + k, zz + 2);
            if (rr) ru_nn = get3(u, n, rx, ry, zz + 2);
            if (ro) o_nn = get3(u, n, ox0 + oi, oy0 + oj, zz + 2);
        }
        // residual of plane zz at the thread's four tile points
        T up = T(0), dn = T(0);
        if (!ZERO_U) {
            up = su[buf][(j0 + 1) * kT3U + i + 2];           // row j0 - 1
            dn = su[buf][(j0 + kS3Pts + 2) * kT3U + i + 2];  // row j0 + 4
        }
#pragma unroll
        for (int k = 0; k < kS3Pts; ++k) {
            T bb = b_next[k];
            b_next[k] = get3(b, n, px, oy0 + j0 + k, zz + 1);
            if (UNSCALED_B) bb = scale2(bb, hk);  // h^2 b, exact
            T r;
            if (!ZERO_U) {
                const T *row = &su[buf][(j0 + k + 2) * kT3U + i + 2];
                const T us = k == 0 ? up : u_cur[k - 1];
                const T un = k == kS3Pts - 1 ? dn : u_cur[k + 1];
                const T s = radd(radd(radd(row[-1], row[1]), radd(us, un)), radd(u_prev[k], u_next[k]));
                r = radd(rfma(m6, u_cur[k], bb), s);
                su[1 - buf][(j0 + k + 2) * kT3U + i + 2] = u_next[k];
            } else {
                r = bb;
            }
            if (!(own[k] && zin)) r = T(0);
            if (NORM && own[k] && zz >= z0 && zz < z1) sq_add(acc, r);
            r_n[k] = r;
            sr[buf][(j0 + k + 1) * kT3R + i + 1] = r;
        }
        if (NORM && (zz & 7) == 7) sq_flush(acc);  // at most 32 terms pending
        if (rr) {
            T bb = rb_next;
            rb_next = get3(b, n, rx, ry, zz + 1);
            if (UNSCALED_B) bb = scale2(bb, hk);
            T r;
            if (!ZERO_U) {
                const T *row = &su[buf][(rj + 2) * kT3U + ri + 2];
                const T s = radd(radd(radd(row[-1], row[1]), radd(row[-kT3U], row[kT3U])), radd(ru_prev, ru_next));
                r = radd(rfma(m6, ru_cur, bb), s);
                su[1 - buf][(rj + 2) * kT3U + ri + 2] = ru_next;
            } else {
                r = bb;
            }
            if (!(r_in && zin)) r = T(0);
            sr[buf][(rj + 1) * kT3R + ri + 1] = r;
        }
        if (ro) su[1 - buf][(oj + 2) * kT3U + oi + 2] = o_next;
        __syncthreads();
        {
            // x-pair sums of rows j0 - 1 .. j0 + 4 of the residual plane
            const T *rp = sr[buf];
            T hp[kS3Pts + 2], rv[kS3Pts + 2];
#pragma unroll
            for (int q = 0; q < kS3Pts + 2; ++q) {
                const T *row = &rp[(j0 + q) * kT3R + i + 1];  // row j0 - 1 + q, column i
                hp[q] = radd(row[-1], row[1]);
                rv[q] = q >= 1 && q <= kS3Pts ? r_n[q - 1] : row[0];
            }
#pragma unroll
            for (int k = 0; k < kS3Pts; ++k) {
                const T p1 = radd(hp[k + 1], radd(rv[k], rv[k + 2]));
                const T p2 = radd(hp[k], hp[k + 2]);
                if (own[k] && zz - 1 >= z0) {
                    const T F = radd(p1_c[k], radd(r_m[k], r_n[k]));
                    const T E = radd(p2_c[k], radd(p1_m[k], p1));
                    const T C = radd(p2_m[k], p2);
                    const T base = ZERO_U ? rmul(c0, r_c[k]) : rfma(c0, r_c[k], u_prev[k]);
                    out[(size_t)(zz - 1) * plane + (size_t)(oy0 + j0 + k) * n + px] =
                        rfma(c3, C, rfma(c2, E, rfma(c1, F, base)));
                }
                p1_m[k] = p1_c[k];
                p1_c[k] = p1;
                p2_m[k] = p2_c[k];
                p2_c[k] = p2;
            }
        }
#pragma unroll
        for (int k = 0; k < kS3Pts; ++k) {
            r_m[k] = r_c[k];
            r_c[k] = r_n[k];
            if (!ZERO_U) {
                u_prev[k] = u_cur[k];
                u_cur[k] = u_next[k];
                u_next[k] = u_nn[k];
            }
        }
        ru_prev = ru_cur;
        ru_cur = ru_next;
        ru_next = ru_nn;
        o_next = o_nn;
    }
    __syncthreads();  // the next segment refills both buffers
}

// persistent like sweep3d_kernel (same (tile, plane) runs, same partials)
template <typename T, bool ZERO_U, bool UNSCALED_B, bool NORM>
__global__ void __launch_bounds__(kS3Threads, 1)
sweep27_kernel(const T *__restrict__ u, const T *__restrict__ b, T *__restrict__ out, int n, int bx, long total,
               long per, T c0, T c1, T c2, T c3, int hk, double *__restrict__ partials)
{
    __shared__ T su[2][kT3U * kT3U];
    __shared__ T sr[2][kT3R * kT3R];
    SqSum acc;
    const long w0 = (long)blockIdx.x * per, w1 = w0 + per < total ? w0 + per : total;
    for (long w = w0; w < w1;) {
        const int tile = (int)(w / n), z0 = (int)(w - (long)tile * n);
        const int z1 = (int)(z0 + (w1 - w) < (long)n ? z0 + (w1 - w) : (long)n);
        sweep27_segment<T, ZERO_U, UNSCALED_B, NORM>(su, sr, u, b, out, n, tile % bx, tile / bx, z0, z1, c0, c1, c2,
                                                     c3, hk, acc);
        w += z1 - z0;
    }
    if (NORM) block_sum_store<kS3Threads>(sq_value(acc), &partials[blockIdx.x]);
}

// ---------------------------------------------------------------------------
// Residual + full weighting. Coarse point (ic, jc, kc) has fine centre
// (2ic+1, 2jc+1, 2kc+1) (0-based):
//   along x: t1 = (rh(2ic) + rh(2ic+2)) + 2 rh(2ic+1)
//   along y: t2 = (t1(2jc) + t1(2jc+2)) + 2 t1(2jc+1)
//   along z: v  = (t2(2kc) + t2(2kc+2)) + 2 t2(2kc+1)
//   bh_c = 0.0625 v        (= 4 R rh, R = (1,2,1)/4 per axis)
// Block: 16x16 coarse columns; per fine plane the residual on the 33x33 fine
// patch is formed in shared memory from a ring of three u planes.
// (The load of a plane into the ring happens one step after its global read.)
// ---------------------------------------------------------------------------
constexpr int kR3 = 16;              // coarse tile edge
constexpr int kR3F = 2 * kR3 + 1;    // fine residual patch edge (33)
constexpr int kR3U = kR3F + 2;       // u patch edge incl. halo (35)
constexpr int kR3Threads = kR3 * kR3;

// at most 4 blocks per SM (measured fastest for the FP64 form against 2, 3 and 5)
template <typename T, bool UNSCALED_B>
__global__ void __launch_bounds__(kR3Threads, 4)
resrestrict3d_kernel(const T *__restrict__ u, const T *__restrict__ b, T *__restrict__ bc, int n, int Zc,
                     int hk)
{
    __shared__ T su[3][kR3U * kR3U];
    __shared__ T sr[kR3F * kR3F];
    __shared__ T st1[kR3F * kR3];
    const T m6 = in_reg(T(-6)), two = in_reg(T(2));
    const int nc = (n - 1) / 2;
    const int t = threadIdx.x;
    const int tic = t % kR3, tjc = t / kR3;
    const int ic0 = blockIdx.x * kR3, jc0 = blockIdx.y * kR3;
    const int ic = ic0 + tic, jc = jc0 + tjc;
    const int fx0 = 2 * ic0, fy0 = 2 * jc0;  // fine patch origin (0-based)
    const int kc0 = blockIdx.z * Zc, kc1 = min(kc0 + Zc, nc);
    const int f0 = 2 * kc0, f1 = 2 * kc1;
    const size_t plane = (size_t)n * n;

    // each thread moves the same (at most 5) points of every u plane and b
    // plane; the copies of plane f + 2 (u) and f + 1 (b) are loaded into
    // registers at step f, so their latency overlaps a step of work
    constexpr int kLU = (kR3U * kR3U + kR3Threads - 1) / kR3Threads;
    constexpr int kLB = (kR3F * kR3F + kR3Threads - 1) / kR3Threads;
    T upre[kLU], bpre[kLB];
    auto fetch_u = [&](int fz) {
#pragma unroll
        for (int k = 0; k < kLU; ++k) {
            const int q = t + k * kR3Threads;
            upre[k] = q < kR3U * kR3U ? get3(u, n, fx0 + q % kR3U - 1, fy0 + q / kR3U - 1, fz) : T(0);
        }
    };
    auto store_u = [&](int slot) {
#pragma unroll
        for (int k = 0; k < kLU; ++k) {
            const int q = t + k * kR3Threads;
            if (q < kR3U * kR3U) su[slot][q] = upre[k];
        }
    };
    auto fetch_b = [&](int fz) {
#pragma unroll
        for (int k = 0; k < kLB; ++k) {
            const int q = t + k * kR3Threads;
            const int x = fx0 + q % kR3F, y = fy0 + q / kR3F;
            bpre[k] = (q < kR3F * kR3F && x < n && y < n && fz < n) ? b[(size_t)fz * plane + (size_t)y * n + x] : T(0);
        }
    };
    fetch_u(f0 - 1);
    store_u((f0 - 1 + 3) % 3);
    fetch_u(f0);
    store_u(f0 % 3);
    fetch_u(f0 + 1);
    fetch_b(f0);
    T t2a = T(0), t2b = T(0);  // y-pass of fine planes f-2, f-1
    for (int f = f0; f <= f1; ++f) {
        store_u((f + 1) % 3);
        T bb_k[kLB];
#pragma unroll
        for (int k = 0; k < kLB; ++k) bb_k[k] = bpre[k];
        fetch_u(f + 2);
        fetch_b(f + 1);
        __syncthreads();
        const T *um = su[(f + 2) % 3], *uc = su[f % 3], *up = su[(f + 1) % 3];
#pragma unroll
        for (int k = 0; k < kLB; ++k) {
            const int q = t + k * kR3Threads;
            if (q >= kR3F * kR3F) break;
            const int i = q % kR3F, j = q / kR3F;
            const int x = fx0 + i, y = fy0 + j;
            const int p = (j + 1) * kR3U + (i + 1);
            T r = T(0);
            if (x < n && y < n && f < n) {
                T bb = bb_k[k];
                if (UNSCALED_B) bb = scale2(bb, hk);
                const T s = radd(radd(radd(uc[p - 1], uc[p + 1]), radd(uc[p - kR3U], uc[p + kR3U])),
                                 radd(um[p], up[p]));
                r = radd(rfma(m6, uc[p], bb), s);
            }
            sr[q] = r;
        }
        __syncthreads();
        for (int q = t; q < kR3F * kR3; q += kR3Threads) {
            const int k = q % kR3, j = q / kR3;
            const T *row = &sr[j * kR3F + 2 * k];
            st1[q] = rfma(two, row[1], radd(row[0], row[2]));
        }
        __syncthreads();
        const T t2 = rfma(two, st1[(2 * tjc + 1) * kR3 + tic], radd(st1[2 * tjc * kR3 + tic], st1[(2 * tjc + 2) * kR3 + tic]));
        if (f >= f0 + 2 && (f & 1) == 0 && ic < nc && jc < nc) {
            const int kc = f / 2 - 1;
            const T v = rfma(two, t2b, radd(t2a, t2));
            bc[((size_t)kc * nc + jc) * nc + ic] = scale2<-4>(v);  // 0.0625 v
        }
        t2a = t2b;
        t2b = t2;
        __syncthreads();  // the ring slot of plane f - 1 is reloaded next
    }
}

// ---------------------------------------------------------------------------
// Trilinear interpolation + correction u += P e: the value at fine point
// (fx, fy, fz) (0-based) is built along x, then y, then z:
//   along x: fx = 2k+1 -> e(k);  fx = 2k -> 0.5 (e(k-1) + e(k))
//   same along y on the x-values, then along z; u = u + value.
// Thread per fine (x, y) column of a 32x8 tile, marching over coarse planes.
// ---------------------------------------------------------------------------
constexpr int kP3X = 32, kP3Y = 8;

template <typename T>
__device__ __forceinline__ T p3_interp_x(const T *e, int nc, int fx, int jc, int kc)
{
    if (fx & 1) return get3(e, nc, fx >> 1, jc, kc);
    const int k = fx >> 1;
    return scale2<-1>(radd(get3(e, nc, k - 1, jc, kc), get3(e, nc, k, jc, kc)));
}

template <typename T>
__device__ __forceinline__ T p3_interp_xy(const T *e, int nc, int fx, int fy, int kc)
{
    if (fy & 1) return p3_interp_x(e, nc, fx, fy >> 1, kc);
    const int m = fy >> 1;
    return scale2<-1>(radd(p3_interp_x(e, nc, fx, m - 1, kc), p3_interp_x(e, nc, fx, m, kc)));
}

template <typename T>
__global__ void __launch_bounds__(kP3X * kP3Y)
prolong3d_kernel(const T *__restrict__ e, T *__restrict__ u, int n, int Zc)
{
    const int nc = (n - 1) / 2;
    const int fx = blockIdx.x * kP3X + threadIdx.x % kP3X;
    const int fy = blockIdx.y * kP3Y + threadIdx.x / kP3X;
    if (fx >= n || fy >= n) return;
    const int m0 = blockIdx.z * Zc, m1 = min(m0 + Zc, nc + 1);
    const size_t plane = (size_t)n * n;
    T *col = u + (size_t)fy * n + fx;
    // software pipeline: the coarse values and the two u values of step m + 1
    // are loaded before step m is written (this thread owns its column, the
    // block its fine planes 2 m0 .. 2 m1 - 1)
    T prev = p3_interp_xy(e, nc, fx, fy, m0 - 1);
    T cur = p3_interp_xy(e, nc, fx, fy, m0);
    T ue = col[(size_t)(2 * m0) * plane];
    T uo = m0 < nc ? col[(size_t)(2 * m0 + 1) * plane] : T(0);
    for (int m = m0; m < m1; ++m) {
        T nxt = T(0), ue_n = T(0), uo_n = T(0);
        if (m + 1 < m1) {
            nxt = p3_interp_xy(e, nc, fx, fy, m + 1);
            ue_n = col[(size_t)(2 * m + 2) * plane];
            if (m + 1 < nc) uo_n = col[(size_t)(2 * m + 3) * plane];
        }
        col[(size_t)(2 * m) * plane] = radd(ue, scale2<-1>(radd(prev, cur)));
        if (m < nc) col[(size_t)(2 * m + 1) * plane] = radd(uo, cur);
        prev = cur;
        cur = nxt;
        ue = ue_n;
        uo = uo_n;
    }
}

// ---------------------------------------------------------------------------
// Scaled residual rh = fma(-6, u, bh) + s (as in the sweep), InT arithmetic,
// written as OutT, with one squared partial sum per block. A block owns a
// 64 x 8 tile of (x, y) columns, thread t the two adjacent columns
// 2 (t % 32), 2 (t % 32) + 1 of row t / 32, and marches along z; the
// in-plane neighbours come from a double-buffered shared plane (tile plus a
// one-point ring), one barrier per plane, every global load one plane ahead.
// ---------------------------------------------------------------------------
constexpr int kQX = 64, kQY = 8, kQThreads = 256, kQW = kQX + 2;
constexpr int kQRing = 2 * kQX + 2 * kQY;  // 144 ring points, one per thread t < 144

// at most 6 blocks per SM (42 registers; measured fastest for the FP64 form)
template <typename InT, typename OutT>
__global__ void __launch_bounds__(kQThreads, 5)
residual3d_kernel(const InT *__restrict__ u, const InT *__restrict__ b, OutT *__restrict__ rh_out, int n,
                  int Z, int hk, bool unscaled, double *__restrict__ partials, long opitch, long oplane, long ooff)
{
    __shared__ InT su[2][(kQY + 2) * kQW];  // [(j + 1) * kQW + i + 1]: tile point (i, j), i in -1 .. 64
    const int t = threadIdx.x;
    const int tx = t % (kQX / 2), ty = t / (kQX / 2);
    const int X0 = blockIdx.x * kQX, Y0 = blockIdx.y * kQY;
    const int xa = X0 + 2 * tx, xb = xa + 1, y = Y0 + ty;
    const int z0 = blockIdx.z * Z, z1 = min(z0 + Z, n);
    const bool owna = xa < n && y < n, ownb = xb < n && y < n;
    const int ia = (ty + 1) * kQW + 2 * tx + 1;  // shared index of column xa
    // ring point of this thread (tile-relative (ri, rj))
    const bool ring = t < kQRing;
    int ri = 0, rj = 0;
    if (t < kQX) { ri = t; rj = -1; }
    else if (t < 2 * kQX) { ri = t - kQX; rj = kQY; }
    else if (t < 2 * kQX + kQY) { ri = -1; rj = t - 2 * kQX; }
    else { ri = kQX; rj = t - 2 * kQX - kQY; }
    const int ir = (rj + 1) * kQW + ri + 1;

    InT ap = get3(u, n, xa, y, z0 - 1), bp = get3(u, n, xb, y, z0 - 1);
    InT ac = get3(u, n, xa, y, z0), bc = get3(u, n, xb, y, z0);
    InT an = get3(u, n, xa, y, z0 + 1), bn = get3(u, n, xb, y, z0 + 1);
    InT fa_next = get3(b, n, xa, y, z0), fb_next = get3(b, n, xb, y, z0);
    InT ring_next = InT(0);
    su[z0 & 1][ia] = ac;
    su[z0 & 1][ia + 1] = bc;
    if (ring) {
        su[z0 & 1][ir] = get3(u, n, X0 + ri, Y0 + rj, z0);
        ring_next = get3(u, n, X0 + ri, Y0 + rj, z0 + 1);
    }
    __syncthreads();
    // -6 from a register: a DFMA with a constant-bank operand issues at the
    // DADD rate (measured 2D: no gain, its register budget is tighter)
    const InT m6 = in_reg(InT(-6));
    SqSum acc;
    for (int z = z0; z < z1; ++z) {
        const int buf = z & 1;
        InT fa = fa_next, fb = fb_next;
        fa_next = get3(b, n, xa, y, z + 1);
        fb_next = get3(b, n, xb, y, z + 1);
        const InT ann = get3(u, n, xa, y, z + 2), bnn = get3(u, n, xb, y, z + 2);
        const InT ring_nn = ring ? get3(u, n, X0 + ri, Y0 + rj, z + 2) : InT(0);
        if (unscaled) {
            fa = scale2(fa, hk);
            fb = scale2(fb, hk);
        }
        const InT *P = su[buf];
        const InT sa = radd(radd(radd(P[ia - 1], bc), radd(P[ia - kQW], P[ia + kQW])), radd(ap, an));
        const InT sb = radd(radd(radd(ac, P[ia + 2]), radd(P[ia + 1 - kQW], P[ia + 1 + kQW])), radd(bp, bn));
        const InT ra = radd(rfma(m6, ac, fa), sa);
        const InT rb = radd(rfma(m6, bc, fb), sb);
        if (owna) {
            sq_add(acc, ra);
            if (rh_out)
                rh_out[opitch ? ooff + z * oplane + (long)y * opitch + xa : ((long)z * n + y) * n + xa] =
                    to_out<OutT>(ra);
        }
        if (ownb) {
            sq_add(acc, rb);
            if (rh_out)
                rh_out[opitch ? ooff + z * oplane + (long)y * opitch + xb : ((long)z * n + y) * n + xb] =
                    to_out<OutT>(rb);
        }
        if ((z & 15) == 15) sq_flush(acc);  // at most 32 terms pending
        su[1 - buf][ia] = an;
        su[1 - buf][ia + 1] = bn;
        if (ring) su[1 - buf][ir] = ring_next;
        __syncthreads();
        ap = ac;
        ac = an;
        an = ann;
        bp = bc;
        bc = bn;
        bn = bnn;
        ring_next = ring_nn;
    }
    if (partials)
        block_sum_store<kQThreads>(sq_value(acc), &partials[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x]);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// One block per resident slot, runs of at least 2 planes (small levels need
// the blocks more than they mind the two extra residual planes of a run).
// The 7- and 27-point sweeps share the tiles and the plan.
S3Plan sweep3d_plan(int n, int elem_bytes)
{
    S3Plan g;
    g.bx = (n + kT3 - 1) / kT3;
    g.total = (long)g.bx * g.bx * n;
    const long most = std::min<long>((long)sweep3d_blocks_per_sm(elem_bytes) * num_sms(), (g.total + 1) / 2);
    g.per = (g.total + most - 1) / most;
    g.blocks = (int)((g.total + g.per - 1) / g.per);
    return g;
}

Grid3 residual3d_grid(int n)
{
    Grid3 g;
    g.bx = (n + kQX - 1) / kQX;
    g.by = (n + kQY - 1) / kQY;
    g.Z = chunk_rows(g.bx * g.by, n, 8 * num_sms(), 2, 64);
    g.bz = (n + g.Z - 1) / g.Z;
    return g;
}

template <typename T>
cudaError_t launch_sweep3d(const T *u, const T *b, bool unscaled, T *out, int n, const double *c,
                           double *partials, cudaStream_t s)
{
    const bool wide = c[2] != 0.0 || c[3] != 0.0;  // 27-point M (edge or corner weights)
    const S3Plan g = sweep3d_plan(n, (int)sizeof(T));
    const int hk = h2_exponent(n);
    const T c0 = T(c[0]), c1 = T(c[1]), c2 = T(c[2]), c3 = T(c[3]);
#define MG_SWEEP(ZU, UB, NRM)                                                                                     \
    do {                                                                                                          \
        if (wide)                                                                                                 \
            sweep27_kernel<T, ZU, UB, NRM><<<g.blocks, kS3Threads, 0, s>>>(u, b, out, n, g.bx, g.total, g.per, c0, \
                                                                           c1, c2, c3, hk, partials);              \
        else                                                                                                      \
            sweep3d_kernel<T, ZU, UB, NRM><<<g.blocks, kS3Threads, 0, s>>>(u, b, out, n, g.bx, g.total, g.per, c0, \
                                                                           c1, hk, partials);                      \
    } while (0)
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
cudaError_t launch_resrestrict3d(const T *u, const T *b, bool unscaled, T *bc, int n, cudaStream_t s)
{
    const int nc = (n - 1) / 2;
    const int bxy = (nc + kR3 - 1) / kR3;
    const int Zc = chunk_rows(bxy * bxy, nc, 8 * num_sms(), 1, 32);
    const dim3 grid(bxy, bxy, (nc + Zc - 1) / Zc);
    const int hk = h2_exponent(n);
    if (unscaled)
        resrestrict3d_kernel<T, true><<<grid, kR3Threads, 0, s>>>(u, b, bc, n, Zc, hk);
    else
        resrestrict3d_kernel<T, false><<<grid, kR3Threads, 0, s>>>(u, b, bc, n, Zc, hk);
    count_launch(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong3d(const T *e, T *u, int n, cudaStream_t s)
{
    const int nc = (n - 1) / 2;
    const int bx = (n + kP3X - 1) / kP3X, by = (n + kP3Y - 1) / kP3Y;
    const int Zc = chunk_rows(bx * by, nc + 1, 8 * num_sms(), 1, 32);
    const dim3 grid(bx, by, (nc + 1 + Zc - 1) / Zc);
    prolong3d_kernel<T><<<grid, kP3X * kP3Y, 0, s>>>(e, u, n, Zc);
    count_launch(1);
    return cudaGetLastError();
}

template <typename InT, typename OutT>
cudaError_t launch_residual3d(const InT *u, const InT *b, bool unscaled, OutT *rh, int n, double *partials,
                              cudaStream_t s, long out_pitch, long out_plane, long out_off)
{
    const Grid3 g = residual3d_grid(n);
    residual3d_kernel<InT, OutT><<<dim3(g.bx, g.by, g.bz), kQThreads, 0, s>>>(
        u, b, rh, n, g.Z, h2_exponent(n), unscaled, partials, out_pitch, out_plane, out_off);
    count_launch(1);
    return cudaGetLastError();
}

#define MG_INST(T)                                                                                   \
    template cudaError_t launch_sweep3d<T>(const T *, const T *, bool, T *, int, const double *,     \
                                           double *, cudaStream_t);                                  \
    template cudaError_t launch_resrestrict3d<T>(const T *, const T *, bool, T *, int, cudaStream_t); \
    template cudaError_t launch_prolong3d<T>(const T *, T *, int, cudaStream_t);
MG_INST(double)
MG_INST(float)
#undef MG_INST
template cudaError_t launch_residual3d<double, double>(const double *, const double *, bool, double *, int,
                                                       double *, cudaStream_t, long, long, long);
template cudaError_t launch_residual3d<double, float>(const double *, const double *, bool, float *, int,
                                                      double *, cudaStream_t, long, long, long);
template cudaError_t launch_residual3d<float, float>(const float *, const float *, bool, float *, int,
                                                     double *, cudaStream_t, long, long, long);

}  // namespace mg
