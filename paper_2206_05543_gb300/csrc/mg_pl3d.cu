// mg_pl3d.cu -- FP32 3D kernels on the padded level layout (internal levels
// of the 3D refinement cycle).
//
// Layout (Pitch3): element (x, y, z), each in [-1, n], at
// off + z*plane + y*pitch + x, with a zero ghost ring and 16-byte-aligned,
// padded rows, so threads move four x-columns with one float4 and read no
// bounds-checked element. Formulas and operation order as in
// mg_kernels3d.cu (the results equal the compact FP32 kernels bit for bit).
#include "mg_common.cuh"
#include "mg_internal.h"

namespace mg {

constexpr int kP3TX = 32;                 // threads along x (4 columns each)
constexpr int kP3Cols = 4 * kP3TX;        // 128 columns per tile
constexpr int kP3TY = 14;                 // output rows per tile
constexpr int kP3Rows = kP3TY + 2;        // residual rows per tile (with halo)
constexpr int kP3Threads = kP3TX * kP3Rows;  // 512
constexpr int kP3W = kP3Cols + 8;         // shared row width (4 halo columns each side)

__device__ __forceinline__ float4 ld4g(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4g(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float &e4(float4 &v, int k) { return (&v.x)[k]; }
__device__ __forceinline__ float ce4(const float4 &v, int k) { return (&v.x)[k]; }

// ---------------------------------------------------------------------------
// SPAI sweep (formula as sweep3d_kernel): the block computes the residual on
// 128 columns x 16 rows (output 128 x 14) per plane, marching over z.
// ACC64: the refinement epilogue, u64 (compact FP64) += result.
// ---------------------------------------------------------------------------
template <bool ZERO_U, bool ACC64>
__global__ void __launch_bounds__(kP3Threads)
sweep3d_pl_kernel(const float *__restrict__ u, const float *__restrict__ b, float *__restrict__ out,
                  double *__restrict__ u64, Pitch3 g, int Z, float c0, float c1)
{
    __shared__ __align__(16) float su[2][kP3Rows + 2][kP3W];
    __shared__ __align__(16) float sr[3][kP3Rows][kP3W];
    const int n = g.n;
    const int tx = threadIdx.x % kP3TX, ty = threadIdx.x / kP3TX;
    const int x0 = blockIdx.x * kP3Cols, y0 = blockIdx.y * kP3TY;
    const int x = x0 + 4 * tx, yr = y0 - 1 + ty;
    const int z0 = blockIdx.z * Z, z1 = min(z0 + Z, n);
    const float *U = u + g.off, *Bp = b + g.off;
    const long P = g.pitch, S = g.plane;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    auto ok = [&](int y, int z) { return y >= -1 && y <= n && z >= -1 && z <= n; };
    auto at4 = [&](const float *a, int xx, int y, int z) { return ok(y, z) ? ld4g(a + z * S + y * P + xx) : z4; };
    auto at1 = [&](const float *a, int xx, int y, int z) { return ok(y, z) ? a[z * S + y * P + xx] : 0.f; };
    const bool lt = tx == 0, rt = tx == kP3TX - 1;
    const int xh = lt ? x0 - 1 : x0 + kP3Cols;  // halo column of the edge threads
    const bool yin = yr >= 0 && yr < n;
    const bool own_row = ty >= 1 && ty <= kP3TY && yin;

    float4 um = z4, uc = z4, un = z4, rm = z4, rc = z4, bn;
    float hm = 0.f, hc = 0.f, hn = 0.f, hb, rhm = 0.f, rhc = 0.f;
    if (!ZERO_U) {
        um = at4(U, x, yr, z0 - 2);
        uc = at4(U, x, yr, z0 - 1);
        if (lt || rt) {
            hm = at1(U, xh, yr, z0 - 2);
            hc = at1(U, xh, yr, z0 - 1);
        }
    }
    bn = at4(Bp, x, yr, z0 - 1);
    hb = (lt || rt) ? at1(Bp, xh, yr, z0 - 1) : 0.f;
    (void)rhm;
    (void)rhc;
    for (int zz = z0 - 1; zz <= z1; ++zz) {
        const int buf = zz & 1;
        const float4 bc = bn;
        const float hbc = hb;
        bn = at4(Bp, x, yr, zz + 1);
        if (lt || rt) hb = at1(Bp, xh, yr, zz + 1);
        const bool zin = zz >= 0 && zz < n;
        float4 r;
        float rh = 0.f;
        if (!ZERO_U) {
            un = at4(U, x, yr, zz + 1);
            if (lt || rt) hn = at1(U, xh, yr, zz + 1);
            float(*s)[kP3W] = su[buf];
            st4g(&s[ty + 1][4 + 4 * tx], uc);
            if (lt) st4g(&s[ty + 1][0], at4(U, x0 - 4, yr, zz));
            if (rt) st4g(&s[ty + 1][kP3Cols + 4], at4(U, x0 + kP3Cols, yr, zz));
            if (ty == 0 || ty == kP3Rows - 1) {  // the two extra rows y0 - 2 and y0 + 15
                const int er = ty == 0 ? 0 : kP3Rows + 1, ey = ty == 0 ? y0 - 2 : y0 + kP3Rows - 1;
                st4g(&s[er][4 + 4 * tx], at4(U, x, ey, zz));
                if (lt) st4g(&s[er][0], at4(U, x0 - 4, ey, zz));
                if (rt) st4g(&s[er][kP3Cols + 4], at4(U, x0 + kP3Cols, ey, zz));
            }
            __syncthreads();
            const float *row = &s[ty + 1][4 + 4 * tx], *rs = &s[ty][4 + 4 * tx], *rn = &s[ty + 2][4 + 4 * tx];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float ss = radd(radd(radd(row[k - 1], row[k + 1]), radd(rs[k], rn[k])), radd(e4(um, k), e4(un, k)));
                e4(r, k) = radd(rfma(-6.f, e4(uc, k), ce4(bc, k)), ss);
            }
            if (lt || rt) {
                const int c = lt ? 3 : kP3Cols + 4;
                const float ss = radd(radd(radd(s[ty + 1][c - 1], s[ty + 1][c + 1]), radd(s[ty][c], s[ty + 2][c])),
                                      radd(hm, hn));
                rh = radd(rfma(-6.f, hc, hbc), ss);
            }
        } else {
            r = bc;
            rh = hbc;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (!(zin && yin && x + k < n)) e4(r, k) = 0.f;
        if ((lt || rt) && !(zin && yin && xh >= 0 && xh < n)) rh = 0.f;
        float(*q)[kP3W] = sr[(zz + 3) % 3];
        st4g(&q[ty][4 + 4 * tx], r);
        if (lt) q[ty][3] = rh;
        if (rt) q[ty][kP3Cols + 4] = rh;
        __syncthreads();
        if (zz - 1 >= z0 && own_row) {
            float(*p)[kP3W] = sr[(zz + 2) % 3];  // plane zz - 1
            const float *row = &p[ty][4 + 4 * tx], *rs = &p[ty - 1][4 + 4 * tx], *rn = &p[ty + 1][4 + 4 * tx];
            float4 o;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float E = radd(radd(radd(row[k - 1], row[k + 1]), radd(rs[k], rn[k])), radd(e4(rm, k), e4(r, k)));
                const float base = ZERO_U ? rmul(c0, e4(rc, k)) : rfma(c0, e4(rc, k), e4(um, k));
                e4(o, k) = rfma(c1, E, base);
            }
            if (ACC64) {
                double *ur = u64 + ((long)(zz - 1) * n + yr) * n + x;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (x + k < n) ur[k] = __dadd_rn(ur[k], (double)e4(o, k));
            } else {
                float *dst = out + g.off + (long)(zz - 1) * S + (long)yr * P + x;
                if (x + 3 < n) {
                    st4g(dst, o);
                } else {
                    for (int k = 0; k < 4; ++k)
                        if (x + k < n) dst[k] = e4(o, k);
                }
            }
        }
        rm = rc;
        rc = r;
        if (!ZERO_U) {
            um = uc;
            uc = un;
            hm = hc;
            hc = hn;
        }
    }
}

// ---------------------------------------------------------------------------
// Residual + full weighting (formula as resrestrict3d_kernel): 16 x 16 coarse
// columns per block, fine residual patch 33 x 33 per fine plane from a ring of
// three u planes (patch rows loaded as aligned float4 from column 2 ic0 - 4).
// ---------------------------------------------------------------------------
constexpr int kQ = 16;                  // coarse tile edge
constexpr int kQF = 2 * kQ + 1;         // 33 fine residual points per row
constexpr int kQU = 40;                 // u patch row width (10 float4, columns 2 ic0 - 4 ..)
constexpr int kQR = kQF + 2;            // 35 u patch rows
constexpr int kQThreads = kQ * kQ;

__global__ void __launch_bounds__(kQThreads)
resrestrict3d_pl_kernel(const float *__restrict__ u, const float *__restrict__ b, float *__restrict__ bc, Pitch3 g,
                        Pitch3 gc, int Zc)
{
    __shared__ __align__(16) float su[3][kQR][kQU];
    __shared__ float sr[kQF][kQF + 1];
    __shared__ float st1[kQF][kQ + 1];
    const int n = g.n, nc = gc.n, t = threadIdx.x;
    const int tic = t % kQ, tjc = t / kQ;
    const int ic0 = blockIdx.x * kQ, jc0 = blockIdx.y * kQ;
    const int ic = ic0 + tic, jc = jc0 + tjc;
    const int fx0 = 2 * ic0, fy0 = 2 * jc0;
    const int kc0 = blockIdx.z * Zc, kc1 = min(kc0 + Zc, nc);
    const int f0 = 2 * kc0, f1 = 2 * kc1;
    const float *U = u + g.off, *Bp = b + g.off;
    const long P = g.pitch, S = g.plane;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // u patch: rows fy0 - 1 .. fy0 + 33, columns fx0 - 4 .. fx0 + 35
    auto load_plane = [&](int slot, int fz) {
        for (int q = t; q < kQR * (kQU / 4); q += kQThreads) {
            const int r = q / (kQU / 4), c4 = q % (kQU / 4);
            const int y = fy0 - 1 + r;
            float4 v = z4;
            if (y <= n && fz >= -1 && fz <= n) v = ld4g(U + fz * S + y * P + fx0 - 4 + 4 * c4);
            st4g(&su[slot][r][4 * c4], v);
        }
    };
    load_plane((f0 - 1 + 3) % 3, f0 - 1);
    load_plane(f0 % 3, f0);
    float t2a = 0.f, t2b = 0.f;
    for (int f = f0; f <= f1; ++f) {
        load_plane((f + 1) % 3, f + 1);
        __syncthreads();
        const int sm = (f + 2) % 3, sc = f % 3, sp = (f + 1) % 3;
        for (int q = t; q < kQF * kQF; q += kQThreads) {
            const int i = q % kQF, j = q / kQF;
            const int x = fx0 + i, y = fy0 + j;
            float r = 0.f;
            if (x < n && y < n) {
                const int cx = i + 4, ry = j + 1;  // patch coordinates
                const float bb = Bp[(long)f * S + (long)y * P + x];
                const float s = radd(radd(radd(su[sc][ry][cx - 1], su[sc][ry][cx + 1]),
                                          radd(su[sc][ry - 1][cx], su[sc][ry + 1][cx])),
                                     radd(su[sm][ry][cx], su[sp][ry][cx]));
                r = radd(rfma(-6.f, su[sc][ry][cx], bb), s);
            }
            sr[j][i] = r;
        }
        __syncthreads();
        for (int q = t; q < kQF * kQ; q += kQThreads) {
            const int k = q % kQ, j = q / kQ;
            st1[j][k] = rfma(2.f, sr[j][2 * k + 1], radd(sr[j][2 * k], sr[j][2 * k + 2]));
        }
        __syncthreads();
        const float t2 = rfma(2.f, st1[2 * tjc + 1][tic], radd(st1[2 * tjc][tic], st1[2 * tjc + 2][tic]));
        if (f >= f0 + 2 && (f & 1) == 0 && ic < nc && jc < nc) {
            const int kc = f / 2 - 1;
            bc[gc.off + (long)kc * gc.plane + (long)jc * gc.pitch + ic] = scale2<-4>(rfma(2.f, t2b, radd(t2a, t2)));
        }
        t2a = t2b;
        t2b = t2;
        __syncthreads();  // the ring slot of plane f - 1 is reloaded next
    }
}

// ---------------------------------------------------------------------------
// Trilinear interpolation + correction (formula as prolong3d_kernel): thread
// per 4 fine x-columns of one fine row, marching over coarse planes.
// ---------------------------------------------------------------------------
constexpr int kR3X = 32, kR3Y = 8;

__global__ void __launch_bounds__(kR3X * kR3Y)
prolong3d_pl_kernel(const float *__restrict__ e, float *__restrict__ u, Pitch3 g, Pitch3 gc, int Zc)
{
    const int n = g.n, nc = gc.n;
    const int qx = blockIdx.x * kR3X + threadIdx.x % kR3X;  // fine columns 4 qx .. 4 qx + 3
    const int fy = blockIdx.y * kR3Y + threadIdx.x / kR3X;
    const int fx = 4 * qx;
    if (fx >= n || fy >= n) return;
    const int m0 = blockIdx.z * Zc, m1 = min(m0 + Zc, nc + 1);
    const float *E = e + gc.off;
    float *Uf = u + g.off;
    // x-pass of coarse row jc, plane kc at the thread's 4 fine columns:
    // 4q -> 0.5 (e[2q-1] + e[2q]), 4q+1 -> e[2q], 4q+2 -> 0.5 (e[2q] + e[2q+1]), 4q+3 -> e[2q+1]
    auto xpass = [&](int jc, int kc, float *v) {
        const float *row = E + (long)kc * gc.plane + (long)jc * gc.pitch;
        const float em = row[2 * qx - 1], a = row[2 * qx], bq = row[2 * qx + 1];
        v[0] = scale2<-1>(radd(em, a));
        v[1] = a;
        v[2] = scale2<-1>(radd(a, bq));
        v[3] = bq;
    };
    auto xypass = [&](int kc, float *v) {
        if (fy & 1) {
            xpass(fy >> 1, kc, v);
        } else {
            float va[4], vb[4];
            const int m = fy >> 1;
            xpass(m - 1, kc, va);
            xpass(m, kc, vb);
            for (int k = 0; k < 4; ++k) v[k] = scale2<-1>(radd(va[k], vb[k]));
        }
    };
    float pv[4], cv[4];
    xypass(m0 - 1, pv);
    for (int m = m0; m < m1; ++m) {
        xypass(m, cv);
        {   // fine plane 2m
            float *p = Uf + (long)(2 * m) * g.plane + (long)fy * g.pitch + fx;
            float4 w = ld4g(p);
            for (int k = 0; k < 4; ++k) e4(w, k) = radd(e4(w, k), scale2<-1>(radd(pv[k], cv[k])));
            if (fx + 3 < n) st4g(p, w);
            else for (int k = 0; k < 4; ++k) if (fx + k < n) p[k] = e4(w, k);
        }
        if (m < nc) {  // fine plane 2m+1
            float *p = Uf + (long)(2 * m + 1) * g.plane + (long)fy * g.pitch + fx;
            float4 w = ld4g(p);
            for (int k = 0; k < 4; ++k) e4(w, k) = radd(e4(w, k), cv[k]);
            if (fx + 3 < n) st4g(p, w);
            else for (int k = 0; k < 4; ++k) if (fx + k < n) p[k] = e4(w, k);
        }
        for (int k = 0; k < 4; ++k) pv[k] = cv[k];
    }
}

// compact <-> padded
__global__ void pack3d_kernel(const float *__restrict__ in, float *__restrict__ out, Pitch3 g, bool to_padded)
{
    const int n = g.n;
    const long np = (long)n * n * n;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < np; i += (long)gridDim.x * blockDim.x) {
        const long x = i % n, y = (i / n) % n, z = i / ((long)n * n);
        const long p = g.off + z * g.plane + y * g.pitch + x;
        if (to_padded) out[p] = in[i];
        else out[i] = in[p];
    }
}

// u (compact FP64) += e (padded FP32)
__global__ void add_pl3d_kernel(double *__restrict__ u, const float *__restrict__ e, Pitch3 g)
{
    const int n = g.n;
    for (long r = blockIdx.y; r < (long)n * n; r += gridDim.y) {  // row r = z * n + y
        const long z = r / n, y = r % n;
        double *ur = u + r * n;
        const float *er = e + g.off + z * g.plane + y * g.pitch;
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
            ur[x] = __dadd_rn(ur[x], (double)er[x]);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
Pitch3 pitch3(int n)
{
    Pitch3 g;
    g.n = n;
    const int strips = (n + kP3Cols - 1) / kP3Cols;
    // the restriction reads patch rows up to column 2 ic0 + 35 <= n + 32
    g.pitch = ((std::max(strips * kP3Cols + 8, n + 44) + 31) / 32) * 32;
    g.plane = (long)(n + 2) * g.pitch;
    g.off = g.plane + g.pitch + 4;
    return g;
}

size_t pitch3_floats(int n)
{
    const Pitch3 g = pitch3(n);
    return (size_t)(n + 2) * g.plane + 64;
}

cudaError_t launch_sweep3d_pl(const float *u, const float *b, float *out, double *u64, int n, const double *c,
                              cudaStream_t s)
{
    const Pitch3 g = pitch3(n);
    const int bx = (n + kP3Cols - 1) / kP3Cols, by = (n + kP3TY - 1) / kP3TY;
    const int Z = chunk_rows(bx * by, n, 3 * num_sms(), 4, 128);
    const dim3 grid(bx, by, (n + Z - 1) / Z);
    const float c0 = (float)c[0], c1 = (float)c[1];
    if (u64)
        sweep3d_pl_kernel<false, true><<<grid, kP3Threads, 0, s>>>(u, b, nullptr, u64, g, Z, c0, c1);
    else if (u)
        sweep3d_pl_kernel<false, false><<<grid, kP3Threads, 0, s>>>(u, b, out, nullptr, g, Z, c0, c1);
    else
        sweep3d_pl_kernel<true, false><<<grid, kP3Threads, 0, s>>>(u, b, out, nullptr, g, Z, c0, c1);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_resrestrict3d_pl(const float *u, const float *b, float *bc, int n, cudaStream_t s)
{
    const Pitch3 g = pitch3(n), gc = pitch3((n - 1) / 2);
    const int nc = gc.n;
    const int bxy = (nc + kQ - 1) / kQ;
    const int Zc = chunk_rows(bxy * bxy, nc, 8 * num_sms(), 2, 32);
    resrestrict3d_pl_kernel<<<dim3(bxy, bxy, (nc + Zc - 1) / Zc), kQThreads, 0, s>>>(u, b, bc, g, gc, Zc);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_prolong3d_pl(const float *e, float *u, int n, cudaStream_t s)
{
    const Pitch3 g = pitch3(n), gc = pitch3((n - 1) / 2);
    const int nc = gc.n;
    const int qxs = (n + 3) / 4;
    const int bx = (qxs + kR3X - 1) / kR3X, by = (n + kR3Y - 1) / kR3Y;
    const int Zc = chunk_rows(bx * by, nc + 1, 8 * num_sms(), 2, 32);
    prolong3d_pl_kernel<<<dim3(bx, by, (nc + 1 + Zc - 1) / Zc), kR3X * kR3Y, 0, s>>>(e, u, g, gc, Zc);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_pack3d(const float *in, float *out, int n, bool to_padded, cudaStream_t s)
{
    const long np = (long)n * n * n;
    const int blocks = (int)std::min<long>((np + 255) / 256, 8L * num_sms());
    pack3d_kernel<<<blocks, 256, 0, s>>>(in, out, pitch3(n), to_padded);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_add_pl3d(double *u, const float *e, int n, cudaStream_t s)
{
    const int bx = (n + 255) / 256;
    const int by = (int)std::min<long>((long)n * n, std::max<long>(1, (long)num_sms() * 16 / bx));
    add_pl3d_kernel<<<dim3(bx, by), 256, 0, s>>>(u, e, pitch3(n));
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace mg
