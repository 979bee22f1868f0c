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

// x strips of the sweep (mg_tma3d.cu): 128 columns each; rows are padded to
// whole strips plus the 4-column margins its tiles read on both sides
constexpr int kP3Cols = 128;

__device__ __forceinline__ float4 ld4g(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4g(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float &e4(float4 &v, int k) { return (&v.x)[k]; }

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
            ur[x] = __dadd_rn(ur[x], widen(er[x]));
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

cudaError_t launch_prolong3d_pl(const float *e, float *u, int n, cudaStream_t s)
{
    const Pitch3 g = pitch3(n), gc = pitch3((n - 1) / 2);
    const int nc = gc.n;
    const int qxs = (n + 3) / 4;
    const int bx = (qxs + kR3X - 1) / kR3X, by = (n + kR3Y - 1) / kR3Y;
    const int Zc = chunk_rows(bx * by, nc + 1, 8 * num_sms(), 1, 32);
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
