// mg_noalloc.cu -- one SPAI sweep with the squared residual norm of its input,
// for callers that cannot allocate device memory.
//
// The allocating form (mg_op_sweep with a norm output) gets its per-block
// partial sums from cudaMalloc on every call. Some callers cannot do that:
// code that lives under a framework's own memory pool (a caching allocator
// that owns the device heap and must not be bypassed), services that run
// with a fixed device-memory budget decided at start-up, and latency-bound
// loops where cudaMalloc/cudaFree would synchronise the whole device. This
// entry point takes its scratch from a fixed array in device memory instead
// and allocates nothing.
//
// The scratch is a file-scope __device__ array of kMaxPartials doubles
// (256 KiB). Every GPU that loads the library holds it until the process
// exits. Host code never uses the array's name as an address: the device
// address is looked up once per device with cudaGetSymbolAddress.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mg.h"
#include "mg_ctx.h"
#include "mg_internal.h"

namespace {

// one partial sum per block of the sweep: enough for 2D grids up to
// n = 16383 and 3D grids up to n = 1023 points per axis on a 152-SM GB300
constexpr int kMaxPartials = 32768;

static __device__ __align__(256) double g_sweep_partials[kMaxPartials];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on
// the first call for that device, with the device current).
mg_status scratch_on_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return mg::cuda_fail(e);
    if (dev < 0 || dev >= kMaxDevices) return mg::cuda_fail(cudaErrorInvalidDevice);
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sweep_partials);
        if (e != cudaSuccess) return mg::cuda_fail(e);
        if (!p) return mg::cuda_fail(cudaErrorInvalidSymbol);
        g_addr[dev] = (double *)p;
    }
    *out = g_addr[dev];
    return MG_OK;
}

int partials_needed(int d, int n, int elem_bytes)
{
    if (d == 2) {
        const mg::Grid2 g = mg::sweep2d_grid(n);
        return g.bx * g.by;
    }
    return mg::sweep3d_plan(n, elem_bytes).blocks;
}

template <typename T>
mg_status run(int d, int n, const double *c, const void *u, const void *bh, int unscaled, void *u_out,
              double *norm2_dev, cudaStream_t s, double *partials, int np)
{
    cudaError_t e = d == 2 ? mg::launch_sweep2d<T>((const T *)u, (const T *)bh, unscaled != 0, (T *)u_out, n, c,
                                                   partials, s)
                           : mg::launch_sweep3d<T>((const T *)u, (const T *)bh, unscaled != 0, (T *)u_out, n, c,
                                                   partials, s);
    if (e == cudaSuccess) e = mg::launch_sum_partials(partials, np, norm2_dev, s);
    return e == cudaSuccess ? MG_OK : mg::cuda_fail(e);
}

}  // namespace

extern "C" mg_status mg_op_sweep_norm_noalloc(int d, int n, mg_prec prec, const double *spai_coeffs, int ncoeffs,
                                              const void *u, const void *bh, int b_unscaled, void *u_out,
                                              double *rnorm2_dev_out, void *stream)
{
    // every argument, including the size limit, is checked before any CUDA call
    if ((d != 2 && d != 3) || n < 3 || !(n & 1) || ((n + 1) & n) != 0 || !spai_coeffs || ncoeffs < 1 ||
        ncoeffs > (d == 2 ? 3 : 2) || !bh || !u_out || !rnorm2_dev_out || (prec != MG_FP64 && prec != MG_FP32_IR))
        return MG_EINVAL;
    if ((d == 2 && n > 16383) || (d == 3 && n > 1023)) return MG_EINVAL;
    const int np = partials_needed(d, n, prec == MG_FP64 ? 8 : 4);
    if (np > kMaxPartials) return MG_EINVAL;
    double c[4] = {0, 0, 0, 0};
    for (int j = 0; j < ncoeffs; ++j) c[j] = spai_coeffs[j];
    double *partials = nullptr;
    mg_status st = scratch_on_current_device(&partials);
    if (st != MG_OK) return st;
    // every block overwrites its own partial, so nothing needs clearing
    return prec == MG_FP64 ? run<double>(d, n, c, u, bh, b_unscaled, u_out, rnorm2_dev_out, (cudaStream_t)stream,
                                         partials, np)
                           : run<float>(d, n, c, u, bh, b_unscaled, u_out, rnorm2_dev_out, (cudaStream_t)stream,
                                        partials, np);
}
