// mg_host.cu -- solver contexts, cycle scheduling, CUDA-graph capture and the
// C ABI declared in include/mg.h (He, Liu, Wang, arXiv:2206.05543, Sec. 4).
//
// A context owns the level hierarchy N, N/2, ..., 4 of one problem. The
// cycle is recorded once into CUDA graphs on a private stream:
//   pre  - the first smoothing sweep on the finest level, which also yields
//          ||b - A u_k|| of its input (or the FP64 residual in refinement
//          mode), the fixed-order reduction and the copy of the norm to
//          pinned host memory;
//   rest - the remainder of the cycle: restriction, coarse levels (the last
//          ones inside one block, see mg_tail.cu), interpolation and the
//          post-smoothing sweeps;
//   meas - plain cycles only: the norm of ||b - A u_k|| alone, used for the
//          test that is predicted to end the solve (see mg_solve).
// mg_solve replays rest + pre once per cycle and reads one double back, so
// the stopping test costs one synchronisation per cycle and a converged u is
// never touched again (the pre sweep writes to the ping-pong buffer).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/mg.h"
#include "mg_common.cuh"
#include "mg_internal.h"
#include "mg_ctx.h"

namespace mg {

static std::atomic<unsigned long long> g_launches{0};
static thread_local unsigned long long *g_capture_counter = nullptr;
static thread_local char g_last_error[256] = "";

void count_launch(unsigned long long k)
{
    if (g_capture_counter)
        *g_capture_counter += k;
    else
        g_launches += k;
}

int num_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            sms = v;
        else
            sms = 152;
    }
    return sms;
}

mg_status cuda_fail(cudaError_t e)
{
    snprintf(g_last_error, sizeof g_last_error, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return MG_ECUDA;
}

#define MG_CUDA(call)                                    \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_);     \
    } while (0)

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------
__global__ void sum_partials_kernel(const double *__restrict__ p, int np, double *__restrict__ out)
{
    double v = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) v += p[i];
    block_sum_store<256>(v, out);
}

cudaError_t launch_sum_partials(const double *partials, int np, double *out, cudaStream_t s)
{
    sum_partials_kernel<<<1, 256, 0, s>>>(partials, np, out);
    count_launch(1);
    return cudaGetLastError();
}

// dst = src (src null: dst = 0) over n 4-byte words; 16-byte vectors where
// both pointers allow them
__global__ void __launch_bounds__(256) words_kernel(unsigned *__restrict__ dst, const unsigned *__restrict__ src,
                                                    size_t n, int vec)
{
    const size_t stride = (size_t)gridDim.x * 256;
    size_t i = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (vec) {
        const size_t n4 = n / 4;
        uint4 *d4 = (uint4 *)dst;
        const uint4 *s4 = (const uint4 *)src;
        for (size_t j = i; j < n4; j += stride) d4[j] = src ? s4[j] : make_uint4(0, 0, 0, 0);
        for (size_t j = n4 * 4 + i; j < n; j += stride) dst[j] = src ? src[j] : 0u;
    } else {
        for (size_t j = i; j < n; j += stride) dst[j] = src ? src[j] : 0u;
    }
}

static cudaError_t launch_words(void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    if (bytes % 4 || ((uintptr_t)dst | (uintptr_t)src) % 4) return cudaErrorInvalidValue;
    const size_t n = bytes / 4;
    if (!n) return cudaSuccess;
    const int vec = ((uintptr_t)dst | (uintptr_t)src) % 16 == 0;
    const size_t want = (n / (vec ? 4 : 1) + 255) / 256;
    const int blocks = (int)std::min<size_t>(std::max<size_t>(want, 1), (size_t)8 * num_sms());
    words_kernel<<<blocks, 256, 0, s>>>((unsigned *)dst, (const unsigned *)src, n, vec);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_zero_words(void *p, size_t bytes, cudaStream_t s) { return launch_words(p, nullptr, bytes, s); }

cudaError_t launch_copy_words(void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    return launch_words(dst, src, bytes, s);
}

// The same sum, and the kNormBytes that start at out (the sum and the error
// word after it) stored into mapped pinned host memory as well. The host
// reads them after the stream synchronises (mg_residual_norm). A
// device-to-host copy would do the same but can queue behind a caller's
// large copy on a copy engine.
__global__ void sum_partials_host_kernel(const double *__restrict__ p, int np, double *__restrict__ out,
                                         unsigned long long *__restrict__ host)
{
    double v = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) v += p[i];
    block_sum_store<256>(v, out);  // thread 0 stores out[0]
    if (threadIdx.x == 0) {
        const unsigned long long *o = (const unsigned long long *)out;
        host[0] = o[0];
        host[1] = o[1];
    }
}

// The first refinement residual of a solve from u = 0: rh = h^2 b rounded to
// FP32 once, the value the FP64 residual kernel forms there (fma(-2d, 0, h^2 b)
// plus a zero neighbour sum, which turns -0 into +0), written to the padded
// level-0 layout, with the squared norm of h^2 b: one partial per block.
template <int D>
__global__ void __launch_bounds__(256) refine_rhs_zero_kernel(const double *__restrict__ b, float *__restrict__ rh,
                                                               int n, int hk, long pitch, long plane, long off,
                                                               double *__restrict__ partials)
{
    SqSum acc;
    const long np = D == 2 ? (long)n * n : (long)n * n * n;
    int cnt = 0;
    for (long i = blockIdx.x * 256L + threadIdx.x; i < np; i += (long)gridDim.x * 256L) {
        double r = scale2(b[i], hk);
        if ((__double_as_longlong(r) << 1) == 0) r = 0.0;  // -0 -> +0
        sq_add(acc, r);
        if (++cnt == 32) {
            sq_flush(acc);
            cnt = 0;
        }
        const long x = i % n, yz = i / n;
        rh[D == 2 ? off + yz * pitch + x : off + (yz / n) * plane + (yz % n) * pitch + x] = narrow_rn(r);
    }
    block_sum_store<256>(sq_value(acc), &partials[blockIdx.x]);
}

static cudaError_t launch_sum_partials_host(const mg_ctx *c, int np, cudaStream_t s)
{
    static_assert(kNormBytes == 2 * sizeof(unsigned long long), "sum and error word");
    sum_partials_host_kernel<<<1, 256, 0, s>>>(c->partials, np, c->d_norm2, c->h_norm2_dev);
    count_launch(1);
    return cudaGetLastError();
}

// The squared residual norm of a pre or norm-only graph: also into mapped
// host memory for the host-driven loop of mg_solve (and mg_vcycle's graphs),
// device memory only inside the device-side loop graph, which writes nothing
// to host memory while it runs.
static cudaError_t launch_norm_sum(const mg_ctx *c, int np)
{
    return c->norm_to_host ? launch_sum_partials_host(c, np, c->s)
                           : launch_sum_partials(c->partials, np, c->d_norm2, c->s);
}

// ---------------------------------------------------------------------------
// the cycle loop of a solve on the device: the stop test ||r_k|| <= tol ||r_0||
// of Sec. 4 decided by one-thread kernels that set the condition values of the
// loop graph's conditional nodes, so that a solve synchronises with the host
// once instead of once per cycle. Every decision is the host loop's, in the
// same IEEE double arithmetic (round to nearest, no contraction).
// ---------------------------------------------------------------------------
// ||r||_2 = sqrt(sum rh^2) / h^2 from the summed squares, formed as
// sqrt(s) * N * N
__device__ __forceinline__ double loop_norm(const double *norm2, double nd)
{
    return __dmul_rn(__dmul_rn(__dsqrt_rn(norm2[0]), nd), nd);
}

// whether another cycle runs; MG_ENOCONV once max_cycles cycles ran
__device__ __forceinline__ bool loop_continue(LoopState &s)
{
    if (s.status != MG_OK || s.rk <= __dmul_rn(s.a.tol, s.r0)) return false;
    if (s.k == s.a.max_cycles) {
        s.status = MG_ENOCONV;
        return false;
    }
    return true;
}

// whether the coming cycle ends with the norm-only graph: the last
// convergence factor, carried one cycle forward, puts its residual under the
// tolerance
__device__ __forceinline__ bool loop_guess(const LoopState &s)
{
    return s.guessing && s.k >= 1 && s.rprev > 0.0 &&
           __dmul_rn(s.rk, __ddiv_rn(s.rk, s.rprev)) <= __dmul_rn(s.a.tol, s.r0);
}

// The solve's outcome and the launch count, stored once when the loop ends:
// while the loop runs, nothing is written to host memory (a kernel's writes
// to host memory must land before the next kernel starts, and they can wait
// behind a large transfer a caller runs meanwhile on the same link).
__device__ __forceinline__ void loop_finish(const LoopState &s, unsigned long long *launched)
{
    mg_solve_info *info = s.a.info;
    info->r0 = s.r0;
    info->rk = s.rk;
    info->cycles = s.k;
    info->status = s.status;
    *launched = s.launched;
}

__device__ __forceinline__ bool wait_expired(const int *err) { return *(volatile const int *)err != 0; }

// a solve's arguments, by value, stored for its loop graph
__global__ void loop_args_kernel(LoopState *st, LoopArgs a) { st->a = a; }

// the first graph of the solve: the from-zero pre graph or the pre graph
__global__ void loop_head_kernel(const LoopState *st, cudaGraphConditionalHandle from_zero)
{
    cudaGraphSetConditional(from_zero, st->a.zero_start ? 1u : 0u);
}

// after the first pre graph: r_0, the history's first entry, the loop's
// state; zero_u is set when a solve from u = 0 runs no cycle (u would stay
// unwritten otherwise). n_pre0, n_pre: kernels of the two first graphs.
__global__ void loop_init_kernel(LoopState *st, const double *norm2, const int *err, double nd, int guessing,
                                 unsigned n_pre0, unsigned n_pre, cudaGraphConditionalHandle loop,
                                 cudaGraphConditionalHandle zero_u, unsigned long long *launched)
{
    LoopState s = *st;
    s.r0 = s.rk = loop_norm(norm2, nd);
    s.rprev = 0.0;
    s.k = s.guess = s.rerun = 0;
    s.guessing = guessing;
    s.status = wait_expired(err) ? MG_ETIMEOUT : (isfinite(s.r0) ? MG_OK : MG_ENAN);
    if (s.a.hist) s.a.hist[0] = s.r0;
    const bool more = loop_continue(s);
    const bool zero = s.a.zero_start && !more;
    // the head kernel, the first graph, this kernel, the zeroing of u
    s.launched += 2 + (s.a.zero_start ? n_pre0 : n_pre) + (zero ? 1 : 0);
    *st = s;
    if (!more) loop_finish(s, launched);
    cudaGraphSetConditional(zero_u, zero ? 1u : 0u);
    cudaGraphSetConditional(loop, more ? 1u : 0u);
}

// The end of a cycle: the count, the history, NaN, a wrong guess (the pre
// graph runs at the start of the next cycle and guessing stops for this
// solve), the stop test, and the choice of the next cycle's last graph.
// n_rest, n_pre, n_meas: kernels of those graphs; has_meas: the body chooses
// between the pre and norm-only graphs (else it always runs pre).
__global__ void loop_after_kernel(LoopState *st, const double *norm2, const int *err, double nd, int has_meas,
                                  unsigned n_rest, unsigned n_pre, unsigned n_meas, cudaGraphConditionalHandle loop,
                                  cudaGraphConditionalHandle rerun_pre, cudaGraphConditionalHandle use_meas,
                                  unsigned long long *launched)
{
    LoopState s = *st;
    s.launched += 1 + n_rest + (s.rerun ? n_pre : 0) + (s.guess ? n_meas : n_pre);
    s.rerun = 0;
    if (wait_expired(err)) {
        s.status = MG_ETIMEOUT;
    } else {
        ++s.k;
        s.rprev = s.rk;
        s.rk = loop_norm(norm2, nd);
        if (s.a.hist) s.a.hist[s.k] = s.rk;
        if (!isfinite(s.rk)) s.status = MG_ENAN;
        s.rerun = s.status == MG_OK && s.guess && !(s.rk <= __dmul_rn(s.a.tol, s.r0)) && s.k < s.a.max_cycles;
        if (s.rerun) s.guessing = 0;
    }
    const bool more = loop_continue(s);
    s.guess = more && loop_guess(s);
    *st = s;
    if (!more) loop_finish(s, launched);
    if (has_meas) {
        cudaGraphSetConditional(rerun_pre, s.rerun ? 1u : 0u);
        cudaGraphSetConditional(use_meas, s.guess ? 1u : 0u);
    }
    cudaGraphSetConditional(loop, more ? 1u : 0u);
}

// refine_rhs_zero_kernel over the context's level 0 (padded FP32 rhs BH[0]);
// nb: the blocks launched (partials to sum), at most the context's partials
static cudaError_t launch_refine_rhs_zero(const mg_ctx *c, const double *b, int &nb)
{
    const int n = c->n[0];
    nb = std::max(1, std::min(c->npartials, 8 * num_sms()));
    const int hk = h2_exponent(n);
    if (c->d == 2) {
        const Pitch2 g = pitch2(n);
        refine_rhs_zero_kernel<2><<<nb, 256, 0, c->s>>>(b, (float *)c->BH[0], n, hk, g.pitch, 0, g.off, c->partials);
    } else {
        const Pitch3 g = pitch3(n);
        refine_rhs_zero_kernel<3><<<nb, 256, 0, c->s>>>(b, (float *)c->BH[0], n, hk, g.pitch, g.plane, g.off,
                                                         c->partials);
    }
    count_launch(1);
    return cudaGetLastError();
}

template <typename T>
__global__ void add_to_f64_kernel(double *__restrict__ u, const T *__restrict__ e, size_t np)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < np; i += (size_t)gridDim.x * blockDim.x)
        u[i] = __dadd_rn(u[i], to_out<double>(e[i]));
}

template <typename T>
cudaError_t launch_add_to_f64(double *u, const T *e, size_t np, cudaStream_t s)
{
    const int blocks = (int)std::min<size_t>((np + 255) / 256, (size_t)num_sms() * 8);
    add_to_f64_kernel<T><<<blocks, 256, 0, s>>>(u, e, np);
    count_launch(1);
    return cudaGetLastError();
}

// u (compact FP64) += e (padded FP32 layout); block y = row, x-threads = columns
__global__ void add_pl2d_kernel(double *__restrict__ u, const float *__restrict__ e, Pitch2 g)
{
    const int n = g.n;
    for (int y = blockIdx.y; y < n; y += gridDim.y) {
        double *ur = u + (long)y * n;
        const float *er = e + g.off + (long)y * g.pitch;
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
            ur[x] = __dadd_rn(ur[x], widen(er[x]));
    }
}

cudaError_t launch_add_pl2d(double *u, const float *e, int n, cudaStream_t s)
{
    const int bx = (n + 255) / 256;
    const int by = (int)std::min<long>(n, std::max<long>(1, (long)num_sms() * 16 / bx));
    add_pl2d_kernel<<<dim3(bx, by), 256, 0, s>>>(u, e, pitch2(n));
    count_launch(1);
    return cudaGetLastError();
}

template <typename InT, typename T>
__global__ void scale_copy_kernel(const InT *__restrict__ b, T *__restrict__ bh, size_t np, InT h2)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < np; i += (size_t)gridDim.x * blockDim.x)
        bh[i] = (T)rmul(h2, b[i]);  // exact: h2 is a power of two
}

template <typename InT, typename T>
cudaError_t launch_scale_copy(const InT *b, T *bh, size_t np, double h2, cudaStream_t s)
{
    const int blocks = (int)std::min<size_t>((np + 255) / 256, (size_t)num_sms() * 8);
    scale_copy_kernel<InT, T><<<blocks, 256, 0, s>>>(b, bh, np, (InT)h2);
    count_launch(1);
    return cudaGetLastError();
}
template cudaError_t launch_scale_copy<double, double>(const double *, double *, size_t, double, cudaStream_t);
template cudaError_t launch_scale_copy<float, float>(const float *, float *, size_t, double, cudaStream_t);

// ---------------------------------------------------------------------------
// dispatch on the dimension
// ---------------------------------------------------------------------------
template <typename T>
static cudaError_t op_sweep(int d, const T *u, const T *b, bool unscaled, T *out, int n, const double *c,
                            double *partials, cudaStream_t s)
{
    return d == 2 ? launch_sweep2d<T>(u, b, unscaled, out, n, c, partials, s)
                  : launch_sweep3d<T>(u, b, unscaled, out, n, c, partials, s);
}
template <typename T>
static cudaError_t op_resrestrict(int d, const T *u, const T *b, bool unscaled, T *bc, int n, cudaStream_t s)
{
    return d == 2 ? launch_resrestrict2d<T>(u, b, unscaled, bc, n, s)
                  : launch_resrestrict3d<T>(u, b, unscaled, bc, n, s);
}
template <typename T>
static cudaError_t op_prolong(int d, const T *e, T *u, int n, cudaStream_t s)
{
    return d == 2 ? launch_prolong2d<T>(e, u, n, s) : launch_prolong3d<T>(e, u, n, s);
}
template <typename InT, typename OutT>
static cudaError_t op_residual(int d, const InT *u, const InT *b, bool unscaled, OutT *rh, int n,
                               double *partials, cudaStream_t s)
{
    return d == 2 ? launch_residual2d<InT, OutT>(u, b, unscaled, rh, n, partials, s)
                  : launch_residual3d<InT, OutT>(u, b, unscaled, rh, n, partials, s);
}
static int sweep_partials(int d, int n, int elem_bytes)
{
    if (d == 2) {
        const Grid2 g = sweep2d_grid(n);
        return g.bx * g.by;
    }
    return sweep3d_plan(n, elem_bytes).blocks;
}
static int residual_partials(int d, int n)
{
    if (d == 2) {
        const Grid2 g = sweep2d_grid(n);
        return g.bx * g.by;
    }
    const Grid3 g = residual3d_grid(n);
    return g.bx * g.by * g.bz;
}

static size_t npoints(int d, int n) { return d == 2 ? (size_t)n * n : (size_t)n * n * n; }

// 3D weights with a non-zero edge or corner weight: the 27-point M
static bool wide_weights(int d, const double *w, int nw)
{
    if (d != 3) return false;
    for (int j = 2; j < nw; ++j)
        if (w[j] != 0.0) return true;
    return false;
}

static bool valid_N(int N)
{
    if (N < 4 || N > (1 << 20)) return false;
    return (N & (N - 1)) == 0;
}

mg_status capture_graph(mg_ctx *c, cudaGraphExec_t *out, unsigned long long *nodes,
                        const std::function<cudaError_t()> &body)
{
    cudaGraph_t graph = nullptr;
    unsigned long long counter = 0;
    cudaError_t e = cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e);
    g_capture_counter = &counter;
    e = body();
    g_capture_counter = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->s, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(e != cudaSuccess ? e : e2);
    }
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e);
    *nodes = counter;
    return MG_OK;
}

// Capture the work issued by body() on the context's stream into graph g,
// after the nodes in deps; on return deps holds the nodes the work ends with.
cudaError_t capture_into(mg_ctx *c, cudaGraph_t g, std::vector<cudaGraphNode_t> &deps,
                         const std::function<cudaError_t()> &body, unsigned long long *nodes)
{
    cudaError_t e = cudaStreamBeginCaptureToGraph(c->s, g, deps.empty() ? nullptr : deps.data(), nullptr,
                                                  deps.size(), cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    unsigned long long counter = 0;
    g_capture_counter = &counter;
    e = body();
    g_capture_counter = nullptr;
    if (nodes) *nodes = counter;
    if (e == cudaSuccess) {
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *tail = nullptr;
        size_t ntail = 0;
        e = cudaStreamGetCaptureInfo(c->s, &cs, nullptr, nullptr, &tail, nullptr, &ntail);
        if (e == cudaSuccess) deps.assign(tail, tail + ntail);
    }
    cudaGraph_t out = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(c->s, &out);
    return e != cudaSuccess ? e : e2;
}

// Add a conditional node of the given type after deps (then deps = {node});
// bodies[0 .. size-1] receive its body graphs.
cudaError_t add_conditional(cudaGraph_t g, std::vector<cudaGraphNode_t> &deps, cudaGraphConditionalHandle h,
                            cudaGraphConditionalNodeType type, unsigned size, cudaGraph_t *bodies)
{
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = size;
    cudaGraphNode_t node = nullptr;
    const cudaError_t e = cudaGraphAddNode(&node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &p);
    if (e != cudaSuccess) return e;
    for (unsigned i = 0; i < size; ++i) bodies[i] = p.conditional.phGraph_out[i];
    deps.assign(1, node);
    return cudaSuccess;
}

}  // namespace mg

using namespace mg;

// Contexts whose device-side loops count their kernels in mapped memory;
// mg_kernel_launch_count adds their counts, and a destroyed context's count
// moves into g_launches.
static std::mutex g_reg_mu;
static std::vector<mg_ctx *> g_reg;

static void register_ctx(mg_ctx *c)
{
    std::lock_guard<std::mutex> lock(g_reg_mu);
    g_reg.push_back(c);
}

static void unregister_ctx(mg_ctx *c)
{
    std::lock_guard<std::mutex> lock(g_reg_mu);
    for (size_t i = 0; i < g_reg.size(); ++i)
        if (g_reg[i] == c) {
            g_reg.erase(g_reg.begin() + (long)i);
            if (c->h_launched) g_launches += *(volatile unsigned long long *)c->h_launched;
            return;
        }
}

static unsigned long long registered_launches()
{
    std::lock_guard<std::mutex> lock(g_reg_mu);
    unsigned long long n = 0;
    for (mg_ctx *c : g_reg) n += *(volatile unsigned long long *)c->h_launched;
    return n;
}

// (an executable graph still running when destroyed is freed when it ends)
static void destroy_set(GraphPair &g)
{
    for (cudaGraphExec_t x : {g.pre, g.rest, g.meas, g.pre0, g.loop})
        if (x) cudaGraphExecDestroy(x);
    g = GraphPair{};
}

static void free_graphs(mg_ctx *c)
{
    destroy_set(c->g);
    for (GraphPair &g : c->other) destroy_set(g);
    c->other.clear();
    if (c->adj && c->adj->graph) {  // the adjoint's graph holds the weights too
        cudaGraphExecDestroy(c->adj->graph);
        c->adj->graph = nullptr;
    }
}

static void destroy_ctx(mg_ctx *c)
{
    if (!c) return;
    free_batch(c);
    free_adjoint(c);
    free_graphs(c);
    for (void *p : c->owned) cudaFree(p);
    unregister_ctx(c);
    if (c->h_norm2) cudaFreeHost(c->h_norm2);
    if (c->h_launched) cudaFreeHost(c->h_launched);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->s) cudaStreamDestroy(c->s);
    delete c;
}

static mg_status dalloc(mg_ctx *c, void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return MG_ENOMEM;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    c->owned.push_back(*p);
    return MG_OK;
}

// ---------------------------------------------------------------------------
// cycle recording
// ---------------------------------------------------------------------------
namespace {

// bytes of one buffer of level l in the context's layout
size_t level_bytes(const mg_ctx *c, int l)
{
    const int n = c->n[l];
    if (c->pl) return (c->d == 2 ? pitch2_floats(n) : pitch3_floats(n)) * sizeof(float);
    return npoints(c->d, n) * c->esize;
}

template <typename T>
struct Recorder {
    mg_ctx *c;
    const T *b0;       // finest-level right-hand side (unscaled in FP64 mode)
    bool b0_unscaled;
    T *A0;             // finest-level primary buffer
    double *acc64 = nullptr;    // refinement: FP64 solution the last sweep adds into
    bool fused_update = false;  // set when that addition was recorded

    T *A(int l) { return l == 0 ? A0 : (T *)c->A[l]; }
    bool pl() const { return c->pl; }
    cudaError_t sweep(const T *u, const T *b, bool unsc, T *out, int n)
    {
        if (pl() && c->d == 2)
            return launch_sweep2d_pl((const float *)u, (const float *)b, (float *)out, n, c->c, nullptr, c->s);
        if (pl()) return launch_sweep3d_tma((const float *)u, (const float *)b, (float *)out, n, c->c, c->d_err, c->s);
        return op_sweep<T>(c->d, u, b, unsc, out, n, c->c, nullptr, c->s);
    }
    cudaError_t resrestrict(const T *u, const T *b, bool unsc, T *bc, int n)
    {
        if (pl() && c->d == 2) return launch_resrestrict2d_pl((const float *)u, (const float *)b, (float *)bc, n, c->s);
        if (pl()) return launch_resrestrict3d_tma((const float *)u, (const float *)b, (float *)bc, n, c->d_err, c->s);
        return op_resrestrict<T>(c->d, u, b, unsc, bc, n, c->s);
    }
    cudaError_t prolong(const T *e, T *u, int n)
    {
        if (pl() && c->d == 2) return launch_prolong2d_pl((const float *)e, (float *)u, n, c->s);
        if (pl()) return launch_prolong3d_pl((const float *)e, (float *)u, n, c->s);
        return op_prolong<T>(c->d, e, u, n, c->s);
    }
    size_t bytes(int l) const { return level_bytes(c, l); }
    T *B(int l) { return (T *)c->B[l]; }
    const T *BH(int l) { return l == 0 ? b0 : (const T *)c->BH[l]; }
    bool unsc(int l) { return l == 0 && b0_unscaled; }

    // ops of the tail kernel for a visit of level l (host recursion, the same
    // order as the reference cycle)
    void tail_ops(TailArgs &a, int l, bool &ok)
    {
        auto push = [&](int kind, int lev) {
            if (a.nops >= kMaxTailOps) {
                ok = false;
                return;
            }
            a.ops[a.nops].kind = (short)kind;
            a.ops[a.nops].level = (short)(lev - c->lt);
            ++a.nops;
        };
        if (c->n[l] == 3) {
            push(TAIL_SOLVE, l);
            return;
        }
        for (int s = 0; s < c->nu1; ++s) push(TAIL_SWEEP, l);
        push(TAIL_RESTRICT, l);
        push(TAIL_ZERO, l + 1);
        for (int g = 0; g < c->gamma; ++g) tail_ops(a, l + 1, ok);
        push(TAIL_PROLONG, l);
        for (int s = 0; s < c->nu2; ++s) push(TAIL_SWEEP, l);
    }

    cudaError_t tail(int l, bool zero_start)
    {
        TailArgs a;
        memset(&a, 0, sizeof a);
        a.d = c->d;
        a.lu = c->lu;
        for (int j = 0; j < 4; ++j) a.c[j] = c->c[j];
        for (int k = c->lt; k < c->L; ++k) {
            // the tail always reads a scaled rhs buffer
            a.lv[k - c->lt] = tail_level(A(k), B(k), (void *)c->BH[k], c->RH[k], c->n[k]);
            if (c->pl && c->d == 2) {
                const Pitch2 g = pitch2(c->n[k]);
                a.lv[k - c->lt].pitch = g.pitch;
                a.lv[k - c->lt].off = g.off;
            } else if (c->pl) {
                const Pitch3 g = pitch3(c->n[k]);
                a.lv[k - c->lt].pitch = g.pitch;
                a.lv[k - c->lt].plane = g.plane;
                a.lv[k - c->lt].off = g.off;
            }
        }
        bool ok = true;
        if (zero_start) {
            a.ops[a.nops].kind = TAIL_ZERO;
            a.ops[a.nops].level = (short)(l - c->lt);
            ++a.nops;
        }
        tail_ops(a, l, ok);
        if (!ok) return cudaErrorInvalidValue;
        return launch_tail<T>(a, c->s);
    }

    // Record the remainder of a visit of level l whose current value is in
    // A(l) (or zero when zero_start). `skip_first` says the first pre-sweep
    // A(l) -> B(l) was already recorded elsewhere. On return the new value
    // is in A(l).
    cudaError_t visit(int l, bool zero_start, bool skip_first)
    {
        cudaError_t e;
        if (l >= c->lt) {
            if (l == 0 && b0_unscaled) {
                // finest level inside the tail: form the scaled rhs first
                e = launch_scale_copy<T, T>(b0, (T *)c->BH[0], npoints(c->d, c->n[0]),
                                            1.0 / ((double)c->N * c->N), c->s);
                if (e) return e;
            }
            return tail(l, zero_start);
        }
        const int n = c->n[l];
        T *buf[2] = {A(l), B(l)};
        int cur = 0;
        bool zero = zero_start;
        if (pl() && c->d == 2 && c->nu1 == 1 && c->nu2 == 1 && !skip_first) {
            // V(1,1) on an FP32 2D level in two temporally blocked passes:
            // pre-sweep + residual + restriction, then interpolation +
            // correction + post-sweep (the last one of a refinement cycle
            // adds into the FP64 solution)
            e = launch_sweep_restrict2d_pl(zero ? nullptr : (const float *)buf[0], (const float *)BH(l),
                                           (float *)buf[1], (float *)c->BH[l + 1], n, c->c, c->s);
            if (e) return e;
            for (int g = 0; g < c->gamma; ++g) {
                e = visit(l + 1, g == 0, false);
                if (e) return e;
            }
            if (l == 0 && acc64) {
                fused_update = true;
                return launch_prolong_sweep2d_pl((const float *)buf[1], (const float *)A(l + 1), (const float *)BH(l),
                                                 nullptr, acc64, n, c->c, c->s);
            }
            return launch_prolong_sweep2d_pl((const float *)buf[1], (const float *)A(l + 1), (const float *)BH(l),
                                             (float *)buf[0], nullptr, n, c->c, c->s);
        }
        for (int s = 0; s < c->nu1; ++s) {
            if (s == 0 && skip_first) {
                cur = 1;
                zero = false;
                continue;
            }
            e = sweep(zero ? nullptr : buf[cur], BH(l), unsc(l), buf[1 - cur], n);
            if (e) return e;
            cur = 1 - cur;
            zero = false;
        }
        if (zero) {
            e = launch_zero_words(buf[cur], bytes(l), c->s);
            if (e) return e;
        }
        e = resrestrict(buf[cur], BH(l), unsc(l), (T *)c->BH[l + 1], n);
        if (e) return e;
        for (int g = 0; g < c->gamma; ++g) {
            e = visit(l + 1, g == 0, false);
            if (e) return e;
        }
        e = prolong(A(l + 1), buf[cur], n);
        if (e) return e;
        for (int s = 0; s < c->nu2; ++s) {
            if (l == 0 && acc64 && pl() && s == c->nu2 - 1) {
                // refinement: the last finest sweep adds its result to the FP64 u
                fused_update = true;
                if (c->d == 2)
                    return launch_sweep2d_pl_acc64((const float *)buf[cur], (const float *)BH(l), acc64, n, c->c,
                                                   c->s);
                return launch_sweep3d_tma_acc64((const float *)buf[cur], (const float *)BH(l), acc64, n, c->c,
                                                c->d_err, c->s);
            }
            e = sweep(buf[cur], BH(l), unsc(l), buf[1 - cur], n);
            if (e) return e;
            cur = 1 - cur;
        }
        if (cur != 0) {
            e = launch_copy_words(buf[0], buf[1], bytes(l), c->s);
            if (e) return e;
        }
        return cudaSuccess;
    }
};

template <typename F>
static mg_status capture(mg_ctx *c, cudaGraphExec_t *out, unsigned long long *nodes, F &&body)
{
    return mg::capture_graph(c, out, nodes, std::function<cudaError_t()>(body));
}

using CaptureFn = std::function<cudaError_t()>;

// The graphs of a solve. pre: the residual norm of u (with a fused pre-sweep
// when the cycle starts with one); pre0: the same for u = 0 without reading
// u; meas: the norm alone (only with a fused pre-sweep); rest: the rest of the
// cycle. loop: a whole solve with its stop test on the device,
//   head -> [IF from_zero: pre0 ELSE pre] -> init -> [IF zero_u: u = 0] ->
//   WHILE loop { [IF rerun_pre: pre] -> rest -> [IF use_meas: meas ELSE pre]
//                -> after }
// (without meas: WHILE loop { rest -> pre -> after }), where the one-thread
// kernels head, init and after set the condition values.
static mg_status record_graphs(mg_ctx *c, void *u, const CaptureFn &pre, const CaptureFn &pre0,
                               const CaptureFn *meas, const CaptureFn &rest)
{
    // the plain graphs (mg_vcycle, the host-driven loop of mg_solve); their
    // norms also go to mapped host memory
    mg_status st;
    c->norm_to_host = true;
    if ((st = capture(c, &c->g.pre, &c->g.pre_nodes, pre)) != MG_OK) return st;
    if ((st = capture(c, &c->g.pre0, &c->g.pre0_nodes, pre0)) != MG_OK) return st;
    if (meas && (st = capture(c, &c->g.meas, &c->g.meas_nodes, *meas)) != MG_OK) return st;
    if ((st = capture(c, &c->g.rest, &c->g.rest_nodes, rest)) != MG_OK) return st;
    // the loop graph of mg_solve_async, with its own copies of the same work
    cudaGraph_t G = nullptr;
    cudaError_t e = cudaGraphCreate(&G, 0);
    if (e) return cuda_fail(e);
    const double nd = (double)c->N;
    const int has_meas = meas != nullptr;
    const size_t ubytes = npoints(c->d, c->n[0]) * (c->prec == MG_FP32 ? sizeof(float) : sizeof(double));
    c->norm_to_host = false;
    auto build = [&]() -> cudaError_t {
        // every handle belongs to the top graph and is reset at each launch
        cudaGraphConditionalHandle from_zero, loop, zero_u, rerun_pre = 0, use_meas = 0;
        cudaError_t e = cudaGraphConditionalHandleCreate(&from_zero, G, 0, cudaGraphCondAssignDefault);
        if (!e) e = cudaGraphConditionalHandleCreate(&loop, G, 0, cudaGraphCondAssignDefault);
        if (!e) e = cudaGraphConditionalHandleCreate(&zero_u, G, 0, cudaGraphCondAssignDefault);
        if (!e && has_meas) e = cudaGraphConditionalHandleCreate(&rerun_pre, G, 0, cudaGraphCondAssignDefault);
        if (!e && has_meas) e = cudaGraphConditionalHandleCreate(&use_meas, G, 0, cudaGraphCondAssignDefault);
        std::vector<cudaGraphNode_t> top, body, none;
        if (!e) e = capture_into(c, G, top, [&]() {
            loop_head_kernel<<<1, 1, 0, c->s>>>(c->d_loop, from_zero);
            return cudaGetLastError();
        }, nullptr);
        unsigned long long n_pre0 = 0, n_pre_head = 0;
        cudaGraph_t first[2] = {nullptr, nullptr};  // [0]: from zero, [1]: else
        if (!e) e = add_conditional(G, top, from_zero, cudaGraphCondTypeIf, 2, first);
        if (!e) e = capture_into(c, first[0], none, pre0, &n_pre0);
        none.clear();
        if (!e) e = capture_into(c, first[1], none, pre, &n_pre_head);
        none.clear();
        if (!e) e = capture_into(c, G, top, [&]() {
            loop_init_kernel<<<1, 1, 0, c->s>>>(c->d_loop, c->d_norm2, c->d_err, nd, has_meas, (unsigned)n_pre0,
                                                (unsigned)n_pre_head, loop, zero_u, c->h_launched_dev);
            return cudaGetLastError();
        }, nullptr);
        cudaGraph_t Z = nullptr, B = nullptr;
        if (!e) e = add_conditional(G, top, zero_u, cudaGraphCondTypeIf, 1, &Z);
        if (!e) e = capture_into(c, Z, none, [&]() { return launch_zero_words(u, ubytes, c->s); }, nullptr);
        if (!e) e = add_conditional(G, top, loop, cudaGraphCondTypeWhile, 1, &B);
        unsigned long long n_rest = 0, n_pre = 0, n_meas = 0;
        if (!e && has_meas) {
            cudaGraph_t R = nullptr;  // a wrong guess: the pre graph after all
            e = add_conditional(B, body, rerun_pre, cudaGraphCondTypeIf, 1, &R);
            none.clear();
            if (!e) e = capture_into(c, R, none, pre, nullptr);
        }
        if (!e) e = capture_into(c, B, body, rest, &n_rest);
        if (!e && has_meas) {
            cudaGraph_t two[2] = {nullptr, nullptr};  // [0]: condition set, [1]: else
            e = add_conditional(B, body, use_meas, cudaGraphCondTypeIf, 2, two);
            none.clear();
            if (!e) e = capture_into(c, two[0], none, *meas, &n_meas);
            none.clear();
            if (!e) e = capture_into(c, two[1], none, pre, &n_pre);
        } else if (!e) {
            e = capture_into(c, B, body, pre, &n_pre);
        }
        if (!e) e = capture_into(c, B, body, [&]() {
            loop_after_kernel<<<1, 1, 0, c->s>>>(c->d_loop, c->d_norm2, c->d_err, nd, has_meas, (unsigned)n_rest,
                                                 (unsigned)n_pre, (unsigned)n_meas, loop, rerun_pre, use_meas,
                                                 c->h_launched_dev);
            return cudaGetLastError();
        }, nullptr);
        if (!e) e = cudaGraphInstantiate(&c->g.loop, G, 0);
        return e;
    };
    e = build();
    c->norm_to_host = true;
    cudaGraphDestroy(G);
    return e ? cuda_fail(e) : MG_OK;
}

// Plain cycles in precision T on the caller's arrays (level 0 = caller's u, b).
template <typename T>
static mg_status record_plain(mg_ctx *c, void *u, const void *b)
{
    const int d = c->d, n0 = c->n[0];
    Recorder<T> R{c, (const T *)b, true, (T *)u};
    const bool fused = c->nu1 >= 1 && c->lt > 0;
    const CaptureFn pre = [&]() -> cudaError_t {
        cudaError_t e;
        if (fused)
            e = op_sweep<T>(d, (const T *)u, (const T *)b, true, (T *)c->B[0], n0, c->c, c->partials, c->s);
        else
            e = op_residual<T, T>(d, (const T *)u, (const T *)b, true, (T *)nullptr, n0, c->partials, c->s);
        if (e) return e;
        const int np = fused ? sweep_partials(d, n0, (int)sizeof(T)) : residual_partials(d, n0);
        return launch_norm_sum(c, np);
    };
    // solve from u = 0: the first pre-sweep in its from-zero form (u is not
    // read; the rest of the cycle writes it); without a fused pre-sweep, u is
    // zeroed and the pre graph's residual follows
    const CaptureFn pre0 = [&]() -> cudaError_t {
        cudaError_t e;
        if (fused) {
            e = op_sweep<T>(d, (const T *)nullptr, (const T *)b, true, (T *)c->B[0], n0, c->c, c->partials, c->s);
        } else {
            e = launch_zero_words(u, npoints(d, n0) * sizeof(T), c->s);
            if (!e) e = op_residual<T, T>(d, (const T *)u, (const T *)b, true, (T *)nullptr, n0, c->partials, c->s);
        }
        if (e) return e;
        const int np = fused ? sweep_partials(d, n0, (int)sizeof(T)) : residual_partials(d, n0);
        return launch_norm_sum(c, np);
    };
    const CaptureFn meas = [&]() -> cudaError_t {
        cudaError_t e = op_residual<T, T>(d, (const T *)u, (const T *)b, true, (T *)nullptr, n0, c->partials, c->s);
        if (e) return e;
        return launch_norm_sum(c, residual_partials(d, n0));
    };
    const CaptureFn rest = [&]() -> cudaError_t { return R.visit(0, false, fused); };
    return record_graphs(c, u, pre, pre0, fused ? &meas : nullptr, rest);
}

// graph sets kept per context: the current one and this many others
constexpr size_t kOtherGraphSets = 3;

// Make c->g the graphs for the caller's arrays u and b: the current set, a
// kept one, or a new recording (the oldest kept set is dropped).
static mg_status record(mg_ctx *c, void *u, const void *b)
{
    if (c->g.pre && c->g.cap_u == u && c->g.cap_b == b) return MG_OK;
    if (c->g.pre) c->other.push_back(c->g);
    c->g = GraphPair{};
    for (size_t i = 0; i < c->other.size(); ++i)
        if (c->other[i].cap_u == u && c->other[i].cap_b == b) {
            c->g = c->other[i];
            c->other.erase(c->other.begin() + (long)i);
            return MG_OK;
        }
    while (c->other.size() > kOtherGraphSets) {
        destroy_set(c->other.front());
        c->other.erase(c->other.begin());
    }
    const int d = c->d, n0 = c->n[0];
    const size_t np0 = npoints(d, n0);
    mg_status st;
    if (c->prec == MG_FP64) {
        st = record_plain<double>(c, u, b);
    } else if (c->prec == MG_FP32) {
        st = record_plain<float>(c, u, b);
    } else {
        // refinement: FP64 residual -> FP32 scaled rhs of level 0; FP32 cycle
        // from zero; u += e in FP64
        Recorder<float> R{c, (const float *)c->BH[0], false, (float *)c->A[0]};
        const CaptureFn pre = [&]() -> cudaError_t {
            cudaError_t e;
            if (c->pl && d == 2) {
                const Pitch2 g = pitch2(n0);
                e = launch_residual2d<double, float>((const double *)u, (const double *)b, true, (float *)c->BH[0],
                                                     n0, c->partials, c->s, g.pitch, g.off);
            } else if (c->pl) {
                const Pitch3 g = pitch3(n0);
                e = launch_residual3d<double, float>((const double *)u, (const double *)b, true, (float *)c->BH[0],
                                                     n0, c->partials, c->s, g.pitch, g.plane, g.off);
            } else {
                e = op_residual<double, float>(d, (const double *)u, (const double *)b, true, (float *)c->BH[0], n0,
                                               c->partials, c->s);
            }
            if (e) return e;
            return launch_norm_sum(c, residual_partials(d, n0));
        };
        // solve from u = 0: u zeroed (the FP64 updates add into it) and the
        // first residual is h^2 b itself, rounded to FP32, without FP64 work
        const CaptureFn pre0 = [&]() -> cudaError_t {
            cudaError_t e = launch_zero_words(u, np0 * sizeof(double), c->s);
            int nb = 0;
            if (!e) e = launch_refine_rhs_zero(c, (const double *)b, nb);
            if (e) return e;
            return launch_norm_sum(c, nb);
        };
        const CaptureFn rest = [&]() -> cudaError_t {
            cudaError_t e = cudaSuccess;
            R.fused_update = false;
            for (int k = 0; k < c->inner && !e; ++k) {
                // only the last cycle of the iteration may fuse the FP64 update
                R.acc64 = k == c->inner - 1 ? (double *)u : nullptr;
                e = R.visit(0, k == 0, false);
            }
            if (e || R.fused_update) return e;
            if (c->pl && d == 2) return launch_add_pl2d((double *)u, (const float *)c->A[0], n0, c->s);
            if (c->pl) return launch_add_pl3d((double *)u, (const float *)c->A[0], n0, c->s);
            return launch_add_to_f64<float>((double *)u, (const float *)c->A[0], np0, c->s);
        };
        st = record_graphs(c, u, pre, pre0, nullptr, rest);
    }
    if (st != MG_OK) {
        destroy_set(c->g);
        return st;
    }
    c->g.cap_u = u;
    c->g.cap_b = b;
    return MG_OK;
}

// Order the context's stream after the caller's and clear the error word, so
// that an expired wait of an earlier call does not fail this one.
static mg_status enter(mg_ctx *c)
{
    MG_CUDA(cudaSetDevice(c->dev));
    MG_CUDA(cudaEventRecord(c->ev_in, c->user));
    MG_CUDA(cudaStreamWaitEvent(c->s, c->ev_in, 0));
    MG_CUDA(launch_zero_words(c->d_err, sizeof(int), c->s));
    return MG_OK;
}

static mg_status leave(mg_ctx *c)
{
    MG_CUDA(cudaEventRecord(c->ev_out, c->s));
    MG_CUDA(cudaStreamWaitEvent(c->user, c->ev_out, 0));
    return MG_OK;
}

static mg_status launch_graph(mg_ctx *c, cudaGraphExec_t g, unsigned long long nodes)
{
    MG_CUDA(cudaGraphLaunch(g, c->s));
    g_launches += nodes;
    return MG_OK;
}

// ||r||_2 from the last pre graph: sqrt(sum rh^2) / h^2
static double norm_from_host(mg_ctx *c)
{
    return std::sqrt(*c->h_norm2) * (double)c->N * (double)c->N;
}

// a kernel of this call gave up on a bounded wait (bit 0); bit 1: its drain
// of the copies still in flight gave up too, so a copy may have landed after
// the block ended and the context's buffers are no longer trustworthy
static bool timed_out_word(int e)
{
    if (e & 2)
        snprintf(g_last_error, sizeof g_last_error,
                 "a bounded device wait and the drain of its copies both expired: destroy the context");
    return e != 0;
}

static bool timed_out(const mg_ctx *c)
{
    int e;
    std::memcpy(&e, c->h_norm2 + 1, sizeof e);
    return timed_out_word(e);
}

static mg_status setup_impl(int d, int N, const double *coeffs, int ncoeffs, int nu1, int nu2, int gamma,
                            mg_prec prec, void *stream, mg_ctx **out)
{
    if (!out) return MG_EINVAL;
    *out = nullptr;
    if ((d != 2 && d != 3) || !valid_N(N) || !coeffs || ncoeffs < 1 || ncoeffs > (d == 2 ? 3 : 4) ||
        nu1 < 0 || nu2 < 0 || nu1 + nu2 < 1 || gamma < 1 || gamma > 2 ||
        (prec != MG_FP64 && prec != MG_FP32_IR && prec != MG_FP32))
        return MG_EINVAL;
    for (int j = 0; j < ncoeffs; ++j)
        if (!std::isfinite(coeffs[j])) return MG_EINVAL;
    // the 27-point M (edge or corner weights) runs on the compact-layout
    // kernels: FP64 and plain FP32 cycles, not the padded FP32 refinement levels
    if (wide_weights(d, coeffs, ncoeffs) && prec == MG_FP32_IR) return MG_EINVAL;
    if (d == 3 && (size_t)(N - 1) * (N - 1) * (N - 1) > (size_t)1 << 34) return MG_EINVAL;
    mg_ctx *c = new (std::nothrow) mg_ctx;
    if (!c) return MG_ENOMEM;
    c->d = d;
    c->N = N;
    c->nu1 = nu1;
    c->nu2 = nu2;
    c->gamma = gamma;
    c->prec = prec;
    c->ncoef = ncoeffs;
    for (int j = 0; j < ncoeffs; ++j) c->c[j] = coeffs[j];
    c->user = (cudaStream_t)stream;
    c->esize = prec == MG_FP64 ? sizeof(double) : sizeof(float);
    mg_status st = MG_OK;
#define MG_TRY(x)                      \
    do {                               \
        st = (x);                      \
        if (st != MG_OK) goto fail;    \
    } while (0)
#define MG_TRYC(x)                              \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) {                \
            st = cuda_fail(e_);                 \
            goto fail;                          \
        }                                       \
    } while (0)
    {
        MG_TRYC(cudaGetDevice(&c->dev));
        MG_TRYC(cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking));
        MG_TRYC(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
        MG_TRYC(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
        for (int m = N; m >= 4; m /= 2) c->n.push_back(m - 1);
        c->L = (int)c->n.size();
        // levels with n <= 15 (2D) / 7 (3D) run inside the one-block tail
        const int tail_n = d == 2 ? 15 : 7;
        c->lt = c->L;
        for (int l = 0; l < c->L; ++l)
            if (c->n[l] <= tail_n) {
                c->lt = l;
                break;
            }
        if (c->L - c->lt > kMaxTailLevels) c->lt = c->L - kMaxTailLevels;
        c->A.assign(c->L, nullptr);
        c->B.assign(c->L, nullptr);
        c->BH.assign(c->L, nullptr);
        c->RH.assign(c->L, nullptr);
        c->pl = prec == MG_FP32_IR;
        for (int l = 0; l < c->L; ++l) {
            const size_t bytes = level_bytes(c, l);
            const bool caller_level = l == 0 && prec != MG_FP32_IR;
            if (!caller_level) MG_TRY(dalloc(c, &c->A[l], bytes));
            MG_TRY(dalloc(c, &c->B[l], bytes));
            if (!caller_level || c->lt == 0) MG_TRY(dalloc(c, &c->BH[l], bytes));
            if (l >= c->lt) MG_TRY(dalloc(c, &c->RH[l], bytes));
            if (c->pl)  // ghost rings and row padding must read as zero
                for (void *p : {c->A[l], c->B[l], c->BH[l], c->RH[l]})
                    if (p) MG_TRYC(cudaMemset(p, 0, bytes));
        }
        int np = std::max({sweep_partials(d, c->n[0], 8), sweep_partials(d, c->n[0], 4), residual_partials(d, c->n[0])});
        c->npartials = np;
        MG_TRY(dalloc(c, (void **)&c->partials, (size_t)np * sizeof(double)));
        MG_TRY(dalloc(c, (void **)&c->d_norm2, kNormBytes));
        MG_TRYC(cudaMemset(c->d_norm2, 0, kNormBytes));
        c->d_err = (int *)(c->d_norm2 + 1);
        MG_TRY(dalloc(c, (void **)&c->lu, 27 * 27 * sizeof(double)));
        {
            double lu[27 * 27];
            coarse_inverse(d, lu);
            const int m = d == 2 ? 9 : 27;
            MG_TRYC(cudaMemcpy(c->lu, lu, (size_t)m * m * sizeof(double), cudaMemcpyHostToDevice));
        }
        MG_TRYC(cudaHostAlloc((void **)&c->h_norm2, kNormBytes, cudaHostAllocMapped));
        MG_TRYC(cudaHostGetDevicePointer((void **)&c->h_norm2_dev, c->h_norm2, 0));
        std::memset(c->h_norm2, 0, kNormBytes);
        MG_TRYC(cudaHostAlloc((void **)&c->h_launched, sizeof(unsigned long long), cudaHostAllocMapped));
        MG_TRYC(cudaHostGetDevicePointer((void **)&c->h_launched_dev, c->h_launched, 0));
        *c->h_launched = 0;
        MG_TRY(dalloc(c, (void **)&c->d_loop, sizeof(LoopState)));
        MG_TRYC(cudaMemset(c->d_loop, 0, sizeof(LoopState)));
        register_ctx(c);
    }
    *out = c;
    return MG_OK;
fail:
    destroy_ctx(c);
    return st;
#undef MG_TRY
#undef MG_TRYC
}

}  // namespace

// ---------------------------------------------------------------------------
// single operators
// ---------------------------------------------------------------------------
static bool valid_level(int d, int n)
{
    return (d == 2 || d == 3) && n >= 3 && (n & 1) && valid_N(n + 1);
}

// FP32 2D single operators run the padded-layout kernels of the FP32 cycles:
// the compact arrays are packed into zero-ringed temporaries and unpacked.
struct PaddedTmp {
    int d = 2;
    std::vector<float *> bufs;
    explicit PaddedTmp(int dim) : d(dim) {}
    ~PaddedTmp()
    {
        for (float *p : bufs) cudaFree(p);
    }
    float *make(int n, const void *compact, cudaStream_t s, cudaError_t &e)
    {
        float *p = nullptr;
        const size_t bytes = (d == 2 ? pitch2_floats(n) : pitch3_floats(n)) * sizeof(float);
        if (e == cudaSuccess) e = cudaMalloc(&p, bytes);
        if (e == cudaSuccess) bufs.push_back(p);
        if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, bytes, s);
        if (e == cudaSuccess && compact) e = pack((const float *)compact, p, n, true, s);
        return p;
    }
    cudaError_t pack(const float *in, float *out, int n, bool to_padded, cudaStream_t s)
    {
        return d == 2 ? launch_pack2d(in, out, n, to_padded, s) : launch_pack3d(in, out, n, to_padded, s);
    }
};

static mg_status op_sweep_pl(int d, int n, const double *c, const void *u, const void *bh, int unscaled, void *out,
                             double *rnorm2, cudaStream_t s)
{
    if (unscaled) return MG_EINVAL;  // the FP32 cycles only see scaled right-hand sides
    if (d == 3 && rnorm2) return MG_EINVAL;  // the 3D FP32 sweep has no fused norm
    cudaError_t e = cudaSuccess;
    PaddedTmp tmp(d);
    float *pu = u ? tmp.make(n, u, s, e) : nullptr;
    float *pb = tmp.make(n, bh, s, e), *po = tmp.make(n, nullptr, s, e);
    double *partials = nullptr;
    int *err = nullptr, h_err = 0;
    const int np = d == 2 ? sweep2d_pl_blocks(n, sweep2d_pl_H(n)) : 0;
    if (!e && rnorm2) e = cudaMalloc(&partials, (size_t)(np + 1) * sizeof(double));
    if (!e && d == 3) e = cudaMalloc(&err, sizeof(int));
    if (!e && d == 3) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (!e) e = d == 2 ? launch_sweep2d_pl(pu, pb, po, n, c, partials, s) : launch_sweep3d_tma(pu, pb, po, n, c, err, s);
    if (!e) e = tmp.pack(po, (float *)out, n, false, s);
    if (!e && rnorm2) {
        e = launch_sum_partials(partials, np, partials + np, s);
        if (!e) e = cudaMemcpyAsync(rnorm2, partials + np, sizeof(double), cudaMemcpyDeviceToHost, s);
    }
    if (!e && err) e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (partials) cudaFree(partials);
    if (err) cudaFree(err);
    if (e) return cuda_fail(e);
    return h_err ? MG_ETIMEOUT : MG_OK;
}

template <typename T>
static mg_status op_sweep_t(int d, int n, const double *c, const void *u, const void *bh, int unscaled, void *out,
                            double *rnorm2, cudaStream_t s)
{
    if (sizeof(T) == 4 && !unscaled && !(d == 3 && rnorm2)) return op_sweep_pl(d, n, c, u, bh, unscaled, out, rnorm2, s);
    double *partials = nullptr, *sum = nullptr;
    cudaError_t e;
    if (rnorm2) {
        const int np = sweep_partials(d, n, (int)sizeof(T));
        if ((e = cudaMalloc(&partials, (size_t)np * sizeof(double) + sizeof(double)))) return cuda_fail(e);
        sum = partials + np;
    }
    e = op_sweep<T>(d, (const T *)u, (const T *)bh, unscaled != 0, (T *)out, n, c, partials, s);
    if (!e && rnorm2) {
        e = launch_sum_partials(partials, sweep_partials(d, n, (int)sizeof(T)), sum, s);
        if (!e) e = cudaMemcpyAsync(rnorm2, sum, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
    }
    if (partials) cudaFree(partials);
    return e ? cuda_fail(e) : MG_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

mg_status mg_setup_ex(int d, int N, const double *spai_coeffs, int ncoeffs, int nu1, int nu2, int gamma,
                      mg_prec prec, void *cuda_stream, mg_ctx **out)
{
    return setup_impl(d, N, spai_coeffs, ncoeffs, nu1, nu2, gamma, prec, cuda_stream, out);
}

mg_status mg_setup(int d, int N, const double *spai_coeffs, int ncoeffs, int nu1, int nu2, mg_prec prec,
                   void *cuda_stream, mg_ctx **out)
{
    return setup_impl(d, N, spai_coeffs, ncoeffs, nu1, nu2, 1, prec, cuda_stream, out);
}

void mg_destroy(mg_ctx *ctx)
{
    if (ctx) {
        cudaSetDevice(ctx->dev);
        if (ctx->s) cudaStreamSynchronize(ctx->s);
        destroy_ctx(ctx);
    }
}

mg_status mg_vcycle(mg_ctx *ctx, void *u, const void *b)
{
    if (!ctx || !u || !b || ctx->batch) return MG_EINVAL;
    mg_status st = enter(ctx);
    if (st != MG_OK) return st;
    if ((st = record(ctx, u, b)) == MG_OK && (st = launch_graph(ctx, ctx->g.pre, ctx->g.pre_nodes)) == MG_OK)
        st = launch_graph(ctx, ctx->g.rest, ctx->g.rest_nodes);
    // every exit after enter() orders the caller's stream after the work queued here
    const mg_status st2 = leave(ctx);
    return st != MG_OK ? st : st2;
}

// wait for the context's stream; MG_ETIMEOUT when a kernel's bounded wait expired
static mg_status sync_ctx(mg_ctx *ctx)
{
    const cudaError_t e = cudaStreamSynchronize(ctx->s);
    if (e != cudaSuccess) return cuda_fail(e);
    return timed_out(ctx) ? MG_ETIMEOUT : MG_OK;
}

// Queue one solve on the context's stream, between enter() and leave(): its
// arguments (by value, in a kernel's parameters) and the loop graph, which
// runs the first pre graph, the cycles and the stop test on the device. The
// pre graph smooths the next cycle's input speculatively while it measures
// the residual, so the measurement that ends the solve would pay for a sweep
// nobody uses: when the last convergence factor, carried one cycle forward,
// puts the coming residual under the tolerance, the cycle ends with the
// norm-only graph instead; if the guess was wrong, the pre graph runs after
// it and guessing stops for this solve. Either way u, the cycle count and
// the history are those of the speculative schedule.
static mg_status queue_solve(mg_ctx *ctx, const void *b, void *u, double tol, int max_cycles, bool zero_start,
                             mg_solve_info *info, double *hist)
{
    mg_status st;
    if ((st = record(ctx, u, b)) != MG_OK) return st;
    LoopArgs a;
    a.tol = tol;
    a.hist = hist;
    a.info = info;
    a.max_cycles = max_cycles;
    a.zero_start = zero_start ? 1 : 0;
    loop_args_kernel<<<1, 1, 0, ctx->s>>>(ctx->d_loop, a);
    count_launch(1);
    MG_CUDA(cudaGetLastError());
    MG_CUDA(cudaGraphLaunch(ctx->g.loop, ctx->s));
    return MG_OK;
}

// mg_solve_ex between enter() and leave(): the same schedule driven from the
// host, one synchronisation per cycle (the norm comes through mapped host
// memory). On small grids this is faster than the device-side loop, whose
// conditional nodes cost a few microseconds per cycle more than the round
// trip, and every kernel of it is visible to profilers that cannot look
// inside graphs with conditional nodes. Its iterates, counts and history are
// those of mg_solve_async bit for bit.
static mg_status solve_loop(mg_ctx *ctx, const void *b, void *u, double tol, int max_cycles, bool zero_start,
                            int *cycles_out, double *relres_out, double *hist_out)
{
    mg_status st;
    if ((st = record(ctx, u, b)) != MG_OK) return st;
    if ((st = zero_start ? launch_graph(ctx, ctx->g.pre0, ctx->g.pre0_nodes)
                         : launch_graph(ctx, ctx->g.pre, ctx->g.pre_nodes)) != MG_OK)
        return st;
    if ((st = sync_ctx(ctx)) != MG_OK) return st;
    const double r0 = norm_from_host(ctx);
    double rk = r0, rprev = 0.0;
    int k = 0;
    if (hist_out) hist_out[0] = r0;
    st = std::isfinite(r0) ? MG_OK : MG_ENAN;
    bool guessing = ctx->g.meas != nullptr;
    while (st == MG_OK && !(rk <= tol * r0)) {
        if (k == max_cycles) {
            st = MG_ENOCONV;
            break;
        }
        const bool guess = guessing && k >= 1 && rprev > 0.0 && rk * (rk / rprev) <= tol * r0;
        mg_status ls;
        if ((ls = launch_graph(ctx, ctx->g.rest, ctx->g.rest_nodes)) != MG_OK) return ls;
        ls = guess ? launch_graph(ctx, ctx->g.meas, ctx->g.meas_nodes) : launch_graph(ctx, ctx->g.pre, ctx->g.pre_nodes);
        if (ls != MG_OK) return ls;
        if ((ls = sync_ctx(ctx)) != MG_OK) return ls;
        ++k;
        rprev = rk;
        rk = norm_from_host(ctx);
        if (hist_out) hist_out[k] = rk;
        if (!std::isfinite(rk)) st = MG_ENAN;
        if (st == MG_OK && guess && !(rk <= tol * r0) && k < max_cycles) {
            guessing = false;
            if ((ls = launch_graph(ctx, ctx->g.pre, ctx->g.pre_nodes)) != MG_OK) return ls;
            if ((ls = sync_ctx(ctx)) != MG_OK) return ls;
        }
    }
    if (zero_start && k == 0) {
        // no cycle ran (zero rhs, max_cycles = 0, a non-finite r0): u is the
        // zero initial guess, which a zero start never wrote
        const size_t bytes = npoints(ctx->d, ctx->n[0]) * (ctx->prec == MG_FP32 ? sizeof(float) : sizeof(double));
        MG_CUDA(launch_zero_words(u, bytes, ctx->s));
    }
    if (cycles_out) *cycles_out = k;
    if (relres_out) *relres_out = r0 > 0.0 ? rk / r0 : 0.0;
    return st;
}

mg_status mg_solve_ex(mg_ctx *ctx, const void *b, void *u, double tol, int max_cycles, unsigned flags,
                      int *cycles_out, double *relres_out, double *hist_out)
{
    if (!ctx || !u || !b || max_cycles < 0 || !(tol >= 0.0) || ctx->batch || (flags & ~MG_SOLVE_ZERO_START))
        return MG_EINVAL;
    mg_status st = enter(ctx);
    if (st != MG_OK) return st;
    st = solve_loop(ctx, b, u, tol, max_cycles, (flags & MG_SOLVE_ZERO_START) != 0, cycles_out, relres_out,
                    hist_out);
    const mg_status st2 = leave(ctx);
    return st != MG_OK ? st : st2;
}

mg_status mg_solve_async(mg_ctx *ctx, const void *b, void *u, double tol, int max_cycles, unsigned flags,
                         mg_solve_info *info, double *hist)
{
    if (!ctx || !u || !b || !info || max_cycles < 0 || !(tol >= 0.0) || ctx->batch ||
        (flags & ~MG_SOLVE_ZERO_START))
        return MG_EINVAL;
    mg_status st = enter(ctx);
    if (st != MG_OK) return st;
    st = queue_solve(ctx, b, u, tol, max_cycles, (flags & MG_SOLVE_ZERO_START) != 0, info, hist);
    const mg_status st2 = leave(ctx);
    return st != MG_OK ? st : st2;
}

mg_status mg_solve(mg_ctx *ctx, const void *b, void *u, double tol, int max_cycles, int *cycles_out,
                   double *relres_out, double *hist_out)
{
    return mg_solve_ex(ctx, b, u, tol, max_cycles, 0u, cycles_out, relres_out, hist_out);
}

mg_status mg_set_coeffs(mg_ctx *ctx, const double *spai_coeffs, int ncoeffs)
{
    if (!ctx || !spai_coeffs || ncoeffs < 1 || ncoeffs > (ctx->d == 2 ? 3 : 4)) return MG_EINVAL;
    for (int j = 0; j < ncoeffs; ++j)
        if (!std::isfinite(spai_coeffs[j])) return MG_EINVAL;
    if (wide_weights(ctx->d, spai_coeffs, ncoeffs) && (ctx->prec == MG_FP32_IR || ctx->batch)) return MG_EINVAL;
    if (cudaSetDevice(ctx->dev) != cudaSuccess || cudaStreamSynchronize(ctx->s) != cudaSuccess)
        return cuda_fail(cudaGetLastError());
    for (int j = 0; j < 4; ++j) ctx->c[j] = j < ncoeffs ? spai_coeffs[j] : 0.0;
    ctx->ncoef = ncoeffs;
    free_graphs(ctx);
    return MG_OK;
}

mg_status mg_set_refinement_cycles(mg_ctx *ctx, int cycles)
{
    if (ctx && ctx->batch) return batch_set_inner(ctx, cycles);
    if (!ctx || ctx->prec != MG_FP32_IR || cycles < 1 || cycles > 8) return MG_EINVAL;
    if (cudaSetDevice(ctx->dev) != cudaSuccess || cudaStreamSynchronize(ctx->s) != cudaSuccess)
        return cuda_fail(cudaGetLastError());
    ctx->inner = cycles;
    free_graphs(ctx);
    return MG_OK;
}

mg_status mg_residual_norm(mg_ctx *ctx, const void *u, const void *b, double *norm_out)
{
    if (!ctx || !u || !b || !norm_out || ctx->batch) return MG_EINVAL;
    mg_status st = enter(ctx);
    if (st != MG_OK) return st;
    const int n0 = ctx->n[0];
    cudaError_t e = ctx->prec == MG_FP32
                        ? op_residual<float, float>(ctx->d, (const float *)u, (const float *)b, true, (float *)nullptr,
                                                    n0, ctx->partials, ctx->s)
                        : op_residual<double, double>(ctx->d, (const double *)u, (const double *)b, true,
                                                      (double *)nullptr, n0, ctx->partials, ctx->s);
    if (!e) e = launch_sum_partials_host(ctx, residual_partials(ctx->d, n0), ctx->s);
    st = e ? cuda_fail(e) : sync_ctx(ctx);
    if (st == MG_OK) *norm_out = norm_from_host(ctx);
    const mg_status st2 = leave(ctx);
    return st != MG_OK ? st : st2;
}

mg_status mg_op_sweep(int d, int n, mg_prec prec, const double *spai_coeffs, int ncoeffs, const void *u,
                      const void *bh, int b_unscaled, void *u_out, double *rnorm2_out, void *stream)
{
    if (!valid_level(d, n) || !spai_coeffs || ncoeffs < 1 || ncoeffs > (d == 2 ? 3 : 4) || !bh || !u_out)
        return MG_EINVAL;
    // the FP32 operators run the padded-layout refinement kernels (7-point M in 3D)
    if (wide_weights(d, spai_coeffs, ncoeffs) && prec != MG_FP64) return MG_EINVAL;
    double c[4] = {0, 0, 0, 0};
    for (int j = 0; j < ncoeffs; ++j) c[j] = spai_coeffs[j];
    if (prec == MG_FP64)
        return op_sweep_t<double>(d, n, c, u, bh, b_unscaled, u_out, rnorm2_out, (cudaStream_t)stream);
    if (prec == MG_FP32_IR)
        return op_sweep_t<float>(d, n, c, u, bh, b_unscaled, u_out, rnorm2_out, (cudaStream_t)stream);
    return MG_EINVAL;
}

mg_status mg_op_residual(int d, int n, mg_prec prec, const void *u, const void *bh, int b_unscaled, void *rh_out,
                         void *stream)
{
    if (!valid_level(d, n) || !u || !bh || !rh_out) return MG_EINVAL;
    cudaError_t e;
    if (prec == MG_FP64)
        e = op_residual<double, double>(d, (const double *)u, (const double *)bh, b_unscaled != 0, (double *)rh_out,
                                        n, nullptr, (cudaStream_t)stream);
    else if (prec == MG_FP32_IR)
        e = op_residual<float, float>(d, (const float *)u, (const float *)bh, b_unscaled != 0, (float *)rh_out, n,
                                      nullptr, (cudaStream_t)stream);
    else
        return MG_EINVAL;
    return e ? cuda_fail(e) : MG_OK;
}

mg_status mg_op_residual_refine(int d, int n, const double *u, const double *bh, int b_unscaled, float *rh32_out,
                                double *rnorm2_out, void *stream)
{
    if (!valid_level(d, n) || !u || !bh || !rh32_out) return MG_EINVAL;
    const cudaStream_t s = (cudaStream_t)stream;
    double *partials = nullptr;
    const int np = residual_partials(d, n);
    cudaError_t e = cudaSuccess;
    if (rnorm2_out) e = cudaMalloc(&partials, (size_t)(np + 1) * sizeof(double));
    if (!e) e = op_residual<double, float>(d, u, bh, b_unscaled != 0, rh32_out, n, partials, s);
    if (!e && rnorm2_out) {
        e = launch_sum_partials(partials, np, partials + np, s);
        if (!e) e = cudaMemcpyAsync(rnorm2_out, partials + np, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
    }
    if (partials) cudaFree(partials);
    return e ? cuda_fail(e) : MG_OK;
}

mg_status mg_op_residual_restrict(int d, int n, mg_prec prec, const void *u, const void *bh, int b_unscaled,
                                  void *bh_coarse_out, void *stream)
{
    if (!valid_level(d, n) || n < 7 || !u || !bh || !bh_coarse_out) return MG_EINVAL;
    cudaError_t e;
    if (prec == MG_FP64)
        e = op_resrestrict<double>(d, (const double *)u, (const double *)bh, b_unscaled != 0,
                                   (double *)bh_coarse_out, n, (cudaStream_t)stream);
    else if (prec == MG_FP32_IR && !b_unscaled) {
        PaddedTmp tmp(d);
        e = cudaSuccess;
        const cudaStream_t s = (cudaStream_t)stream;
        float *pu = tmp.make(n, u, s, e), *pb = tmp.make(n, bh, s, e), *pc = tmp.make((n - 1) / 2, nullptr, s, e);
        int *err = nullptr, h_err = 0;
        if (!e && d == 3) e = cudaMalloc(&err, sizeof(int));
        if (!e && d == 3) e = cudaMemsetAsync(err, 0, sizeof(int), s);
        if (!e) e = d == 2 ? launch_resrestrict2d_pl(pu, pb, pc, n, s) : launch_resrestrict3d_tma(pu, pb, pc, n, err, s);
        if (!e) e = tmp.pack(pc, (float *)bh_coarse_out, (n - 1) / 2, false, s);
        if (!e && err) e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (err) cudaFree(err);
        if (!e && h_err) return MG_ETIMEOUT;
    } else if (prec == MG_FP32_IR)
        e = op_resrestrict<float>(d, (const float *)u, (const float *)bh, b_unscaled != 0, (float *)bh_coarse_out,
                                  n, (cudaStream_t)stream);
    else
        return MG_EINVAL;
    return e ? cuda_fail(e) : MG_OK;
}

mg_status mg_op_prolong_correct(int d, int n, mg_prec prec, const void *e_coarse, void *u, void *stream)
{
    if (!valid_level(d, n) || n < 7 || !e_coarse || !u) return MG_EINVAL;
    cudaError_t e;
    if (prec == MG_FP64)
        e = op_prolong<double>(d, (const double *)e_coarse, (double *)u, n, (cudaStream_t)stream);
    else if (prec == MG_FP32_IR) {
        PaddedTmp tmp(d);
        e = cudaSuccess;
        const cudaStream_t s = (cudaStream_t)stream;
        float *pe = tmp.make((n - 1) / 2, e_coarse, s, e), *pu = tmp.make(n, u, s, e);
        if (!e) e = d == 2 ? launch_prolong2d_pl(pe, pu, n, s) : launch_prolong3d_pl(pe, pu, n, s);
        if (!e) e = tmp.pack(pu, (float *)u, n, false, s);
        if (!e) e = cudaStreamSynchronize(s);
    } else if (prec == MG_FP32_IR)
        e = op_prolong<float>(d, (const float *)e_coarse, (float *)u, n, (cudaStream_t)stream);
    else
        return MG_EINVAL;
    return e ? cuda_fail(e) : MG_OK;
}

// the temporally blocked V(1,1) passes of the FP32 2D levels, on padded copies
static mg_status fused_args_ok(int d, int n, mg_prec prec, const double *w, int nw, double *c)
{
    if (d != 2 || prec != MG_FP32_IR || !valid_level(d, n) || n < 7 || !w || nw < 1 || nw > 3) return MG_EINVAL;
    for (int j = 0; j < 4; ++j) c[j] = j < nw ? w[j] : 0.0;
    return MG_OK;
}

mg_status mg_op_sweep_restrict(int d, int n, mg_prec prec, const double *spai_coeffs, int ncoeffs, const void *u,
                               const void *bh, void *u_out, void *bh_coarse_out, void *stream)
{
    double c[4];
    if (fused_args_ok(d, n, prec, spai_coeffs, ncoeffs, c) != MG_OK || !bh || !u_out || !bh_coarse_out)
        return MG_EINVAL;
    const cudaStream_t s = (cudaStream_t)stream;
    const int nc = (n - 1) / 2;
    cudaError_t e = cudaSuccess;
    PaddedTmp tmp(d);
    float *pu = u ? tmp.make(n, u, s, e) : nullptr;
    float *pb = tmp.make(n, bh, s, e), *po = tmp.make(n, nullptr, s, e), *pc = tmp.make(nc, nullptr, s, e);
    if (!e) e = launch_sweep_restrict2d_pl(pu, pb, po, pc, n, c, s);
    if (!e) e = tmp.pack(po, (float *)u_out, n, false, s);
    if (!e) e = tmp.pack(pc, (float *)bh_coarse_out, nc, false, s);
    if (!e) e = cudaStreamSynchronize(s);
    return e ? cuda_fail(e) : MG_OK;
}

mg_status mg_op_prolong_sweep(int d, int n, mg_prec prec, const double *spai_coeffs, int ncoeffs,
                              const void *e_coarse, const void *u, const void *bh, void *u_out, double *u64_acc,
                              void *stream)
{
    double c[4];
    if (fused_args_ok(d, n, prec, spai_coeffs, ncoeffs, c) != MG_OK || !e_coarse || !u || !bh ||
        (!u_out && !u64_acc))
        return MG_EINVAL;
    const cudaStream_t s = (cudaStream_t)stream;
    const int nc = (n - 1) / 2;
    cudaError_t e = cudaSuccess;
    PaddedTmp tmp(d);
    float *pe = tmp.make(nc, e_coarse, s, e), *pu = tmp.make(n, u, s, e), *pb = tmp.make(n, bh, s, e);
    float *po = u64_acc ? nullptr : tmp.make(n, nullptr, s, e);
    if (!e) e = launch_prolong_sweep2d_pl(pu, pe, pb, po, u64_acc, n, c, s);
    if (!e && !u64_acc) e = tmp.pack(po, (float *)u_out, n, false, s);
    if (!e) e = cudaStreamSynchronize(s);
    return e ? cuda_fail(e) : MG_OK;
}

mg_status mg_op_coarse_solve(int d, mg_prec prec, const void *bh, void *x_out, void *stream)
{
    if ((d != 2 && d != 3) || !bh || !x_out || (prec != MG_FP64 && prec != MG_FP32_IR)) return MG_EINVAL;
    double lu[27 * 27];
    coarse_inverse(d, lu);
    double *dlu = nullptr;
    cudaError_t e = cudaMalloc(&dlu, sizeof lu);
    if (e) return cuda_fail(e);
    e = cudaMemcpy(dlu, lu, sizeof lu, cudaMemcpyHostToDevice);
    TailArgs a;
    memset(&a, 0, sizeof a);
    a.d = d;
    a.lu = dlu;
    a.lv[0] = tail_level(x_out, nullptr, (void *)bh, nullptr, 3);
    a.ops[0].kind = TAIL_SOLVE;
    a.ops[0].level = 0;
    a.nops = 1;
    if (!e) e = prec == MG_FP64 ? launch_tail<double>(a, (cudaStream_t)stream) : launch_tail<float>(a, (cudaStream_t)stream);
    if (!e) e = cudaStreamSynchronize((cudaStream_t)stream);
    cudaFree(dlu);
    return e ? cuda_fail(e) : MG_OK;
}

const char *mg_strerror(mg_status s)
{
    switch (s) {
    case MG_OK: return "success";
    case MG_EINVAL: return "invalid argument";
    case MG_ENOMEM: return "out of memory";
    case MG_ECUDA: return "CUDA error";
    case MG_ENOCONV: return "not converged within max_cycles";
    case MG_ENAN: return "residual norm is NaN or Inf";
    case MG_ETIMEOUT: return "device-side wait timed out";
    }
    return "unknown status";
}

const char *mg_last_cuda_error(void) { return g_last_error; }

unsigned long long mg_kernel_launch_count(void) { return g_launches.load() + registered_launches(); }

}  // extern "C"
