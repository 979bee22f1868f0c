// mg_ctx.h -- the solver context shared by the host translation units
// (cycle recording in mg_host.cu, the adjoint in mg_adjoint.cu).
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <vector>

#include "../../include/mg.h"

// device workspace of the adjoint (allocated on first use for a given K):
// the cycle inputs u_1 .. u_{K-1} (finest level), and per level the inputs of
// the sweeps of the cycle being reversed, that level's right-hand side and
// the adjoint fields; the whole evaluation is recorded into one CUDA graph
struct AdjointWork {
    int K = 0;
    std::vector<void *> ck;                    // [k], k = 1 .. K-1 (ck[0] unused: u_0 = 0)
    std::vector<std::vector<void *>> sw;       // [level][sweep]: outputs of the visit's sweeps
    std::vector<void *> bh;                    // [level], level >= 1
    std::vector<void *> G, GB, T;              // per level
    double *partials = nullptr;                // per-block coefficient partials of every reverse sweep
    size_t npartials = 0;                      // doubles
    double *acc = nullptr;                     // 3 coefficient gradients (device)
    double *h_acc = nullptr;                   // pinned copy
    cudaGraphExec_t graph = nullptr;
    unsigned long long nodes = 0;
    const void *cap_b = nullptr, *cap_g = nullptr, *cap_gb = nullptr;
    size_t bytes = 0;                          // device bytes of this workspace
    std::vector<void *> owned;
};

struct BatchWork;  // mg_batched.cu

struct GraphPair {
    cudaGraphExec_t pre = nullptr, rest = nullptr;
    cudaGraphExec_t meas = nullptr;  // residual norm only (plain cycles with a fused pre graph)
    cudaGraphExec_t pre0 = nullptr;  // the first pre graph of a solve from u = 0 (u not read)
    // the cycle loop of a solve with its stop test on the device: conditional
    // nodes around rest, the norm step and one loop kernel per cycle
    cudaGraphExec_t loop = nullptr;
    unsigned long long pre_nodes = 0, rest_nodes = 0, meas_nodes = 0, pre0_nodes = 0;
    const void *cap_u = nullptr, *cap_b = nullptr;  // the arrays the graphs were recorded for
};

// The arguments of one solve, stored on the device by a kernel launched
// before the solve's graphs (stream-ordered, so solves queued back to back
// on one context do not share them).
struct LoopArgs {
    double tol;
    double *hist;          // device-accessible history, or null
    mg_solve_info *info;   // device-accessible result
    int max_cycles;
    int zero_start;
};

// the device-side loop's working state (device memory, one per context)
struct LoopState {
    LoopArgs a;
    double r0, rk, rprev;
    int k, status, guessing, guess, rerun;
    unsigned long long launched;  // kernels the loop graphs ran on this context
};

struct mg_ctx {
    int d = 2, N = 0, L = 0, nu1 = 1, nu2 = 1, gamma = 1, lt = 0, dev = 0;
    int inner = 1;  // FP32 cycles per refinement iteration (MG_FP32_IR)
    mg_prec prec = MG_FP64;
    double c[4] = {0, 0, 0, 0};  // omega-folded weights (3D: centre, face, edge, corner)
    int ncoef = 0;
    cudaStream_t user = nullptr, s = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // hierarchy in the cycle's precision (double or float); level 0 of an
    // FP64 context uses the caller's u and (unscaled) b for A and BH
    std::vector<int> n;
    std::vector<void *> A, B, BH, RH;
    size_t esize = 8;
    bool pl = false;  // FP32 levels in the padded layout (refinement, 2D)
    double *lu = nullptr;  // exact inverse of the coarsest operator (device)
    double *partials = nullptr;
    int npartials = 0;
    // d_norm2[0]: squared norm of the last residual; the word after it
    // (d_err) is set by a kernel whose bounded device-side wait gave up. Both
    // reach the host together (kNormBytes) in mapped pinned h_norm2, stored
    // there by the kernel that forms the sum (h_norm2_dev: its device address).
    double *d_norm2 = nullptr;
    double *h_norm2 = nullptr;  // mapped pinned
    unsigned long long *h_norm2_dev = nullptr;
    int *d_err = nullptr;
    bool norm_to_host = true;  // while recording: the pre graphs' norms also to h_norm2
    LoopState *d_loop = nullptr;
    // mapped pinned: the count of kernels the loop graphs ran
    unsigned long long *h_launched = nullptr, *h_launched_dev = nullptr;
    GraphPair g;                  // the graphs for the arrays of the last call
    std::vector<GraphPair> other; // graphs recorded for other arrays, oldest first
    std::vector<void *> owned;  // device allocations to free
    AdjointWork *adj = nullptr;
    BatchWork *batch = nullptr;  // set for batched contexts
};


namespace mg {
constexpr size_t kNormBytes = 2 * sizeof(double);
mg_status cuda_fail(cudaError_t e);
void free_adjoint(mg_ctx *c);
void free_batch(mg_ctx *c);
// batched contexts: FP32 cycles per refinement iteration (re-records the cycle graph)
mg_status batch_set_inner(mg_ctx *c, int inner);
// Record the work issued by body() on the context's stream into a CUDA graph;
// *nodes receives the number of kernels it launches per replay.
mg_status capture_graph(mg_ctx *c, cudaGraphExec_t *out, unsigned long long *nodes,
                        const std::function<cudaError_t()> &body);
// Capture the work issued by body() on the context's stream into graph g
// after the nodes in deps; on return deps holds the nodes the work ends with;
// *nodes (nullable) receives the number of kernels it launches.
cudaError_t capture_into(mg_ctx *c, cudaGraph_t g, std::vector<cudaGraphNode_t> &deps,
                         const std::function<cudaError_t()> &body, unsigned long long *nodes);
// Add a conditional node of the given type to g after deps (then deps =
// {node}); bodies[0 .. size-1] receive its body graphs.
cudaError_t add_conditional(cudaGraph_t g, std::vector<cudaGraphNode_t> &deps, cudaGraphConditionalHandle h,
                            cudaGraphConditionalNodeType type, unsigned size, cudaGraph_t *bodies);
}  // namespace mg
