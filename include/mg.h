/*
 * mg.h -- C ABI of the GB300 (sm_103a) geometric-multigrid library for the
 * Dirichlet Poisson problem with the SPAI smoothers of He, Liu and Wang,
 * "Optimized sparse approximate inverse smoothers for solving Laplacian
 * linear systems" (arXiv:2206.05543).
 *
 * Problem (Sec. 1, Eqs. (1.1)-(1.3)): A_h u_h = b_h on the interior points of
 * (0,1)^d, d = 2 (5-point stencil) or d = 3 (7-point stencil), h = 1/N, N a
 * power of two >= 4. Non-zero boundary data g is folded into b by the caller.
 *
 * Smoother (Sec. 2, Eq. (2.1)): u <- u + omega M_h (b_h - A_h u) with M_h a
 * symmetric stencil proportional to h^2 (Sec. 3). The library takes the
 * omega-folded, h-free weights
 *     2D: c = (c0, c1, c2)     = omega * (centre, edge, corner) / h^2
 *     3D: c = (c0, c1, c2, c3) = omega * (centre, face, edge, corner) / h^2
 * e.g. M9 = Upsilon(44,10,3)/24 with omega = (309 - 12 sqrt 10)/1720
 * (Theorem 3.1) gives c = omega*(44, 10, 3)/24; M7 = T(8/5, 2/5) with
 * omega = 20/73 (Theorem 3.2) gives c = (16/73, 2/73). Fewer weights than
 * the maximum leave the rest zero (Jacobi: one weight, M5 and M7: two). A 3D
 * M with a non-zero edge or corner weight is the symmetric 27-point stencil
 * (19-point without corners) that Sec. 3.2 mentions as a wider SPAI
 * smoother; it runs on the FP64 and plain FP32 cycles (MG_FP64, MG_FP32) and
 * the FP64 single operators; MG_FP32_IR contexts and the adjoint take the
 * 7-point M only (MG_EINVAL otherwise).
 *
 * Cycle (Sec. 4): re-discretised coarse operators (H = 2h), full-weighting
 * restriction, bilinear/trilinear interpolation, nu1 pre- and nu2
 * post-smoothing sweeps, coarsest grid h0 = 1/4 solved exactly, stopping on
 * ||b - A u_k||_2 <= tol ||b - A u_0||_2.
 *
 * Layout of every grid array crossing this ABI: interior points only,
 * row-major with x fastest, (N-1)^d elements: a[y*(N-1) + x] in 2D,
 * a[(z*(N-1) + y)*(N-1) + x] in 3D; index i is the grid point (i+1)h.
 * Grid arrays are DEVICE pointers unless stated otherwise; the caller owns
 * them, and they must stay valid until the work queued on the context's
 * stream has finished.
 *
 * Errors: every call returns an mg_status; no exception crosses the ABI.
 * On MG_ECUDA the CUDA error text is available from mg_last_cuda_error().
 * All work runs on the stream given to mg_setup; calls that return numbers
 * to the host (norms, cycle counts) synchronise that stream.
 */
#ifndef MG_H
#define MG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_ctx mg_ctx; /* opaque; owns every coarse-level buffer */

typedef enum {
    MG_OK = 0,
    MG_EINVAL = -1,   /* bad argument: d, N, weights, nu, null pointer ... */
    MG_ENOMEM = -2,   /* device or pinned host allocation failed */
    MG_ECUDA = -3,    /* a CUDA runtime call or kernel launch failed */
    MG_ENOCONV = -4,  /* max_cycles ran out; u and the history are still written */
    MG_ENAN = -5,     /* the residual norm became NaN or Inf */
    MG_ETIMEOUT = -6  /* a bounded device-side wait gave up */
} mg_status;

typedef enum {
    MG_FP64 = 0,    /* every level and every operation in FP64; u, b are double */
    MG_FP32_IR = 1, /* FP32 cycle inside FP64 iterative refinement: the outer
                       residual b - A u and the update u += e in FP64; u, b double */
    MG_FP32 = 2     /* every level and every operation in FP32; u, b are float */
} mg_prec;

/* ---------------------------------------------------------------------- */
/* solver context                                                         */
/* ---------------------------------------------------------------------- */

/* Create a solver for dimension d (2 or 3) and grid N (power of two, >= 4).
 * spai_coeffs: HOST array of ncoeffs omega-folded weights (see above;
 * 1..3 in 2D, 1..4 in 3D). nu1, nu2 >= 0 sweeps, nu1 + nu2 >= 1.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Allocates the level hierarchy on the current device. MG_EINVAL, MG_ENOMEM
 * or MG_ECUDA on failure (*out is then NULL). */
mg_status mg_setup(int d, int N, const double *spai_coeffs, int ncoeffs, int nu1, int nu2,
                   mg_prec prec, void *cuda_stream, mg_ctx **out);

/* Like mg_setup, with gamma coarse-grid visits per level: 1 = V cycle,
 * 2 = W cycle (Sec. 4 tests W(1+0) and V(1+1)). */
mg_status mg_setup_ex(int d, int N, const double *spai_coeffs, int ncoeffs, int nu1, int nu2,
                      int gamma, mg_prec prec, void *cuda_stream, mg_ctx **out);

/* One cycle in place on u for right-hand side b (device arrays, (N-1)^d,
 * double for MG_FP64 / MG_FP32_IR, float for MG_FP32). MG_FP64, MG_FP32: one
 * V/W cycle. MG_FP32_IR: one refinement step (FP64 residual, FP32 cycle for
 * the correction, FP64 update). Asynchronous. */
mg_status mg_vcycle(mg_ctx *ctx, void *u, const void *b);

/* Solve from the initial guess in u until ||b - A u_k||_2 <= tol ||b - A u_0||_2
 * or max_cycles cycles ran (Sec. 4). b, u: device arrays of the context's
 * type (see mg_vcycle); residual norms are accumulated in FP64. cycles_out,
 * relres_out (= ||r_k||/||r_0||): nullable HOST pointers. hist_out: nullable
 * HOST array of max_cycles + 1 doubles receiving ||r_k||_2, k = 0..cycles.
 * Returns MG_OK, MG_ENOCONV (u and outputs still written) or MG_ENAN.
 * Synchronises the stream once per cycle: the host applies the stop test
 * (see mg_solve_async for the same solve with the test on the device). */
mg_status mg_solve(mg_ctx *ctx, const void *b, void *u, double tol, int max_cycles, int *cycles_out,
                   double *relres_out, double *hist_out);

/* mg_solve with options. flags: 0 or MG_SOLVE_ZERO_START: the initial guess
 * is zero and u is output only (its prior contents are never read). The
 * first cycle then starts with the from-zero form of its first operation (a
 * sweep of u = 0, or for MG_FP32_IR the residual h^2 b rounded to FP32 once),
 * which gives the same iterates as a solve from an explicitly zeroed u (up to
 * the sign of exact zeros) without the FP64 work of A u_0. Other bits:
 * MG_EINVAL. */
#define MG_SOLVE_ZERO_START 1u
mg_status mg_solve_ex(mg_ctx *ctx, const void *b, void *u, double tol, int max_cycles, unsigned flags,
                      int *cycles_out, double *relres_out, double *hist_out);

/* The outcome of a solve, as the device writes it. */
typedef struct mg_solve_info {
    double r0;   /* ||b - A u_0||_2 */
    double rk;   /* ||b - A u_k||_2 after the last cycle (relres = rk / r0) */
    int cycles;  /* k */
    int status;  /* MG_OK, MG_ENOCONV, MG_ENAN or MG_ETIMEOUT */
} mg_solve_info;

/* mg_solve_ex without any synchronisation: the whole solve, its stop test
 * included, is queued on the context's stream (after the work queued on the
 * caller's stream so far; the caller's stream waits for it) and the call
 * returns. info: DEVICE-ACCESSIBLE memory (device memory, or page-locked host
 * memory on a system with unified addressing), written when the solve ends;
 * it must stay valid until then. hist: nullable device-accessible array of
 * max_cycles + 1 doubles (||r_k||_2, k = 0..cycles). The cycles and the stop
 * test run on the device: a CUDA graph whose conditional loop node repeats
 * the cycle while a one-thread kernel finds the test unmet; nothing is
 * written to host memory before the solve ends. Iterates, cycle count and
 * history equal mg_solve_ex's bit for bit. The return value reports errors found before
 * queueing (arguments, graph recording); the solve's own status is
 * info->status. Solves queued back to back on one context run one after the
 * other; their arrays may differ (the graphs of the last few (u, b) pairs
 * are kept). */
mg_status mg_solve_async(mg_ctx *ctx, const void *b, void *u, double tol, int max_cycles, unsigned flags,
                         mg_solve_info *info, double *hist);

/* ||b - A_h u||_2 of device arrays u, b (context's type, norm accumulated in
 * FP64); result in *norm_out (HOST). */
mg_status mg_residual_norm(mg_ctx *ctx, const void *u, const void *b, double *norm_out);

void mg_destroy(mg_ctx *ctx);

/* Replace the omega-folded weights of a context (HOST array, same rules as
 * mg_setup); the recorded cycle is re-recorded on the next call. */
mg_status mg_set_coeffs(mg_ctx *ctx, const double *spai_coeffs, int ncoeffs);

/* MG_FP32_IR contexts and batched contexts: the number of FP32 cycles per
 * refinement iteration (1..8; default 1). Each iteration still forms
 * r = b - A u in FP64 once, rounds it to FP32, runs `cycles` FP32 cycles on
 * A e = r from e = 0 (the later ones starting from the current e) and adds e
 * to u in FP64; more cycles per iteration mean fewer FP64 residuals per
 * solve (the residual reduction per iteration is about the cycle's
 * contraction to that power). MG_EINVAL for other precisions, and for
 * batched contexts with cycles > 1 unless nu1 + nu2 is even and every
 * N >= 32. Single-problem contexts re-record on the next call; batched
 * contexts re-record here (synchronises). */
mg_status mg_set_refinement_cycles(mg_ctx *ctx, int cycles);

/* ---------------------------------------------------------------------- */
/* batched solves (many right-hand sides, uneven grid sizes)              */
/* ---------------------------------------------------------------------- */

/* A context for `count` independent 2D problems with grid sizes Ns[0..count-1]
 * (HOST array; each a power of two, 4 <= N <= 32768), solved by FP32 V(nu1,nu2)
 * cycles inside FP64 iterative refinement (prec must be MG_FP32_IR; d must
 * be 2; 1 <= nu1 <= 4, 0 <= nu2 <= 4). The cycles of all problems are aligned
 * by grid size (Sec. 4 cycle): one launch per operator and size serves every
 * problem that has a level of that size; the levels with at most 15 points
 * per axis run in one block per problem. The row-chunk height of each launch
 * is chosen by timing at setup (cached per device and size; persisted when
 * the environment variable MG_AUTOTUNE_CACHE names a file). */
mg_status mg_setup_batched(int d, int count, const int *Ns, const double *spai_coeffs, int ncoeffs,
                           int nu1, int nu2, mg_prec prec, void *cuda_stream, mg_ctx **out);

/* Solve every problem i to ||b_i - A u_i||_2 <= tol ||b_i - A u_i^0||_2:
 * b[i], u[i] are device FP64 arrays ((Ns[i]-1)^2, u[i] holds the initial
 * guess), passed as HOST arrays of device pointers. A problem that has
 * converged is masked out of later iterations. cycles_out, relres_out:
 * nullable HOST arrays of count entries. MG_OK when all converged,
 * MG_ENOCONV if some ran out of max_cycles, MG_ENAN if some norm became
 * NaN/Inf. Synchronises once per refinement iteration. */
mg_status mg_solve_batched(mg_ctx *ctx, const void *const *b, void *const *u, double tol, int max_cycles,
                           int *cycles_out, double *relres_out);

/* mg_solve_batched with options (see mg_solve_ex): MG_SOLVE_ZERO_START: every
 * initial guess is zero and the u[i] are output only; the first residuals
 * are h^2 b_i rounded to FP32 without FP64 work. Same iterates as from
 * explicitly zeroed u[i] (up to the sign of exact zeros). */
mg_status mg_solve_batched_ex(mg_ctx *ctx, const void *const *b, void *const *u, double tol, int max_cycles,
                              unsigned flags, int *cycles_out, double *relres_out);

/* ---------------------------------------------------------------------- */
/* adjoint of K cycles                                                    */
/* ---------------------------------------------------------------------- */

/* Reverse-mode derivative of u_K = K cycles from u_0 = 0 for right-hand
 * side b (the transpose of each step of Sec. 4's cycle: the sweep
 * u' = u + W (bh - Ah u) of Eq. (2.1) becomes g <- g - Ah (W g) with
 * dL/dbh += W g and dL/dc_j += <g, N_j rh>; restriction and interpolation
 * swap roles, R^T = P / 2^d; the coarsest solve is symmetric).
 * Inputs: b and grad_uK = dL/du_K, device arrays of the context's type
 * (double for MG_FP64, float for MG_FP32; MG_FP32_IR is rejected).
 * Outputs: grad_b_out = dL/db (device, same type) and grad_coeffs_out =
 * dL/dc (HOST, ncoeffs doubles, summed over every sweep of every level and
 * cycle, accumulated in FP64). Requires a V cycle (gamma = 1), nu1 >= 1, N >= 8
 * and, in 3D, a context made with at most 2 weights (the 7-point M).
 * Checkpointing: a first forward pass keeps only the cycle inputs
 * u_1 .. u_{K-1}; each cycle is replayed from its input just before it is
 * reversed, keeping per level the inputs of that visit's sweeps and its
 * right-hand side. Device workspace (owned by the context, allocated on the
 * first call for a given K, size from mg_adjoint_workspace_bytes):
 * (K - 1) finest fields + per level (nu1 + nu2 + 5) fields (the finest
 * nu1 + nu2 + 4, the coarsest 6) + 24 bytes per block of the reverse sweeps;
 * e.g. 3D N = 512 FP64, K = 4, V(1,1): about 11 GB. The evaluation is
 * recorded into a CUDA graph and replayed while b, grad_uK and grad_b_out
 * stay the same arrays. Synchronises. */
mg_status mg_vcycles_adjoint(mg_ctx *ctx, int K, const void *b, const void *grad_uK, void *grad_b_out,
                             double *grad_coeffs_out);

/* Device bytes of the workspace mg_vcycles_adjoint uses for K cycles on this
 * context (HOST *bytes_out). No GPU work. */
mg_status mg_adjoint_workspace_bytes(mg_ctx *ctx, int K, unsigned long long *bytes_out);

/* ---------------------------------------------------------------------- */
/* single operators on one level (each step of the cycle, for checking)    */
/* ---------------------------------------------------------------------- */
/* n = points per axis of the level (N_l - 1, odd, >= 3); arrays in the
 * interior layout of that level, device pointers. prec selects the element
 * type: MG_FP64 -> double, MG_FP32_IR -> float. bh is the scaled right-hand
 * side h_l^2 b_l unless b_unscaled != 0, in which case b is unscaled and the
 * kernel forms h^2 b itself (h = 1/(n+1)). stream: cudaStream_t.
 * These are checking paths, not the solver's hot path: they allocate
 * temporaries with cudaMalloc and synchronise the stream whenever they return
 * a number to the host (a norm), run an FP32 operator (the FP32 kernels work
 * on zero-ringed padded copies made for the call) or solve the coarsest grid
 * (a copy of the exact inverse); only the FP64 operators without a norm are
 * asynchronous and allocation-free. */

/* One SPAI sweep u_out = u + W (bh - h^2 A u) (Sec. 2, Eq. (2.1)); u == NULL
 * means u = 0. If rnorm2_out (HOST) is non-NULL it receives the sum of the
 * squared scaled residuals h^4 |b - A u|^2 of the input u; this synchronises. */
mg_status mg_op_sweep(int d, int n, mg_prec prec, const double *spai_coeffs, int ncoeffs, const void *u,
                      const void *bh, int b_unscaled, void *u_out, double *rnorm2_out, void *stream);

/* Scaled residual rh = bh - h^2 A u (Sec. 1, Eq. (1.3)). */
mg_status mg_op_residual(int d, int n, mg_prec prec, const void *u, const void *bh, int b_unscaled,
                         void *rh_out, void *stream);

/* The outer step of the FP32-in-FP64 refinement: the scaled residual
 * rh = bh - h^2 A u (Sec. 1, Eq. (1.3)) of FP64 u and bh, evaluated in FP64
 * in the order of mg_op_residual and rounded once to FP32 (round to nearest,
 * ties to even) into rh32_out, the right-hand side of the FP32 cycle. u, bh:
 * double, rh32_out: float, all device arrays of n^d points (interior
 * layout). If rnorm2_out (HOST) is non-NULL it receives sum(rh^2) of the
 * FP64 residual, summed in FP64; this synchronises. */
mg_status mg_op_residual_refine(int d, int n, const double *u, const double *bh, int b_unscaled, float *rh32_out,
                                double *rnorm2_out, void *stream);

/* Coarse right-hand side bh_c = 4 R (bh - h^2 A u), full weighting R
 * (Sec. 4); bh_c has ((n-1)/2)^d points. */
mg_status mg_op_residual_restrict(int d, int n, mg_prec prec, const void *u, const void *bh, int b_unscaled,
                                  void *bh_coarse_out, void *stream);

/* u += P e, P = bilinear/trilinear interpolation of the coarse correction
 * e (((n-1)/2)^d points) (Sec. 4), in place on u. */
mg_status mg_op_prolong_correct(int d, int n, mg_prec prec, const void *e_coarse, void *u, void *stream);

/* The two temporally blocked passes of a V(1,1) visit of an FP32 2D level
 * (the FP32 cycles of MG_FP32_IR contexts run them), for checking against
 * the single steps; d must be 2, prec MG_FP32_IR (float arrays), n >= 7,
 * 1..3 weights, bh scaled. Results equal the unfused steps bit for bit.
 * mg_op_sweep_restrict: u_out = one SPAI sweep of u (Sec. 2, Eq. (2.1);
 * u == NULL: from zero) and bh_coarse_out = 4 R (bh - h^2 A u_out), full
 * weighting R (Sec. 4), ((n-1)/2)^2 points. */
mg_status mg_op_sweep_restrict(int d, int n, mg_prec prec, const double *spai_coeffs, int ncoeffs, const void *u,
                               const void *bh, void *u_out, void *bh_coarse_out, void *stream);

/* mg_op_prolong_sweep: v = u + P e_coarse (bilinear interpolation and
 * correction, Sec. 4), then one SPAI sweep of v (Sec. 2, Eq. (2.1)) into
 * u_out (float); if u64_acc (DEVICE, n^2 doubles, compact) is non-NULL the
 * sweep's result is instead added to it in FP64 (the update of the FP64
 * solution that ends an FP32 refinement cycle) and u_out may be NULL. */
mg_status mg_op_prolong_sweep(int d, int n, mg_prec prec, const double *spai_coeffs, int ncoeffs,
                              const void *e_coarse, const void *u, const void *bh, void *u_out, double *u64_acc,
                              void *stream);

/* Exact solve of h0^2 A_h0 x = bh on the coarsest grid (n = 3, 3^d points). */
mg_status mg_op_coarse_solve(int d, mg_prec prec, const void *bh, void *x_out, void *stream);

/* One SPAI sweep with the squared residual norm of its input, allocating
 * nothing. The paper has no counterpart: this is a service for callers that
 * cannot call cudaMalloc -- code confined to a framework's own memory pool
 * (whose caching allocator owns the device heap), services with a device
 * memory budget fixed at start-up, or loops that cannot afford the
 * device-wide synchronisation of cudaMalloc/cudaFree.
 * Arguments as for mg_op_sweep, except that the norm goes to DEVICE memory:
 * rnorm2_dev_out (one double, caller-owned) receives sum(rh^2) of the input
 * u, written by a kernel on `stream`; nothing is copied to the host and the
 * call does not synchronise.
 * Scratch: the per-block partial sums live in a fixed 256 KiB array in device
 * memory inside the library (every GPU that loads the library holds it until
 * the process exits). Sizes beyond it are rejected with MG_EINVAL before any
 * CUDA work: n <= 16383 in 2D, n <= 1023 in 3D (and at most 32768 blocks).
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.
 * All calls share the one array: calls whose work overlaps on the GPU (other
 * streams, other threads) race on it and must be serialised by the caller.
 * Every block overwrites its own partial sum, so no clearing is needed. */
mg_status mg_op_sweep_norm_noalloc(int d, int n, mg_prec prec, const double *spai_coeffs, int ncoeffs,
                                   const void *u, const void *bh, int b_unscaled, void *u_out,
                                   double *rnorm2_dev_out, void *stream);

/* ---------------------------------------------------------------------- */
/* diagnostics                                                            */
/* ---------------------------------------------------------------------- */
const char *mg_strerror(mg_status status);
const char *mg_last_cuda_error(void);
/* Number of kernels the library launched (directly or as graph nodes)
 * since the process started; graph replays count every node. The kernels of
 * a solve's device-side cycle loop are counted by the device and appear here
 * once they have run. */
unsigned long long mg_kernel_launch_count(void);

/* Measured issue rate of the FP64 pipe on the current device, for the
 * roofline of the FP64 kernels (which are bound by that pipe, not by HBM).
 * The paper has no counterpart. One wave of blocks runs 8 independent chains
 * per thread of one instruction kind: 0 = DFMA with all operands in
 * registers, 1 = DADD, 2 = DMUL, 3 = DFMA with one operand from the constant
 * bank. *ops_per_sm_clk (HOST) receives thread-level operations per SM per
 * SM clock (the nominal rate of this part is 2); *sm_mhz (HOST, nullable) the
 * SM clock seen during the run (cycles / elapsed time). Allocates a few
 * bytes and synchronises; takes tens of milliseconds. */
mg_status mg_measure_fp64_rate(int kind, double *ops_per_sm_clk, double *sm_mhz);

/* Test hook for the bounded device-side waits (the TMA-staged 3D FP32
 * kernels wait on mbarriers for their copies). The next `launches` such
 * launches make their first copy's barrier expect 16 bytes more than the copy
 * delivers, so that wait expires after its bound (about one second); the
 * block then records the expiry, drains its other copies and returns, and
 * the synchronising call that follows reports MG_ETIMEOUT. Nothing faults,
 * traps or hangs. A launch armed while a cycle is being recorded into the
 * context's CUDA graph stays armed in every replay of that graph. 0 disarms;
 * returns the number of launches still armed before the call. */
int mg_test_arm_wait_expiry(int launches);

#ifdef __cplusplus
}
#endif
#endif /* MG_H */
