// mg_internal.h -- declarations shared by the library's translation units
// (launchers of the kernels, launch accounting, device properties).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

namespace mg {

// Streaming multiprocessors of the current device (grid sizing only).
int num_sms();
// Launch accounting behind mg_kernel_launch_count().
void count_launch(unsigned long long k);

// Rows per block for the marching kernels: enough blocks to fill the GPU
// (target_blocks), clamped to [lo, hi].
inline int chunk_rows(int nblk_x, int nrows, int target_blocks, int lo, int hi)
{
    long want = ((long)nblk_x * nrows + target_blocks - 1) / target_blocks;
    return (int)std::min<long>(std::max<long>(want, lo), hi);
}

struct Grid2 {
    int bx, by, H;
};
Grid2 sweep2d_grid(int n);

// 2D level operators; arrays in the interior layout of a level with n points
// per axis. c = omega-folded weights (c0, c1, c2). u == nullptr: u = 0.
// partials != nullptr: one squared-residual partial sum per block
// (sweep2d_grid(n).bx * .by doubles).
template <typename T>
cudaError_t launch_sweep2d(const T *u, const T *b, bool unscaled, T *out, int n, const double *c,
                           double *partials, cudaStream_t s);
template <typename T>
cudaError_t launch_resrestrict2d(const T *u, const T *b, bool unscaled, T *bc, int n, cudaStream_t s);
template <typename T>
cudaError_t launch_prolong2d(const T *e, T *u, int n, cudaStream_t s);

// Scaled residual rh = bh - h^2 A u in InT (bh = h^2 b formed in the kernel
// when `unscaled`), written as OutT when rh != nullptr, plus squared partial
// sums (one per block of sweep2d_grid(n)) when partials != nullptr.
template <typename InT, typename OutT>
cudaError_t launch_residual2d(const InT *u, const InT *b, bool unscaled, OutT *rh, int n, double *partials,
                              cudaStream_t s, long out_pitch = 0, long out_off = 0);

struct Grid3 {
    int bx, by, bz, Z;
};
// persistent 3D sweep: bx x bx tiles x n planes = total items, `per` per block;
// resident blocks per SM by element size (FP64 2: no register cap that forces
// spills; FP32 4)
struct S3Plan {
    int bx, blocks;
    long total, per;
};
constexpr int sweep3d_blocks_per_sm(int elem_bytes) { return elem_bytes == 8 ? 2 : 3; }
S3Plan sweep3d_plan(int n, int elem_bytes);
Grid3 residual3d_grid(int n);

// 3D level operators (same conventions as the 2D ones; c = (c0, c1, c2, c3):
// centre, face, edge, corner weights; the sweep takes the 27-point form when
// c2 or c3 is non-zero).
template <typename T>
cudaError_t launch_sweep3d(const T *u, const T *b, bool unscaled, T *out, int n, const double *c,
                           double *partials, cudaStream_t s);
template <typename T>
cudaError_t launch_resrestrict3d(const T *u, const T *b, bool unscaled, T *bc, int n, cudaStream_t s);
template <typename T>
cudaError_t launch_prolong3d(const T *e, T *u, int n, cudaStream_t s);
template <typename InT, typename OutT>
cudaError_t launch_residual3d(const InT *u, const InT *b, bool unscaled, OutT *rh, int n, double *partials,
                              cudaStream_t s, long out_pitch = 0, long out_plane = 0, long out_off = 0);

// ---- batched 2D operators (one launch per grid size across problems) -------
template <typename T>
struct BItem {  // one problem's level in a batched launch
    const T *u;   // input (sweep), residual input (restrict), coarse e (interpolation)
    const T *b;   // scaled right-hand side of the level
    T *out;       // sweep output, coarse rhs (restrict), fine u corrected in place (interpolation)
    int problem;  // index into the active flags
    int flags;    // bit 0: b is the unscaled caller array
};
template <typename OutT>
struct BRes {  // FP64 residual of one problem's caller arrays
    const double *u, *b;
    OutT *out;
    double *partials;  // residual2d_batched_tiles(n) partial sums
    int problem, pad;
};
template <typename OutT>
cudaError_t launch_residual2d_batched(const BRes<OutT> *tab, int nprob, const int *active, int n, cudaStream_t s,
                                      long opitch = 0, long ooff = 0);
// The batched FP64 residual of every finest size in one persistent launch:
// group g holds the problems whose finest level has n points per axis (table
// tab), its items are item0 .. item0 + nprob * bx * by - 1, written to the
// padded FP32 layout (pitch, off) of that size. Groups in descending n.
struct BResGroup {
    const BRes<float> *tab;
    long pitch, off;
    int n, H, bx, by, hk, item0;
};
// fills g's launch geometry from g.n; returns its item count for nprob problems
int residual2d_batched_group(BResGroup &g, int nprob);
cudaError_t launch_residual2d_batched_all(const BResGroup *groups, int ngroups, int items, const int *active,
                                          cudaStream_t s);
// the same items for u = 0 (rh = h^2 b rounded to FP32, norm partials), every problem
cudaError_t launch_residual2d_batched_zero(const BResGroup *groups, int ngroups, int items, cudaStream_t s);
int residual2d_batched_tiles(int n);
// mode 0: every item from its u; 1: from zero; 2: per item (u == nullptr: from zero)
cudaError_t launch_sweep2d_pl_batched(const BItem<float> *tab, int nprob, const int *active, int n, int H, int mode,
                                      const double *c, cudaStream_t s);
cudaError_t launch_resrestrict2d_pl_batched(const BItem<float> *tab, int nprob, const int *active, int n, int Hc,
                                            cudaStream_t s);
cudaError_t launch_prolong2d_pl_batched(const BItem<float> *tab, int nprob, const int *active, int n, int Hc,
                                        cudaStream_t s);

// ---- padded FP32 layout (mg_pl2d.cu) ---------------------------------------
// A level with n points per axis stored with a zero ghost ring and padded,
// 16-byte-aligned rows: element (x, y), x, y in [-1, n], at off + y*pitch + x.
struct Pitch2 {
    int n, pitch, rows;
    long off;
};
Pitch2 pitch2(int n);
size_t pitch2_floats(int n);
cudaError_t launch_sweep2d_pl(const float *u, const float *b, float *out, int n, const double *c, double *partials,
                              cudaStream_t s);
cudaError_t launch_resrestrict2d_pl(const float *u, const float *b, float *bc, int n, cudaStream_t s);
cudaError_t launch_prolong2d_pl(const float *e, float *u, int n, cudaStream_t s);
cudaError_t launch_pack2d(const float *in, float *out, int n, bool to_padded, cudaStream_t s);
cudaError_t launch_add_pl2d(double *u, const float *e, int n, cudaStream_t s);
cudaError_t launch_sweep2d_pl_acc64(const float *u, const float *b, double *u64, int n, const double *c, cudaStream_t s);
int sweep2d_pl_blocks(int n, int H);
// temporally blocked V(1,1) passes (mg_fused2d.cu), bit-identical to the
// unfused kernels: (A) u1 = sweep of u0 (nullptr: from zero) and
// bc = 4 R (bh - A u1); (B) out = sweep of u1 + P e, or, with u64 != nullptr,
// u64 (compact FP64) += that sweep (out unused)
cudaError_t launch_sweep_restrict2d_pl(const float *u0, const float *bh, float *u1, float *bc, int n, const double *c,
                                       cudaStream_t s);
cudaError_t launch_prolong_sweep2d_pl(const float *u1, const float *e, const float *bh, float *out, double *u64, int n,
                                      const double *c, cudaStream_t s);
// batched forms (one launch per level size across problems)
struct FItem {
    const float *u;  // A: start (nullptr: zero); B: the pre-smoothed field
    const float *e;  // B: the coarse correction
    const float *b;  // the level's scaled right-hand side
    float *out;      // A: the smoothed field; B: the visit's result
    float *out2;     // A: the coarse right-hand side
    int problem, pad;
};
cudaError_t launch_sweep_restrict2d_pl_batched(const FItem *tab, int nprob, const int *active, int n, int Hc,
                                               const double *c, cudaStream_t s);
cudaError_t launch_prolong_sweep2d_pl_batched(const FItem *tab, int nprob, const int *active, int n, int H,
                                              const double *c, cudaStream_t s);

// 3D: element (x, y, z), each in [-1, n], at off + z*plane + y*pitch + x.
struct Pitch3 {
    int n, pitch;
    long plane, off;
};
Pitch3 pitch3(int n);
size_t pitch3_floats(int n);
// SPAI sweep with TMA-staged tiles; u == nullptr: zero start. A copy that
// does not land within about a second sets *err (device int) to nonzero.
cudaError_t launch_sweep3d_tma(const float *u, const float *b, float *out, int n, const double *c, int *err,
                               cudaStream_t s);
// the same sweep with the refinement epilogue u64 (compact FP64) += result
cudaError_t launch_sweep3d_tma_acc64(const float *u, const float *b, double *u64, int n, const double *c, int *err,
                                     cudaStream_t s);
// residual + full weighting on TMA-staged planes (*err as for the sweep)
cudaError_t launch_resrestrict3d_tma(const float *u, const float *b, float *bc, int n, int *err, cudaStream_t s);
cudaError_t launch_prolong3d_pl(const float *e, float *u, int n, cudaStream_t s);
cudaError_t launch_pack3d(const float *in, float *out, int n, bool to_padded, cudaStream_t s);
cudaError_t launch_add_pl3d(double *u, const float *e, int n, cudaStream_t s);
int sweep2d_pl_H(int n);

// ---- coarse tail (one block runs the last levels of a cycle) --------------
constexpr int kTailThreads = 256;
constexpr int kMaxTailLevels = 8;
constexpr int kMaxTailOps = 480;
enum TailOpKind : int { TAIL_ZERO = 0, TAIL_SWEEP = 1, TAIL_RESTRICT = 2, TAIL_SOLVE = 3, TAIL_PROLONG = 4 };
struct TailLevel {
    void *u, *tmp, *bh, *rh;  // element type = the kernel's T
    int n, pitch;             // element (x, y, z) at off + z*plane + y*pitch + x
    long plane, off;          // compact: pitch = n, plane = n*n, off = 0
};
struct TailOp {
    short kind, level;  // level indexes TailArgs::lv
};
struct TailArgs {
    TailLevel lv[kMaxTailLevels];
    TailOp ops[kMaxTailOps];
    double c[4];  // 2D: centre, edge, corner; 3D: centre, face, edge, corner
    const double *lu;  // exact inverse of the coarsest operator (device, coarse_inverse)
    int d, nops;
};
inline TailLevel tail_level(void *u, void *tmp, void *bh, void *rh, int n)
{
    TailLevel t;
    t.u = u;
    t.tmp = tmp;
    t.bh = bh;
    t.rh = rh;
    t.n = n;
    t.pitch = n;
    t.plane = (long)n * n;
    t.off = 0;
    return t;
}
template <typename T>
cudaError_t launch_tail(const TailArgs &a, cudaStream_t s);
// lv: count x kMaxTailLevels levels; problem p runs ops[op_off[p] .. + op_cnt[p]]
template <typename T>
cudaError_t launch_tail_batched(const TailLevel *lv, const TailOp *ops, const int *op_off, const int *op_cnt,
                                const int *active, int count, int d, const double *c, const double *lu, cudaStream_t s);
// exact inverse of h0^2 A_h0 (m x m row-major, m = 3^d) for the coarsest solve
void coarse_inverse(int d, double *inv);

// ---- small helpers (mg_host.cu) -------------------------------------------
cudaError_t launch_sum_partials(const double *partials, int np, double *out, cudaStream_t s);
// Zero / copy `bytes` (a multiple of 4; 4-byte aligned pointers) with a
// kernel. The solve paths use these instead of cudaMemsetAsync and
// cudaMemcpyAsync, which a copy engine may run and queue behind a caller's
// large host transfer on the same engine.
cudaError_t launch_zero_words(void *p, size_t bytes, cudaStream_t s);
cudaError_t launch_copy_words(void *dst, const void *src, size_t bytes, cudaStream_t s);
template <typename T>
cudaError_t launch_add_to_f64(double *u, const T *e, size_t np, cudaStream_t s);
template <typename T>
cudaError_t launch_scale_copy(const double *b, T *bh, size_t np, double h2, cudaStream_t s);

}  // namespace mg
