// mg_batched.cu -- many independent 2D problems of uneven sizes solved
// together: FP32 V cycles inside FP64 iterative refinement (He, Liu, Wang,
// arXiv:2206.05543, Sec. 4 cycle).
//
// Every problem i has the levels N_i, N_i/2, ..., 4. The cycles of all
// problems are aligned by grid size: going down, the launch for size s covers
// every problem with N_i >= s (for those with N_i > s it is a coarse level);
// one launch per operator and size serves the whole batch, and the levels
// with n <= 15 run inside one block per problem. Each launch is persistent
// (a fixed number of blocks loops over (problem, tile) items) and skips the
// items of problems that have converged (device flags). The row-chunk height
// of each launch is chosen by timing candidates once per size (autotuner,
// cached per device and size; optionally persisted to the JSON file named by
// MG_AUTOTUNE_CACHE).
//
// One refinement iteration for all active problems:
//   pre  : r_i = b_i - A u_i in FP64 (one launch per distinct N), written as
//          the FP32 scaled right-hand side of level 0, per-problem ||r_i||^2,
//          stored by the summing kernel into mapped pinned host memory;
//   rest : the FP32 V cycle from zero on every level size, then u_i += e_i.
// The host reads the norms once per iteration, retires converged problems
// and uploads the new flags before the next launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/mg.h"
#include "mg_common.cuh"
#include "mg_ctx.h"
#include "mg_internal.h"

namespace mg {

// ---------------------------------------------------------------------------
// small batched kernels
// ---------------------------------------------------------------------------
// per active problem: the sum of its partials into norm2[p] and into the
// mapped pinned host array h_norm2 (read after the stream synchronises; no
// device-to-host copy that could queue behind a caller's large copies)
__global__ void batched_sums(const double *__restrict__ partials, const int *__restrict__ off,
                             const int *__restrict__ cnt, const int *__restrict__ active, double *__restrict__ norm2,
                             double *__restrict__ h_norm2)
{
    const int p = blockIdx.x;
    if (!active[p]) return;
    double v = 0.0;
    for (int i = threadIdx.x; i < cnt[p]; i += blockDim.x) v += partials[off[p] + i];
    block_sum_store<256>(v, &norm2[p]);  // thread 0 stores it
    if (threadIdx.x == 0) h_norm2[p] = norm2[p];
}

struct UpdItem {
    double *u;        // compact FP64 caller array
    const float *e;   // padded FP32 level 0 result
    long long np;     // n * n
    int n, pitch;
    long long off;
};

constexpr int kUpdChunk = 8192;

// u_i += e_i for problem blockIdx.y, chunk blockIdx.x
__global__ void batched_update(const UpdItem *__restrict__ tab, const int *__restrict__ active)
{
    const int p = blockIdx.y;
    if (!active[p]) return;
    const UpdItem it = tab[p];
    // chunk = kUpdChunk / n_pad rows of the problem (whole rows)
    const int rows = max(1, kUpdChunk / it.n);
    const int y0 = blockIdx.x * rows;
    if (y0 >= it.n) return;
    const int y1 = min(y0 + rows, it.n);
    constexpr int kUnroll = 4;  // loads in flight per thread and row
    for (int y = y0; y < y1; ++y) {
        double *ur = it.u + (long long)y * it.n;
        const float *er = it.e + it.off + (long long)y * it.pitch;
        for (int x0 = threadIdx.x; x0 < it.n; x0 += kUnroll * blockDim.x) {
            double uv[kUnroll];
            float ev[kUnroll];
#pragma unroll
            for (int q = 0; q < kUnroll; ++q) {
                const int x = x0 + q * blockDim.x;
                if (x < it.n) {
                    uv[q] = ur[x];
                    ev[q] = er[x];
                }
            }
#pragma unroll
            for (int q = 0; q < kUnroll; ++q) {
                const int x = x0 + q * blockDim.x;
                if (x < it.n) ur[x] = __dadd_rn(uv[q], widen(ev[q]));
            }
        }
    }
}

// u_i = 0 for problem blockIdx.y, chunk blockIdx.x (a solve from zero)
__global__ void batched_zero(const UpdItem *__restrict__ tab)
{
    const UpdItem it = tab[blockIdx.y];
    const int rows = max(1, kUpdChunk / it.n);
    const int y0 = blockIdx.x * rows;
    if (y0 >= it.n) return;
    const long i1 = (long)min(y0 + rows, it.n) * it.n;
    for (long i = (long)y0 * it.n + threadIdx.x; i < i1; i += blockDim.x) it.u[i] = 0.0;
}

// ---------------------------------------------------------------------------
// autotune cache
// ---------------------------------------------------------------------------
static std::mutex g_tune_mutex;
static std::map<std::string, int> g_tune;
static bool g_tune_loaded = false;

static void tune_load()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("MG_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    // flat JSON object {"key": int, ...}
    char key[256];
    int v, c;
    while ((c = fgetc(f)) != EOF) {
        if (c != '"') continue;
        int k = 0;
        while ((c = fgetc(f)) != EOF && c != '"' && k < 255) key[k++] = (char)c;
        key[k] = 0;
        if (fscanf(f, " : %d", &v) == 1) g_tune[key] = v;
    }
    fclose(f);
}

static void tune_save()
{
    const char *path = getenv("MG_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "w");
    if (!f) return;
    fprintf(f, "{\n");
    size_t i = 0;
    for (auto &kv : g_tune) fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++i < g_tune.size() ? "," : "");
    fprintf(f, "}\n");
    fclose(f);
}

}  // namespace mg

using namespace mg;

struct BatchSize {
    int n = 0;
    std::vector<int> probs, lev;
    std::vector<BItem<float> *> pre, post;
    BItem<float> *rr = nullptr, *pro = nullptr;
    // first pre-sweep of the later cycles of a refinement iteration: finest
    // levels from the previous cycle's result, coarse levels from zero
    BItem<float> *again = nullptr;
    // V(1,1): the two temporally blocked passes (mg_fused2d.cu) per level:
    // sweep + residual + restriction (fa; fagain for the later cycles of an
    // iteration), interpolation + correction + sweep (fb)
    FItem *fa = nullptr, *fagain = nullptr, *fb = nullptr;
    int H = 16, Hrr = 8, Hpro = 8, Hfa = 16, Hfb = 32;
};

struct BatchGroup {
    int n = 0;  // finest n of the group
    std::vector<int> probs;
    BRes<float> *res = nullptr;
    std::vector<BRes<float>> host;
    int tiles = 0;
};

struct BatchWork {
    int count = 0, d = 2;
    std::vector<int> N;
    std::vector<std::vector<int>> n;
    std::vector<std::vector<float *>> A, B, BH, RH;
    std::vector<int> lt;  // first tail level per problem
    std::vector<BatchSize> sizes;
    std::vector<BatchGroup> groups;
    TailLevel *tail_lv = nullptr;
    TailOp *tail_ops = nullptr;
    int *op_off = nullptr, *op_cnt = nullptr;
    double *partials = nullptr;
    int *part_off = nullptr, *part_cnt = nullptr;
    BResGroup *rgroups = nullptr;  // the groups for the one-launch residual, descending n
    int res_items = 0;
    double *norm2 = nullptr, *h_norm2 = nullptr;  // h_norm2: mapped pinned
    double *h_norm2_dev = nullptr;                 // its device address
    int *active = nullptr, *h_active = nullptr;  // h_active: mapped pinned
    int *h_active_dev = nullptr;
    UpdItem *upd = nullptr;
    std::vector<UpdItem> upd_host;
    int upd_chunks = 1;
    char *arena = nullptr;
    cudaGraphExec_t pre = nullptr, rest = nullptr, pre0 = nullptr;  // pre0: the first pre of a zero start
    unsigned long long pre_nodes = 0, rest_nodes = 0, pre0_nodes = 0;
    std::vector<const void *> cap_u, cap_b;
};

namespace {

struct Arena {
    char *base = nullptr;
    size_t off = 0, cap = 0;
    void *take(size_t bytes)
    {
        off = (off + 255) & ~(size_t)255;
        void *p = base ? base + off : nullptr;
        off += bytes ? bytes : 16;
        return p;
    }
};

void tail_ops_for(std::vector<TailOp> &out, const std::vector<int> &n, int l, int lt, int nu1, int nu2)
{
    auto push = [&](int kind, int lev) { out.push_back(TailOp{(short)kind, (short)(lev - lt)}); };
    if (n[l] == 3) {
        push(TAIL_SOLVE, l);
        return;
    }
    for (int s = 0; s < nu1; ++s) push(TAIL_SWEEP, l);
    push(TAIL_RESTRICT, l);
    push(TAIL_ZERO, l + 1);
    tail_ops_for(out, n, l + 1, lt, nu1, nu2);
    push(TAIL_PROLONG, l);
    for (int s = 0; s < nu2; ++s) push(TAIL_SWEEP, l);
}

// result buffer of a level visit of problem p at level l
float *result_buf(const BatchWork *w, int p, int l, int nu)
{
    if (l >= w->lt[p]) return w->A[p][l];
    return nu % 2 ? w->B[p][l] : w->A[p][l];
}

float time_ms(cudaStream_t s, cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

// choose the row-chunk heights of every size by timing candidates
mg_status autotune(mg_ctx *c, BatchWork *w)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_load();
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, c->dev) != cudaSuccess) return cuda_fail(cudaGetLastError());
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    bool changed = false;
    for (BatchSize &S : w->sizes) {
        const int np = (int)S.probs.size();
        char kb[200];
        auto tune = [&](const char *op, const int *cands, int ncand, int &best, auto &&run) {
            snprintf(kb, sizeof kb, "%s|d%d|n%d|p%d|f32|%s", prop.name, w->d, S.n, np, op);
            auto it = g_tune.find(kb);
            if (it != g_tune.end()) {
                best = it->second;
                return;
            }
            float best_ms = 1e30f;
            for (int i = 0; i < ncand; ++i) {
                const int H = cands[i];
                if (H > S.n) continue;
                run(H);  // warm up
                cudaEventRecord(e0, c->s);
                for (int r = 0; r < 3; ++r) run(H);
                cudaEventRecord(e1, c->s);
                const float ms = time_ms(c->s, e0, e1);
                if (ms < best_ms) {
                    best_ms = ms;
                    best = H;
                }
            }
            g_tune[kb] = best;
            changed = true;
        };
        static const int sweep_c[] = {4, 8, 16, 32, 64};
        static const int rr_c[] = {2, 4, 8, 16, 32};
        if (c->nu1 == 1 && c->nu2 == 1) {
            static const int fa_c[] = {4, 8, 16, 32, 64};
            static const int fb_c[] = {8, 16, 32, 64, 128};
            tune("fused-a", fa_c, 5, S.Hfa, [&](int H) {
                launch_sweep_restrict2d_pl_batched(S.fa, np, w->active, S.n, H, c->c, c->s);
            });
            tune("fused-b", fb_c, 5, S.Hfb, [&](int H) {
                launch_prolong_sweep2d_pl_batched(S.fb, np, w->active, S.n, H, c->c, c->s);
            });
            continue;
        }
        tune("sweep", sweep_c, 5, S.H, [&](int H) {
            launch_sweep2d_pl_batched(S.pre[0], np, w->active, S.n, H, 1, c->c, c->s);
        });
        tune("restrict", rr_c, 5, S.Hrr, [&](int H) {
            launch_resrestrict2d_pl_batched(S.rr, np, w->active, S.n, H, c->s);
        });
        tune("prolong", rr_c, 5, S.Hpro, [&](int H) {
            launch_prolong2d_pl_batched(S.pro, np, w->active, S.n, H, c->s);
        });
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaError_t e = cudaStreamSynchronize(c->s);
    if (e != cudaSuccess) return cuda_fail(e);
    if (changed) tune_save();
    return MG_OK;
}

cudaError_t record_cycle(mg_ctx *c, BatchWork *w, bool first)
{
    cudaError_t e;
    const int nu1 = c->nu1, nu2 = c->nu2;
    if (nu1 == 1 && nu2 == 1) {
        // V(1,1) in two temporally blocked passes per level size
        for (BatchSize &S : w->sizes)
            if ((e = launch_sweep_restrict2d_pl_batched(first ? S.fa : S.fagain, (int)S.probs.size(), w->active, S.n,
                                                        S.Hfa, c->c, c->s)))
                return e;
        if ((e = launch_tail_batched<float>(w->tail_lv, w->tail_ops, w->op_off, w->op_cnt, w->active, w->count, w->d,
                                            c->c, c->lu, c->s)))
            return e;
        for (auto it = w->sizes.rbegin(); it != w->sizes.rend(); ++it)
            if ((e = launch_prolong_sweep2d_pl_batched(it->fb, (int)it->probs.size(), w->active, it->n, it->Hfb, c->c,
                                                       c->s)))
                return e;
        return cudaSuccess;
    }
    // descend
    for (BatchSize &S : w->sizes) {
        const int np = (int)S.probs.size();
        for (int k = 0; k < nu1; ++k) {
            if (k == 0 && !first)
                e = launch_sweep2d_pl_batched(S.again, np, w->active, S.n, S.H, 2, c->c, c->s);
            else
                e = launch_sweep2d_pl_batched(S.pre[k], np, w->active, S.n, S.H, k == 0 ? 1 : 0, c->c, c->s);
            if (e) return e;
        }
        if (nu1 == 0) {
            // no pre-sweep: the level's value is zero
            for (size_t j = 0; j < S.probs.size(); ++j) {
                const int p = S.probs[j], l = S.lev[j];
                const size_t bytes = pitch2_floats(S.n) * sizeof(float);
                if ((e = launch_zero_words(w->A[p][l], bytes, c->s))) return e;
            }
        }
        if ((e = launch_resrestrict2d_pl_batched(S.rr, np, w->active, S.n, S.Hrr, c->s))) return e;
    }
    // tails, one block per problem
    if ((e = launch_tail_batched<float>(w->tail_lv, w->tail_ops, w->op_off, w->op_cnt, w->active, w->count, w->d, c->c,
                                        c->lu, c->s)))
        return e;
    // ascend
    for (auto it = w->sizes.rbegin(); it != w->sizes.rend(); ++it) {
        BatchSize &S = *it;
        const int np = (int)S.probs.size();
        if ((e = launch_prolong2d_pl_batched(S.pro, np, w->active, S.n, S.Hpro, c->s))) return e;
        for (int k = 0; k < nu2; ++k)
            if ((e = launch_sweep2d_pl_batched(S.post[k], np, w->active, S.n, S.H, 0, c->c, c->s))) return e;
    }
    return cudaSuccess;
}

cudaError_t record_rest(mg_ctx *c, BatchWork *w)
{
    cudaError_t e;
    for (int k = 0; k < c->inner; ++k)
        if ((e = record_cycle(c, w, k == 0))) return e;
    // u_i += e_i in FP64
    batched_update<<<dim3(w->upd_chunks, w->count), 256, 0, c->s>>>(w->upd, w->active);
    count_launch(1);
    return cudaGetLastError();
}

// a solve from u = 0: every u_i zeroed (the FP64 updates add into it), the
// first residual h^2 b_i rounded to FP32 without FP64 work
cudaError_t record_pre0(mg_ctx *c, BatchWork *w)
{
    cudaError_t e;
    batched_zero<<<dim3(w->upd_chunks, w->count), 256, 0, c->s>>>(w->upd);
    count_launch(1);
    if ((e = cudaGetLastError())) return e;
    if ((e = launch_residual2d_batched_zero(w->rgroups, (int)w->groups.size(), w->res_items, c->s))) return e;
    batched_sums<<<w->count, 256, 0, c->s>>>(w->partials, w->part_off, w->part_cnt, w->active, w->norm2,
                                             w->h_norm2_dev);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t record_pre(mg_ctx *c, BatchWork *w)
{
    cudaError_t e;
    if ((e = launch_residual2d_batched_all(w->rgroups, (int)w->groups.size(), w->res_items, w->active, c->s)))
        return e;
    batched_sums<<<w->count, 256, 0, c->s>>>(w->partials, w->part_off, w->part_cnt, w->active, w->norm2,
                                             w->h_norm2_dev);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace

namespace mg {
mg_status batch_set_inner(mg_ctx *c, int inner)
{
    BatchWork *w = c->batch;
    if (!w || inner < 1 || inner > 8) return MG_EINVAL;
    if (inner > 1) {
        // later cycles continue level 0 in place of the first pre-sweep's
        // input: it must be the buffer the cycle ends in, and not a tail level
        if ((c->nu1 + c->nu2) % 2) return MG_EINVAL;
        for (int p = 0; p < w->count; ++p)
            if (w->lt[p] == 0) return MG_EINVAL;
    }
    if (cudaSetDevice(c->dev) != cudaSuccess || cudaStreamSynchronize(c->s) != cudaSuccess)
        return cuda_fail(cudaGetLastError());
    if (w->rest) cudaGraphExecDestroy(w->rest);
    w->rest = nullptr;
    c->inner = inner;
    return capture_graph(c, &w->rest, &w->rest_nodes, [&]() { return record_rest(c, w); });
}

void free_batch(mg_ctx *c)
{
    BatchWork *w = c->batch;
    if (!w) return;
    if (w->pre) cudaGraphExecDestroy(w->pre);
    if (w->pre0) cudaGraphExecDestroy(w->pre0);
    if (w->rest) cudaGraphExecDestroy(w->rest);
    if (w->arena) cudaFree(w->arena);
    if (w->h_norm2) cudaFreeHost(w->h_norm2);
    if (w->h_active) cudaFreeHost(w->h_active);
    delete w;
    c->batch = nullptr;
}
}  // namespace mg

extern "C" mg_status mg_setup_batched(int d, int count, const int *Ns, const double *spai_coeffs, int ncoeffs, int nu1,
                                      int nu2, mg_prec prec, void *cuda_stream, mg_ctx **out)
{
    if (!out) return MG_EINVAL;
    *out = nullptr;
    if (d != 2 || count < 1 || !Ns || prec != MG_FP32_IR || nu1 < 1 || nu2 < 0 || nu1 > 4 || nu2 > 4) return MG_EINVAL;
    int Nmax = 0;
    for (int i = 0; i < count; ++i) {
        const int N = Ns[i];
        if (N < 4 || N > (1 << 15) || (N & (N - 1))) return MG_EINVAL;
        Nmax = std::max(Nmax, N);
    }
    // the shared parts (stream, events, coarsest LU, weights) come from a
    // one-problem context of the largest size
    mg_ctx *c = nullptr;
    mg_status st = mg_setup(d, 4, spai_coeffs, ncoeffs, nu1, nu2, MG_FP32, cuda_stream, &c);
    if (st != MG_OK) return st;
    c->prec = MG_FP32_IR;
    BatchWork *w = new (std::nothrow) BatchWork;
    if (!w) {
        mg_destroy(c);
        return MG_ENOMEM;
    }
    c->batch = w;
    w->count = count;
    w->d = d;
    w->N.assign(Ns, Ns + count);
    w->n.resize(count);
    w->A.resize(count);
    w->B.resize(count);
    w->BH.resize(count);
    w->RH.resize(count);
    w->lt.resize(count);
    for (int p = 0; p < count; ++p) {
        for (int m = Ns[p]; m >= 4; m /= 2) w->n[p].push_back(m - 1);
        w->lt[p] = (int)w->n[p].size();
        for (int l = 0; l < (int)w->n[p].size(); ++l)
            if (w->n[p][l] <= 15) {
                w->lt[p] = l;
                break;
            }
    }
    // sizes handled by the batched marching kernels (n > 15), descending
    for (int s = Nmax; s >= 32; s /= 2) {
        BatchSize S;
        S.n = s - 1;
        for (int p = 0; p < count; ++p)
            if (Ns[p] >= s) {
                S.probs.push_back(p);
                int l = 0;
                while ((Ns[p] >> l) != s) ++l;
                S.lev.push_back(l);
            }
        if (!S.probs.empty()) w->sizes.push_back(S);
    }
    // distinct finest sizes -> outer residual groups
    std::vector<int> finest(Ns, Ns + count);
    std::sort(finest.begin(), finest.end());
    finest.erase(std::unique(finest.begin(), finest.end()), finest.end());
    for (int N : finest) {
        BatchGroup G;
        G.n = N - 1;
        G.tiles = residual2d_batched_tiles(G.n);
        for (int p = 0; p < count; ++p)
            if (Ns[p] == N) G.probs.push_back(p);
        w->groups.push_back(G);
    }
    // ---- one arena: plan, allocate, carve ----
    std::vector<int> part_off(count), part_cnt(count);
    int tot_parts = 0;
    for (BatchGroup &G : w->groups)
        for (int p : G.probs) {
            part_off[p] = tot_parts;
            part_cnt[p] = G.tiles;
            tot_parts += G.tiles;
        }
    std::vector<TailOp> ops_all;
    std::vector<int> op_off(count), op_cnt(count);
    for (int p = 0; p < count; ++p) {
        op_off[p] = (int)ops_all.size();
        const int lt = w->lt[p];
        ops_all.push_back(TailOp{(short)TAIL_ZERO, 0});
        tail_ops_for(ops_all, w->n[p], lt, lt, nu1, nu2);
        op_cnt[p] = (int)ops_all.size() - op_off[p];
    }
    auto carve = [&](Arena &a, bool real) {
        for (int p = 0; p < count; ++p) {
            const int L = (int)w->n[p].size();
            if (real) {
                w->A[p].assign(L, nullptr);
                w->B[p].assign(L, nullptr);
                w->BH[p].assign(L, nullptr);
                w->RH[p].assign(L, nullptr);
            }
            for (int l = 0; l < L; ++l) {
                const size_t bytes = pitch2_floats(w->n[p][l]) * sizeof(float);
                float *A = (float *)a.take(bytes), *B = (float *)a.take(bytes), *BH = (float *)a.take(bytes);
                float *RH = l >= w->lt[p] ? (float *)a.take(bytes) : nullptr;
                if (real) {
                    w->A[p][l] = A;
                    w->B[p][l] = B;
                    w->BH[p][l] = BH;
                    w->RH[p][l] = RH;
                }
            }
        }
        for (BatchSize &S : w->sizes) {
            const size_t tb = S.probs.size() * sizeof(BItem<float>);
            std::vector<BItem<float> *> pre, post;
            for (int k = 0; k < nu1; ++k) pre.push_back((BItem<float> *)a.take(tb));
            for (int k = 0; k < nu2; ++k) post.push_back((BItem<float> *)a.take(tb));
            BItem<float> *rr = (BItem<float> *)a.take(tb), *pro = (BItem<float> *)a.take(tb);
            BItem<float> *again = (BItem<float> *)a.take(tb);
            const size_t fbytes = S.probs.size() * sizeof(FItem);
            FItem *fa = (FItem *)a.take(fbytes), *fagain = (FItem *)a.take(fbytes), *fb = (FItem *)a.take(fbytes);
            if (real) {
                S.pre = pre;
                S.post = post;
                S.rr = rr;
                S.pro = pro;
                S.again = again;
                S.fa = fa;
                S.fagain = fagain;
                S.fb = fb;
            }
        }
        for (BatchGroup &G : w->groups) {
            BRes<float> *r = (BRes<float> *)a.take(G.probs.size() * sizeof(BRes<float>));
            if (real) G.res = r;
        }
        BResGroup *rg = (BResGroup *)a.take(w->groups.size() * sizeof(BResGroup));
        if (real) w->rgroups = rg;
        TailLevel *tl = (TailLevel *)a.take((size_t)count * kMaxTailLevels * sizeof(TailLevel));
        TailOp *to = (TailOp *)a.take(ops_all.size() * sizeof(TailOp));
        int *oo = (int *)a.take(count * sizeof(int)), *oc = (int *)a.take(count * sizeof(int));
        double *pa = (double *)a.take((size_t)tot_parts * sizeof(double));
        int *po = (int *)a.take(count * sizeof(int)), *pc = (int *)a.take(count * sizeof(int));
        double *nrm = (double *)a.take(count * sizeof(double));
        int *act = (int *)a.take(count * sizeof(int));
        UpdItem *up = (UpdItem *)a.take(count * sizeof(UpdItem));
        if (real) {
            w->tail_lv = tl;
            w->tail_ops = to;
            w->op_off = oo;
            w->op_cnt = oc;
            w->partials = pa;
            w->part_off = po;
            w->part_cnt = pc;
            w->norm2 = nrm;
            w->active = act;
            w->upd = up;
        }
    };
    Arena plan;
    carve(plan, false);
    cudaError_t ce = cudaMalloc((void **)&w->arena, plan.off);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        mg_destroy(c);
        return ce == cudaErrorMemoryAllocation ? MG_ENOMEM : cuda_fail(ce);
    }
    Arena real;
    real.base = w->arena;
    carve(real, true);
    // ghost rings and row padding of every padded level must read as zero
    if ((ce = cudaMemset(w->arena, 0, plan.off)) != cudaSuccess) {
        mg_destroy(c);
        return cuda_fail(ce);
    }
    if (cudaHostAlloc((void **)&w->h_norm2, count * sizeof(double), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&w->h_norm2_dev, w->h_norm2, 0) != cudaSuccess ||
        cudaHostAlloc((void **)&w->h_active, count * sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&w->h_active_dev, w->h_active, 0) != cudaSuccess) {
        cudaGetLastError();
        mg_destroy(c);
        return MG_ENOMEM;
    }
    // ---- fill the device tables ----
    std::vector<cudaError_t> errs;
    auto up = [&](void *dst, const void *src, size_t bytes) { errs.push_back(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice)); };
    for (BatchSize &S : w->sizes) {
        const size_t np = S.probs.size();
        std::vector<BItem<float>> tab(np);
        for (int k = 0; k < nu1; ++k) {
            for (size_t j = 0; j < np; ++j) {
                const int p = S.probs[j], l = S.lev[j];
                float *buf[2] = {w->A[p][l], w->B[p][l]};
                tab[j] = BItem<float>{k ? buf[k % 2] : nullptr, w->BH[p][l], buf[(k + 1) % 2], p, 0};
            }
            up(S.pre[k], tab.data(), np * sizeof(BItem<float>));
        }
        // later cycles of an iteration: level 0 continues from the previous
        // cycle's result (buffer A when nu1 + nu2 is even), coarse levels from zero
        for (size_t j = 0; j < np; ++j) {
            const int p = S.probs[j], l = S.lev[j];
            float *buf[2] = {w->A[p][l], w->B[p][l]};
            tab[j] = BItem<float>{l == 0 ? result_buf(w, p, 0, nu1 + nu2) : nullptr, w->BH[p][l], buf[1], p, 0};
        }
        up(S.again, tab.data(), np * sizeof(BItem<float>));
        for (size_t j = 0; j < np; ++j) {
            const int p = S.probs[j], l = S.lev[j];
            float *buf[2] = {w->A[p][l], w->B[p][l]};
            tab[j] = BItem<float>{buf[nu1 % 2], w->BH[p][l], w->BH[p][l + 1], p, 0};
        }
        up(S.rr, tab.data(), np * sizeof(BItem<float>));
        for (size_t j = 0; j < np; ++j) {
            const int p = S.probs[j], l = S.lev[j];
            float *buf[2] = {w->A[p][l], w->B[p][l]};
            tab[j] = BItem<float>{result_buf(w, p, l + 1, nu1 + nu2), nullptr, buf[nu1 % 2], p, 0};
        }
        up(S.pro, tab.data(), np * sizeof(BItem<float>));
        for (int k = 0; k < nu2; ++k) {
            for (size_t j = 0; j < np; ++j) {
                const int p = S.probs[j], l = S.lev[j];
                float *buf[2] = {w->A[p][l], w->B[p][l]};
                const int cur = (nu1 + k) % 2;
                tab[j] = BItem<float>{buf[cur], w->BH[p][l], buf[1 - cur], p, 0};
            }
            up(S.post[k], tab.data(), np * sizeof(BItem<float>));
        }
        // the fused V(1,1) passes: the pre-smoothed field in B, the visit's
        // result in A (as for the unfused V(1,1))
        std::vector<FItem> fa(np), fagain(np), fb(np);
        for (size_t j = 0; j < np; ++j) {
            const int p = S.probs[j], l = S.lev[j];
            fa[j] = FItem{nullptr, nullptr, w->BH[p][l], w->B[p][l], w->BH[p][l + 1], p, 0};
            fagain[j] = fa[j];
            if (l == 0) fagain[j].u = result_buf(w, p, 0, nu1 + nu2);
            fb[j] = FItem{w->B[p][l], result_buf(w, p, l + 1, nu1 + nu2), w->BH[p][l], w->A[p][l], nullptr, p, 0};
        }
        up(S.fa, fa.data(), np * sizeof(FItem));
        up(S.fagain, fagain.data(), np * sizeof(FItem));
        up(S.fb, fb.data(), np * sizeof(FItem));
    }
    {
        std::vector<TailLevel> tl((size_t)count * kMaxTailLevels);
        for (int p = 0; p < count; ++p)
            for (int l = w->lt[p]; l < (int)w->n[p].size(); ++l) {
                TailLevel &t = tl[(size_t)p * kMaxTailLevels + (l - w->lt[p])];
                t = tail_level(w->A[p][l], w->B[p][l], w->BH[p][l], w->RH[p][l], w->n[p][l]);
                const Pitch2 g = pitch2(w->n[p][l]);
                t.pitch = g.pitch;
                t.off = g.off;
            }
        up(w->tail_lv, tl.data(), tl.size() * sizeof(TailLevel));
        up(w->tail_ops, ops_all.data(), ops_all.size() * sizeof(TailOp));
        up(w->op_off, op_off.data(), count * sizeof(int));
        up(w->op_cnt, op_cnt.data(), count * sizeof(int));
        up(w->part_off, part_off.data(), count * sizeof(int));
        up(w->part_cnt, part_cnt.data(), count * sizeof(int));
        std::vector<int> ones(count, 1);
        up(w->active, ones.data(), count * sizeof(int));
    }
    for (BatchGroup &G : w->groups) {
        G.host.resize(G.probs.size());
        for (size_t j = 0; j < G.probs.size(); ++j) {
            const int p = G.probs[j];
            G.host[j] = BRes<float>{nullptr, nullptr, w->BH[p][0], w->partials + part_off[p], p, 0};
        }
    }
    {
        // groups of the one-launch residual, descending n
        std::vector<BResGroup> rg;
        int items = 0;
        for (auto it = w->groups.rbegin(); it != w->groups.rend(); ++it) {
            const Pitch2 g = pitch2(it->n);
            BResGroup q{it->res, g.pitch, g.off, it->n, 0, 0, 0, 0, items};
            items += residual2d_batched_group(q, (int)it->probs.size());
            rg.push_back(q);
        }
        w->res_items = items;
        errs.push_back(cudaMemcpy(w->rgroups, rg.data(), rg.size() * sizeof(BResGroup), cudaMemcpyHostToDevice));
    }
    w->upd_host.resize(count);
    for (int p = 0; p < count; ++p) {
        const long long np = (long long)w->n[p][0] * w->n[p][0];
        const Pitch2 g = pitch2(w->n[p][0]);
        w->upd_host[p] = UpdItem{nullptr, result_buf(w, p, 0, nu1 + nu2), np, w->n[p][0], g.pitch, g.off};
    }
    int maxchunks = 1;
    for (int p = 0; p < count; ++p) {
        const int n = w->n[p][0], rows = std::max(1, kUpdChunk / n);
        maxchunks = std::max(maxchunks, (n + rows - 1) / rows);
    }
    w->upd_chunks = maxchunks;
    for (cudaError_t e : errs)
        if (e != cudaSuccess) {
            mg_destroy(c);
            return cuda_fail(e);
        }
    st = autotune(c, w);
    if (st == MG_OK) st = capture_graph(c, &w->rest, &w->rest_nodes, [&]() { return record_rest(c, w); });
    if (st == MG_OK) st = capture_graph(c, &w->pre, &w->pre_nodes, [&]() { return record_pre(c, w); });
    if (st == MG_OK) st = capture_graph(c, &w->pre0, &w->pre0_nodes, [&]() { return record_pre0(c, w); });
    if (st != MG_OK) {
        mg_destroy(c);
        return st;
    }
    *out = c;
    return MG_OK;
}

extern "C" mg_status mg_solve_batched(mg_ctx *ctx, const void *const *b, void *const *u, double tol, int max_cycles,
                                      int *cycles_out, double *relres_out)
{
    return mg_solve_batched_ex(ctx, b, u, tol, max_cycles, 0u, cycles_out, relres_out);
}

extern "C" mg_status mg_solve_batched_ex(mg_ctx *ctx, const void *const *b, void *const *u, double tol,
                                         int max_cycles, unsigned flags, int *cycles_out, double *relres_out)
{
    if (!ctx || !ctx->batch || !b || !u || max_cycles < 0 || !(tol >= 0.0) || (flags & ~MG_SOLVE_ZERO_START))
        return MG_EINVAL;
    const bool zero_start = (flags & MG_SOLVE_ZERO_START) != 0;
    BatchWork *w = ctx->batch;
    const int count = w->count;
    for (int p = 0; p < count; ++p)
        if (!b[p] || !u[p]) return MG_EINVAL;
    if (cudaSetDevice(ctx->dev) != cudaSuccess) return cuda_fail(cudaGetLastError());
    if (cudaEventRecord(ctx->ev_in, ctx->user) != cudaSuccess || cudaStreamWaitEvent(ctx->s, ctx->ev_in, 0) != cudaSuccess)
        return cuda_fail(cudaGetLastError());
    // caller arrays -> device tables (only when they changed)
    bool changed = (int)w->cap_u.size() != count;
    for (int p = 0; !changed && p < count; ++p) changed = w->cap_u[p] != u[p] || w->cap_b[p] != b[p];
    if (changed) {
        for (BatchGroup &G : w->groups) {
            for (size_t j = 0; j < G.probs.size(); ++j) {
                G.host[j].u = (const double *)u[G.probs[j]];
                G.host[j].b = (const double *)b[G.probs[j]];
            }
            if (cudaMemcpyAsync(G.res, G.host.data(), G.host.size() * sizeof(BRes<float>), cudaMemcpyHostToDevice,
                                ctx->s) != cudaSuccess)
                return cuda_fail(cudaGetLastError());
        }
        for (int p = 0; p < count; ++p) w->upd_host[p].u = (double *)u[p];
        if (cudaMemcpyAsync(w->upd, w->upd_host.data(), count * sizeof(UpdItem), cudaMemcpyHostToDevice, ctx->s) !=
            cudaSuccess)
            return cuda_fail(cudaGetLastError());
        if (cudaStreamSynchronize(ctx->s) != cudaSuccess) return cuda_fail(cudaGetLastError());
        w->cap_u.assign(u, u + count);
        w->cap_b.assign(b, b + count);
    }
    std::vector<double> r0(count, 0.0), rk(count, 0.0);
    std::vector<int> cyc(count, 0), state(count, 0);  // 0 active, 1 converged, 2 out of cycles, 3 NaN
    for (int p = 0; p < count; ++p) w->h_active[p] = 1;
    auto upload_flags = [&]() {
        // a kernel reads the flags from mapped memory: a copy engine could
        // queue this behind a caller's large transfer
        return launch_copy_words(w->active, w->h_active_dev, count * sizeof(int), ctx->s);
    };
    if (upload_flags() != cudaSuccess || cudaGraphLaunch(zero_start ? w->pre0 : w->pre, ctx->s) != cudaSuccess ||
        cudaStreamSynchronize(ctx->s) != cudaSuccess)
        return cuda_fail(cudaGetLastError());
    count_launch(zero_start ? w->pre0_nodes : w->pre_nodes);
    for (int k = 0;; ++k) {
        int nactive = 0;
        for (int p = 0; p < count; ++p) {
            if (state[p]) continue;
            const double r = std::sqrt(w->h_norm2[p]) * (double)w->N[p] * (double)w->N[p];
            if (k == 0) r0[p] = r;
            rk[p] = r;
            cyc[p] = k;
            if (!std::isfinite(r))
                state[p] = 3;
            else if (r <= tol * r0[p])
                state[p] = 1;
            else if (k == max_cycles)
                state[p] = 2;
            if (state[p]) w->h_active[p] = 0;
            else ++nactive;
        }
        if (!nactive) break;
        if (upload_flags() != cudaSuccess || cudaGraphLaunch(w->rest, ctx->s) != cudaSuccess ||
            cudaGraphLaunch(w->pre, ctx->s) != cudaSuccess || cudaStreamSynchronize(ctx->s) != cudaSuccess)
            return cuda_fail(cudaGetLastError());
        count_launch(w->rest_nodes + w->pre_nodes);
    }
    mg_status st = MG_OK;
    for (int p = 0; p < count; ++p) {
        if (cycles_out) cycles_out[p] = cyc[p];
        if (relres_out) relres_out[p] = r0[p] > 0.0 ? rk[p] / r0[p] : 0.0;
        if (state[p] == 3) st = MG_ENAN;
        else if (state[p] == 2 && st == MG_OK) st = MG_ENOCONV;
    }
    if (cudaEventRecord(ctx->ev_out, ctx->s) != cudaSuccess || cudaStreamWaitEvent(ctx->user, ctx->ev_out, 0) != cudaSuccess)
        return cuda_fail(cudaGetLastError());
    return st;
}
