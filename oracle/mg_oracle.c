/*
 * mg_oracle.c -- plain, slow FP64 CPU oracle for the SPAI-smoothed geometric
 * multigrid method of He, Liu and Wang, "Optimized sparse approximate inverse
 * smoothers for solving Laplacian linear systems" (arXiv:2206.05543).
 *
 * TEST INFRASTRUCTURE. This file is the checker, not the product: only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it. It shares no code with the CUDA library and the CUDA library never
 * calls it.
 *
 * What it computes (paper passages in brackets):
 *   - the Dirichlet Poisson system A_h u_h = b_h on the interior points of the
 *     unit square/cube, 5-point (2D) / 7-point (3D) stencil, h = 1/N [Sec. 1,
 *     Eqs. (1.1)-(1.3)];
 *   - the preconditioned Richardson smoother u <- u + omega M_h (b_h - A_h u)
 *     with stencil-pattern SPAI matrices M_h [Sec. 2, Eq. (2.1); Sec. 3];
 *   - the multigrid cycle of Sec. 4: re-discretised coarse operators (H = 2h),
 *     full-weighting restriction, linear interpolation, nu1 pre- and nu2
 *     post-smoothing sweeps, coarsest mesh h0 = 1/4, V (gamma = 1) or W
 *     (gamma = 2) cycle, stopping on the relative residual 2-norm;
 *   - the residual-norm history behind the rate rho^(k) = (|r_k|/|r_0|)^(1/k)
 *     [Sec. 4, Eq. (4.1)].
 *
 * Scaled form. Every level stores its right-hand side multiplied by its own
 * h^2 ("bh"), so that the scaled residual rh = h^2 (b - A u) reads
 *     rh = bh - (2d u - sum of the 2d neighbours of u),
 * and omega M_h rh / h^2 becomes a stencil with dimensionless weights c_j:
 *     2D: u' = u + c0 rh + c1 (edge sum of rh) + c2 (corner sum of rh)
 *     3D: u' = u + c0 rh + c1 (face sum of rh).
 * Since h is a power of two every h^2 scaling is exact in binary floating
 * point. The coarse right-hand side becomes bh_c = (H^2/h^2) R rh = 4 R rh.
 *
 * Rounding order. Each formula is evaluated in one fixed order, spelled out
 * below, with fused multiply-adds only where written as fma(). The file must
 * be compiled with -ffp-contract=off so that the compiler adds none of its
 * own. Any order is a valid evaluation of the formulas; fixing one makes the
 * FP64 results reproducible to the last bit by any implementation that
 * follows the same order.
 *
 * Layout. A level with n = N-1 interior points per axis stores its interior
 * only, row-major with x fastest: u[y*n + x] (2D), u[(z*n + y)*n + x] (3D),
 * where array index i stands for the grid point (i+1)h. Values outside the
 * interior (the Dirichlet boundary) are zero.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ENOCONV (-4)

/* ------------------------------------------------------------------ */
/* grid access                                                        */
/* ------------------------------------------------------------------ */

/* Value of a level array at integer coordinates, zero outside the interior
 * (Dirichlet), or wrapped around (periodic, used only by the Fourier check). */
static double at2(const double *a, int n, int periodic, int x, int y)
{
    if (periodic) {
        x = (x % n + n) % n;
        y = (y % n + n) % n;
    } else if (x < 0 || x >= n || y < 0 || y >= n) {
        return 0.0;
    }
    return a[(long)y * n + x];
}

static double at3(const double *a, int n, int periodic, int x, int y, int z)
{
    if (periodic) {
        x = (x % n + n) % n;
        y = (y % n + n) % n;
        z = (z % n + n) % n;
    } else if (x < 0 || x >= n || y < 0 || y >= n || z < 0 || z >= n) {
        return 0.0;
    }
    return a[((long)z * n + y) * n + x];
}

static long npoints(int d, int n)
{
    return d == 2 ? (long)n * n : (long)n * n * n;
}

/* ------------------------------------------------------------------ */
/* residual                                                           */
/* ------------------------------------------------------------------ */

/* Scaled residual rh = bh - h^2 A_h u of the 5-point / 7-point operator
 * [Eq. (1.3)]:
 *   2D: s  = (u_W + u_E) + (u_S + u_N)
 *       rh = fma(-4, u, bh) + s
 *   3D: s  = ((u_W + u_E) + (u_S + u_N)) + (u_D + u_U)
 *       rh = fma(-6, u, bh) + s
 * (W/E: x-1/x+1, S/N: y-1/y+1, D/U: z-1/z+1). */
void orc_residual_scaled(int d, int n, int periodic, const double *u,
                         const double *bh, double *rh)
{
    if (d == 2) {
#pragma omp parallel for schedule(static)
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x) {
                long p = (long)y * n + x;
                double s = (at2(u, n, periodic, x - 1, y) + at2(u, n, periodic, x + 1, y)) +
                           (at2(u, n, periodic, x, y - 1) + at2(u, n, periodic, x, y + 1));
                rh[p] = fma(-4.0, u[p], bh[p]) + s;
            }
    } else {
#pragma omp parallel for schedule(static)
        for (int z = 0; z < n; ++z)
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x) {
                    long p = ((long)z * n + y) * n + x;
                    double s = ((at3(u, n, periodic, x - 1, y, z) + at3(u, n, periodic, x + 1, y, z)) +
                                (at3(u, n, periodic, x, y - 1, z) + at3(u, n, periodic, x, y + 1, z))) +
                               (at3(u, n, periodic, x, y, z - 1) + at3(u, n, periodic, x, y, z + 1));
                    rh[p] = fma(-6.0, u[p], bh[p]) + s;
                }
    }
}

/* Timing only: the number of threads the grid loops above use (each point is
 * computed by one thread in the same order, so results do not depend on it;
 * norms are summed by one thread). Returns the count in effect, 1 when the
 * library was built without OpenMP. */
#ifdef _OPENMP
#include <omp.h>
#endif
int orc_set_threads(int threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
    return omp_get_max_threads();
#else
    (void)threads;
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* SPAI smoothing sweep                                               */
/* ------------------------------------------------------------------ */

/* In-plane sums of rh around (x, y) in plane z, for the 27-point stencil:
 *   hp = rh_W + rh_E                    (the pair along x)
 *   p1 = hp + (rh_S + rh_N)             (the 4 in-plane edge neighbours)
 *   p2 = hp(y - 1) + hp(y + 1)          (the 4 in-plane corner neighbours)
 * Outside the grid every rh is zero, so are these sums. */
static double hp3(const double *rh, int n, int periodic, int x, int y, int z)
{
    return at3(rh, n, periodic, x - 1, y, z) + at3(rh, n, periodic, x + 1, y, z);
}

static double p1_3(const double *rh, int n, int periodic, int x, int y, int z)
{
    return hp3(rh, n, periodic, x, y, z) + (at3(rh, n, periodic, x, y - 1, z) + at3(rh, n, periodic, x, y + 1, z));
}

static double p2_3(const double *rh, int n, int periodic, int x, int y, int z)
{
    return hp3(rh, n, periodic, x, y - 1, z) + hp3(rh, n, periodic, x, y + 1, z);
}

/* Apply the omega-folded SPAI stencil to rh and add it to u [Eq. (2.1)]:
 *   2D: E = (rh_W + rh_E) + (rh_S + rh_N)
 *       C = (rh_SW + rh_SE) + (rh_NW + rh_NE)
 *       out = fma(c2, C, fma(c1, E, fma(c0, rh, u)))
 *   3D, 7-point M (the family T of Sec. 3.2; c2 = c3 = 0):
 *       E = ((rh_W + rh_E) + (rh_S + rh_N)) + (rh_D + rh_U)
 *       out = fma(c1, E, fma(c0, rh, u))
 *   3D, 27-point M (Sec. 3.2, closing remark; weights c0 centre, c1 the 6
 *   faces, c2 the 12 edges, c3 the 8 corners; used when c2 or c3 != 0):
 *       F = p1(z) + (rh_D + rh_U)                 (faces)
 *       E = p2(z) + (p1(z - 1) + p1(z + 1))       (edges)
 *       C = p2(z - 1) + p2(z + 1)                 (corners)
 *       out = fma(c3, C, fma(c2, E, fma(c1, F, fma(c0, rh, u))))
 *   (p1, p2 as above; for c2 = c3 = 0 the face sum F is the 7-point E.)
 * rh is zero outside the interior, i.e. M_h is the stencil matrix restricted
 * to the interior points. */
static void apply_spai(int d, int n, int periodic, const double *c,
                       const double *rh, const double *u, double *out)
{
    if (d == 2) {
#pragma omp parallel for schedule(static)
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x) {
                long p = (long)y * n + x;
                double E = (at2(rh, n, periodic, x - 1, y) + at2(rh, n, periodic, x + 1, y)) +
                           (at2(rh, n, periodic, x, y - 1) + at2(rh, n, periodic, x, y + 1));
                double C = (at2(rh, n, periodic, x - 1, y - 1) + at2(rh, n, periodic, x + 1, y - 1)) +
                           (at2(rh, n, periodic, x - 1, y + 1) + at2(rh, n, periodic, x + 1, y + 1));
                out[p] = fma(c[2], C, fma(c[1], E, fma(c[0], rh[p], u[p])));
            }
    } else if (c[2] == 0.0 && c[3] == 0.0) {
#pragma omp parallel for schedule(static)
        for (int z = 0; z < n; ++z)
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x) {
                    long p = ((long)z * n + y) * n + x;
                    double E = ((at3(rh, n, periodic, x - 1, y, z) + at3(rh, n, periodic, x + 1, y, z)) +
                                (at3(rh, n, periodic, x, y - 1, z) + at3(rh, n, periodic, x, y + 1, z))) +
                               (at3(rh, n, periodic, x, y, z - 1) + at3(rh, n, periodic, x, y, z + 1));
                    out[p] = fma(c[1], E, fma(c[0], rh[p], u[p]));
                }
    } else {
#pragma omp parallel for schedule(static)
        for (int z = 0; z < n; ++z)
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x) {
                    long p = ((long)z * n + y) * n + x;
                    double F = p1_3(rh, n, periodic, x, y, z) +
                               (at3(rh, n, periodic, x, y, z - 1) + at3(rh, n, periodic, x, y, z + 1));
                    double E = p2_3(rh, n, periodic, x, y, z) +
                               (p1_3(rh, n, periodic, x, y, z - 1) + p1_3(rh, n, periodic, x, y, z + 1));
                    double C = p2_3(rh, n, periodic, x, y, z - 1) + p2_3(rh, n, periodic, x, y, z + 1);
                    out[p] = fma(c[3], C, fma(c[2], E, fma(c[1], F, fma(c[0], rh[p], u[p]))));
                }
    }
}

/* One smoothing sweep u_out = u + omega M_h (b_h - A_h u), out of place.
 * c holds the omega-folded weights: 2D (centre, edge, corner), 3D (centre,
 * face, edge, corner); 4 entries are read in 3D, 3 in 2D. rh_work must hold
 * n^d doubles. */
void orc_sweep(int d, int n, int periodic, const double *c, const double *u,
               const double *bh, double *u_out, double *rh_work)
{
    orc_residual_scaled(d, n, periodic, u, bh, rh_work);
    apply_spai(d, n, periodic, c, rh_work, u, u_out);
}

/* ------------------------------------------------------------------ */
/* grid transfers                                                     */
/* ------------------------------------------------------------------ */

/* Full-weighting restriction [Sec. 4], in tensor-product form: the 1D weights
 * (1, 2, 1)/4 per axis. With the scaled right-hand sides the coarse value is
 * bh_c = 4 R rh, evaluated per coarse point J (fine centre F = 2J, 1-based):
 *   along x: t = (rh(F_x-1) + rh(F_x+1)) + 2 rh(F_x)       (weights sum 4)
 *   along y: t = (t(F_y-1) + t(F_y+1)) + 2 t(F_y)            (sum 16)
 *   [3D, along z: same]                                       (sum 64)
 *   bh_c = 0.25 t (2D) or 0.0625 t (3D), i.e. 4/16 and 4/64.
 * All fine points F +- 1 are interior, so no boundary values enter. */
void orc_restrict(int d, int nf, const double *rh, double *bh_c)
{
    int nc = (nf - 1) / 2;
    if (d == 2) {
#pragma omp parallel for schedule(static)
        for (int J = 1; J <= nc; ++J)
            for (int I = 1; I <= nc; ++I) {
                int fx = 2 * I - 1, fy = 2 * J - 1; /* 0-based index of fine point 2I, 2J */
                double t[3];
                for (int k = 0; k < 3; ++k) {
                    const double *row = rh + (long)(fy - 1 + k) * nf;
                    t[k] = (row[fx - 1] + row[fx + 1]) + 2.0 * row[fx];
                }
                double v = (t[0] + t[2]) + 2.0 * t[1];
                bh_c[(long)(J - 1) * nc + (I - 1)] = 0.25 * v;
            }
    } else {
#pragma omp parallel for schedule(static)
        for (int K = 1; K <= nc; ++K)
            for (int J = 1; J <= nc; ++J)
                for (int I = 1; I <= nc; ++I) {
                    int fx = 2 * I - 1, fy = 2 * J - 1, fz = 2 * K - 1;
                    double t2[3];
                    for (int kz = 0; kz < 3; ++kz) {
                        double t1[3];
                        for (int ky = 0; ky < 3; ++ky) {
                            const double *row = rh + ((long)(fz - 1 + kz) * nf + (fy - 1 + ky)) * nf;
                            t1[ky] = (row[fx - 1] + row[fx + 1]) + 2.0 * row[fx];
                        }
                        t2[kz] = (t1[0] + t1[2]) + 2.0 * t1[1];
                    }
                    double v = (t2[0] + t2[2]) + 2.0 * t2[1];
                    bh_c[((long)(K - 1) * nc + (J - 1)) * nc + (I - 1)] = 0.0625 * v;
                }
    }
}

/* Coarse value at 1-based coarse coordinates, zero on the boundary. */
static double ec2(const double *e, int nc, int I, int J)
{
    if (I < 1 || I > nc || J < 1 || J > nc) return 0.0;
    return e[(long)(J - 1) * nc + (I - 1)];
}

static double ec3(const double *e, int nc, int I, int J, int K)
{
    if (I < 1 || I > nc || J < 1 || J > nc || K < 1 || K > nc) return 0.0;
    return e[((long)(K - 1) * nc + (J - 1)) * nc + (I - 1)];
}

/* Linear interpolation [Sec. 4], read as the tensor product of 1D linear
 * interpolation (bilinear / trilinear, P = 2^d R^T), followed by the
 * coarse-grid correction u += P e. Per fine point (1-based coordinates):
 *   along x: v(x) = e(x/2)                        if x is even
 *                   0.5 (e((x-1)/2) + e((x+1)/2)) if x is odd
 *   then the same along y (and z), applied to the values of the previous
 *   axis; finally u = u + v. */
static double interp_x2(const double *e, int nc, int x, int Jy)
{
    if (x % 2 == 0) return ec2(e, nc, x / 2, Jy);
    return 0.5 * (ec2(e, nc, (x - 1) / 2, Jy) + ec2(e, nc, (x + 1) / 2, Jy));
}

static double interp_xy2(const double *e, int nc, int x, int y)
{
    if (y % 2 == 0) return interp_x2(e, nc, x, y / 2);
    return 0.5 * (interp_x2(e, nc, x, (y - 1) / 2) + interp_x2(e, nc, x, (y + 1) / 2));
}

static double interp_x3(const double *e, int nc, int x, int Jy, int Jz)
{
    if (x % 2 == 0) return ec3(e, nc, x / 2, Jy, Jz);
    return 0.5 * (ec3(e, nc, (x - 1) / 2, Jy, Jz) + ec3(e, nc, (x + 1) / 2, Jy, Jz));
}

static double interp_xy3(const double *e, int nc, int x, int y, int Jz)
{
    if (y % 2 == 0) return interp_x3(e, nc, x, y / 2, Jz);
    return 0.5 * (interp_x3(e, nc, x, (y - 1) / 2, Jz) + interp_x3(e, nc, x, (y + 1) / 2, Jz));
}

static double interp_xyz3(const double *e, int nc, int x, int y, int z)
{
    if (z % 2 == 0) return interp_xy3(e, nc, x, y, z / 2);
    return 0.5 * (interp_xy3(e, nc, x, y, (z - 1) / 2) + interp_xy3(e, nc, x, y, (z + 1) / 2));
}

void orc_prolong_add(int d, int nf, const double *e_c, double *u)
{
    int nc = (nf - 1) / 2;
    if (d == 2) {
#pragma omp parallel for schedule(static)
        for (int y = 1; y <= nf; ++y)
            for (int x = 1; x <= nf; ++x) {
                long p = (long)(y - 1) * nf + (x - 1);
                u[p] = u[p] + interp_xy2(e_c, nc, x, y);
            }
    } else {
#pragma omp parallel for schedule(static)
        for (int z = 1; z <= nf; ++z)
            for (int y = 1; y <= nf; ++y)
                for (int x = 1; x <= nf; ++x) {
                    long p = ((long)(z - 1) * nf + (y - 1)) * nf + (x - 1);
                    u[p] = u[p] + interp_xyz3(e_c, nc, x, y, z);
                }
    }
}

/* ------------------------------------------------------------------ */
/* coarsest-level solve                                               */
/* ------------------------------------------------------------------ */

/* Gaussian elimination without pivoting (the matrix is symmetric positive
 * definite) on the scaled coarsest operator h0^2 A_h0, unknowns in the
 * natural order, applied to the augmented system with right-hand side rhs:
 *   for k: for i > k: l = a_ik / a_kk; a_ij -= l a_kj (j > k); y_i -= l y_k
 *   for i = m-1 .. 0: y_i -= a_ij x_j for j = i+1 .. m-1 in increasing j;
 *                     x_i = y_i / a_ii.
 * Products are rounded before each subtraction (no fma). */
static void coarse_eliminate(int d, const double *rhs, double *x)
{
    const int n = 3;
    const int m = d == 2 ? 9 : 27;
    double a[27][27];
    double y[27];
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < m; ++j) a[i][j] = 0.0;
        y[i] = rhs[i];
    }
    for (int i = 0; i < m; ++i) {
        int xi = i % n, yi = (i / n) % n, zi = i / (n * n);
        a[i][i] = 2.0 * d;
        for (int j = 0; j < m; ++j) {
            int xj = j % n, yj = (j / n) % n, zj = j / (n * n);
            int dist = abs(xi - xj) + abs(yi - yj) + abs(zi - zj);
            if (dist == 1) a[i][j] = -1.0;
        }
    }
    for (int k = 0; k < m; ++k)
        for (int i = k + 1; i < m; ++i) {
            double l = a[i][k] / a[k][k];
            for (int j = k + 1; j < m; ++j) a[i][j] = a[i][j] - l * a[k][j];
            y[i] = y[i] - l * y[k];
        }
    for (int i = m - 1; i >= 0; --i) {
        double s = y[i];
        for (int j = i + 1; j < m; ++j) s = s - a[i][j] * x[j];
        x[i] = s / a[i][i];
    }
}

/* Exact solve on the coarsest grid h0 = 1/4 (3^d interior unknowns)
 * [Sec. 4; the solver is not named there]: x = B bh with B the inverse of
 * h0^2 A_h0, whose column j is the elimination above applied to the unit
 * vector e_j; the product is summed in increasing j, each product rounded
 * before the addition:  x_i = (...((0 + B_i0 bh_0) + B_i1 bh_1) ...). */
void orc_coarse_solve(int d, const double *bh, double *x)
{
    const int m = d == 2 ? 9 : 27;
    double inv[27][27], e[27], col[27];
    for (int j = 0; j < m; ++j) {
        for (int i = 0; i < m; ++i) e[i] = i == j ? 1.0 : 0.0;
        coarse_eliminate(d, e, col);
        for (int i = 0; i < m; ++i) inv[i][j] = col[i];
    }
    for (int i = 0; i < m; ++i) {
        double s = 0.0;
        for (int j = 0; j < m; ++j) s = s + inv[i][j] * bh[j];
        x[i] = s;
    }
}

/* ------------------------------------------------------------------ */
/* multigrid cycle                                                    */
/* ------------------------------------------------------------------ */

typedef struct {
    int d, N, L;      /* dimension, finest N, number of levels (N = 4 -> 1) */
    int nu1, nu2, gamma;
    double c[4];
    double **u, **bh, **rh, **tmp; /* per level, index 0 = finest */
} orc_mg;

static int nlevels(int N)
{
    int L = 0;
    while (N >= 4) {
        ++L;
        if (N == 4) break;
        N /= 2;
    }
    return L;
}

static int valid_N(int N)
{
    if (N < 4) return 0;
    while (N > 4) {
        if (N % 2) return 0;
        N /= 2;
    }
    return N == 4;
}

static void mg_free(orc_mg *g)
{
    if (!g->u) return;
    for (int l = 0; l < g->L; ++l) {
        free(g->u[l]);
        free(g->bh[l]);
        free(g->rh[l]);
        free(g->tmp[l]);
    }
    free(g->u);
    free(g->bh);
    free(g->rh);
    free(g->tmp);
    g->u = NULL;
}

static int mg_init(orc_mg *g, int d, int N, const double *c, int ncoef, int nu1,
                   int nu2, int gamma)
{
    memset(g, 0, sizeof *g);
    if ((d != 2 && d != 3) || !valid_N(N) || nu1 < 0 || nu2 < 0 || gamma < 1 ||
        ncoef < 1 || ncoef > (d == 2 ? 3 : 4))
        return ORC_EINVAL;
    g->d = d;
    g->N = N;
    g->L = nlevels(N);
    g->nu1 = nu1;
    g->nu2 = nu2;
    g->gamma = gamma;
    for (int j = 0; j < 4; ++j) g->c[j] = j < ncoef ? c[j] : 0.0;
    g->u = calloc(g->L, sizeof(double *));
    g->bh = calloc(g->L, sizeof(double *));
    g->rh = calloc(g->L, sizeof(double *));
    g->tmp = calloc(g->L, sizeof(double *));
    if (!g->u || !g->bh || !g->rh || !g->tmp) return ORC_ENOMEM;
    for (int l = 0; l < g->L; ++l) {
        long np = npoints(d, (N >> l) - 1);
        g->u[l] = calloc(np, sizeof(double));
        g->bh[l] = calloc(np, sizeof(double));
        g->rh[l] = calloc(np, sizeof(double));
        g->tmp[l] = calloc(np, sizeof(double));
        if (!g->u[l] || !g->bh[l] || !g->rh[l] || !g->tmp[l]) {
            mg_free(g);
            return ORC_ENOMEM;
        }
    }
    return ORC_OK;
}

static void smooth(orc_mg *g, int l, int sweeps)
{
    int n = (g->N >> l) - 1;
    long np = npoints(g->d, n);
    for (int s = 0; s < sweeps; ++s) {
        orc_sweep(g->d, n, 0, g->c, g->u[l], g->bh[l], g->tmp[l], g->rh[l]);
        memcpy(g->u[l], g->tmp[l], np * sizeof(double));
    }
}

/* One multigrid cycle on level l for u[l], bh[l] [Sec. 4]. */
static void cycle(orc_mg *g, int l)
{
    int n = (g->N >> l) - 1;
    if (n == 3) {
        orc_coarse_solve(g->d, g->bh[l], g->u[l]);
        return;
    }
    smooth(g, l, g->nu1);
    orc_residual_scaled(g->d, n, 0, g->u[l], g->bh[l], g->rh[l]);
    orc_restrict(g->d, n, g->rh[l], g->bh[l + 1]);
    memset(g->u[l + 1], 0, npoints(g->d, (n - 1) / 2) * sizeof(double));
    for (int k = 0; k < g->gamma; ++k) cycle(g, l + 1);
    orc_prolong_add(g->d, n, g->u[l + 1], g->u[l]);
    smooth(g, l, g->nu2);
}

/* Sum of squares with compensated (Neumaier) summation, so that the norm is
 * accurate to a few ulps whatever the grid size; a plain running sum of n
 * positive terms can be off by up to ~n eps relative. */
static double sum_squares(const double *a, long np)
{
    double s = 0.0, comp = 0.0;
    for (long i = 0; i < np; ++i) {
        double x = a[i] * a[i];
        double t = s + x;
        if (fabs(s) >= fabs(x))
            comp += (s - t) + x;
        else
            comp += (x - t) + s;
        s = t;
    }
    return s + comp;
}

static double resnorm_scaled(orc_mg *g)
{
    int n = g->N - 1;
    long np = npoints(g->d, n);
    orc_residual_scaled(g->d, n, 0, g->u[0], g->bh[0], g->rh[0]);
    return sqrt(sum_squares(g->rh[0], np));
}

static void load_rhs(orc_mg *g, const double *b)
{
    long np = npoints(g->d, g->N - 1);
    double h2 = 1.0 / ((double)g->N * (double)g->N); /* exact: N is a power of two */
    for (long i = 0; i < np; ++i) g->bh[0][i] = h2 * b[i];
}

/* ||b - A_h u||_2 (unweighted Euclidean norm [Eq. (4.1)]), from the scaled
 * residual: ||r|| = N^2 ||rh||. */
double orc_residual_norm(int d, int N, const double *u, const double *b)
{
    orc_mg g;
    double zero[4] = {0, 0, 0, 0};
    if (mg_init(&g, d, N, zero, 1, 0, 0, 1) != ORC_OK) return -1.0;
    load_rhs(&g, b);
    memcpy(g.u[0], u, npoints(d, N - 1) * sizeof(double));
    double r = resnorm_scaled(&g) * (double)N * (double)N;
    mg_free(&g);
    return r;
}

/* Run `cycles` multigrid cycles on u in place (b unscaled, finest level). */
int orc_cycles(int d, int N, const double *c, int ncoef, int nu1, int nu2, int gamma,
               int cycles, const double *b, double *u)
{
    orc_mg g;
    int st = mg_init(&g, d, N, c, ncoef, nu1, nu2, gamma);
    if (st != ORC_OK) return st;
    load_rhs(&g, b);
    memcpy(g.u[0], u, npoints(d, N - 1) * sizeof(double));
    for (int k = 0; k < cycles; ++k) cycle(&g, 0);
    memcpy(u, g.u[0], npoints(d, N - 1) * sizeof(double));
    mg_free(&g);
    return ORC_OK;
}

/* Multigrid solve [Sec. 4]: cycle from the initial guess in u until
 * ||r_k|| <= tol ||r_0|| or max_cycles cycles ran.
 * hist (nullable, max_cycles + 1 entries) receives ||r_k||_2 for
 * k = 0 .. *cycles_out. Returns ORC_OK on convergence, ORC_ENOCONV when
 * max_cycles ran out (u and hist are still written). */
int orc_solve(int d, int N, const double *c, int ncoef, int nu1, int nu2, int gamma,
              const double *b, double *u, double tol, int max_cycles, double *hist,
              int *cycles_out, double *relres_out)
{
    orc_mg g;
    int st = mg_init(&g, d, N, c, ncoef, nu1, nu2, gamma);
    if (st != ORC_OK) return st;
    if (max_cycles < 0) {
        mg_free(&g);
        return ORC_EINVAL;
    }
    double scale = (double)N * (double)N;
    load_rhs(&g, b);
    memcpy(g.u[0], u, npoints(d, N - 1) * sizeof(double));
    double r0 = resnorm_scaled(&g), rk = r0;
    int k = 0;
    if (hist) hist[0] = r0 * scale;
    st = ORC_OK;
    while (!(rk <= tol * r0)) {
        if (k == max_cycles) {
            st = ORC_ENOCONV;
            break;
        }
        cycle(&g, 0);
        ++k;
        rk = resnorm_scaled(&g);
        if (hist) hist[k] = rk * scale;
    }
    memcpy(u, g.u[0], npoints(d, N - 1) * sizeof(double));
    if (cycles_out) *cycles_out = k;
    if (relres_out) *relres_out = r0 > 0.0 ? rk / r0 : 0.0;
    mg_free(&g);
    return st;
}
