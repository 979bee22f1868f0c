"""Local Fourier analysis of the SPAI smoothers (Sec. 2, Sec. 3, Table 1).

TEST INFRASTRUCTURE (see the package docstring).

All symbols are written in the cosine variables x_i = cos(theta_i), h = 1
(every symbol below is invariant under the h^2 scaling of the oracle):

    A~(x)  = 2 (d - sum_i x_i)                               [Eq. (3.1), 3D analogue]
    M~(x)  = c0 + 2 c1 sum_i x_i (+ 4 c2 x_1 x_2 in 2D)       [symbols of Upsilon, T]
    S~(x)  = 1 - A~(x) M~(x)        (omega already folded into the weights c)

The high frequencies T^H = [-pi/2, 3pi/2)^d minus [-pi/2, pi/2)^d map to the
cosine set X^H = [-1, 1]^d minus (0, 1]^d (Appendix A and the proof of
Theorem 3.2). The smoothing factor is mu = max_{X^H} |S~| (Sec. 2); for a
positive product A~M~ in [l0, l1] the optimum is mu_opt = (l1 - l0)/(l1 + l0)
at omega_opt = 2/(l0 + l1) (Eqs. (2.6), (2.7)).
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.optimize import minimize


def product_symbol(d: int, w, x) -> np.ndarray:
    """A~ M~ at cosine points x (shape (..., d)); w = stencil weights (units h^2)."""
    x = np.asarray(x, dtype=np.float64)
    sx = x.sum(axis=-1)
    a = 2.0 * (d - sx)
    m = w[0] + 2.0 * w[1] * sx
    if d == 2 and len(w) > 2:
        m = m + 4.0 * w[2] * x[..., 0] * x[..., 1]
    return a * m


def _high_grid(d: int, k: int) -> np.ndarray:
    """Points of X^H on a uniform cosine grid with k points per axis (+ 0)."""
    g = np.union1d(np.linspace(-1.0, 1.0, k), [0.0])
    mesh = np.stack(np.meshgrid(*([g] * d), indexing="ij"), axis=-1).reshape(-1, d)
    return mesh[mesh.min(axis=1) <= 0.0]


def _refine(d: int, w, sign: float, x0) -> float:
    """Polish an extremum of sign*A~M~ over X^H (box [-1,1]^d, one coordinate <= 0)."""
    best = sign * product_symbol(d, w, x0)
    for j in range(d):  # keep coordinate j non-positive
        bounds = [(-1.0, 1.0)] * d
        bounds[j] = (-1.0, 0.0)
        start = np.clip(x0, [b[0] for b in bounds], [b[1] for b in bounds])
        res = minimize(lambda x: -sign * product_symbol(d, w, x), start, bounds=bounds,
                       method="L-BFGS-B", options={"ftol": 1e-15, "gtol": 1e-12})
        best = max(best, -res.fun)
    return sign * best


def extremes(d: int, w, k: int | None = None):
    """(lambda_0, lambda_1) = (min, max) of A~ M~ over X^H."""
    k = k or (1201 if d == 2 else 121)
    pts = _high_grid(d, k)
    vals = product_symbol(d, w, pts)
    lo = _refine(d, w, -1.0, pts[np.argmin(vals)])
    hi = _refine(d, w, +1.0, pts[np.argmax(vals)])
    return min(lo, vals.min()), max(hi, vals.max())


def optimal(d: int, w):
    """(mu_opt, omega_opt) of Eqs. (2.6), (2.7) for the stencil weights w."""
    l0, l1 = extremes(d, w)
    if l0 <= 0.0:
        raise ValueError("product symbol not positive on X^H: no convergent omega")
    return (l1 - l0) / (l1 + l0), 2.0 / (l0 + l1)


def smoothing_factor(d: int, wfold, k: int | None = None) -> float:
    """mu = max_{X^H} |1 - A~ M~| for omega-folded weights."""
    l0, l1 = extremes(d, wfold, k)
    return max(abs(1.0 - l0), abs(1.0 - l1))


# ---------------------------------------------------------------------------
# Appendix A and Theorem 3.2 quantities
# ---------------------------------------------------------------------------

def f_ab(x1, x2, a, b):
    """f_{a,b}(x1, x2) = [b + a (x1 + x2) + x1 x2] (2 - x1 - x2) (Appendix A)."""
    return (b + a * (x1 + x2) + x1 * x2) * (2.0 - x1 - x2)


def f_ab_extremes(a: float, b: float):
    """(m_{a,b}, chi_{a,b}): min and max of f_{a,b} over X^H (2D)."""
    # with 8 gamma = 1, b = 2 alpha, a = 4 beta the product A~M~ of
    # Upsilon(alpha, beta, gamma) equals f_{a,b} (Sec. 3.1)
    w = (b / 2.0, a / 4.0, 1.0 / 8.0)
    return extremes(2, w)


# ---------------------------------------------------------------------------
# two-grid analysis (Sec. 4, Table 1)
# ---------------------------------------------------------------------------

def two_grid_factor(d: int, wfold, nu: int, n: int = 256, coarse: str = "rediscretised") -> float:
    """LFA two-grid factor rho_h(nu): the largest spectral radius of the
    2^d x 2^d symbol S^nu K over the low frequencies theta = 2 pi k / n in
    T^L, theta != 0, where K = I - P~ (A~_H)^{-1} R~ A~_h with full weighting
    (symbol prod (1 + cos theta_i)/2 per harmonic) and linear interpolation
    (the same symbol). The harmonics of theta are theta + pi alpha, alpha in
    {0,1}^d. coarse: "rediscretised" (A_H the same stencil on H = 2h, as in
    the cycle of Sec. 4) or "galerkin" (A_H = R A_h P, whose symbol is the sum
    over the harmonics of R~ A~_h P~). Table 1 (Sec. 4) does not say which it
    uses; its 2D M_5 and M_9 rows are the Galerkin values and its other rows
    the rediscretised ones (both reproduced to the printed digits)."""
    if coarse not in ("rediscretised", "galerkin"):
        raise ValueError(coarse)
    ks = np.arange(-n // 4, n // 4)
    theta = np.stack(np.meshgrid(*([2.0 * np.pi * ks / n] * d), indexing="ij"), -1).reshape(-1, d)
    theta = theta[np.any(theta != 0.0, axis=1)]
    alphas = np.array(list(itertools.product((0, 1), repeat=d)), dtype=np.float64)  # (2^d, d)
    cos = np.cos(theta[:, None, :] + np.pi * alphas[None, :, :])  # (T, 2^d, d)
    sx = cos.sum(axis=-1)
    a_h = 2.0 * (d - sx)
    m = wfold[0] + 2.0 * wfold[1] * sx
    if d == 2 and len(wfold) > 2:
        m = m + 4.0 * wfold[2] * cos[..., 0] * cos[..., 1]
    s = (1.0 - a_h * m) ** nu
    r = np.prod((1.0 + cos) / 2.0, axis=-1)  # (T, 2^d)
    if coarse == "galerkin":
        a_H = (r * a_h * r).sum(axis=-1)
    else:
        a_H = 2.0 * (d - np.cos(2.0 * theta).sum(axis=-1)) / 4.0  # H = 2h relative to h = 1
    K = np.eye(2 ** d)[None] - r[:, :, None] * (r * a_h)[:, None, :] / a_H[:, None, None]
    T = s[:, :, None] * K
    return float(np.max(np.abs(np.linalg.eigvals(T))))


# ---------------------------------------------------------------------------
# numerical min-max over a symmetric stencil family (Sec. 3.1, Sec. 3.2)
# ---------------------------------------------------------------------------
# A symmetric stencil family is given by one weight per class of offsets: the
# offsets with j non-zero components (centre, edges/faces, corners in 2D;
# centre, faces, edges, corners in 3D). The symbol of class j, in the cosine
# variables, is 2^j e_j(x) with e_j the j-th elementary symmetric polynomial
# (Sec. 3.1 for Upsilon, Sec. 3.2 for T and its 19/27-point extensions).
# The paper minimises over a family the smoothing factor
#     mu(w) = min_omega max_{X^H} |1 - omega A~ M~_w| = (l1 - l0) / (l1 + l0)
# (Eqs. (2.6), (2.7)); since omega absorbs a common factor of the weights,
# the centre weight is fixed to 1 and the others are searched.

#: family name -> (dimension, number of weight classes)
FAMILIES = {
    "jacobi2": (2, 1),      # M_J (Sec. 3.1)
    "five": (2, 2),         # 5-point stencils (Sec. 3.1, M_5)
    "nine": (2, 3),         # Upsilon(alpha, beta, gamma) (Sec. 3.1, Theorem 3.1)
    "jacobi3": (3, 1),      # M_J (Sec. 3.2)
    "seven": (3, 2),        # T(alpha, beta) (Sec. 3.2, Theorem 3.2)
    "nineteen": (3, 3),     # + the 12 edge offsets (Sec. 3.2, closing remark)
    "twentyseven": (3, 4),  # + the 8 corner offsets (Sec. 3.2, closing remark)
}


def _elementary(x: np.ndarray, j: int) -> np.ndarray:
    """e_j of the last axis of x (j = 0..d)."""
    d = x.shape[-1]
    out = np.zeros(x.shape[:-1])
    for sub in itertools.combinations(range(d), j):
        out = out + (np.prod(x[..., list(sub)], axis=-1) if sub else 1.0)
    return out


def class_symbol(d: int, w, x) -> np.ndarray:
    """M~ = sum_j w_j 2^j e_j(x) for class weights w (h = 1)."""
    x = np.asarray(x, dtype=np.float64)
    return sum(wj * 2.0 ** j * _elementary(x, j) for j, wj in enumerate(w))


def class_product(d: int, w, x) -> np.ndarray:
    """A~ M~ for class weights w."""
    x = np.asarray(x, dtype=np.float64)
    return 2.0 * (d - x.sum(axis=-1)) * class_symbol(d, w, x)


def _class_product_grad(d: int, w, x: np.ndarray) -> np.ndarray:
    """Gradient of A~ M~ in x (product rule; d e_j / d x_i = e_{j-1} of the others)."""
    a = 2.0 * (d - x.sum())
    m = class_symbol(d, w, x)
    g = np.empty(d)
    for i in range(d):
        rest = np.delete(x, i)
        dm = sum(wj * 2.0 ** j * (_elementary(rest, j - 1) if j >= 1 else 0.0) for j, wj in enumerate(w))
        g[i] = -2.0 * m + a * dm
    return g


_GRIDS = {}


def _sym_grid(d: int):
    """Uniform grid of the box x_1 in [-1, 0], x_2.. in [-1, 1]: for a symbol
    symmetric under permutations of the axes this box holds every value the
    symbol takes on X^H (each point of X^H has some coordinate <= 0)."""
    if d not in _GRIDS:
        k1, k = (201, 401) if d == 2 else (25, 49)
        axes = [np.linspace(-1.0, 0.0, k1)] + [np.linspace(-1.0, 1.0, k)] * (d - 1)
        mesh = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1)
        _GRIDS[d] = (mesh, [(-1.0, 0.0)] + [(-1.0, 1.0)] * (d - 1))
    return _GRIDS[d]


def _grid_local_extrema(vals: np.ndarray, sign: float) -> np.ndarray:
    """Indices (flat) of grid points no smaller (sign=+1) / no larger than
    every axis neighbour."""
    v = sign * vals
    keep = np.ones(v.shape, dtype=bool)
    for ax in range(v.ndim):
        for sh in (1, -1):
            nb = np.roll(v, sh, axis=ax)
            edge = [slice(None)] * v.ndim
            edge[ax] = 0 if sh == 1 else -1
            nb[tuple(edge)] = -np.inf
            keep &= v >= nb
    return np.flatnonzero(keep)


def class_extremes(d: int, w):
    """(l0, l1) = (min, max) of A~ M~ over X^H for symmetric class weights w:
    grid local extrema of the box of _sym_grid, each polished by L-BFGS-B with
    the analytic gradient inside the box."""
    mesh, bounds = _sym_grid(d)
    vals = class_product(d, w, mesh)
    flat = mesh.reshape(-1, d)
    out = []
    for sign in (-1.0, 1.0):
        idx = _grid_local_extrema(vals, sign)
        idx = idx[np.argsort(-sign * vals.ravel()[idx])][:12]
        best = sign * vals.ravel()[idx[0]]
        for i in idx:
            res = minimize(lambda x: -sign * float(class_product(d, w, x)), flat[i],
                           jac=lambda x: -sign * _class_product_grad(d, w, x), bounds=bounds,
                           method="L-BFGS-B", options={"ftol": 1e-16, "gtol": 1e-14, "maxiter": 200})
            best = max(best, -res.fun)
        out.append(sign * best)
    return out[0], out[1]


def class_mu(d: int, w) -> float:
    """mu(w) = (l1 - l0)/(l1 + l0) (Eq. (2.6)); 1 + |l0| when A~ M~ is not
    positive on X^H (no omega makes the sweep smooth)."""
    l0, l1 = class_extremes(d, w)
    if l0 <= 0.0:
        return 1.0 + abs(l0)
    return (l1 - l0) / (l1 + l0)


def optimise_family(name: str, starts=None, seed: int = 0):
    """Numerical min-max over a family: minimise mu over the class weights
    (centre weight 1) by Nelder-Mead from several starts, then polish from the
    best point. Returns (w, mu, omega) with w the unfolded class weights
    (w_0 = 1) and omega = 2/(l0 + l1) (Eq. (2.7)), so that the folded weights
    of the sweep are omega * w."""
    from scipy.optimize import minimize as _min

    d, nclass = FAMILIES[name]
    if nclass == 1:
        w = (1.0,)
        l0, l1 = class_extremes(d, w)
        return w, (l1 - l0) / (l1 + l0), 2.0 / (l0 + l1)
    rng = np.random.default_rng(seed)
    if starts is None:
        starts = [np.zeros(nclass - 1)] + [rng.uniform(0.0, 0.3, nclass - 1) for _ in range(3)]
    f = lambda p: class_mu(d, (1.0, *p))  # noqa: E731
    best = None
    for p0 in starts:
        r = _min(f, np.asarray(p0, dtype=np.float64), method="Nelder-Mead",
                 options={"xatol": 1e-7, "fatol": 1e-12, "maxiter": 4000, "maxfev": 8000})
        if best is None or r.fun < best.fun:
            best = r
    for _ in range(3):  # restart from the best point with a fresh simplex
        r = _min(f, best.x, method="Nelder-Mead",
                 options={"xatol": 1e-11, "fatol": 1e-15, "maxiter": 4000, "maxfev": 8000,
                          "initial_simplex": np.vstack([best.x] + [best.x + 1e-4 * e for e in np.eye(nclass - 1)])})
        if r.fun <= best.fun:
            best = r
    w = (1.0, *best.x)
    l0, l1 = class_extremes(d, w)
    return w, (l1 - l0) / (l1 + l0), 2.0 / (l0 + l1)
