"""FP64 CPU oracle for the SPAI-smoothed multigrid method of He, Liu and Wang,
"Optimized sparse approximate inverse smoothers for solving Laplacian linear
systems" (arXiv:2206.05543).

TEST INFRASTRUCTURE. This package is the checker, not the product: only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it. It shares no code with the CUDA library
(``paper_2206_05543_gb300``) and imports nothing from it.

Contents
--------
``mg_oracle.c``  plain C, FP64: residual, SPAI sweep, full weighting, linear
                 interpolation, coarsest Gaussian elimination, V/W cycle and
                 the solve loop (Sec. 2 Eq. (2.1), Sec. 4), loaded here via
                 ctypes.
``coeffs.py``    the smoothers of Sec. 3 as omega-folded stencil weights.
``lfa.py``       local Fourier analysis: symbols, smoothing factors, the
                 closed forms of Sec. 2/3 and the two-grid factor of Table 1.
``exact.py``     exact discrete solutions (sine transform, dense solve) and
                 the dense/sparse matrices used to pin the stencil code.
``adjoint.py``   reverse-mode derivative of K cycles (see its header).

The grid functions use the interior-only layout: a level with n = N-1
interior points per axis is an array of shape (n, n) or (n, n, n), indexed
[y, x] / [z, y, x], x fastest in memory.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK = 0
ORC_EINVAL = -1
ORC_ENOMEM = -2
ORC_ENOCONV = -4

# Strict IEEE evaluation: no contraction of a*b+c into fma, no fast-math.
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile mg_oracle.c into _build/liboracle.so (gcc, no GPU needed)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        # OpenMP only spreads the per-point grid loops over threads (timing);
        # without it the same source builds single-threaded
        cmd = ["gcc", *CFLAGS, "-fopenmp", "-o", tmp, _SRC, "-lm"]
        if subprocess.run(cmd, capture_output=True).returncode != 0:
            subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            i, d = ctypes.c_int, ctypes.c_double
            L.orc_residual_scaled.argtypes = [i, i, i, dp, dp, dp]
            L.orc_sweep.argtypes = [i, i, i, dp, dp, dp, dp, dp]
            L.orc_restrict.argtypes = [i, i, dp, dp]
            L.orc_prolong_add.argtypes = [i, i, dp, dp]
            L.orc_coarse_solve.argtypes = [i, dp, dp]
            L.orc_residual_norm.argtypes = [i, i, dp, dp]
            L.orc_residual_norm.restype = d
            L.orc_cycles.argtypes = [i, i, dp, i, i, i, i, i, dp, dp]
            L.orc_solve.argtypes = [i, i, dp, i, i, i, i, dp, dp, d, i, dp, ip, dp]
            L.orc_set_threads.argtypes = [i]
            L.orc_set_threads.restype = i
            L.orc_set_threads(1)  # single-threaded unless a timing asks otherwise
            for f in (L.orc_cycles, L.orc_solve):
                f.restype = i
            _lib = L
    return _lib


def set_threads(threads: int) -> int:
    """Threads for the grid loops (timing only; results do not depend on it)."""
    return int(lib().orc_set_threads(int(threads)))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dim_n(a: np.ndarray):
    if a.ndim not in (2, 3) or any(s != a.shape[0] for s in a.shape):
        raise ValueError("expected a square (n, n) or cubic (n, n, n) grid array")
    return a.ndim, a.shape[0]


def _coeffs(d: int, c) -> np.ndarray:
    c = _f64(c).ravel()
    if not 1 <= c.size <= (3 if d == 2 else 4):
        raise ValueError("2D takes up to 3 weights (centre, edge, corner), 3D up to 4 (centre, face, edge, corner)")
    full = np.zeros(4)
    full[: c.size] = c
    return full


# ---------------------------------------------------------------------------
# single operators (Sec. 1 Eq. (1.3), Sec. 2 Eq. (2.1), Sec. 4)
# ---------------------------------------------------------------------------

def residual_scaled(u, bh, periodic: bool = False) -> np.ndarray:
    """rh = bh - h^2 A_h u (zero Dirichlet boundary, or periodic)."""
    u, bh = _f64(u), _f64(bh)
    d, n = _dim_n(u)
    rh = np.empty_like(u)
    lib().orc_residual_scaled(d, n, int(periodic), _p(u), _p(bh), _p(rh))
    return rh


def sweep(u, bh, c, periodic: bool = False) -> np.ndarray:
    """One SPAI sweep u + omega M_h (b_h - A_h u) in scaled form (weights c)."""
    u, bh = _f64(u), _f64(bh)
    d, n = _dim_n(u)
    cc = _coeffs(d, c)
    out = np.empty_like(u)
    work = np.empty_like(u)
    lib().orc_sweep(d, n, int(periodic), _p(cc), _p(u), _p(bh), _p(out), _p(work))
    return out


def restrict(rh) -> np.ndarray:
    """Coarse scaled right-hand side 4 R rh (full weighting)."""
    rh = _f64(rh)
    d, n = _dim_n(rh)
    nc = (n - 1) // 2
    out = np.empty((nc,) * d)
    lib().orc_restrict(d, n, _p(rh), _p(out))
    return out


def prolong_add(e_c, u) -> np.ndarray:
    """u + P e_c (bilinear / trilinear interpolation), returned as a new array."""
    e_c = _f64(e_c)
    d, nc = _dim_n(e_c)
    out = _f64(u).copy()
    if out.shape != (2 * nc + 1,) * d:
        raise ValueError("fine array must have 2 nc + 1 points per axis")
    lib().orc_prolong_add(d, out.shape[0], _p(e_c), _p(out))
    return out


def coarse_solve(bh) -> np.ndarray:
    """Exact solve of h0^2 A_h0 x = bh on the 3^d coarsest grid."""
    bh = _f64(bh)
    d, n = _dim_n(bh)
    if n != 3:
        raise ValueError("the coarsest grid has 3 interior points per axis")
    x = np.empty_like(bh)
    lib().orc_coarse_solve(d, _p(bh), _p(x))
    return x


# ---------------------------------------------------------------------------
# cycles and solve (Sec. 4)
# ---------------------------------------------------------------------------

def _N_of(u) -> int:
    return u.shape[0] + 1


def residual_norm(u, b) -> float:
    """||b - A_h u||_2 on the finest grid (b unscaled)."""
    u, b = _f64(u), _f64(b)
    d, n = _dim_n(u)
    return float(lib().orc_residual_norm(d, n + 1, _p(u), _p(b)))


def cycles(b, u0, c, ncycles: int, nu1: int = 1, nu2: int = 1, gamma: int = 1) -> np.ndarray:
    """Apply `ncycles` V (gamma=1) or W (gamma=2) cycles to u0."""
    b = _f64(b)
    u = _f64(u0).copy()
    d, n = _dim_n(b)
    cc = _coeffs(d, c)
    st = lib().orc_cycles(d, n + 1, _p(cc), 3 if d == 2 else 4, nu1, nu2, gamma, ncycles, _p(b), _p(u))
    if st != ORC_OK:
        raise ValueError(f"orc_cycles failed with status {st}")
    return u


class SolveResult:
    def __init__(self, u, status, cycles, relres, hist):
        self.u = u
        self.status = status
        self.cycles = cycles
        self.relres = relres
        self.hist = hist

    @property
    def converged(self) -> bool:
        return self.status == ORC_OK

    def rate(self) -> float:
        """rho^(k) = (||r_k|| / ||r_0||)^(1/k) at the last cycle (Eq. (4.1))."""
        k = self.cycles
        return float((self.hist[k] / self.hist[0]) ** (1.0 / k)) if k > 0 else 0.0


def solve(b, c, u0=None, tol: float = 1e-10, max_cycles: int = 100, nu1: int = 1, nu2: int = 1,
          gamma: int = 1) -> SolveResult:
    b = _f64(b)
    d, n = _dim_n(b)
    u = np.zeros_like(b) if u0 is None else _f64(u0).copy()
    cc = _coeffs(d, c)
    hist = np.zeros(max_cycles + 1)
    cyc = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = lib().orc_solve(d, n + 1, _p(cc), 3 if d == 2 else 4, nu1, nu2, gamma, _p(b), _p(u), tol,
                         max_cycles, _p(hist), ctypes.byref(cyc), ctypes.byref(rel))
    if st not in (ORC_OK, ORC_ENOCONV):
        raise ValueError(f"orc_solve failed with status {st}")
    return SolveResult(u, st, cyc.value, rel.value, hist[: cyc.value + 1].copy())


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
