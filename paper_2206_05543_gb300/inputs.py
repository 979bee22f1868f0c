"""Seeded synthetic right-hand sides for the Poisson workloads.

This module only draws numbers and evaluates the source terms f of the model
problems; it holds none of the multigrid arithmetic. Both the CUDA library's
tests/benchmark and the CPU oracle are fed from it, so it imports neither.

Layout: interior points only, row-major with x fastest, shape (n,)*d with
n = N - 1; array index i is the grid point (i + 1)/N.

Workloads (sizes of the paper's experiments, Sec. 4):
  - uniform(d, N, seed):   b ~ U[-1, 1] i.i.d., numpy default_rng(seed), FP64;
  - gaussian(d, N, seed):  b ~ N(0, 1) i.i.d.;
  - sine(d, N):            f = d pi^2 prod sin(pi x_i), u = prod sin(pi x_i), g = 0
                           (Example 3 in 3D; its 2D analogue);
  - example1(N):           Example 1, f = 2(1-6x^2)(y^2-y^4) + 2(1-6y^2)(x^2-x^4), g = 0;
  - example2(N):           Example 2, f = -x ln(x)/y - y ln(y)/x, g = 0;
  - batch_sizes(count, seed): grid sizes drawn from {64, 128, 256, 512, 1024}.
"""
from __future__ import annotations

import numpy as np


def _axis(N: int) -> np.ndarray:
    return np.arange(1, N, dtype=np.float64) / N


def uniform(d: int, N: int, seed: int = 0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(N - 1,) * d)


def gaussian(d: int, N: int, seed: int = 0) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(size=(N - 1,) * d)


def sine(d: int, N: int) -> np.ndarray:
    s = np.sin(np.pi * _axis(N))
    out = s
    for _ in range(d - 1):
        out = np.multiply.outer(s, out)
    return d * np.pi ** 2 * out


def example1(N: int) -> np.ndarray:
    x = _axis(N)[None, :]
    y = _axis(N)[:, None]
    return 2 * (1 - 6 * x ** 2) * (y ** 2 - y ** 4) + 2 * (1 - 6 * y ** 2) * (x ** 2 - x ** 4)


def example2(N: int) -> np.ndarray:
    x = _axis(N)[None, :]
    y = _axis(N)[:, None]
    return -x * np.log(x) / y - y * np.log(y) / x


def batch_sizes(count: int = 256, seed: int = 0) -> np.ndarray:
    return np.random.default_rng(seed).choice([64, 128, 256, 512, 1024], count)


def batch_rhs(sizes, first_seed: int = 1):
    """Problem i gets b_i ~ U[-1, 1] from default_rng(first_seed + i)."""
    return [uniform(2, int(N), first_seed + i) for i, N in enumerate(sizes)]
