"""Exact discrete solutions and matrix forms of the operators (oracle side).

TEST INFRASTRUCTURE (see the package docstring).

- ``laplacian``: A_h of Eq. (1.3) assembled from Kronecker products of the 1D
  second difference T = tridiag(-1, 2, -1) (independent of the stencil loops
  in mg_oracle.c), as a scipy sparse matrix.
- ``spai_matrix``: the omega-folded SPAI stencil restricted to the interior,
  c0 I + c1 (edge/face sum) + c2 (corner sum) in 2D, c0 I + c1 (faces) +
  c2 (edges) + c3 (corners) in 3D, from the 1D neighbour-sum matrix
  Z = tridiag(1, 0, 1).
- ``restriction`` / ``prolongation``: full weighting R = kron of the 1D
  (1, 2, 1)/4 matrix, P = 2^d R^T (Sec. 4).
- ``dst_solve``: the exact discrete solution of A_h u = b by the sine
  transform that diagonalises A_h (eigenvalues (2/h^2) sum (1 - cos k pi h)).
- ``manufactured_factor``: for u = prod sin(pi x_i) the grid function is an
  eigenvector of A_h, so u_h = [pi^2 h^2 / (2 (1 - cos pi h))] u on the grid
  (the O(h^2) statement of Sec. 1 with an exact target).
"""
from __future__ import annotations

from functools import reduce

import numpy as np
import scipy.fft
import scipy.sparse as sp


def _kron_all(mats):
    return reduce(lambda a, b: sp.kron(a, b, format="csr"), mats)


def _second_difference(n: int):
    return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")


def _neighbour_sum(n: int):
    return sp.diags([np.ones(n - 1), np.ones(n - 1)], [-1, 1], format="csr")


def laplacian(d: int, N: int):
    """Sparse A_h (h = 1/N) on (N-1)^d interior points, x fastest."""
    n = N - 1
    T, I = _second_difference(n), sp.identity(n, format="csr")
    terms = []
    for axis in range(d):
        # axis 0 is x (fastest) => last Kronecker factor
        mats = [I] * d
        mats[d - 1 - axis] = T
        terms.append(_kron_all(mats))
    return (float(N) ** 2) * reduce(lambda a, b: a + b, terms)


def spai_matrix(d: int, N: int, c):
    """Interior-restricted stencil: 2D c0 I + c1 (edges) + c2 (corners); 3D c0 I +
    c1 (faces) + c2 (edges) + c3 (corners)."""
    n = N - 1
    Z, I = _neighbour_sum(n), sp.identity(n, format="csr")
    W = c[0] * _kron_all([I] * d)
    faces = []
    for axis in range(d):
        mats = [I] * d
        mats[d - 1 - axis] = Z
        faces.append(_kron_all(mats))
    W = W + c[1] * reduce(lambda a, b: a + b, faces)
    if d == 2 and len(c) > 2 and c[2] != 0.0:
        W = W + c[2] * sp.kron(Z, Z, format="csr")
    if d == 3 and len(c) > 2:
        # 12 edge offsets: Z on two of the three axes; 8 corners: Z on all three
        edges = [_kron_all([Z if k != skip else I for k in range(3)]) for skip in range(3)]
        W = W + c[2] * reduce(lambda a, b: a + b, edges)
        if len(c) > 3:
            W = W + c[3] * _kron_all([Z, Z, Z])
    return W


def restriction_1d(nf: int):
    nc = (nf - 1) // 2
    R = sp.lil_matrix((nc, nf))
    for J in range(1, nc + 1):  # coarse J <-> fine 2J (1-based)
        R[J - 1, 2 * J - 2] = 0.25
        R[J - 1, 2 * J - 1] = 0.5
        R[J - 1, 2 * J] = 0.25
    return R.tocsr()


def restriction(d: int, nf: int):
    return _kron_all([restriction_1d(nf)] * d)


def prolongation(d: int, nf: int):
    return (2 ** d) * restriction(d, nf).T.tocsr()


def dst_solve(b: np.ndarray) -> np.ndarray:
    """Exact u = A_h^{-1} b for an (n,)*d array b (n = N-1), via DST-I."""
    b = np.asarray(b, dtype=np.float64)
    d, n = b.ndim, b.shape[0]
    N = n + 1
    k = np.arange(1, n + 1)
    # eigenvalues of the 1D operator, 2 (1 - cos(k pi h)) / h^2 = 4 sin^2(k pi h / 2) / h^2
    lam1 = 4.0 * np.sin(np.pi * k / (2.0 * N)) ** 2 * N * N
    lam = reduce(np.add.outer, [lam1] * d)
    # DST-I with orthonormal scaling is its own inverse
    bt = scipy.fft.dstn(b, type=1, norm="ortho")
    return scipy.fft.idstn(bt / lam, type=1, norm="ortho")


def grid_coords(d: int, N: int):
    x = np.arange(1, N) / N
    return np.meshgrid(*([x] * d), indexing="ij")[::-1]  # (x, y[, z]) with x fastest


def sine_product(d: int, N: int) -> np.ndarray:
    """prod_i sin(pi x_i) on the interior grid, array order [y, x] / [z, y, x]."""
    xs = np.arange(1, N) / N
    s = np.sin(np.pi * xs)
    return reduce(np.multiply.outer, [s] * d)


def manufactured_rhs(d: int, N: int) -> np.ndarray:
    """b_h = f on the grid for u = prod sin(pi x_i): f = d pi^2 u, g = 0."""
    return d * np.pi ** 2 * sine_product(d, N)


def manufactured_factor(N: int) -> float:
    """u_h / u on the grid for the sine manufactured solution (any d)."""
    h = 1.0 / N
    # 1 - cos(pi h) = 2 sin^2(pi h / 2), written without cancellation
    return np.pi ** 2 * h * h / (4.0 * np.sin(np.pi * h / 2.0) ** 2)
