"""Pins of the oracle's adjoint of K cycles (oracle/adjoint.py).

- its taped forward equals the C cycles bit for bit;
- dot-product identity <M b, g> = <b, M^T g> for the linear map b -> u_K;
- for V(nu, nu) cycles the map M is symmetric (symmetric sweep error
  operator, P = 2^d R^T, symmetric coarsest solve), so M^T g = M g: the
  adjoint w.r.t. b equals K forward cycles applied to g;
- FP64 central finite differences of L = 1/2 ||u_K - u*||^2 (u* the exact
  discrete solution, held fixed) w.r.t. entries of b and every weight c_j,
  relative error <= 1e-5 (L is exactly quadratic in b, so the differences
  in b only carry rounding error).
"""
import numpy as np
import pytest

import oracle
from oracle import adjoint, coeffs, exact


def _setup(d, N, seed=0):
    b = np.random.default_rng(seed).standard_normal((N - 1,) * d)
    return b, coeffs.default(d)


@pytest.mark.parametrize("d,N,nu1,nu2", [(2, 16, 1, 1), (2, 32, 2, 1), (3, 16, 1, 1), (3, 8, 1, 2)])
def test_taped_forward_matches_c_cycles(d, N, nu1, nu2):
    b, c = _setup(d, N)
    u, _ = adjoint.forward(b, c, 3, nu1, nu2)
    assert np.array_equal(u, oracle.cycles(b, np.zeros_like(b), c, 3, nu1, nu2))


@pytest.mark.parametrize("d,N,nu1,nu2", [(2, 32, 1, 1), (2, 16, 2, 1), (3, 16, 1, 1), (3, 8, 1, 2)])
def test_dot_product_identity(d, N, nu1, nu2):
    b, c = _setup(d, N, 1)
    rng = np.random.default_rng(2)
    g, b2 = rng.standard_normal(b.shape), rng.standard_normal(b.shape)
    Mb2 = oracle.cycles(b2, np.zeros_like(b2), c, 4, nu1, nu2)
    gb, _ = adjoint.vcycles_adjoint(b, c, 4, g, nu1, nu2)
    lhs, rhs = float(np.vdot(Mb2, g)), float(np.vdot(b2, gb))
    assert lhs == pytest.approx(rhs, rel=1e-12)


@pytest.mark.parametrize("d,N", [(2, 32), (3, 16)])
def test_symmetric_cycle_adjoint_is_forward(d, N):
    b, c = _setup(d, N, 3)
    g = np.random.default_rng(4).standard_normal(b.shape)
    gb, _ = adjoint.vcycles_adjoint(b, c, 4, g)
    Mg = oracle.cycles(g, np.zeros_like(g), c, 4)
    np.testing.assert_allclose(gb, Mg, rtol=0, atol=1e-13 * np.abs(Mg).max())


def _loss(b, c, K, ustar):
    u = oracle.cycles(b, np.zeros_like(b), c, K)
    return 0.5 * float(np.sum((u - ustar) ** 2))


@pytest.mark.parametrize("d,N", [(2, 32), (3, 16)])
def test_finite_differences(d, N):
    K = 4
    b, c = _setup(d, N, 5)
    ustar = exact.dst_solve(b)
    uK = oracle.cycles(b, np.zeros_like(b), c, K)
    gb, gc = adjoint.vcycles_adjoint(b, c, K, uK - ustar)
    rng = np.random.default_rng(6)
    flat = rng.choice(b.size, 6, replace=False)
    for i in flat:
        eps = 1e-2
        bp, bm = b.copy(), b.copy()
        bp.flat[i] += eps
        bm.flat[i] -= eps
        fd = (_loss(bp, c, K, ustar) - _loss(bm, c, K, ustar)) / (2 * eps)
        assert gb.flat[i] == pytest.approx(fd, rel=1e-5, abs=1e-12 * np.abs(gb).max())
    for j in range(len(c)):
        eps = 1e-6 * abs(c[j])
        cp, cm = list(c), list(c)
        cp[j] += eps
        cm[j] -= eps
        fd = (_loss(b, cp, K, ustar) - _loss(b, cm, K, ustar)) / (2 * eps)
        assert gc[j] == pytest.approx(fd, rel=1e-5)
