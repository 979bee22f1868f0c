"""Pins of the oracle's grid operators and cycle against independent forms.

Each operator of mg_oracle.c (stencil loops) is checked against a matrix
assembled from Kronecker products of 1D matrices (oracle/exact.py), the
multigrid solution against a dense Cholesky solve (N <= 16) and the sine
transform, the discretisation against the closed-form discrete solution of
the sine manufactured problem (O(h^2), Sec. 1), and the cycle's convergence
rates against LFA-consistent bands (Sec. 4, Table 1).
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import coeffs, exact
from paper_2206_05543_gb300 import inputs

SMOOTHERS = [(2, "m9"), (2, "jacobi"), (2, "m5"), (2, "vanka"), (2, "tw5"), (3, "m7"), (3, "jacobi")]


def _rand(d, n, seed):
    return np.random.default_rng(seed).uniform(-1, 1, (n,) * d)


@pytest.mark.parametrize("d,N", [(2, 4), (2, 16), (2, 32), (3, 4), (3, 8), (3, 16)])
def test_residual_matches_matrix(d, N):
    u, b = _rand(d, N - 1, 1), _rand(d, N - 1, 2)
    h2 = 1.0 / N ** 2
    rh = oracle.residual_scaled(u, h2 * b)
    ref = b.ravel() - exact.laplacian(d, N) @ u.ravel()
    np.testing.assert_allclose(rh.ravel() / h2, ref, rtol=0, atol=1e-12 * np.abs(ref).max() * N ** 2)
    assert oracle.residual_norm(u, b) == pytest.approx(np.linalg.norm(ref), rel=1e-12)


@pytest.mark.parametrize("d,name", SMOOTHERS)
@pytest.mark.parametrize("N", [8, 16])
def test_sweep_matches_matrix(d, name, N):
    """u' = u + omega M_h (b - A_h u) with M_h the stencil restricted to the
    interior (Sec. 2 Eq. (2.1)); weights folded as c_j = omega m_j / h^2."""
    c = coeffs.weights(d, name)
    u, b = _rand(d, N - 1, 3), _rand(d, N - 1, 4)
    h2 = 1.0 / N ** 2
    out = oracle.sweep(u, h2 * b, c)
    A = exact.laplacian(d, N)
    W = exact.spai_matrix(d, N, c)
    ref = u.ravel() + W @ (h2 * (b.ravel() - A @ u.ravel()))
    np.testing.assert_allclose(out.ravel(), ref, rtol=1e-13, atol=1e-15)


def test_sweep_symmetric_error_operator():
    """M_h and A_h commute (both are diagonalised by the sine basis), so the
    error operator S = I - omega M A of one sweep is symmetric."""
    for d, N in ((2, 8), (3, 4)):
        c = coeffs.default(d)
        n = N - 1
        m = n ** d
        S = np.empty((m, m))
        zero = np.zeros((n,) * d)
        for j in range(m):
            e = np.zeros(m)
            e[j] = 1.0
            S[:, j] = oracle.sweep(e.reshape((n,) * d), zero, c).ravel()
        np.testing.assert_allclose(S, S.T, atol=1e-15)


@pytest.mark.parametrize("d,N", [(2, 8), (2, 32), (3, 8), (3, 16)])
def test_restriction_and_prolongation_match_matrices(d, N):
    n = N - 1
    rh = _rand(d, n, 5)
    bc = oracle.restrict(rh)
    np.testing.assert_allclose(bc.ravel(), 4.0 * (exact.restriction(d, n) @ rh.ravel()), rtol=1e-14,
                               atol=1e-15)
    e = _rand(d, (n - 1) // 2, 6)
    u = _rand(d, n, 7)
    out = oracle.prolong_add(e, u)
    np.testing.assert_allclose(out.ravel(), u.ravel() + exact.prolongation(d, n) @ e.ravel(),
                               rtol=1e-14, atol=1e-15)


def test_transfer_scaling_is_variational():
    """P = 2^d R^T: <restrict(r), e> 2^d / 4 = <r, P e> for random r, e."""
    for d, N in ((2, 16), (3, 8)):
        n = N - 1
        r, e = _rand(d, n, 8), _rand(d, (n - 1) // 2, 9)
        lhs = np.vdot(oracle.restrict(r), e) * 2 ** d / 4.0
        rhs = np.vdot(r, oracle.prolong_add(e, np.zeros_like(r)))
        assert lhs == pytest.approx(rhs, rel=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_coarse_solve(d):
    bh = _rand(d, 3, 10)
    x = oracle.coarse_solve(bh)
    A = exact.laplacian(d, 4) / 16.0  # h0^2 A_h0
    np.testing.assert_allclose(A @ x.ravel(), bh.ravel(), rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("d,N", [(2, 4), (2, 8), (2, 16), (3, 8), (3, 16)])
def test_multigrid_matches_dense_cholesky(d, N):
    b = _rand(d, N - 1, 11)
    res = oracle.solve(b, coeffs.default(d), tol=1e-13, max_cycles=60)
    assert res.converged
    A = exact.laplacian(d, N).toarray()
    ref = scipy.linalg.cho_solve(scipy.linalg.cho_factor(A), b.ravel())
    np.testing.assert_allclose(res.u.ravel(), ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_dst_solver_is_exact():
    b = _rand(2, 31, 12)
    u = exact.dst_solve(b)
    r = b.ravel() - exact.laplacian(2, 32) @ u.ravel()
    assert np.abs(r).max() < 1e-11


@pytest.mark.parametrize("d,Ns", [(2, (16, 32, 64, 128)), (3, (8, 16, 32))])
def test_second_order_accuracy(d, Ns):
    """Sec. 1: ||u_h - u||_inf = O(h^2); for u = prod sin(pi x_i) the discrete
    solution is known in closed form, which pins the solve itself."""
    errs = []
    for N in Ns:
        b = exact.manufactured_rhs(d, N)
        res = oracle.solve(b, coeffs.default(d), tol=1e-12, max_cycles=60)
        u = exact.sine_product(d, N)
        uh = exact.manufactured_factor(N) * u
        assert np.abs(res.u - uh).max() <= 1e-10 * np.abs(uh).max()
        errs.append(np.abs(res.u - u).max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    np.testing.assert_allclose(ratios, 4.0, rtol=0.02)


def test_manufactured_rhs_of_inputs_module():
    """The shared input generator's sine workload is d pi^2 prod sin."""
    for d, N in ((2, 16), (3, 8)):
        np.testing.assert_allclose(inputs.sine(d, N), exact.manufactured_rhs(d, N), rtol=1e-15)


# V-cycle rates from zero start, uniform b, to 1e-10 (Sec. 4 setting): the
# measured rho^(k) must sit near the LFA two-grid factors of Table 1.
RATE_BANDS = [
    # d, N, smoother, nu1, nu2, gamma, cycles range, rate range
    (2, 64, "m9", 1, 1, 1, (9, 11), (0.08, 0.12)),
    (2, 256, "m9", 1, 1, 1, (9, 11), (0.08, 0.12)),
    (2, 64, "jacobi", 1, 1, 1, (19, 23), (0.30, 0.37)),
    (2, 64, "m5", 1, 1, 1, (10, 14), (0.10, 0.16)),
    (2, 64, "m9", 1, 0, 2, (11, 15), (0.13, 0.19)),  # W(1+0)
    (3, 32, "m7", 1, 1, 1, (11, 13), (0.12, 0.17)),
    (3, 32, "m7", 2, 2, 1, (8, 10), (0.06, 0.09)),
    (3, 32, "jacobi", 1, 1, 1, (20, 40), (0.35, 0.60)),
]


@pytest.mark.parametrize("d,N,name,nu1,nu2,gamma,cyc,rate", RATE_BANDS)
def test_cycle_rates(d, N, name, nu1, nu2, gamma, cyc, rate):
    b = inputs.uniform(d, N, 0)
    res = oracle.solve(b, coeffs.weights(d, name), tol=1e-10, max_cycles=100, nu1=nu1, nu2=nu2, gamma=gamma)
    assert res.converged
    assert cyc[0] <= res.cycles <= cyc[1]
    assert rate[0] <= res.rate() <= rate[1]
    # the history is monotone and ends below the tolerance
    assert np.all(np.diff(res.hist) < 0)
    assert res.hist[-1] <= 1e-10 * res.hist[0]


def test_residual_norm_is_accurately_summed():
    """||b - A u||_2 (Eq. (4.1)) on a 1M-point grid agrees with an exactly
    rounded sum (math.fsum) of the squared residual to 1e-14."""
    import math
    N = 1024
    u, b = _rand(2, N - 1, 21), _rand(2, N - 1, 22)
    r = b.ravel() - exact.laplacian(2, N) @ u.ravel()
    ref = math.sqrt(math.fsum(r * r))
    assert oracle.residual_norm(u, b) == pytest.approx(ref, rel=1e-14)


def test_oracle_results_do_not_depend_on_thread_count():
    """The grid loops may run on several threads (timing); every point is
    still computed by one thread in the same order, so cycles are identical."""
    import os
    for d, N in ((2, 64), (3, 16)):
        b = np.random.default_rng(11).uniform(-1, 1, (N - 1,) * d)
        c = coeffs.default(d)
        try:
            oracle.set_threads(1)
            one = oracle.cycles(b, np.zeros_like(b), c, 2)
            oracle.set_threads(max(2, os.cpu_count() or 2))
            many = oracle.cycles(b, np.zeros_like(b), c, 2)
        finally:
            oracle.set_threads(1)
        assert np.array_equal(one, many)
