"""Pins of the oracle's numerical min-max over stencil families (Sec. 3) and
of its 27-point 3D sweep.

- From scratch (centre weight 1, the other class weights searched), the
  min-max recovers the paper's optima: M9 = Upsilon(44, 10, 3)/24 with
  omega = (309 - 12 sqrt 10)/1720 (Theorem 3.1), M7 = T(8/5, 2/5) with
  omega = 20/73 (Theorem 3.2), the best 5-point M5 with omega = 1/4 and the
  weighted Jacobi factors 3/5 and 5/7 (Sec. 3.1, 3.2): folded weights to
  1e-6, smoothing factors to 1e-9.
- The 19- and 27-point 3D optima (Sec. 3.2 names them, prints no weights;
  tests/golden/wide_smoothers.txt, written by make_wide_smoothers.py) are
  reproduced by a fresh run, are local minima of mu, improve on M7, and equal
  the library's constants.
- The 27-point oracle sweep equals u + W (bh - h^2 A u) with W assembled from
  Kronecker products (independent of the stencil loops), its error operator
  is symmetric, and power iteration of the periodic sweep on the high
  frequencies gives the LFA smoothing factor of the same weights.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import coeffs, exact, lfa
from conftest import read_golden
from paper_2206_05543_gb300 import smoothers

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

SQRT10 = math.sqrt(10.0)


def _folded(w, om):
    return np.array([om * x for x in w])


@pytest.mark.parametrize("family,expect_c,expect_mu", [
    ("nine", coeffs.default(2), (9 + 8 * SQRT10) / 215),   # Theorem 3.1
    ("seven", coeffs.default(3), 25 / 73),                 # Theorem 3.2
    ("five", coeffs.weights(2, "m5"), 9 / 41),            # Sec. 3.1, M5
    ("jacobi2", coeffs.weights(2, "jacobi"), 3 / 5),       # Sec. 3.1, M_J
    ("jacobi3", coeffs.weights(3, "jacobi"), 5 / 7),       # Sec. 3.2, M_J
])
def test_minmax_recovers_the_papers_optima_from_scratch(family, expect_c, expect_mu):
    w, mu, om = lfa.optimise_family(family)
    assert w[0] == 1.0
    expect = np.array(expect_c)
    # the 5-point family has no corner class: the paper's M5 has a zero corner weight
    assert np.all(expect[len(w):] == 0.0)
    np.testing.assert_allclose(_folded(w, om), expect[: len(w)], rtol=1e-6, atol=0)
    assert mu == pytest.approx(expect_mu, abs=1e-9)


def _wide():
    rows = {}
    for r in read_golden("wide_smoothers.txt"):
        rows.setdefault(r[0], {})[r[1]] = [float(x) for x in r[2:]]
    return rows


@pytest.mark.parametrize("family,const", [("nineteen", smoothers.M19), ("twentyseven", smoothers.M27)])
def test_wide_3d_optima(family, const):
    g = _wide()[family]
    # the library's constants are the golden folded weights
    assert tuple(const) == tuple(g["c"])
    # a fresh run of the min-max reproduces them
    w, mu, om = lfa.optimise_family(family)
    np.testing.assert_allclose(_folded(w, om), g["c"], rtol=1e-8, atol=0)
    assert mu == pytest.approx(g["mu"][0], abs=1e-10)
    # better than M7 (Theorem 3.2's optimum over the 7-point family)
    assert mu < 25 / 73 - 0.1
    # a local minimum: moving any non-centre class weight raises mu
    base = lfa.class_mu(3, g["w"])
    assert base == pytest.approx(mu, abs=1e-10)
    for j in range(1, len(g["w"])):
        for step in (-1e-4, 1e-4):
            p = list(g["w"])
            p[j] += step
            assert lfa.class_mu(3, p) > base
    # the folded weights balance the extremes: |1 - l0| = |1 - l1| = mu
    l0, l1 = lfa.class_extremes(3, g["c"])
    assert 1 - l0 == pytest.approx(mu, abs=1e-10) and l1 - 1 == pytest.approx(mu, abs=1e-10)


def test_the_27_point_family_contains_the_19_point_one():
    assert _wide()["twentyseven"]["mu"][0] < _wide()["nineteen"]["mu"][0]


def test_class_symbol_matches_the_two_2d_and_3d_symbols():
    """class_product with the 7-point / 9-point weights equals the symbols of
    Sec. 3 used by the closed-form checks (product_symbol)."""
    rng = np.random.default_rng(0)
    for d, w in ((2, (1.0, 0.3, 0.07)), (3, (1.0, 0.2))):
        x = rng.uniform(-1, 1, (50, d))
        np.testing.assert_allclose(lfa.class_product(d, w, x), lfa.product_symbol(d, w, x), rtol=1e-14)


@pytest.mark.parametrize("name,c", [("m27", smoothers.M27), ("m19", smoothers.M19)])
@pytest.mark.parametrize("N", [4, 8])
def test_27_point_sweep_matches_matrix(name, c, N):
    d = 3
    rng = np.random.default_rng(N)
    u, b = rng.uniform(-1, 1, (N - 1,) * 3), rng.uniform(-1, 1, (N - 1,) * 3)
    h2 = 1.0 / N ** 2
    out = oracle.sweep(u, h2 * b, c)
    A = exact.laplacian(d, N)
    W = exact.spai_matrix(d, N, c)
    ref = u.ravel() + W @ (h2 * (b.ravel() - A @ u.ravel()))
    np.testing.assert_allclose(out.ravel(), ref, rtol=1e-13, atol=1e-15)


def test_27_point_sweep_error_operator_is_symmetric():
    c = smoothers.M27
    n = 3
    m = n ** 3
    zero = np.zeros((n,) * 3)
    S = np.empty((m, m))
    for j in range(m):
        e = np.zeros(m)
        e[j] = 1.0
        S[:, j] = oracle.sweep(e.reshape((n,) * 3), zero, c).ravel()
    np.testing.assert_allclose(S, S.T, atol=1e-15)


def test_power_iteration_periodic_27_point_sweep():
    """The oracle's periodic 27-point sweep with b = 0 applies S = I - omega M A;
    on the high frequencies its largest |eigenvalue| is mu of the weights."""
    from test_oracle_lfa import _high_projection, _krylov_extreme

    c = smoothers.M27
    n = 64
    rng = np.random.default_rng(3)
    zero = np.zeros((n,) * 3)
    v0 = _high_projection(rng.standard_normal((n,) * 3))
    est = _krylov_extreme(lambda v: _high_projection(oracle.sweep(v, zero, c, periodic=True)), v0, 80)
    l0, l1 = lfa.class_extremes(3, c)
    assert est == pytest.approx(max(abs(1 - l0), abs(1 - l1)), abs=1e-3)


@pytest.mark.parametrize("name,c,nu", [("m27", smoothers.M27, 1), ("m27", smoothers.M27, 2), ("m7", smoothers.M7, 2)])
def test_v_cycle_rates_of_the_wide_smoother(name, c, nu):
    """The oracle's V(nu,nu) cycle with the 27-point smoother converges to
    1e-10 faster per cycle than with M7 (3D N = 32, uniform b)."""
    b = np.random.default_rng(5).uniform(-1, 1, (31,) * 3)
    r = oracle.solve(b, c, tol=1e-10, nu1=nu, nu2=nu)
    assert r.converged
    if name == "m27":
        r7 = oracle.solve(b, smoothers.M7, tol=1e-10, nu1=nu, nu2=nu)
        assert r.cycles < r7.cycles
        assert r.rate() < r7.rate()
