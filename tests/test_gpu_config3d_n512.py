"""Full-size parity of the 3D workload (Example 3 of Sec. 4: N = 512,
511^3 = 133,432,831 unknowns, 7-point Laplacian, M7 smoother of Theorem 3.2,
V(2,2) cycles) against the FP64 oracle, in the launch configurations the
benchmark times.

- Each FP64 3D operator (sweep with and without the fused residual norm, and
  from zero; residual + full weighting; interpolation + correction) is
  compared with the oracle over the WHOLE array, bit for bit, at n = 255 and
  n = 511: the persistent sweep splits (tile, plane) items into z-segments
  whose seams depend on n and on the SM count, so sampled points are not
  enough.
- The FP64 solve on the uniform right-hand side (seed 0): the first two
  cycles' iterates bit for bit and r_0..r_2 within 1e-12 relative.
- The manufactured sine problem u = sin(pi x) sin(pi y) sin(pi z), in FP64
  and in FP32-in-FP64 refinement, solved to 1e-10: the oracle's FP64
  residual of each result; the distance to the exact discrete solution
  u_h = F u (F = pi^2 h^2 / (2 (1 - cos pi h)), F - 1 = 3.137e-6 at N = 512),
  which the residual bounds: b is an eigenvector of A_h for its smallest
  eigenvalue lambda, so ||u - u_h|| <= ||r|| / lambda and ||u_h|| =
  ||b|| / lambda give ||u - u_h|| / ||u_h|| <= ||r|| / ||b||; the distance
  to the continuous solution, F - 1; and the two precisions against each
  other, within the sum of their residual bounds. The computed residual
  carries rounding noise of at most about 12 eps N^2 ||u|| (the stencil's
  terms are up to 6 N^2 |u| each), which is added to the bounds.

The oracle runs its grid loops on every host core here (its results do not
depend on the thread count).
"""
import os

import numpy as np
import pytest

import oracle
from oracle import coeffs, exact
from paper_2206_05543_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_05543_gb300 import binding  # noqa: E402
from paper_2206_05543_gb300.binding import Solver  # noqa: E402

N = 512


@pytest.fixture(scope="module", autouse=True)
def _oracle_threads():
    oracle.set_threads(len(os.sched_getaffinity(0)))
    yield
    oracle.set_threads(1)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float64)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("n", [255, 511])
def test_fp64_3d_operators_whole_array_bitwise(n):
    w = coeffs.default(3)
    rng = np.random.default_rng(n)
    u = rng.uniform(-1, 1, (n,) * 3)
    b = rng.uniform(-1, 1, (n,) * 3)
    h2 = 1.0 / (n + 1) ** 2
    bh = h2 * b
    ref = oracle.sweep(u, bh, w)
    out, nrm = binding.op_sweep(dev(u), dev(b), w, b_unscaled=True, want_norm=True)
    assert np.array_equal(host(out), ref)
    del out
    rh = oracle.residual_scaled(u, bh)
    assert nrm == pytest.approx(float(np.sum(rh * rh)), rel=1e-12)
    out, _ = binding.op_sweep(dev(u), dev(bh), w)
    assert np.array_equal(host(out), ref)
    del out, ref
    out0, _ = binding.op_sweep(None, dev(bh), w)
    assert np.array_equal(host(out0), oracle.sweep(np.zeros_like(u), bh, w))
    del out0
    got = binding.op_residual_restrict(dev(u), dev(b), b_unscaled=True)
    assert np.array_equal(host(got), oracle.restrict(rh))
    del got, rh
    nc = (n - 1) // 2
    e = rng.uniform(-1, 1, (nc,) * 3)
    got = binding.op_prolong_correct(dev(e), dev(u))
    assert np.array_equal(host(got), oracle.prolong_add(e, u))


def test_config_3d_n512_fp64_two_cycles_bitwise():
    """Uniform b (seed 0), zero start, FP64 V(2,2) with M7: u_1, u_2 and
    r_0..r_2 as the benchmark's solver computes them."""
    b = inputs.uniform(3, N, 0)
    w = coeffs.default(3)
    ref = oracle.solve(b, w, tol=0.0, max_cycles=2, nu1=2, nu2=2)
    with Solver(3, N, w, nu1=2, nu2=2) as s:
        info = s.solve(dev(b), tol=0.0, max_cycles=2)
        got = host(info.u)
    assert info.cycles == 2
    np.testing.assert_allclose(info.hist, ref.hist, rtol=1e-12, atol=0)
    assert np.array_equal(got, ref.u)


def test_config_3d_n512_sine_fp64_and_mixed():
    b = inputs.sine(3, N)
    nb = float(np.linalg.norm(b))
    sp_ = exact.sine_product(3, N)
    F = exact.manufactured_factor(N)
    assert F - 1.0 == pytest.approx(3.137e-6, rel=1e-3)
    uh = F * sp_
    nuh, nsp = float(np.linalg.norm(uh)), float(np.linalg.norm(sp_))
    sols, rel = {}, {}
    for prec in ("fp64", "fp32_ir"):
        with Solver(3, N, coeffs.default(3), nu1=2, nu2=2, precision=prec) as s:
            info = s.solve(dev(b), tol=1e-10, max_cycles=40)
            u = host(info.u)
        assert info.converged, prec
        r = oracle.residual_norm(u, b)
        rel[prec] = r / nb
        assert rel[prec] <= 1e-10 * (1 + 1e-6), prec
        noise = 12 * np.finfo(np.float64).eps * N ** 2 * float(np.linalg.norm(u)) / nb
        rel[prec] += noise
        # algebraic error, bounded by the relative residual
        assert np.linalg.norm(u - uh) / nuh <= rel[prec] * (1 + 1e-6), prec
        # discretisation error of the converged solution: F - 1 (Sec. 1, O(h^2))
        assert np.linalg.norm(u - sp_) / nsp == pytest.approx(F - 1.0, abs=2e-10), prec
        sols[prec] = u
    diff = np.linalg.norm(sols["fp32_ir"] - sols["fp64"]) / np.linalg.norm(sols["fp64"])
    assert diff <= (rel["fp64"] + rel["fp32_ir"]) * (1 + 1e-6)
