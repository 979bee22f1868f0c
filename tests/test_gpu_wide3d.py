"""GPU parity of the 27-point (and 19-point) 3D SPAI sweep against the FP64
oracle, through the C ABI.

The weights are the LFA min-max optima of the symmetric 19- and 27-point
families (Sec. 3.2's closing remark; tests/golden/wide_smoothers.txt, pinned
in test_oracle_lfa_optimiser.py). The kernel evaluates the oracle's
operation order (x pairs, in-plane edge and corner sums, then faces, edges
and corners across planes), so FP64 results must be identical: single
sweeps (from u and from zero, scaled and unscaled right-hand side, with the
fused residual norm) up to n = 127 here and the whole n = 255 / 511 arrays in
the slow tests, and whole solves (iterates bit for bit, per-cycle residual
norms within 1e-12 relative).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2206_05543_gb300 import inputs, smoothers

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_05543_gb300 import binding  # noqa: E402
from paper_2206_05543_gb300.binding import MGError, Solver  # noqa: E402

WIDE = {"m27": smoothers.M27, "m19": smoothers.M19}


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


@pytest.mark.parametrize("n", [3, 7, 15, 31, 63, 127])
@pytest.mark.parametrize("name", ["m27", "m19"])
def test_wide_sweep_fp64_bitwise(n, name):
    w = WIDE[name]
    rng = np.random.default_rng(n)
    u, b = rng.uniform(-1, 1, (n,) * 3), rng.uniform(-1, 1, (n,) * 3)
    h2 = 1.0 / (n + 1) ** 2
    ref = oracle.sweep(u, h2 * b, w)
    out, nrm = binding.op_sweep(dev(u), dev(b), w, b_unscaled=True, want_norm=True)
    assert np.array_equal(host(out), ref)
    rh = oracle.residual_scaled(u, h2 * b)
    assert nrm == pytest.approx(float(np.sum(rh * rh)), rel=1e-13)
    out, _ = binding.op_sweep(dev(u), dev(h2 * b), w)
    assert np.array_equal(host(out), ref)
    out0, nrm0 = binding.op_sweep(None, dev(h2 * b), w, want_norm=True)
    assert np.array_equal(host(out0), oracle.sweep(np.zeros_like(u), h2 * b, w))
    assert nrm0 == pytest.approx(float(np.sum((h2 * b) ** 2)), rel=1e-13)


def test_wide_weights_are_refused_where_unsupported():
    """The FP32 refinement levels and the adjoint take the 7-point M only."""
    with pytest.raises(MGError):
        Solver(3, 32, smoothers.M27, precision="fp32_ir")
    u = dev(np.zeros((15,) * 3), torch.float32)
    with pytest.raises(MGError):
        binding.op_sweep(u, u, smoothers.M27)
    with Solver(3, 16, smoothers.M27, precision="fp32") as s:
        b = dev(np.ones((15,) * 3), torch.float32)
        with pytest.raises(MGError):
            s.vcycles_adjoint(b, b, 2)


def _parity(N, b, w, nu, tol=1e-10, max_cycles=60):
    ref = oracle.solve(b, w, tol=tol, max_cycles=max_cycles, nu1=nu, nu2=nu)
    with Solver(3, N, w, nu1=nu, nu2=nu) as s:
        info = s.solve(dev(b), tol=tol, max_cycles=max_cycles)
        got = host(info.u)
    assert info.status == ref.status
    assert info.cycles == ref.cycles
    np.testing.assert_allclose(info.hist, ref.hist, rtol=1e-12, atol=0)
    assert np.array_equal(got, ref.u)
    return info


@pytest.mark.parametrize("N,nu", [(4, 1), (8, 1), (16, 1), (32, 1), (64, 1), (32, 2), (64, 2)])
def test_wide_solve_bitwise(N, nu):
    info = _parity(N, inputs.uniform(3, N, N), smoothers.M27, nu)
    assert info.converged


def test_wide_19_point_solve_and_sine():
    _parity(32, inputs.uniform(3, 32, 7), smoothers.M19, 1)
    _parity(32, inputs.sine(3, 32), smoothers.M27, 1)


def test_wide_plain_fp32_cycles():
    """MG_FP32 contexts run the same kernels in single precision: the solve
    stalls at FP32 rounding, a few 1e-7 of ||b||, and the residual (recomputed
    by the oracle in FP64) agrees with the library's."""
    N = 32
    b = inputs.uniform(3, N, 2)
    with Solver(3, N, smoothers.M27, nu1=1, nu2=1, precision="fp32") as s:
        info = s.solve(dev(b, torch.float32), tol=1e-5, max_cycles=30)
        u = host(info.u)
    assert info.converged
    r = oracle.residual_norm(u, b.astype(np.float32).astype(np.float64))
    assert r <= 1e-5 * np.linalg.norm(b) * 1.01


@pytest.fixture
def _oracle_threads():
    oracle.set_threads(len(os.sched_getaffinity(0)))
    yield
    oracle.set_threads(1)


@pytest.mark.slow
@pytest.mark.parametrize("n", [255, 511])
def test_wide_sweep_whole_array_bitwise(n, _oracle_threads):
    w = smoothers.M27
    rng = np.random.default_rng(n + 1)
    u, b = rng.uniform(-1, 1, (n,) * 3), rng.uniform(-1, 1, (n,) * 3)
    bh = b / (n + 1) ** 2
    out, nrm = binding.op_sweep(dev(u), dev(b), w, b_unscaled=True, want_norm=True)
    assert np.array_equal(host(out), oracle.sweep(u, bh, w))
    del out
    rh = oracle.residual_scaled(u, bh)
    assert nrm == pytest.approx(float(np.sum(rh * rh)), rel=1e-12)


@pytest.mark.slow
def test_wide_config_3d_n512_two_cycles_bitwise(_oracle_threads):
    """N = 512, uniform b (seed 0), FP64 V(1,1) with the 27-point smoother: the
    first two cycles' iterates and r_0..r_2 in the benchmark's configuration."""
    N = 512
    b = inputs.uniform(3, N, 0)
    w = smoothers.M27
    ref = oracle.solve(b, w, tol=0.0, max_cycles=2, nu1=1, nu2=1)
    with Solver(3, N, w, nu1=1, nu2=1) as s:
        info = s.solve(dev(b), tol=0.0, max_cycles=2)
        got = host(info.u)
    assert info.cycles == 2
    np.testing.assert_allclose(info.hist, ref.hist, rtol=1e-12, atol=0)
    assert np.array_equal(got, ref.u)
