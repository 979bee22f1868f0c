"""The bounded device-side waits of the TMA-staged 3D FP32 kernels, made to
expire on purpose without any fault: an armed launch makes its first copy's
mbarrier expect 16 bytes more than the copy delivers, so the bounded wait
(about one second) runs out; the kernel records the expiry, drains its other
copies and returns, and the call reports MG_ETIMEOUT. Afterwards the device
and the library keep working (the same call succeeds and is correct)."""
import numpy as np
import pytest

import oracle
from oracle import coeffs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_05543_gb300 import binding, inputs  # noqa: E402
from paper_2206_05543_gb300.binding import MG_ETIMEOUT, MGError, Solver  # noqa: E402


def _f32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _case(n, seed):
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1, 1, (n,) * 3).astype(np.float32).astype(np.float64)
    bh = (rng.uniform(-1, 1, (n,) * 3) / (n + 1) ** 2).astype(np.float32).astype(np.float64)
    return u, bh


@pytest.fixture(autouse=True)
def _disarm():
    binding.arm_wait_expiry(0)
    yield
    binding.arm_wait_expiry(0)


@pytest.mark.parametrize("zero_start", [False, True])
def test_sweep_wait_expiry_reports_timeout_and_recovers(zero_start):
    n = 15
    u, bh = _case(n, 3)
    w = coeffs.default(3)
    uin = None if zero_start else _f32(u)
    binding.arm_wait_expiry(1)
    with pytest.raises(MGError) as ei:
        binding.op_sweep(uin, _f32(bh), w)
    assert ei.value.status == MG_ETIMEOUT
    assert binding.arm_wait_expiry(0) == 0  # the armed launch was used
    out, _ = binding.op_sweep(uin, _f32(bh), w)
    torch.cuda.synchronize()
    ref = oracle.sweep(np.zeros_like(u) if zero_start else u, bh, w)
    S = np.abs(u).max() * (1 + sum(abs(x) for x in w) * 8 * 8)
    np.testing.assert_allclose(out.double().cpu().numpy(), ref, rtol=0, atol=32 * 2.0 ** -24 * S)


def test_restriction_wait_expiry_reports_timeout_and_recovers():
    n = 15
    u, bh = _case(n, 4)
    binding.arm_wait_expiry(1)
    with pytest.raises(MGError) as ei:
        binding.op_residual_restrict(_f32(u), _f32(bh))
    assert ei.value.status == MG_ETIMEOUT
    out = binding.op_residual_restrict(_f32(u), _f32(bh))
    torch.cuda.synchronize()
    ref = oracle.restrict(oracle.residual_scaled(u, bh))
    S = 7 * np.abs(u).max() * 4 ** 3 / 4
    np.testing.assert_allclose(out.double().cpu().numpy(), ref, rtol=0, atol=32 * 2.0 ** -24 * S)


def test_solve_reports_timeout_then_a_new_context_converges():
    b = inputs.uniform(3, 32, 5)
    binding.arm_wait_expiry(1)  # consumed while the refinement cycle is recorded
    with Solver(3, 32, nu1=2, nu2=2, precision="fp32_ir") as s:
        with pytest.raises(MGError) as ei:
            s.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_cycles=30)
        assert ei.value.status == MG_ETIMEOUT
    with Solver(3, 32, nu1=2, nu2=2, precision="fp32_ir") as s:
        info = s.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_cycles=30)
        u = info.u.cpu().numpy()
    assert info.converged
    assert oracle.residual_norm(u, b) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-6)


def test_solve_reports_timeout_then_the_same_context_converges():
    """The error word is cleared at the start of every call: after a solve
    that reported MG_ETIMEOUT, re-recording the cycle (mg_set_coeffs with the
    same weights; the armed launch lives in the recorded graph) lets the same
    context converge, and its result passes the oracle's FP64 residual check."""
    b = inputs.uniform(3, 32, 6)
    w = coeffs.default(3)
    with Solver(3, 32, w, nu1=2, nu2=2, precision="fp32_ir") as s:
        binding.arm_wait_expiry(1)  # consumed while the refinement cycle is recorded
        with pytest.raises(MGError) as ei:
            s.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_cycles=30)
        assert ei.value.status == MG_ETIMEOUT
        assert binding.arm_wait_expiry(0) == 0
        s.set_coeffs(w)
        info = s.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_cycles=30)
        u = info.u.cpu().numpy()
        # a second solve on the same context and graphs
        info2 = s.solve(torch.from_numpy(b).cuda(), tol=1e-10, max_cycles=30)
        assert info2.converged and np.array_equal(info2.u.cpu().numpy(), u)
    assert info.converged
    assert oracle.residual_norm(u, b) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-6)
