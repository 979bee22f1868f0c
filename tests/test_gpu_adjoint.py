"""GPU adjoint of K cycles (mg_vcycles_adjoint) against the FP64 oracle.

- FP64 contexts: dL/db and dL/dc agree with oracle/adjoint.py to 1e-12
  (relative, norm-wise for dL/db): the two evaluate the same transposed
  operators with different association of the transposed stencils.
- The adjoint workload: 3D, N = 128, b ~ N(0,1) seed 0, K = 4 V(1,1)
  cycles from zero, L = 1/2 ||u_K - u*||^2 with u* the exact discrete
  solution (sine transform) held fixed. In FP64 the GPU gradients meet FP64
  central finite differences to 1e-5; with 127^3 FP32 fields the bounds are
  stated per test from the FP32 arithmetic.
- torch.autograd: the Function wrapper gives the same gradients.
"""
import numpy as np
import pytest

import oracle
from oracle import adjoint, coeffs, exact
from paper_2206_05543_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_05543_gb300.autograd import vcycles  # noqa: E402
from paper_2206_05543_gb300.binding import MGError, Solver  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("d,N,K,nu1,nu2", [(2, 32, 3, 1, 1), (2, 64, 2, 2, 1), (3, 16, 4, 1, 1), (3, 32, 2, 1, 2)])
def test_fp64_adjoint_matches_oracle(d, N, K, nu1, nu2):
    b = inputs.gaussian(d, N, 1)
    g = inputs.gaussian(d, N, 2)
    c = coeffs.default(d)
    gb_ref, gc_ref = adjoint.vcycles_adjoint(b, c, K, g, nu1, nu2)
    with Solver(d, N, c, nu1=nu1, nu2=nu2) as s:
        bt = torch.from_numpy(b).cuda()
        u = s.cycles(bt, K)
        assert np.array_equal(u.cpu().numpy(), oracle.cycles(b, np.zeros_like(b), c, K, nu1, nu2))
        gb, gc = s.vcycles_adjoint(bt, torch.from_numpy(g).cuda(), K)
    assert _rel(gb.cpu().numpy(), gb_ref) <= 1e-12
    np.testing.assert_allclose(gc, gc_ref, rtol=1e-10)


def _fd_checks(b, c, K, ustar, gb, gc):
    """FP64 central differences of the oracle forward (u* fixed), rel 1e-5."""
    def loss(bb, cc):
        u = oracle.cycles(bb, np.zeros_like(bb), cc, K)
        return 0.5 * float(np.sum((u - ustar) ** 2))

    for j in range(len(c)):
        eps = 1e-6 * abs(c[j])
        cp, cm = list(c), list(c)
        cp[j] += eps
        cm[j] -= eps
        fd = (loss(b, cp) - loss(b, cm)) / (2 * eps)
        assert gc[j] == pytest.approx(fd, rel=1e-5)
    rng = np.random.default_rng(9)
    for i in rng.choice(b.size, 3, replace=False):
        eps = 1e-2  # L is exactly quadratic in b: no truncation error
        bp, bm = b.copy(), b.copy()
        bp.flat[i] += eps
        bm.flat[i] -= eps
        fd = (loss(bp, c) - loss(bm, c)) / (2 * eps)
        assert gb.flat[i] == pytest.approx(fd, rel=1e-5, abs=1e-6 * np.abs(gb).max())


def _workload():
    d, N, K = 3, 128, 4
    b = inputs.gaussian(d, N, 0)
    c = coeffs.default(d)
    ustar = exact.dst_solve(b)
    uK_ref = oracle.cycles(b, np.zeros_like(b), c, K)
    return d, N, K, b, c, ustar, uK_ref


def test_adjoint_workload_fp64_3d_n128():
    """The adjoint workload in FP64 on the GPU: oracle adjoint to 1e-12 and
    FP64 central finite differences to 1e-5."""
    d, N, K, b, c, ustar, uK_ref = _workload()
    gb_ref, gc_ref = adjoint.vcycles_adjoint(b, c, K, uK_ref - ustar)
    with Solver(d, N, c) as s:
        bt = torch.from_numpy(b).cuda()
        uK = s.cycles(bt, K)
        assert np.array_equal(uK.cpu().numpy(), uK_ref)
        g = uK - torch.from_numpy(ustar).cuda()
        gb, gc = s.vcycles_adjoint(bt, g.contiguous(), K)
    gbn = gb.cpu().numpy()
    assert _rel(gbn, gb_ref) <= 1e-12
    np.testing.assert_allclose(gc, gc_ref, rtol=1e-10)
    _fd_checks(b, c, K, ustar, gbn, gc)


def test_adjoint_workload_fp32_3d_n128():
    """The adjoint workload with 127^3 FP32 fields.
    (1) the FP32 adjoint operator, fed the same g as the FP64 oracle adjoint:
        relative error <= 1e-5 (FP32 rounding, ~50 transposed sweeps);
    (2) the whole FP32 pipeline (FP32 forward, g = u_K - u* formed in FP32):
        g is ~1e-4 of |u|, so FP32 rounding of u_K is amplified by
        |u_K| / |u_K - u*|; the bound is stated from the measured forward
        error: rel(dL/db) <= 2 |dU_K| / |u_K - u*| + 1e-5, and the forward
        error itself <= 1e-5 relative."""
    d, N, K, b, c, ustar, uK_ref = _workload()
    g64 = uK_ref - ustar
    gb_ref, gc_ref = adjoint.vcycles_adjoint(b, c, K, g64)
    with Solver(d, N, c, precision="fp32") as s:
        bt = torch.from_numpy(b).to("cuda", torch.float32)
        g32 = torch.from_numpy(g64).to("cuda", torch.float32)
        gb, gc = s.vcycles_adjoint(bt, g32, K)
        assert _rel(gb.double().cpu().numpy(), gb_ref) <= 1e-5
        np.testing.assert_allclose(gc, gc_ref, rtol=1e-5)
        uK = s.cycles(bt, K)
        fwd_err = float(np.linalg.norm(uK.double().cpu().numpy() - uK_ref))
        assert fwd_err <= 1e-5 * np.linalg.norm(uK_ref)
        g = (uK - torch.from_numpy(ustar).to("cuda", torch.float32)).contiguous()
        gb2, gc2 = s.vcycles_adjoint(bt, g, K)
    bound = 2 * fwd_err / np.linalg.norm(g64) + 1e-5
    assert _rel(gb2.double().cpu().numpy(), gb_ref) <= bound
    assert np.all(np.abs(np.asarray(gc2) - gc_ref) <= bound * np.abs(gc_ref))


def test_autograd_function():
    d, N, K = 2, 64, 3
    b = inputs.gaussian(d, N, 3)
    c = coeffs.default(d)
    ustar = torch.from_numpy(exact.dst_solve(b)).cuda()
    with Solver(d, N, c) as s:
        bt = torch.from_numpy(b).cuda().requires_grad_(True)
        ct = torch.tensor(c, dtype=torch.float64, requires_grad=True)
        u = vcycles(bt, ct, s, K)
        loss = 0.5 * ((u - ustar) ** 2).sum()
        loss.backward()
        uK = oracle.cycles(b, np.zeros_like(b), c, K)
        gb_ref, gc_ref = adjoint.vcycles_adjoint(b, c, K, uK - ustar.cpu().numpy())
    assert _rel(bt.grad.cpu().numpy(), gb_ref) <= 1e-12
    np.testing.assert_allclose(ct.grad.numpy(), gc_ref, rtol=1e-10)


def test_adjoint_rejects_unsupported_contexts():
    b = torch.zeros((31, 31), dtype=torch.float64, device="cuda")
    with Solver(2, 32, gamma=2, nu1=1, nu2=0) as s:
        with pytest.raises(MGError):
            s.vcycles_adjoint(b, b, 2)
    with Solver(2, 32, precision="fp32_ir") as s:
        with pytest.raises(MGError):
            s.vcycles_adjoint(b, b, 2)


def test_plain_fp32_solve():
    """Plain FP32 cycles (MG_FP32) converge until FP32 rounding (~1e-6)."""
    for d, N in ((2, 256), (3, 64)):
        b = inputs.uniform(d, N, 4)
        with Solver(d, N, precision="fp32") as s:
            info = s.solve(torch.from_numpy(b).to("cuda", torch.float32), tol=1e-5)
            u = info.u.double().cpu().numpy()
        assert info.converged
        # the FP64 residual of the FP32 result is at the FP32 stopping level
        assert oracle.residual_norm(u, b) <= 2e-5 * np.linalg.norm(b)
        ref = oracle.solve(b, coeffs.default(d), tol=1e-10)
        assert _rel(u, ref.u) <= 1e-4


@pytest.mark.slow
def test_fp64_adjoint_3d_n512_fits_and_matches_a_directional_difference():
    """The adjoint at the 3D benchmark size in FP64 (K = 2 V(1,1), 133M
    unknowns): the workspace (cycle inputs plus one cycle's sweep inputs per
    level) is about ten finest fields, and <dL/db, v> matches the central
    difference of L(b) = 1/2 ||u_K(b)||^2 along a random v (L is quadratic
    in b, so the difference has no truncation error; the bound is the FP64
    rounding of the two forward evaluations)."""
    N, K = 512, 2
    rng = np.random.default_rng(4)
    b = torch.from_numpy(rng.standard_normal((N - 1,) * 3)).cuda()
    v = torch.from_numpy(rng.standard_normal((N - 1,) * 3)).cuda()
    with Solver(3, N) as s:
        ws = s.adjoint_workspace_bytes(K)
        field = (N - 1) ** 3 * 8
        assert ws <= 11 * field, ws / field
        uK = s.cycles(b, K)
        gb, gc = s.vcycles_adjoint(b, uK.contiguous(), K)
        torch.cuda.synchronize()
        eps = 1e-3

        def loss(bb):
            u = s.cycles(bb, K)
            return 0.5 * float(torch.sum(u * u))

        fd = (loss(b + eps * v) - loss(b - eps * v)) / (2 * eps)
        dd = float(torch.sum(gb * v))
    assert dd == pytest.approx(fd, rel=1e-6)
