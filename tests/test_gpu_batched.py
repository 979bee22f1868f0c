"""Batched solves of many 2D problems with uneven grid sizes (FP32 cycles in
FP64 refinement), through mg_setup_batched / mg_solve_batched.

The batched launches run the same per-tile code as the one-problem kernels,
so every problem's iterate must equal, bit for bit, the one-problem
refinement solve of the same right-hand side, with the same iteration
count. Against the FP64 oracle: the FP64 residual of each result (recomputed
by the oracle) is below tol * ||b_i||.
"""
import numpy as np
import pytest

import oracle
from paper_2206_05543_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_05543_gb300.binding import MG_ENOCONV, MG_OK, BatchedSolver, MGError, Solver  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_batched_equals_single_problem_solves():
    Ns = [64, 8, 256, 4, 128, 16, 64, 32, 512, 128]
    bs = [inputs.uniform(2, N, 100 + i) for i, N in enumerate(Ns)]
    with BatchedSolver(Ns) as bsolver:
        us, st, cyc, rel = bsolver.solve([_dev(b) for b in bs], tol=1e-10)
        got = [u.cpu().numpy() for u in us]
    assert st == MG_OK
    for i, (N, b) in enumerate(zip(Ns, bs)):
        with Solver(2, N, precision="fp32_ir") as s:
            info = s.solve(_dev(b), tol=1e-10)
        assert info.cycles == cyc[i], (i, N)
        assert np.array_equal(got[i], info.u.cpu().numpy()), (i, N)
        assert oracle.residual_norm(got[i], b) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-6)
        assert rel[i] <= 1e-10


def test_batched_workload_256_problems():
    """256 problems, N drawn (seed 0) from {64, ..., 1024}, b_i ~ U[-1, 1]
    from seed 1 + i, FP32 V(1,1) in FP64 refinement to 1e-10."""
    Ns = [int(N) for N in inputs.batch_sizes(256, 0)]
    bs = inputs.batch_rhs(Ns, 1)
    with BatchedSolver(Ns) as bsolver:
        dev_b = [_dev(b) for b in bs]
        us, st, cyc, rel = bsolver.solve(dev_b, tol=1e-10)
        got = [u.cpu().numpy() for u in us]
    assert st == MG_OK
    assert max(rel) <= 1e-10
    for i in range(0, 256, 1):
        assert oracle.residual_norm(got[i], bs[i]) <= 1e-10 * np.linalg.norm(bs[i]) * (1 + 1e-6), i
    assert 8 <= min(cyc) and max(cyc) <= 12


def test_batched_masking_and_edge_cases():
    Ns = [64, 128, 32]
    bs = [inputs.uniform(2, 64, 1), np.zeros((127, 127)), inputs.uniform(2, 32, 2)]
    with BatchedSolver(Ns) as bsolver:
        us, st, cyc, rel = bsolver.solve([_dev(b) for b in bs], tol=1e-10, max_cycles=2)
        assert st == MG_ENOCONV
        assert cyc == [2, 0, 2]
        assert not us[1].any()
        # solving again with new buffers re-uploads the pointer tables
        us2, st2, cyc2, _ = bsolver.solve([_dev(b) for b in bs], tol=1e-10)
        assert st2 == MG_OK and cyc2[1] == 0 and min(cyc2[0], cyc2[2]) >= 8


def test_batched_two_cycles_per_iteration_equals_single_problem_solves():
    """Two FP32 cycles per refinement iteration: every problem's iterate equals
    the one-problem solve with the same setting, bit for bit."""
    Ns = [64, 256, 32, 128, 64, 512]
    bs = [inputs.uniform(2, N, 200 + i) for i, N in enumerate(Ns)]
    with BatchedSolver(Ns) as bsolver:
        bsolver.set_refinement_cycles(2)
        us, st, cyc, rel = bsolver.solve([_dev(b) for b in bs], tol=1e-10)
        got = [u.cpu().numpy() for u in us]
    assert st == MG_OK
    for i, (N, b) in enumerate(zip(Ns, bs)):
        with Solver(2, N, precision="fp32_ir") as s:
            s.set_refinement_cycles(2)
            info = s.solve(_dev(b), tol=1e-10)
        assert info.cycles == cyc[i], (i, N)
        assert np.array_equal(got[i], info.u.cpu().numpy()), (i, N)
        assert oracle.residual_norm(got[i], b) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-6)
    assert max(cyc) <= 7


def test_batched_several_cycles_needs_no_tail_finest_level():
    with BatchedSolver([64, 16]) as bsolver:
        with pytest.raises(MGError):
            bsolver.set_refinement_cycles(2)
        bsolver.set_refinement_cycles(1)


@pytest.mark.parametrize("inner", [1, 2])
def test_batched_zero_start_equals_explicit_zero_initial_guesses(inner):
    """MG_SOLVE_ZERO_START on a batch: the us are output only (filled with NaN
    before the call); iterates, cycle counts and relative residuals equal
    those of the solve from explicitly zeroed us bit for bit."""
    Ns = [64, 128, 256, 64, 512, 128, 32, 32]
    bs = [torch.from_numpy(b).cuda() for b in inputs.batch_rhs(Ns, 3)]
    with BatchedSolver(Ns, nu1=1, nu2=1) as s:
        if inner > 1:
            s.set_refinement_cycles(inner)
        ref, st_r, cyc_r, rel_r = s.solve(bs, [torch.zeros_like(b) for b in bs], tol=1e-10)
        got, st_g, cyc_g, rel_g = s.solve(bs, [torch.full_like(b, float("nan")) for b in bs], tol=1e-10,
                                          zero_start=True)
        new, _, cyc_n, _ = s.solve(bs, tol=1e-10)  # us None: zero start
    assert st_g == st_r and cyc_g == cyc_r and cyc_n == cyc_r
    for a, r, c in zip(got, ref, new):
        assert torch.equal(a, r) and torch.equal(c, r)
    np.testing.assert_allclose(rel_g, rel_r, rtol=1e-12, atol=0)
