"""Squared residual norms of the FP64 kernels against exactly rounded sums.

The FP64 sweeps and residuals accumulate sum(r^2) without FP64 arithmetic per
point (split of r into FP32 head and tail, float-float accumulator with its
own power-of-two exponent, FP64 flush every 32 terms). The solver's norm
histories are compared with the oracle at 1e-12 elsewhere; these cases stress
what those inputs do not: values spread over 200 orders of magnitude in one
array, uniformly tiny and huge arrays, exact zeros, infinities. The reference
is math.fsum of the FP64 squares (exactly rounded)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_05543_gb300 import binding, smoothers  # noqa: E402
from paper_2206_05543_gb300.binding import Solver  # noqa: E402


def _ref_sumsq(a):
    return math.fsum((np.asarray(a, dtype=np.float64).ravel() ** 2).tolist())


def _fields(shape, seed):
    rng = np.random.default_rng(seed)
    sign = np.where(rng.random(shape) < 0.5, -1.0, 1.0)
    return {
        "spread": sign * 10.0 ** rng.uniform(-100, 100, shape),
        "tiny": sign * rng.uniform(0.5, 1.0, shape) * 1e-150,
        "huge": sign * rng.uniform(0.5, 1.0, shape) * 1e150,
        "sparse": np.where(rng.random(shape) < 0.01, sign * rng.uniform(0.1, 10.0, shape), 0.0),
        "one": np.pad(np.ones((1,) * len(shape)), [(0, s - 1) for s in shape]),
    }


@pytest.mark.parametrize("d,n", [(2, 127), (2, 1023), (3, 31), (3, 127)])
def test_sweep_norm_from_zero_matches_fsum(d, n):
    """Sweep from u = 0: r = bh, so the returned sum is sum(bh^2)."""
    c = smoothers.M9 if d == 2 else smoothers.M7
    for name, bh in _fields((n,) * d, 5).items():
        _, s2 = binding.op_sweep(None, torch.from_numpy(bh).cuda(), c, want_norm=True)
        ref = _ref_sumsq(bh)
        assert s2 == pytest.approx(ref, rel=1e-12, abs=0.0), name


@pytest.mark.parametrize("d,N", [(2, 128), (3, 32)])
def test_residual_norm_matches_fsum(d, N):
    """mg_residual_norm with u = 0 is ||b||: the FP64 residual is h^2 b exactly."""
    n = N - 1
    for name, b in _fields((n,) * d, 6).items():
        with Solver(d, N) as s:
            u = torch.zeros((n,) * d, dtype=torch.float64, device="cuda")
            got = s.residual_norm(u, torch.from_numpy(b).cuda())
        assert got == pytest.approx(math.sqrt(_ref_sumsq(b)), rel=1e-12, abs=0.0), name


def test_norm_of_zero_and_non_finite():
    n = 127
    z = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    _, s2 = binding.op_sweep(None, z, smoothers.M9, want_norm=True)
    assert s2 == 0.0
    bad = np.zeros((n, n))
    bad[40, 50] = np.inf
    _, s2 = binding.op_sweep(None, torch.from_numpy(bad).cuda(), smoothers.M9, want_norm=True)
    assert not math.isfinite(s2)
    bad[40, 50] = np.nan
    _, s2 = binding.op_sweep(None, torch.from_numpy(bad).cuda(), smoothers.M9, want_norm=True)
    assert math.isnan(s2)
