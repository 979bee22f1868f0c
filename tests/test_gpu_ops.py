"""GPU parity of every single operator of the cycle against the FP64 oracle,
through the C ABI (mg_op_*).

FP64: the kernels evaluate each formula in the same operation order as the
oracle (written out in oracle/mg_oracle.c and beside each kernel), so the
results must be identical (np.array_equal; signed zeros compare equal).
FP32: same formulas in single precision; the bound is derived from the
arithmetic: every output is a sum of at most ~25 rounded terms, so
|out32 - out64| <= 32 * 2^-24 * S where S bounds the magnitude of the terms
(plus the rounding of the FP32 inputs themselves, which the oracle sees).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import coeffs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_05543_gb300 import binding  # noqa: E402

EPS32 = 2.0 ** -24


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def rand(shape, seed, lo=-1.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, shape)


SM2 = ["m9", "jacobi", "m5", "vanka", "tw5"]
SIZES2 = [3, 7, 15, 63, 255, 511, 1023]
SIZES3 = [3, 7, 15, 31, 63]


def _w(d, name):
    return coeffs.weights(d, name)


@pytest.mark.parametrize("n", SIZES2)
@pytest.mark.parametrize("name", SM2)
def test_sweep2d_fp64_bitwise(n, name):
    w = _w(2, name)
    u, b = rand((n, n), 1), rand((n, n), 2)
    h2 = 1.0 / (n + 1) ** 2
    ref = oracle.sweep(u, h2 * b, w)
    out, _ = binding.op_sweep(dev(u), dev(b), w, b_unscaled=True)
    assert np.array_equal(host(out), ref)
    out2, _ = binding.op_sweep(dev(u), dev(h2 * b), w, b_unscaled=False)
    assert np.array_equal(host(out2), ref)


@pytest.mark.parametrize("n", SIZES2)
def test_sweep2d_zero_start_and_norm(n):
    w = _w(2, "m9")
    bh = rand((n, n), 3) / (n + 1) ** 2
    ref = oracle.sweep(np.zeros((n, n)), bh, w)
    out, nrm = binding.op_sweep(None, dev(bh), w, want_norm=True)
    assert np.array_equal(host(out), ref)
    assert nrm == pytest.approx(float(np.sum(bh * bh)), rel=1e-13)
    u = rand((n, n), 4)
    _, nrm = binding.op_sweep(dev(u), dev(bh), w, want_norm=True)
    rh = oracle.residual_scaled(u, bh)
    assert nrm == pytest.approx(float(np.sum(rh * rh)), rel=1e-13)


@pytest.mark.parametrize("n", SIZES3)
@pytest.mark.parametrize("name", ["m7", "jacobi"])
def test_sweep3d_fp64_bitwise(n, name):
    w = _w(3, name)
    u, b = rand((n, n, n), 5), rand((n, n, n), 6)
    h2 = 1.0 / (n + 1) ** 2
    ref = oracle.sweep(u, h2 * b, w)
    out, nrm = binding.op_sweep(dev(u), dev(b), w, b_unscaled=True, want_norm=True)
    assert np.array_equal(host(out), ref)
    rh = oracle.residual_scaled(u, h2 * b)
    assert nrm == pytest.approx(float(np.sum(rh * rh)), rel=1e-13)
    out0, _ = binding.op_sweep(None, dev(h2 * b), w)
    assert np.array_equal(host(out0), oracle.sweep(np.zeros_like(u), h2 * b, w))


@pytest.mark.parametrize("d,n", [(2, 3), (2, 15), (2, 255), (2, 1023), (3, 3), (3, 15), (3, 63), (3, 127)])
def test_residual_refine_rounds_the_fp64_residual_once(d, n):
    """Outer refinement step: the FP64 residual, rounded to FP32 (numpy's
    float64 -> float32 cast is IEEE round to nearest even), bit for bit; its
    squared norm summed in FP64 within 1e-12 relative of the exact sum."""
    u, b = rand((n,) * d, 27), rand((n,) * d, 28)
    h2 = 1.0 / (n + 1) ** 2
    ref = oracle.residual_scaled(u, h2 * b)
    for unscaled, bb in ((True, b), (False, h2 * b)):
        rh32, nrm2 = binding.op_residual_refine(dev(u), dev(bb), b_unscaled=unscaled, want_norm=True)
        torch.cuda.synchronize()
        got = rh32.cpu().numpy()
        assert got.dtype == np.float32
        assert np.array_equal(got.view(np.uint32), ref.astype(np.float32).view(np.uint32))
        exact = math.fsum((ref * ref).ravel())
        assert abs(nrm2 - exact) <= 1e-12 * exact


def _narrowing_cases(count, seed):
    """float64 bit patterns that stress binary64 -> binary32 rounding: exact
    ties (odd and even kept part), values just above/below a tie, results at
    the edges of the binary32 exponent range (subnormal, smallest normal,
    largest finite, overflow), zeros and infinities."""
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2 ** 63, count, dtype=np.uint64) | (rng.integers(0, 2, count, dtype=np.uint64) << 63)
    k = np.arange(count) % 8
    low29 = np.uint64((1 << 29) - 1)
    half = np.uint64(1 << 28)
    bits = np.where(k == 0, (bits & ~low29) | half, bits)                 # exact ties
    bits = np.where(k == 1, (bits & ~low29) | (half + np.uint64(1)), bits)  # just above
    bits = np.where(k == 2, (bits & ~low29) | (half - np.uint64(1)), bits)  # just below
    exp = rng.integers(860, 1160, count).astype(np.uint64)  # around binary32's range 897..1150
    sign_frac = bits & np.uint64(0x800FFFFFFFFFFFFF)
    bits = np.where(k >= 3, sign_frac | (exp << np.uint64(52)), bits)
    bits = np.where(k == 3, (bits & ~low29) | half, bits)                 # ties near the range edges
    x = bits.view(np.float64).copy()
    x[np.isnan(x)] = 1.5
    x[:8] = [0.0, -0.0, np.inf, -np.inf, 3.4028235677973366e38, 3.4028235677973362e38, 1.1754943508222875e-38,
             1.401298464324817e-45]
    return x


@pytest.mark.parametrize("d,n", [(2, 255), (3, 63)])
def test_residual_refine_narrowing_is_ieee_round_to_nearest_even(d, n):
    """With u = 0 the residual is bh itself (a zero neighbour sum added to
    it; -0 becomes +0), so the FP32 output is the rounding of arbitrary
    doubles: compared bit for bit with numpy's IEEE conversion."""
    x = _narrowing_cases(n ** d, 5).reshape((n,) * d)
    rh32, _ = binding.op_residual_refine(dev(np.zeros_like(x)), dev(x))
    torch.cuda.synchronize()
    expect = np.where(x == 0.0, 0.0, x)
    with np.errstate(over="ignore"):
        expect32 = expect.astype(np.float32)
    assert np.array_equal(rh32.cpu().numpy().view(np.uint32), expect32.view(np.uint32))


@pytest.mark.parametrize("d,n", [(2, 3), (2, 15), (2, 255), (2, 1023), (3, 3), (3, 15), (3, 63)])
def test_residual_fp64_bitwise(d, n):
    u, b = rand((n,) * d, 7), rand((n,) * d, 8)
    h2 = 1.0 / (n + 1) ** 2
    ref = oracle.residual_scaled(u, h2 * b)
    assert np.array_equal(host(binding.op_residual(dev(u), dev(b), b_unscaled=True)), ref)
    assert np.array_equal(host(binding.op_residual(dev(u), dev(h2 * b))), ref)


@pytest.mark.parametrize("d,n", [(2, 7), (2, 15), (2, 63), (2, 511), (2, 1023), (3, 7), (3, 15), (3, 31), (3, 63)])
def test_residual_restrict_fp64_bitwise(d, n):
    u, b = rand((n,) * d, 9), rand((n,) * d, 10)
    h2 = 1.0 / (n + 1) ** 2
    ref = oracle.restrict(oracle.residual_scaled(u, h2 * b))
    assert np.array_equal(host(binding.op_residual_restrict(dev(u), dev(b), b_unscaled=True)), ref)
    assert np.array_equal(host(binding.op_residual_restrict(dev(u), dev(h2 * b))), ref)


@pytest.mark.parametrize("d,n", [(2, 7), (2, 15), (2, 63), (2, 511), (2, 1023), (3, 7), (3, 15), (3, 31), (3, 63)])
def test_prolong_correct_fp64_bitwise(d, n):
    nc = (n - 1) // 2
    e, u = rand((nc,) * d, 11), rand((n,) * d, 12)
    ref = oracle.prolong_add(e, u)
    out = binding.op_prolong_correct(dev(e), dev(u))
    assert np.array_equal(host(out), ref)


@pytest.mark.parametrize("d", [2, 3])
def test_coarse_solve_fp64_bitwise(d):
    bh = rand((3,) * d, 13)
    assert np.array_equal(host(binding.op_coarse_solve(dev(bh))), oracle.coarse_solve(bh))


# ---------------------------------------------------------------------------
# FP32 versions of the same operators (used inside iterative refinement)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,n,name", [(2, 63, "m9"), (2, 511, "m9"), (2, 1023, "jacobi"), (3, 31, "m7"), (3, 63, "m7"),
                                      (3, 127, "m7"), (3, 255, "jacobi")])
def test_sweep_fp32_within_rounding_bound(d, n, name):
    w = _w(d, name)
    u = rand((n,) * d, 14).astype(np.float32).astype(np.float64)
    bh = (rand((n,) * d, 15) / (n + 1) ** 2).astype(np.float32).astype(np.float64)
    ref = oracle.sweep(u, bh, w)
    out, _ = binding.op_sweep(dev(u, torch.float32), dev(bh, torch.float32), w)
    # terms: |u|, c_j * (sums of up to 8 residuals, each a sum of up to 8 |u| terms)
    S = np.abs(u).max() + sum(abs(x) for x in w) * 8 * (2 * d + 2) * np.abs(u).max()
    np.testing.assert_allclose(host(out), ref, rtol=0, atol=32 * EPS32 * S)


@pytest.mark.parametrize("d,n", [(2, 511), (2, 2047), (3, 63), (3, 127), (3, 255)])
def test_restrict_and_prolong_fp32_within_rounding_bound(d, n):
    u = rand((n,) * d, 16).astype(np.float32).astype(np.float64)
    bh = (rand((n,) * d, 17) / (n + 1) ** 2).astype(np.float32).astype(np.float64)
    ref = oracle.restrict(oracle.residual_scaled(u, bh))
    out = binding.op_residual_restrict(dev(u, torch.float32), dev(bh, torch.float32))
    S = (2 * d + 1) * np.abs(u).max() * 4 ** d / 4
    np.testing.assert_allclose(host(out), ref, rtol=0, atol=32 * EPS32 * S)
    nc = (n - 1) // 2
    e = rand((nc,) * d, 18).astype(np.float32).astype(np.float64)
    ref = oracle.prolong_add(e, u)
    out = binding.op_prolong_correct(dev(e, torch.float32), dev(u, torch.float32))
    np.testing.assert_allclose(host(out), ref, rtol=0, atol=8 * EPS32 * (np.abs(u).max() + np.abs(e).max()))
