"""A float32 model of the squared-norm accumulator the FP64 GPU kernels use
(SqSum in paper_2206_05543_gb300/csrc/mg_common.cuh), checked on the CPU
against exactly rounded sums (math.fsum of the FP64 squares).

The model follows the kernel step by step with numpy float32 arithmetic
(IEEE binary32, round to nearest): each FP64 r is split into h (the top 24
significand bits) and l (the next 23), r^2 2^-2e ~ h^2 + 2hl is formed as the
pair p = hh, q = fma(2h, l, fma(h, h, -p)) (both FMAs emulated exactly: the
products are exact in float64), added to a float-float accumulator that
carries its own power-of-two exponent, and flushed into an FP64 total every
32 terms. This pins the accumulator's design (relative error about 1e-13)
independently of the GPU; tests/test_gpu_norms.py checks the kernels."""
import math
import struct

import numpy as np
import pytest

f32 = np.float32


def _fma32(a, b, c):
    # a * b is exact in float64 for float32 a, b; the sum then rounds once to
    # float64 and once to float32 (the kernel's fma rounds once: the two agree
    # except in rare ties, far below the tolerance checked here)
    return f32(float(a) * float(b) + float(c))


def _split(r):
    bits = struct.unpack("<Q", struct.pack("<d", r))[0]
    ex = (bits >> 52) & 0x7FF
    h = struct.unpack("<f", struct.pack("<I", 0x3F800000 | ((bits >> 29) & 0x7FFFFF)))[0]
    m = struct.unpack("<f", struct.pack("<I", 0x4B000000 | ((bits >> 6) & 0x7FFFFF)))[0] - 8388608.0
    return ex, f32(h), f32(f32(m) * f32(2.0 ** -46))


class SqSumModel:
    def __init__(self):
        self.total = 0.0
        self.hi = f32(0.0)
        self.lo = f32(0.0)
        self.e = -8192
        self.cnt = 0

    def flush(self):
        if self.hi > 0:
            try:  # past the binary64 range the kernel's exponent-field scaling gives infinity
                self.total += math.ldexp(float(self.hi) + float(self.lo), self.e)
            except OverflowError:
                self.total = math.inf
        self.hi, self.lo, self.e, self.cnt = f32(0.0), f32(0.0), -8192, 0

    def add(self, r):
        ex, h, l = _split(r)
        if ex == 0:
            return
        if ex == 0x7FF:
            self.total = math.nan
            return
        p = f32(h * h)
        tq = _fma32(f32(h + h), l, _fma32(h, h, -p))
        tp = p
        et = 2 * (ex - 1023)
        if et > self.e:
            sc = f32(2.0 ** max(self.e - et, -126))
            self.hi, self.lo, self.e = f32(self.hi * sc), f32(self.lo * sc), et
        else:
            sc = f32(2.0 ** max(et - self.e, -126))
            tp, tq = f32(tp * sc), f32(tq * sc)
        sh = f32(self.hi + tp)
        bv = f32(sh - self.hi)
        err = f32(f32(self.hi - f32(sh - bv)) + f32(tp - bv))
        tl = f32(f32(err + self.lo) + tq)
        self.hi = f32(sh + tl)
        self.lo = f32(tl - f32(self.hi - sh))
        self.cnt += 1
        if self.cnt == 32:
            self.flush()

    def value(self):
        self.flush()
        return self.total


def _model_sumsq(a):
    m = SqSumModel()
    for r in np.asarray(a, dtype=np.float64).ravel():
        m.add(float(r))
    return m.value()


def _fsum(a):
    return math.fsum((np.asarray(a, dtype=np.float64).ravel() ** 2).tolist())


@pytest.mark.parametrize("case", ["uniform", "spread", "tiny", "huge", "residual-like", "sparse"])
def test_model_matches_exactly_rounded_sums(case):
    rng = np.random.default_rng(3)
    k = 4000
    sign = np.where(rng.random(k) < 0.5, -1.0, 1.0)
    a = {
        "uniform": rng.uniform(-1, 1, k),
        "spread": sign * 10.0 ** rng.uniform(-100, 100, k),
        "tiny": sign * rng.uniform(0.5, 1, k) * 1e-150,
        "huge": sign * rng.uniform(0.5, 1, k) * 1e150,
        # scaled residuals near convergence on the 2D N = 8192 grid: h^2 r ~ 1e-18
        "residual-like": rng.standard_normal(k) * 1.5e-18,
        "sparse": np.where(rng.random(k) < 0.02, sign * rng.uniform(0.1, 10, k), 0.0),
    }[case]
    assert _model_sumsq(a) == pytest.approx(_fsum(a), rel=1e-12, abs=0.0)


def test_model_edge_values():
    assert _model_sumsq(np.zeros(10)) == 0.0
    assert _model_sumsq([5e-324, -5e-324]) == 0.0  # binary64 subnormals: zero squares in FP64 too
    assert math.isnan(_model_sumsq([1.0, np.inf, 2.0]))
    assert math.isnan(_model_sumsq([1.0, np.nan]))
    # one term: the split loses at most the last six significand bits of r
    for r in (1.0, -3.0, 0.1, 1e-300, 1e300, 2.0 ** 0.5):
        assert _model_sumsq([r]) == pytest.approx(r * r, rel=2.0 ** -44)
