"""GPU parity of the whole solver against the FP64 oracle, through the C ABI.

FP64 contexts: every operator evaluates the oracle's operation order, so the
iterates u_k are bit-identical and the per-cycle residual norms differ only
by the order of the final sum of squares; the test bound is 1e-12 relative
(the tolerance stated for FP64 sweeps and per-cycle residual norms).
Refinement contexts (FP32 cycle inside FP64 refinement): the FP64 residual
of the result, recomputed by the oracle, must be <= tol * ||b||, and the
solution must match the oracle's FP64 solution to the accuracy the common
stopping rule allows (bound stated in each test).
"""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import coeffs, exact
from paper_2206_05543_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_05543_gb300 import binding  # noqa: E402
from paper_2206_05543_gb300.binding import MG_ENAN, MG_ENOCONV, MG_OK, MGError, Solver  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float64)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _parity(d, N, b, name=None, nu1=1, nu2=1, gamma=1, u0=None, tol=1e-10, max_cycles=60):
    w = coeffs.weights(d, name) if name else coeffs.default(d)
    ref = oracle.solve(b, w, u0=u0, tol=tol, max_cycles=max_cycles, nu1=nu1, nu2=nu2, gamma=gamma)
    with Solver(d, N, w, nu1=nu1, nu2=nu2, gamma=gamma) as s:
        u = dev(u0 if u0 is not None else np.zeros_like(b))
        info = s.solve(dev(b), u, tol=tol, max_cycles=max_cycles)
        got = host(info.u)
    assert info.status == ref.status
    assert info.cycles == ref.cycles
    np.testing.assert_allclose(info.hist, ref.hist, rtol=1e-12, atol=0)
    assert np.array_equal(got, ref.u)
    return info, ref


@pytest.mark.parametrize("rhs", ["sine", "uniform"])
def test_config_2d_n64(rhs):
    """2D, N = 64, manufactured sine and uniform[-1, 1] right-hand sides,
    V(1,1) with M9, to 1e-10."""
    b = inputs.sine(2, 64) if rhs == "sine" else inputs.uniform(2, 64, 0)
    info, ref = _parity(2, 64, b)
    assert info.converged and 8 <= info.cycles <= 12
    if rhs == "sine":
        uh = exact.manufactured_factor(64) * exact.sine_product(2, 64)
        assert np.abs(ref.u - uh).max() <= 1e-9 * np.abs(uh).max()


@pytest.mark.parametrize("N", [4, 8, 16, 32, 128, 256, 512, 1024])
def test_2d_sizes(N):
    _parity(2, N, inputs.uniform(2, N, N))


@pytest.mark.parametrize("name", ["jacobi", "m5", "vanka", "tw5"])
def test_2d_other_smoothers(name):
    _parity(2, 128, inputs.uniform(2, 128, 1), name=name, max_cycles=80)


def test_2d_w_cycle_and_random_start():
    """W(1+0) and the paper's uniform (0,1) initial guess (Sec. 4)."""
    b = inputs.uniform(2, 128, 2)
    u0 = np.random.default_rng(7).uniform(0.0, 1.0, b.shape)
    _parity(2, 128, b, nu1=1, nu2=0, gamma=2, u0=u0)
    _parity(2, 128, b, u0=u0)


@pytest.mark.parametrize("N,nu", [(4, 1), (8, 1), (16, 1), (32, 1), (64, 1), (32, 2), (64, 2)])
def test_3d_sizes(N, nu):
    _parity(3, N, inputs.uniform(3, N, N), nu1=nu, nu2=nu)


def test_3d_sine_and_jacobi():
    _parity(3, 32, inputs.sine(3, 32))
    _parity(3, 32, inputs.uniform(3, 32, 3), name="jacobi", max_cycles=80)


@pytest.mark.parametrize("N", [16, 64])
def test_3d_w_cycles_and_random_start(N):
    """W(1+0) and W(2,2) in 3D with M7 and the paper's uniform (0,1)
    initial guess (Sec. 4, Example 3 compares V and W cycles): iterates,
    cycle counts and histories against the oracle."""
    b = inputs.uniform(3, N, 5)
    u0 = np.random.default_rng(11).uniform(0.0, 1.0, b.shape)
    _parity(3, N, b, nu1=1, nu2=0, gamma=2, u0=u0, max_cycles=80)
    _parity(3, N, b, nu1=2, nu2=2, gamma=2)


def test_final_measurement_guess_that_misses():
    """The solver replaces the speculative pre-sweep by a residual-norm-only
    pass when the last convergence factor, carried one cycle forward, puts the
    next residual under the tolerance. The factor of this problem grows from
    cycle to cycle, so with the tolerance between the carried-forward guess
    and the true residual of cycle j the guess misses: the solver must find
    the cycle unconverged, smooth after all and go on. Cycles, history and u
    stay those of the oracle, which never guesses."""
    b = inputs.uniform(2, 64, 64)
    w = coeffs.default(2)
    full = oracle.solve(b, w, tol=0.0, max_cycles=10)
    h = np.asarray(full.hist)
    j = 8
    guess = h[j - 1] ** 2 / h[j - 2]
    assert guess < h[j] * (1 - 1e-3)  # the factor grew at cycle j
    tol = float(np.sqrt(guess * h[j]) / h[0])
    _, ref = _parity(2, 64, b, tol=tol)
    assert ref.cycles == j + 1


def test_final_measurement_guess_that_holds():
    """Tolerance just above the residual of cycle j: the carried-forward guess
    fires at cycle j and the residual-norm-only pass ends the solve there."""
    b = inputs.uniform(3, 32, 5)
    w = coeffs.default(3)
    full = oracle.solve(b, w, tol=0.0, max_cycles=9, nu1=2, nu2=2)
    h = np.asarray(full.hist)
    j = 7
    tol = float(h[j] * (1 + 1e-6) / h[0])
    assert h[j - 1] ** 2 / h[j - 2] <= tol * h[0]
    _, ref = _parity(3, 32, b, nu1=2, nu2=2, tol=tol)
    assert ref.cycles == j


def test_vcycle_single_cycle_bitwise():
    for d, N in ((2, 256), (3, 32)):
        b = inputs.uniform(d, N, 4)
        u0 = np.random.default_rng(5).uniform(0, 1, b.shape)
        ref = oracle.cycles(b, u0, coeffs.default(d), 1)
        with Solver(d, N) as s:
            u = dev(u0)
            s.vcycle(u, dev(b))
            assert np.array_equal(host(u), ref)
            # a second call with other buffers re-records the graphs
            u2, b2 = dev(u0), dev(b.copy())
            s.vcycle(u2, b2)
            assert np.array_equal(host(u2), ref)
            assert s.residual_norm(u2, b2) == pytest.approx(oracle.residual_norm(ref, b), rel=1e-12)


def test_zero_rhs_and_stopping_edge_cases():
    with Solver(2, 64) as s:
        info = s.solve(dev(np.zeros((63, 63))))
        assert info.status == MG_OK and info.cycles == 0 and info.relres == 0.0
        assert not host(info.u).any()
        b = inputs.uniform(2, 64, 6)
        info = s.solve(dev(b), max_cycles=1)
        assert info.status == MG_ENOCONV and info.cycles == 1
        assert np.array_equal(host(info.u), oracle.cycles(b, np.zeros_like(b), coeffs.default(2), 1))
        info = s.solve(dev(b), max_cycles=0)
        assert info.status == MG_ENOCONV and info.cycles == 0
        bad = b.copy()
        bad[10, 10] = np.nan
        info = s.solve(dev(bad))
        assert info.status == MG_ENAN


def test_invalid_arguments_raise():
    with pytest.raises(MGError):
        Solver(2, 48)
    with pytest.raises(MGError):
        Solver(3, 64, coeffs=(0.1, 0.2, 0.3, 0.01, 0.001))
    with Solver(2, 64) as s:
        with pytest.raises(ValueError):
            s.solve(dev(np.zeros((64, 64))))


@pytest.mark.parametrize("d,N,nu,tol_u", [(2, 256, 1, 1e-8), (2, 1024, 1, 1e-8), (3, 32, 2, 1e-8), (3, 64, 2, 1e-8),
                                          (3, 64, 1, 1e-8), (3, 128, 1, 1e-8)])
def test_mixed_precision_refinement(d, N, nu, tol_u):
    """FP32 cycle inside FP64 refinement reaches the FP64 tolerance 1e-10.
    Check: the oracle's FP64 residual of the result and the distance to the
    exact discrete solution (sine transform) against the plain FP64 solve."""
    b = inputs.uniform(d, N, 8)
    with Solver(d, N, nu1=nu, nu2=nu, precision="fp32_ir") as s:
        info = s.solve(dev(b), tol=1e-10, max_cycles=60)
        u = host(info.u)
    assert info.converged
    r = oracle.residual_norm(u, b)
    assert r <= 1e-10 * np.linalg.norm(b) * (1 + 1e-6)
    assert info.hist[-1] == pytest.approx(r, rel=1e-6)
    ustar = exact.dst_solve(b)
    ref = oracle.solve(b, coeffs.default(d), tol=1e-10, nu1=nu, nu2=nu)
    err_mixed = np.linalg.norm(u - ustar) / np.linalg.norm(ustar)
    err_fp64 = np.linalg.norm(ref.u - ustar) / np.linalg.norm(ustar)
    assert err_mixed <= max(tol_u, 10 * err_fp64)


@pytest.mark.parametrize("d,N,nu", [(2, 128, 1), (3, 32, 2)])
def test_refinement_vcycle_equals_the_solves_iterates(d, N, nu):
    """mg_vcycle on a refinement context is one refinement iteration (FP64
    residual, FP32 cycle, u += e in FP64) on the caller's u: one and two calls
    equal solves stopped after one and two iterations, bit for bit, which
    checks that the solve's graphs and the single iteration share their
    arithmetic."""
    b = inputs.uniform(d, N, 11)
    with Solver(d, N, nu1=nu, nu2=nu, precision="fp32_ir") as s:
        u = dev(np.zeros_like(b))
        s.vcycle(u, dev(b))
        one = host(u)
        s.vcycle(u, dev(b))
        two = host(u)
        for k, want in ((1, one), (2, two)):
            info = s.solve(dev(b), tol=0.0, max_cycles=k)
            assert info.status == MG_ENOCONV and info.cycles == k
            assert np.array_equal(host(info.u), want)
    assert not np.array_equal(one, two)


@pytest.mark.parametrize("d,N,nu", [(2, 256, 1), (3, 64, 2)])
def test_refinement_with_several_cycles_per_iteration(d, N, nu):
    """Two and three FP32 cycles per refinement iteration: still the FP64
    tolerance (oracle residual), and the iteration count drops to about the
    single-cycle count divided by the cycles per iteration."""
    b = inputs.uniform(d, N, 9)
    its = {}
    for m in (1, 2, 3):
        with Solver(d, N, nu1=nu, nu2=nu, precision="fp32_ir") as s:
            if m > 1:
                s.set_refinement_cycles(m)
            info = s.solve(dev(b), tol=1e-10, max_cycles=60)
            u = host(info.u)
        assert info.converged, m
        assert oracle.residual_norm(u, b) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-6)
        its[m] = info.cycles
    assert its[2] <= (its[1] + 1) // 2 + 1 and its[3] <= (its[1] + 2) // 3 + 1, its
    with Solver(d, N, nu1=nu, nu2=nu, precision="fp64") as s:
        with pytest.raises(MGError):
            s.set_refinement_cycles(2)


@pytest.mark.slow
def test_config_2d_n8192_two_cycles_bitwise():
    """Full-size 2D workload (N = 8192, 67M unknowns, uniform b seed 0, zero
    start): the first two V(1,1) cycles and the residual norms r_0..r_2 in
    the launch configuration the benchmark times."""
    N = 8192
    b = inputs.uniform(2, N, 0)
    ref = oracle.solve(b, coeffs.default(2), tol=0.0, max_cycles=2)
    with Solver(2, N) as s:
        info = s.solve(dev(b), tol=0.0, max_cycles=2)
        got = host(info.u)
    assert info.cycles == 2
    np.testing.assert_allclose(info.hist, ref.hist, rtol=1e-12, atol=0)
    assert np.array_equal(got, ref.u)


@pytest.mark.slow
def test_config_3d_n512_full_size():
    """Full-size 3D workload (N = 512, 133M unknowns, uniform b seed 0): the
    FP64 sweep in the benchmark's launch configuration equals the oracle at
    sampled points (corners, faces, tile and chunk edges, random) bit for
    bit, and the refinement solves (one and two FP32 cycles per iteration)
    reach an FP64 residual <= 1e-10 ||b||, recomputed by the oracle."""
    N, n = 512, 511
    b = inputs.uniform(3, N, 0)
    w = coeffs.default(3)
    h2 = 1.0 / N ** 2
    u = np.random.default_rng(5).uniform(-1, 1, b.shape)
    out, _ = binding.op_sweep(dev(u), dev(b), w, b_unscaled=True)
    got = host(out)
    rng = np.random.default_rng(6)
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n // 2, n - 1), (255, 29, 127), (256, 30, 128),
           (254, 31, 129)] + [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(60)]
    bh = h2 * b
    for p in pts:
        ref = _residual_sweep_point(u, bh, w, p)
        assert got[p] == ref, (p, got[p], ref)
    del got, out
    for m in (1, 2):
        with Solver(3, N, w, nu1=2, nu2=2, precision="fp32_ir") as s:
            if m > 1:
                s.set_refinement_cycles(m)
            info = s.solve(dev(b), tol=1e-10, max_cycles=40)
            x = host(info.u)
        assert info.converged
        assert oracle.residual_norm(x, b) <= 1e-10 * np.linalg.norm(b) * (1 + 1e-6)


def _residual_sweep_point(u, bh, w, p):
    """One point of the FP64 sweep, in the oracle's operation order, from the
    oracle's scaled residual of the 3^3 neighbourhood boxes of p and its six
    neighbours (every value the stencil reads)."""
    n = u.shape[0]

    def val(a, q):
        return a[q] if all(0 <= c < n for c in q) else 0.0

    def rh(q):
        if not all(0 <= c < n for c in q):
            return 0.0
        box_u = np.array([[[val(u, (q[0] + dz, q[1] + dy, q[2] + dx)) for dx in (-1, 0, 1)]
                           for dy in (-1, 0, 1)] for dz in (-1, 0, 1)])
        box_b = np.zeros((3, 3, 3))
        box_b[1, 1, 1] = bh[q]
        # the 3^3 oracle grid's centre point sees exactly q's six neighbours
        return oracle.residual_scaled(box_u, box_b)[1, 1, 1]

    z, y, x = p
    E = ((rh((z, y, x - 1)) + rh((z, y, x + 1))) + (rh((z, y - 1, x)) + rh((z, y + 1, x)))) + \
        (rh((z - 1, y, x)) + rh((z + 1, y, x)))
    return _fma(w[1], E, _fma(w[0], rh(p), float(u[p])))


def _fma(a, b, c):
    """a * b + c rounded once (exact rational arithmetic, then the nearest double)."""
    from fractions import Fraction
    return float(Fraction(a) * Fraction(b) + Fraction(c))


@pytest.mark.parametrize("d,N,prec,nu", [(2, 128, "fp64", 1), (2, 1024, "fp64", 1), (3, 32, "fp64", 2),
                                         (3, 64, "fp64", 2), (2, 256, "fp32", 1), (3, 32, "fp32", 2),
                                         (2, 256, "fp32_ir", 1), (2, 8, "fp32_ir", 1), (3, 64, "fp32_ir", 2),
                                         (3, 64, "fp32_ir", 1), (2, 4, "fp64", 1)])
def test_zero_start_equals_an_explicit_zero_initial_guess(d, N, prec, nu):
    """MG_SOLVE_ZERO_START: u is output only (here filled with NaN before the
    call) and the solve runs the from-zero form of its first operation; the
    iterates, cycle count and history equal those of a solve from an
    explicitly zeroed u bit for bit (FP64: also the oracle's)."""
    b = inputs.uniform(d, N, 21)
    dt = torch.float32 if prec == "fp32" else torch.float64
    bt = torch.from_numpy(b).to("cuda", dt)
    with Solver(d, N, nu1=nu, nu2=nu, precision=prec) as s:
        ref = s.solve(bt, torch.zeros_like(bt), tol=1e-10 if prec != "fp32" else 1e-5, max_cycles=60)
        garbage = torch.full_like(bt, float("nan"))
        got = s.solve(bt, garbage, tol=1e-10 if prec != "fp32" else 1e-5, max_cycles=60, zero_start=True)
        new = s.solve(bt, tol=1e-10 if prec != "fp32" else 1e-5, max_cycles=60)  # u None: zero start
    assert got.status == ref.status and got.cycles == ref.cycles
    assert torch.equal(got.u, ref.u) and torch.equal(new.u, ref.u)
    np.testing.assert_allclose(got.hist, ref.hist, rtol=1e-12, atol=0)
    if prec == "fp64":
        w = coeffs.default(d)
        o = oracle.solve(b, w, tol=1e-10, max_cycles=60, nu1=nu, nu2=nu)
        assert got.cycles == o.cycles and np.array_equal(host(got.u), o.u)
        np.testing.assert_allclose(got.hist, o.hist, rtol=1e-12, atol=0)


def test_solve_ex_rejects_unknown_flags():
    b = torch.zeros((31, 31), dtype=torch.float64, device="cuda")
    with Solver(2, 32) as s:
        st = binding.lib().mg_solve_ex(s._ctx, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(b.data_ptr()), 1e-10,
                                       10, 2, None, None, None)
    assert st == binding.MG_EINVAL


def test_loop_limits_and_optional_outputs():
    """A solve with tol = 0 runs exactly max_cycles cycles with the oracle's
    history; the outputs are optional."""
    b = inputs.uniform(2, 64, 21)
    w = coeffs.default(2)
    ref = oracle.solve(b, w, tol=0.0, max_cycles=30)
    assert ref.status == MG_ENOCONV and ref.cycles == 30
    with Solver(2, 64) as s:
        info = s.solve(dev(b), tol=0.0, max_cycles=30)
        assert info.status == MG_ENOCONV and info.cycles == 30
        np.testing.assert_allclose(info.hist, ref.hist, rtol=1e-12, atol=0)
        assert np.array_equal(host(info.u), ref.u)
        bt = dev(b)
        u = torch.empty_like(bt)
        cyc = ctypes.c_int(-1)
        lib = binding.lib()
        st = lib.mg_solve_ex(s._ctx, ctypes.c_void_p(bt.data_ptr()), ctypes.c_void_p(u.data_ptr()), 1e-10, 100,
                             binding.MG_SOLVE_ZERO_START, ctypes.byref(cyc), None, None)
        o = oracle.solve(b, w, tol=1e-10, max_cycles=100)
        assert st == MG_OK and cyc.value == o.cycles
        assert np.array_equal(host(u), o.u)
        # no outputs at all; a limit far above the cycles needed
        st = lib.mg_solve_ex(s._ctx, ctypes.c_void_p(bt.data_ptr()), ctypes.c_void_p(u.data_ptr()), 1e-10,
                             1 << 30, binding.MG_SOLVE_ZERO_START, None, None, None)
        assert st == MG_OK and np.array_equal(host(u), o.u)


def test_async_solves_queued_back_to_back():
    """mg_solve_async: solves queued on one context without synchronising,
    over more (u, b) pairs than the context keeps graphs for, each equal to
    the oracle's solve (u bit for bit, cycles, history within the norm
    tolerance); a zero right-hand side from a zero start leaves u = 0."""
    w = coeffs.default(2)
    bs = [inputs.uniform(2, 64, 40 + i) for i in range(6)]
    bs[3] = np.zeros_like(bs[3])
    refs = [oracle.solve(b, w, tol=1e-10, max_cycles=60) for b in bs]
    with Solver(2, 64) as s:
        bds = [dev(b) for b in bs]
        us = [torch.full_like(bd, 7.0) for bd in bds]  # garbage: every solve starts from zero
        pend = [s.solve_async(bd, u, tol=1e-10, max_cycles=60, zero_start=True, history=True)
                for bd, u in zip(bds, us)]
        # the same pairs again: graphs kept or re-recorded, results unchanged
        pend += [s.solve_async(bds[i], us[i], tol=1e-10, max_cycles=60, zero_start=True, history=True)
                 for i in (0, 5, 2)]
        for i, p in zip(list(range(6)) + [0, 5, 2], pend):
            r = p.result()
            ref = refs[i]
            assert r.status == ref.status and r.cycles == ref.cycles
            np.testing.assert_allclose(r.hist, ref.hist, rtol=1e-12, atol=0)
            assert np.array_equal(host(p.u), ref.u)
        assert not host(us[3]).any()


@pytest.mark.parametrize("d,N,prec,nu", [(2, 128, "fp32_ir", 1), (3, 32, "fp32_ir", 2), (3, 32, "fp64", 2)])
def test_async_equals_sync(d, N, prec, nu):
    b = inputs.uniform(d, N, 50)
    with Solver(d, N, nu1=nu, nu2=nu, precision=prec) as s:
        bd = dev(b)
        sync = s.solve(bd, tol=1e-10, max_cycles=60)
        us = host(sync.u)
        p = s.solve_async(bd, tol=1e-10, max_cycles=60, history=True)
        r = p.result()
        assert r.status == sync.status and r.cycles == sync.cycles and r.relres == sync.relres
        assert np.array_equal(r.hist, sync.hist)
        assert np.array_equal(host(p.u), us)
        # the outcome of a limit that runs out
        r = s.solve_async(bd, tol=0.0, max_cycles=3).result()
        assert r.status == MG_ENOCONV and r.cycles == 3


def test_kept_graphs_follow_coefficient_and_refinement_changes():
    """The context keeps the graphs of several (u, b) pairs; a change of the
    smoother weights (or of the FP32 cycles per refinement iteration) must
    reach every kept pair, not only the last one."""
    bA, bB = inputs.uniform(2, 64, 60), inputs.uniform(2, 64, 61)
    w9, w5 = coeffs.default(2), coeffs.weights(2, "m5")
    with Solver(2, 64) as s:
        dA, dB = dev(bA), dev(bB)
        uA, uB = torch.empty_like(dA), torch.empty_like(dB)
        for d, u in ((dA, uA), (dB, uB)):
            s.solve(d, u, tol=1e-10, max_cycles=60, zero_start=True)
        s.set_coeffs(w5)
        for b, d, u in ((bA, dA, uA), (bB, dB, uB)):
            got = s.solve(d, u, tol=1e-10, max_cycles=60, zero_start=True)
            ref = oracle.solve(b, w5, tol=1e-10, max_cycles=60)
            assert got.cycles == ref.cycles and np.array_equal(host(u), ref.u)
    with Solver(2, 128, precision="fp32_ir") as s:
        bA, bB = inputs.uniform(2, 128, 62), inputs.uniform(2, 128, 63)
        dA, dB = dev(bA), dev(bB)
        uA, uB = torch.empty_like(dA), torch.empty_like(dB)
        first = []
        for d, u in ((dA, uA), (dB, uB)):
            f = s.solve(d, u, tol=1e-10, max_cycles=60, zero_start=True)
            first.append((f.cycles, host(u)))
        s.set_refinement_cycles(2)
        for b, d, u, (fc, fu) in zip((bA, bB), (dA, dB), (uA, uB), first):
            got = s.solve(d, u, tol=1e-10, max_cycles=60, zero_start=True)
            assert got.converged and got.cycles <= fc
            # two FP32 cycles per iteration give other iterates than one
            assert not np.array_equal(host(u), fu)
            r = oracle.residual_norm(host(u), b)
            assert r <= 1e-10 * oracle.residual_norm(np.zeros_like(b), b) * (1 + 1e-6)


def test_solve_async_rejects_bad_arguments():
    b = torch.zeros((63, 63), dtype=torch.float64, device="cuda")
    info = torch.zeros(24, dtype=torch.uint8, pin_memory=True)
    lib = binding.lib()
    with Solver(2, 64) as s:
        P = ctypes.c_void_p
        assert lib.mg_solve_async(s._ctx, P(b.data_ptr()), P(b.data_ptr()), 1e-10, 10, 0, None, None) == binding.MG_EINVAL
        assert lib.mg_solve_async(s._ctx, P(b.data_ptr()), P(b.data_ptr()), 1e-10, 10, 4, P(info.data_ptr()),
                                  None) == binding.MG_EINVAL
        assert lib.mg_solve_async(s._ctx, P(b.data_ptr()), P(b.data_ptr()), -1.0, 10, 0, P(info.data_ptr()),
                                  None) == binding.MG_EINVAL
        # a zero right-hand side: no cycle, status OK, written by the device
        p = s.solve_async(b, tol=1e-10, max_cycles=10, info_buf=info)
        r = p.result()
        assert r.status == MG_OK and r.cycles == 0 and not host(p.u).any()
    with pytest.raises(ValueError):
        with Solver(2, 64) as s:
            s.solve_async(b, info_buf=torch.zeros(24, dtype=torch.uint8))  # not page-locked


@pytest.mark.parametrize("case", ["misses", "holds"])
def test_async_final_measurement_guess(case):
    """The device-side loop of mg_solve_async takes the same guesses as the
    host loop: the norm-only graph for the predicted last cycle, and after a
    guess that misses, the pre graph and no more guessing. Cycles, history
    and u equal the oracle's (which never guesses)."""
    if case == "misses":
        d, N, seed, nu, j = 2, 64, 64, 1, 8
        b = inputs.uniform(d, N, seed)
        h = np.asarray(oracle.solve(b, coeffs.default(d), tol=0.0, max_cycles=10).hist)
        guess = h[j - 1] ** 2 / h[j - 2]
        assert guess < h[j] * (1 - 1e-3)
        tol, cycles = float(np.sqrt(guess * h[j]) / h[0]), j + 1
    else:
        d, N, seed, nu, j = 3, 32, 5, 2, 7
        b = inputs.uniform(d, N, seed)
        h = np.asarray(oracle.solve(b, coeffs.default(d), tol=0.0, max_cycles=9, nu1=nu, nu2=nu).hist)
        tol, cycles = float(h[j] * (1 + 1e-6) / h[0]), j
    ref = oracle.solve(b, coeffs.default(d), tol=tol, max_cycles=60, nu1=nu, nu2=nu)
    assert ref.cycles == cycles
    with Solver(d, N, nu1=nu, nu2=nu) as s:
        p = s.solve_async(dev(b), tol=tol, max_cycles=60, history=True)
        r = p.result()
    assert r.status == ref.status and r.cycles == ref.cycles
    np.testing.assert_allclose(r.hist, ref.hist, rtol=1e-12, atol=0)
    assert np.array_equal(host(p.u), ref.u)
