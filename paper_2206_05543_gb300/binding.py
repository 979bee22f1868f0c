"""Thin ctypes binding of the C ABI in include/mg.h (argument marshalling only).

Every numerical step runs inside libmg.so (CUDA, sm_103a); this module only
passes torch tensors' device pointers, the current CUDA stream and sizes
across the ABI and turns status codes into exceptions. There is no fallback:
if the library or a GPU is missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build
from . import smoothers

MG_OK, MG_EINVAL, MG_ENOMEM, MG_ECUDA, MG_ENOCONV, MG_ENAN, MG_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
MG_FP64, MG_FP32_IR, MG_FP32 = 0, 1, 2
MG_SOLVE_ZERO_START = 1
PRECISIONS = {"fp64": MG_FP64, "fp32_ir": MG_FP32_IR, "mixed": MG_FP32_IR, "fp32": MG_FP32}

_lock = threading.Lock()
_lib = None

#: symbols declared in include/mg.h, with (restype, argtypes)
_P, _I, _D, _U = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_ulonglong
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)
SIGNATURES = {
    "mg_setup": (_I, [_I, _I, _DP, _I, _I, _I, _I, _P, ctypes.POINTER(_P)]),
    "mg_setup_ex": (_I, [_I, _I, _DP, _I, _I, _I, _I, _I, _P, ctypes.POINTER(_P)]),
    "mg_vcycle": (_I, [_P, _P, _P]),
    "mg_solve": (_I, [_P, _P, _P, _D, _I, _IP, _DP, _DP]),
    "mg_solve_ex": (_I, [_P, _P, _P, _D, _I, ctypes.c_uint, _IP, _DP, _DP]),
    "mg_solve_async": (_I, [_P, _P, _P, _D, _I, ctypes.c_uint, _P, _P]),
    "mg_residual_norm": (_I, [_P, _P, _P, _DP]),
    "mg_destroy": (None, [_P]),
    "mg_op_sweep": (_I, [_I, _I, _I, _DP, _I, _P, _P, _I, _P, _DP, _P]),
    "mg_op_residual": (_I, [_I, _I, _I, _P, _P, _I, _P, _P]),
    "mg_op_residual_refine": (_I, [_I, _I, _P, _P, _I, _P, _P, _P]),
    "mg_op_residual_restrict": (_I, [_I, _I, _I, _P, _P, _I, _P, _P]),
    "mg_op_prolong_correct": (_I, [_I, _I, _I, _P, _P, _P]),
    "mg_op_coarse_solve": (_I, [_I, _I, _P, _P, _P]),
    "mg_op_sweep_norm_noalloc": (_I, [_I, _I, _I, _DP, _I, _P, _P, _I, _P, _P, _P]),
    "mg_set_coeffs": (_I, [_P, _DP, _I]),
    "mg_set_refinement_cycles": (_I, [_P, _I]),
    "mg_setup_batched": (_I, [_I, _I, _IP, _DP, _I, _I, _I, _I, _P, ctypes.POINTER(_P)]),
    "mg_solve_batched": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _I, _IP, _DP]),
    "mg_solve_batched_ex": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _I, ctypes.c_uint, _IP, _DP]),
    "mg_vcycles_adjoint": (_I, [_P, _I, _P, _P, _P, _DP]),
    "mg_strerror": (ctypes.c_char_p, [_I]),
    "mg_last_cuda_error": (ctypes.c_char_p, []),
    "mg_kernel_launch_count": (_U, []),
    "mg_test_arm_wait_expiry": (_I, [_I]),
    "mg_measure_fp64_rate": (_I, [_I, _DP, _DP]),
    "mg_op_sweep_restrict": (_I, [_I, _I, _I, _DP, _I, _P, _P, _P, _P, _P]),
    "mg_adjoint_workspace_bytes": (_I, [_P, _I, ctypes.POINTER(ctypes.c_ulonglong)]),
    "mg_op_prolong_sweep": (_I, [_I, _I, _I, _DP, _I, _P, _P, _P, _P, _P, _P]),
}


class MGError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {lib().mg_strerror(status).decode()} ({status})"
        if status == MG_ECUDA:
            msg += f": {lib().mg_last_cuda_error().decode()}"
        super().__init__(msg)


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libmg.so (building it with nvcc when stale or missing)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(status: int, where: str, ok=(MG_OK,)):
    if status not in ok:
        raise MGError(status, where)
    return status


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA GPU is required: this library has no CPU path")
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _coeff_array(c):
    arr = (ctypes.c_double * len(c))(*[float(x) for x in c])
    return arr, len(c)


def _dev_ptr(t, dtype, shape, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def kernel_launch_count() -> int:
    return int(lib().mg_kernel_launch_count())


def arm_wait_expiry(launches: int) -> int:
    """Test hook: the next `launches` TMA-staged kernels let their first
    bounded wait expire (the call reports MG_ETIMEOUT). 0 disarms."""
    return int(lib().mg_test_arm_wait_expiry(int(launches)))


FP64_RATE_KINDS = {"dfma_reg": 0, "dadd": 1, "dmul": 2, "dfma_const": 3}


def measure_fp64_rate(kind: str = "dfma_reg"):
    """(FP64 operations issued per SM per clock, SM clock in MHz) of one
    instruction kind on the current device (see mg_measure_fp64_rate)."""
    rate, mhz = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().mg_measure_fp64_rate(FP64_RATE_KINDS[kind], ctypes.byref(rate), ctypes.byref(mhz)),
           "mg_measure_fp64_rate")
    return rate.value, mhz.value


class SolveInfo:
    def __init__(self, u, status, cycles, relres, hist):
        self.u, self.status, self.cycles, self.relres, self.hist = u, status, cycles, relres, hist

    @property
    def converged(self) -> bool:
        return self.status == MG_OK

    def rate(self) -> float:
        """rho^(k) = (||r_k|| / ||r_0||)^(1/k) at the last cycle (Sec. 4, Eq. (4.1))."""
        k = self.cycles
        return float((self.hist[k] / self.hist[0]) ** (1.0 / k)) if k > 0 else 0.0


class MGSolveInfo(ctypes.Structure):
    """mg_solve_info of include/mg.h."""
    _fields_ = [("r0", ctypes.c_double), ("rk", ctypes.c_double), ("cycles", ctypes.c_int), ("status", ctypes.c_int)]


class PendingSolve:
    """A solve queued by Solver.solve_async. The solver's stream (and so the
    torch stream it was created on) is ordered after the solve; result()
    waits for that stream and returns the SolveInfo."""

    def __init__(self, u, info_buf, hist, stream):
        self.u, self._buf, self._hist, self._stream = u, info_buf, hist, stream

    def _info(self) -> MGSolveInfo:
        return MGSolveInfo.from_address(self._buf.data_ptr())

    def result(self) -> SolveInfo:
        self._stream.synchronize()
        r = self._info()
        _check(r.status, "mg_solve_async", ok=(MG_OK, MG_ENOCONV, MG_ENAN))
        hist = None if self._hist is None else self._hist[: r.cycles + 1].cpu().numpy().copy()
        return SolveInfo(self.u, r.status, r.cycles, r.rk / r.r0 if r.r0 > 0 else 0.0, hist)


class Solver:
    """Multigrid solver for A_h u = b on (0,1)^d, h = 1/N (one CUDA context object).

    coeffs: omega-folded SPAI weights (see smoothers.py; default M9 / M7).
    precision: "fp64" (plain FP64 cycle, float64 arrays), "fp32_ir" (FP32 cycle
    inside FP64 iterative refinement, float64 arrays) or "fp32" (plain FP32
    cycle, float32 arrays). gamma = 1: V cycle, 2: W cycle.
    """

    def __init__(self, d: int, N: int, coeffs=None, nu1: int = 1, nu2: int = 1, gamma: int = 1,
                 precision: str = "fp64", stream=None):
        torch = _torch()
        self.d, self.N = int(d), int(N)
        self.n = self.N - 1
        self.shape = (self.n,) * self.d
        self.coeffs = tuple(coeffs if coeffs is not None else smoothers.default(self.d))
        self.precision = precision
        self.nu1, self.nu2, self.gamma = int(nu1), int(nu2), int(gamma)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        arr, nc = _coeff_array(self.coeffs)
        ctx = ctypes.c_void_p()
        _check(lib().mg_setup_ex(self.d, self.N, arr, nc, nu1, nu2, gamma, PRECISIONS[precision],
                                 ctypes.c_void_p(self._stream.cuda_stream), ctypes.byref(ctx)), "mg_setup")
        self._ctx = ctx

    def close(self):
        if getattr(self, "_ctx", None):
            lib().mg_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def dtype(self):
        torch = _torch()
        return torch.float32 if self.precision == "fp32" else torch.float64

    def _args(self, u, b):
        return (_dev_ptr(u, self.dtype, self.shape, "u"), _dev_ptr(b, self.dtype, self.shape, "b"))

    def set_refinement_cycles(self, cycles: int):
        """fp32_ir only: FP32 cycles per refinement iteration (default 1)."""
        _check(lib().mg_set_refinement_cycles(self._ctx, int(cycles)), "mg_set_refinement_cycles")
        self.refinement_cycles = int(cycles)

    def set_coeffs(self, coeffs):
        arr, nc = _coeff_array(coeffs)
        _check(lib().mg_set_coeffs(self._ctx, arr, nc), "mg_set_coeffs")
        self.coeffs = tuple(float(x) for x in coeffs)

    def cycles(self, b, K: int):
        """u_K = K cycles from u_0 = 0 (asynchronous)."""
        torch = _torch()
        u = torch.zeros(self.shape, dtype=self.dtype, device=b.device)
        for _ in range(K):
            self.vcycle(u, b)
        return u

    def vcycles_adjoint(self, b, grad_uK, K: int):
        """(dL/db, dL/dc) of u_K = K cycles from zero, given dL/du_K."""
        torch = _torch()
        gb = torch.empty_like(b)
        gc = (ctypes.c_double * len(self.coeffs))()
        _check(lib().mg_vcycles_adjoint(self._ctx, int(K), _dev_ptr(b, self.dtype, self.shape, "b"),
                                        _dev_ptr(grad_uK, self.dtype, self.shape, "grad_uK"),
                                        ctypes.c_void_p(gb.data_ptr()), gc), "mg_vcycles_adjoint")
        return gb, np.array(list(gc))

    def adjoint_workspace_bytes(self, K: int) -> int:
        """Device bytes mg_vcycles_adjoint uses for K cycles on this context."""
        out = ctypes.c_ulonglong(0)
        _check(lib().mg_adjoint_workspace_bytes(self._ctx, int(K), ctypes.byref(out)), "mg_adjoint_workspace_bytes")
        return int(out.value)

    def vcycle(self, u, b):
        """One cycle in place on u (asynchronous on the solver's stream)."""
        pu, pb = self._args(u, b)
        _check(lib().mg_vcycle(self._ctx, pu, pb), "mg_vcycle")
        return u

    def solve(self, b, u=None, tol: float = 1e-10, max_cycles: int = 100, zero_start=None) -> SolveInfo:
        """Solve from the initial guess in u; u None: from zero into a new
        array. zero_start (default: u is None): the initial guess is zero and
        u is output only (MG_SOLVE_ZERO_START)."""
        torch = _torch()
        if zero_start is None:
            zero_start = u is None
        if u is None:
            u = torch.empty(self.shape, dtype=self.dtype, device=b.device)
        pu, pb = self._args(u, b)
        hist = np.zeros(max_cycles + 1)
        cyc = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        st = lib().mg_solve_ex(self._ctx, pb, pu, float(tol), int(max_cycles), MG_SOLVE_ZERO_START if zero_start else 0,
                               ctypes.byref(cyc), ctypes.byref(rel), hist.ctypes.data_as(_DP))
        _check(st, "mg_solve", ok=(MG_OK, MG_ENOCONV, MG_ENAN))
        return SolveInfo(u, st, cyc.value, rel.value, hist[: cyc.value + 1].copy())

    def solve_async(self, b, u=None, tol: float = 1e-10, max_cycles: int = 100, zero_start=None,
                    info_buf=None, history: bool = False) -> PendingSolve:
        """Queue a solve (mg_solve_async) without synchronising. info_buf: a
        page-locked host tensor of at least 24 bytes to receive the outcome
        (allocated when None); history: also record ||r_k|| on the device."""
        torch = _torch()
        if zero_start is None:
            zero_start = u is None
        if u is None:
            u = torch.empty(self.shape, dtype=self.dtype, device=b.device)
        if info_buf is None:
            info_buf = torch.zeros(ctypes.sizeof(MGSolveInfo), dtype=torch.uint8, pin_memory=True)
        if not info_buf.is_pinned() or info_buf.numel() * info_buf.element_size() < ctypes.sizeof(MGSolveInfo):
            raise ValueError("info_buf: a page-locked host tensor of at least 24 bytes")
        hist = torch.zeros(max_cycles + 1, dtype=torch.float64, device=b.device) if history else None
        pu, pb = self._args(u, b)
        _check(lib().mg_solve_async(self._ctx, pb, pu, float(tol), int(max_cycles),
                                    MG_SOLVE_ZERO_START if zero_start else 0, ctypes.c_void_p(info_buf.data_ptr()),
                                    ctypes.c_void_p(hist.data_ptr()) if hist is not None else None),
               "mg_solve_async")
        return PendingSolve(u, info_buf, hist, self._stream)

    def residual_norm(self, u, b) -> float:
        pu, pb = self._args(u, b)
        out = ctypes.c_double(0.0)
        _check(lib().mg_residual_norm(self._ctx, pu, pb, ctypes.byref(out)), "mg_residual_norm")
        return out.value


class BatchedSolver:
    """Many independent 2D problems of uneven sizes, FP32 V(nu1, nu2) cycles
    inside FP64 refinement, one launch per operator and grid size across the
    batch (mg_setup_batched / mg_solve_batched)."""

    def __init__(self, Ns, coeffs=None, nu1: int = 1, nu2: int = 1, stream=None):
        torch = _torch()
        self.Ns = [int(N) for N in Ns]
        self.count = len(self.Ns)
        self.coeffs = tuple(coeffs if coeffs is not None else smoothers.default(2))
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        arr, nc = _coeff_array(self.coeffs)
        ns = (ctypes.c_int * self.count)(*self.Ns)
        ctx = ctypes.c_void_p()
        _check(lib().mg_setup_batched(2, self.count, ns, arr, nc, int(nu1), int(nu2), MG_FP32_IR,
                                      ctypes.c_void_p(self._stream.cuda_stream), ctypes.byref(ctx)),
               "mg_setup_batched")
        self._ctx = ctx

    def close(self):
        if getattr(self, "_ctx", None):
            lib().mg_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_refinement_cycles(self, cycles: int):
        """FP32 cycles per refinement iteration (default 1; >1 needs nu1 + nu2
        even and every N >= 32)."""
        _check(lib().mg_set_refinement_cycles(self._ctx, int(cycles)), "mg_set_refinement_cycles")
        self.refinement_cycles = int(cycles)

    def solve(self, bs, us=None, tol: float = 1e-10, max_cycles: int = 100, zero_start=None):
        """Returns (us, status, cycles per problem, relres per problem). us
        None: from zero into new arrays. zero_start (default: us is None):
        every initial guess is zero and the us are output only."""
        torch = _torch()
        if len(bs) != self.count:
            raise ValueError(f"expected {self.count} right-hand sides")
        if zero_start is None:
            zero_start = us is None
        if us is None:
            us = [torch.empty_like(b) for b in bs]
        pb = (ctypes.c_void_p * self.count)()
        pu = (ctypes.c_void_p * self.count)()
        for i, (b, u, N) in enumerate(zip(bs, us, self.Ns)):
            pb[i] = _dev_ptr(b, torch.float64, (N - 1, N - 1), f"b[{i}]").value
            pu[i] = _dev_ptr(u, torch.float64, (N - 1, N - 1), f"u[{i}]").value
        cyc = (ctypes.c_int * self.count)()
        rel = (ctypes.c_double * self.count)()
        st = lib().mg_solve_batched_ex(self._ctx, pb, pu, float(tol), int(max_cycles),
                                       MG_SOLVE_ZERO_START if zero_start else 0, cyc, rel)
        _check(st, "mg_solve_batched", ok=(MG_OK, MG_ENOCONV, MG_ENAN))
        return us, st, list(cyc), list(rel)


# ---------------------------------------------------------------------------
# single operators (one level; arrays in that level's interior layout)
# ---------------------------------------------------------------------------

def _prec_of(t):
    torch = _torch()
    if t.dtype == torch.float64:
        return MG_FP64
    if t.dtype == torch.float32:
        return MG_FP32_IR
    raise TypeError("float64 or float32 tensors expected")


def _level(t):
    d = t.dim()
    n = t.shape[0]
    if d not in (2, 3) or any(s != n for s in t.shape):
        raise ValueError("expected an (n, n) or (n, n, n) tensor")
    return d, n


def op_sweep(u, bh, coeffs, b_unscaled: bool = False, want_norm: bool = False, stream=None, out=None):
    """One SPAI sweep; u None = zero initial value. Returns (u_out, sum rh^2 or None)."""
    torch = _torch()
    d, n = _level(bh)
    prec = _prec_of(bh)
    if out is None:
        out = torch.empty_like(bh)
    else:
        _dev_ptr(out, bh.dtype, bh.shape, "out")
    arr, nc = _coeff_array(coeffs)
    pu = ctypes.c_void_p(0) if u is None else _dev_ptr(u, bh.dtype, bh.shape, "u")
    nrm = ctypes.c_double(0.0)
    _check(lib().mg_op_sweep(d, n, prec, arr, nc, pu, _dev_ptr(bh, bh.dtype, bh.shape, "bh"), int(b_unscaled),
                             ctypes.c_void_p(out.data_ptr()), ctypes.byref(nrm) if want_norm else None,
                             _stream_ptr(stream)), "mg_op_sweep")
    return out, (nrm.value if want_norm else None)


def op_residual(u, bh, b_unscaled: bool = False, stream=None):
    torch = _torch()
    d, n = _level(bh)
    out = torch.empty_like(bh)
    _check(lib().mg_op_residual(d, n, _prec_of(bh), _dev_ptr(u, bh.dtype, bh.shape, "u"),
                                _dev_ptr(bh, bh.dtype, bh.shape, "bh"), int(b_unscaled),
                                ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)), "mg_op_residual")
    return out


def op_residual_refine(u, bh, b_unscaled: bool = False, want_norm: bool = False, stream=None):
    """Outer refinement residual: FP64 u, bh -> FP32 rh (one rounding) and,
    if want_norm, sum(rh^2) of the FP64 residual. Returns (rh32, norm2|None)."""
    torch = _torch()
    d, n = _level(bh)
    if bh.dtype != torch.float64:
        raise TypeError("op_residual_refine takes float64 u and bh")
    out = torch.empty(bh.shape, dtype=torch.float32, device=bh.device)
    nrm = ctypes.c_double(0.0)
    _check(lib().mg_op_residual_refine(d, n, _dev_ptr(u, bh.dtype, bh.shape, "u"),
                                       _dev_ptr(bh, bh.dtype, bh.shape, "bh"), int(b_unscaled),
                                       ctypes.c_void_p(out.data_ptr()),
                                       ctypes.byref(nrm) if want_norm else None, _stream_ptr(stream)),
           "mg_op_residual_refine")
    return out, (nrm.value if want_norm else None)


def op_residual_restrict(u, bh, b_unscaled: bool = False, stream=None):
    torch = _torch()
    d, n = _level(bh)
    nc = (n - 1) // 2
    out = torch.empty((nc,) * d, dtype=bh.dtype, device=bh.device)
    _check(lib().mg_op_residual_restrict(d, n, _prec_of(bh), _dev_ptr(u, bh.dtype, bh.shape, "u"),
                                         _dev_ptr(bh, bh.dtype, bh.shape, "bh"), int(b_unscaled),
                                         ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
           "mg_op_residual_restrict")
    return out


def op_prolong_correct(e_coarse, u, stream=None):
    """u += P e_coarse in place; returns u."""
    d, nc = _level(e_coarse)
    n = 2 * nc + 1
    _check(lib().mg_op_prolong_correct(d, n, _prec_of(u), _dev_ptr(e_coarse, u.dtype, (nc,) * d, "e"),
                                       _dev_ptr(u, u.dtype, (n,) * d, "u"), _stream_ptr(stream)),
           "mg_op_prolong_correct")
    return u


def op_coarse_solve(bh, stream=None):
    torch = _torch()
    d, n = _level(bh)
    if n != 3:
        raise ValueError("the coarsest grid has 3 points per axis")
    out = torch.empty_like(bh)
    _check(lib().mg_op_coarse_solve(d, _prec_of(bh), _dev_ptr(bh, bh.dtype, bh.shape, "bh"),
                                    ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)), "mg_op_coarse_solve")
    return out


def op_sweep_restrict(u, bh, coeffs, stream=None):
    """The temporally blocked pass (FP32, 2D): (one sweep of u (None: from
    zero), 4 R of the residual of that sweep)."""
    torch = _torch()
    d, n = _level(bh)
    nc = (n - 1) // 2
    out = torch.empty_like(bh)
    bc = torch.empty((nc,) * d, dtype=bh.dtype, device=bh.device)
    arr, ncf = _coeff_array(coeffs)
    pu = ctypes.c_void_p(0) if u is None else _dev_ptr(u, bh.dtype, bh.shape, "u")
    _check(lib().mg_op_sweep_restrict(d, n, _prec_of(bh), arr, ncf, pu, _dev_ptr(bh, bh.dtype, bh.shape, "bh"),
                                      ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(bc.data_ptr()),
                                      _stream_ptr(stream)), "mg_op_sweep_restrict")
    return out, bc


def op_prolong_sweep(e_coarse, u, bh, coeffs, u64_acc=None, stream=None):
    """The temporally blocked pass (FP32, 2D): one sweep of u + P e_coarse,
    returned as a new tensor, or (u64_acc given, float64) added to u64_acc in
    place (returned)."""
    torch = _torch()
    d, n = _level(bh)
    nc = (n - 1) // 2
    arr, ncf = _coeff_array(coeffs)
    out = None if u64_acc is not None else torch.empty_like(bh)
    pacc = _dev_ptr(u64_acc, torch.float64, bh.shape, "u64_acc") if u64_acc is not None else None
    _check(lib().mg_op_prolong_sweep(d, n, _prec_of(bh), arr, ncf, _dev_ptr(e_coarse, bh.dtype, (nc,) * d, "e"),
                                     _dev_ptr(u, bh.dtype, bh.shape, "u"), _dev_ptr(bh, bh.dtype, bh.shape, "bh"),
                                     ctypes.c_void_p(0 if out is None else out.data_ptr()), pacc,
                                     _stream_ptr(stream)), "mg_op_prolong_sweep")
    return u64_acc if out is None else out
