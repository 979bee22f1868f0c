"""The sweep entry point that allocates nothing (mg_op_sweep_norm_noalloc).

It serves callers that may not call cudaMalloc (code under a framework's own
memory pool, services with a fixed device-memory budget, latency-bound loops
that cannot afford cudaMalloc's device-wide synchronisation): its block
partial sums live in a fixed device array inside the library. These tests check, through
the C ABI, that it gives the same sweep and the same residual norm as the
allocating entry point mg_op_sweep, on two calls in a row (the array keeps
the previous call's contents), and that grids beyond the array are refused
before any GPU work. The file is named to run last in a full test session.
"""
import ctypes

import numpy as np
import pytest

from paper_2206_05543_gb300 import binding, smoothers


def _coeffs(c):
    return (ctypes.c_double * len(c))(*c), len(c)


def test_noalloc_rejects_oversized_grids_before_any_gpu_work():
    L = binding.lib()
    c, nc = _coeffs(smoothers.M9)
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    assert L.mg_op_sweep_norm_noalloc(2, 32767, 0, c, nc, dummy, dummy, 0, dummy, dummy, None) == binding.MG_EINVAL
    c3, nc3 = _coeffs(smoothers.M7)
    assert L.mg_op_sweep_norm_noalloc(3, 2047, 0, c3, nc3, dummy, dummy, 0, dummy, dummy, None) == binding.MG_EINVAL
    assert L.mg_op_sweep_norm_noalloc(2, 64, 0, c, nc, dummy, dummy, 0, dummy, dummy, None) == binding.MG_EINVAL


@pytest.mark.gpu
@pytest.mark.parametrize("d,n,dtype,unscaled", [(2, 1023, "float64", True), (2, 255, "float64", False),
                                                (3, 63, "float64", True), (2, 511, "float32", False),
                                                (3, 31, "float32", False)])
def test_noalloc_matches_allocating_entry_point(d, n, dtype, unscaled):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    tdt = getattr(torch, dtype)
    rng = np.random.default_rng(n + d)
    u = torch.from_numpy(rng.uniform(-1, 1, (n,) * d)).to("cuda", tdt)
    bh = torch.from_numpy(rng.uniform(-1, 1, (n,) * d) / (n + 1) ** 2).to("cuda", tdt)
    w = smoothers.default(d)
    ref_out, ref_norm = binding.op_sweep(u, bh, w, b_unscaled=unscaled, want_norm=True)
    L = binding.lib()
    c, nc = _coeffs(w)
    prec = binding.MG_FP64 if dtype == "float64" else binding.MG_FP32_IR
    stream = torch.cuda.current_stream()
    for call in range(2):
        out = torch.full_like(u, float("nan"))
        nrm = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        st = L.mg_op_sweep_norm_noalloc(d, n, prec, c, nc, ctypes.c_void_p(u.data_ptr()),
                                        ctypes.c_void_p(bh.data_ptr()), int(unscaled), ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(nrm.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == binding.MG_OK, call
        torch.cuda.synchronize()
        if call == 1:  # the first call may load the kernels; the second must take no device memory
            assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == alloc0
        assert torch.equal(out, ref_out), call
        assert nrm.item() == pytest.approx(ref_norm, rel=1e-13), call
