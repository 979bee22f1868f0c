"""The temporally blocked FP32 2D passes of a V(1,1) visit, through the C ABI:
(A) pre-sweep + residual + full weighting, (B) interpolation + correction +
post-sweep (optionally adding into an FP64 solution). They evaluate every
value with the formulas and operation order of the single steps, so their
FP32 outputs must equal the composition of mg_op_sweep,
mg_op_residual_restrict and mg_op_prolong_correct bit for bit (those are
checked against the FP64 oracle within a derived rounding bound in
test_gpu_ops.py), on sizes that span several warp tiles and row chunks and
end in ragged tiles, and for every 2D smoother of Sec. 3.1."""
import numpy as np
import pytest

from paper_2206_05543_gb300 import smoothers

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2206_05543_gb300 import binding  # noqa: E402
from paper_2206_05543_gb300.binding import MGError  # noqa: E402

SIZES = [7, 15, 31, 127, 255, 511, 1023, 4095]
NAMES = ["m9", "jacobi", "m5", "vanka", "tw5"]


def f32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _case(n, seed):
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1, 1, (n, n))
    bh = rng.uniform(-1, 1, (n, n)) / (n + 1) ** 2
    e = rng.uniform(-1, 1, ((n - 1) // 2,) * 2) * 1e-3
    return f32(u), f32(bh), f32(e)


def _bits(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("zero_start", [True, False])
def test_sweep_restrict_equals_the_single_steps(n, name, zero_start):
    w = smoothers.get(2, name)
    u, bh, _ = _case(n, n + 1)
    uin = None if zero_start else u
    u1, bc = binding.op_sweep_restrict(uin, bh, w)
    ref_u1, _ = binding.op_sweep(uin, bh, w)
    ref_bc = binding.op_residual_restrict(ref_u1, bh)
    assert np.array_equal(_bits(u1), _bits(ref_u1))
    assert np.array_equal(_bits(bc), _bits(ref_bc))


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("name", NAMES)
def test_prolong_sweep_equals_the_single_steps(n, name):
    w = smoothers.get(2, name)
    u, bh, e = _case(n, n + 2)
    out = binding.op_prolong_sweep(e, u, bh, w)
    v = binding.op_prolong_correct(e, u.clone())
    ref, _ = binding.op_sweep(v, bh, w)
    assert np.array_equal(_bits(out), _bits(ref))


@pytest.mark.parametrize("n", [15, 255, 1023, 4095])
def test_prolong_sweep_into_fp64(n):
    """The FP64 epilogue: u64 += (FP32 sweep result widened exactly), one
    IEEE double addition per point, on two calls in a row."""
    w = smoothers.M9
    u, bh, e = _case(n, n + 3)
    u64 = torch.from_numpy(np.random.default_rng(n).uniform(-1, 1, (n, n))).cuda()
    start = u64.clone()
    binding.op_prolong_sweep(e, u, bh, w, u64_acc=u64)
    v = binding.op_prolong_correct(e, u.clone())
    ref, _ = binding.op_sweep(v, bh, w)
    torch.cuda.synchronize()
    want = start.cpu().numpy() + ref.cpu().numpy().astype(np.float64)
    assert np.array_equal(u64.cpu().numpy(), want)
    binding.op_prolong_sweep(e, u, bh, w, u64_acc=u64)
    torch.cuda.synchronize()
    assert np.array_equal(u64.cpu().numpy(), want + ref.cpu().numpy().astype(np.float64))


def test_fused_passes_reject_other_forms():
    u, bh, e = _case(15, 1)
    with pytest.raises(MGError):  # FP64 arrays
        binding.op_sweep_restrict(None, bh.double(), smoothers.M9)
    with pytest.raises(MGError):  # 3D
        b3 = torch.zeros((15, 15, 15), dtype=torch.float32, device="cuda")
        binding.op_sweep_restrict(None, b3, smoothers.M7)
