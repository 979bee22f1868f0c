"""The multi-rank path of the benchmark on the CPU: two gloo ranks over
127.0.0.1 run the same cross-rank reduction the GPU ranks run under NCCL
(the slowest rank's time, the sum of the cycles of all replicas), and the
reference arm leaves the work to rank 0."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        ms = [12.5, 20.0][rank]
        cycles = [10, 11][rank]
        out[rank] = bench.reduce_over_ranks(ms, cycles, "cpu")
    finally:
        dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        got = dict(out)
    # every rank sees the slowest time and the total cycles of both replicas
    assert got[0] == got[1] == (20.0, 21.0)


def test_reduce_without_a_process_group_is_the_rank_itself():
    import bench

    assert bench.reduce_over_ranks(3.5, 7, "cpu") == (3.5, 7.0)


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun only rank 0 runs the oracle and prints; rank 1 prints
    nothing and exits 0 (checked here without a process group: the arm reads
    RANK from the environment)."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
