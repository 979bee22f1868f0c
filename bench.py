#!/usr/bin/env python3
"""Throughput benchmark of the SPAI-smoothed multigrid solver on one GB300.

Workload (the headline configuration): 2D Poisson, 5-point stencil, N = 8192
(8191^2 = 67,092,481 unknowns), FP64, b ~ U[-1, 1] (numpy seed 0), zero
initial guess, V(1,1) cycles with the M9 SPAI smoother (Theorem 3.1), full
weighting, bilinear interpolation, 12 levels, solved to a 1e-10 relative
residual. One step = one complete solve (about ten cycles) with b resident
in HBM; every field (537 MB) is larger than L2, so no flush is needed.

value = unknowns x V-cycles / second (DOF/s), summed over ranks; each rank
solves its own replica of the problem (the single-problem path is not
decomposed across GPUs). Printed as one JSON line by rank 0. e2e is the same
metric with every step's b copied in from pinned host memory and its u and
outcome returned to pinned host memory, the solves queued with
mg_solve_async on two alternating device slots so that the copies of one
step overlap the solve of the next.

--impl reference times the FP64 CPU oracle (the checker in oracle/) on this
machine's host cores on the same workload; each step is a bounded sample,
one V(1,1) cycle of the full-size problem.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "V(1,1)-cycles/s & DOF/s, % HBM peak; time-to-1e-10 mixed vs FP64 on GPU"
D, N, TOL, SEED = 2, 8192, 1e-10, 0
NU1 = NU2 = 1
UNKNOWNS = (N - 1) ** D
WORKLOAD = "poisson2d-N8192-fp64-V(1,1)-M9-tol1e-10"
# Algorithmic floating-point operations per point of one 2D sweep
# u' = u + c0 r + c1 E + c2 C with r = bh - 4u + (sum of the 4 neighbours),
# each point's residual formed once: the residual 6 (3 adds for the
# neighbour sum, 1 multiply and 2 adds), the edge and corner sums of r 3 + 3,
# the update 3 multiplies + 3 adds = 18 flops.
SWEEP_FLOPS_PER_POINT = 18
# FP64 instructions the kernel issues per point (add, mul and fma count one
# each): s (3), rh (fma + add), the vertical pair sum reused by neighbouring
# points (1), E (2), C (1), update (3 fma) = 12. (h^2 b is an exact
# power-of-two scaling on the exponent field, done with integer instructions.)
SWEEP_DP_INSTR_PER_POINT = 12
# algorithmic bytes per point of one sweep: read u, read b, write u' (FP64)
SWEEP_BYTES_PER_POINT = 24
# nominal FP64 pipe of this part: 2 operations (add, mul or fma) per SM per
# clock, i.e. 2 x 2 flops per SM per clock for FMAs (1.26 TFLOP/s at 152 SMs
# and 2070 MHz: the part's quoted 1.25 TFLOP/s FP64)
FP64_OPS_PER_SM_CLK = 2
# algorithmic words per finest unknown of one V(1,1) cycle, summed over the
# levels (x 4/3 in 2D): the temporally fused lower bound (pre-sweeps,
# residual and restriction in one pass; interpolation, correction and
# post-sweeps in another: 6 + 2^(1-d) words) and the unfused minimal kernel
# sequence (sweep 3 words, residual + restriction and interpolation +
# correction 2 + 2^-d each: 10 + 2^(1-d) words)
WORDS_FUSED_LOWER = 6 + 2 ** (1 - D)
WORDS_UNFUSED = 10 + 2 ** (1 - D)
LEVEL_SUM = 2 ** D / (2 ** D - 1)
NOMINAL_HBM_GBS = 7900.0


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return {"hbm_gbs": p["hbm_gbs"], "sm_max_mhz": p.get("sm_max_mhz", 2070.0), "source": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() in ("active", "yes", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def run_reference(args):
    """The FP64 CPU oracle on the host cores: one V(1,1) cycle of the
    full-size workload per step (single-threaded C)."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from oracle import coeffs
    from paper_2206_05543_gb300 import inputs

    b = inputs.uniform(D, N, SEED)
    u = np.zeros_like(b)
    w = coeffs.default(D)
    for _ in range(args.warmup):
        oracle.cycles(b, u, w, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u = oracle.cycles(b, u, w, 1)
    dt = time.perf_counter() - t0
    value = UNKNOWNS * args.steps / dt
    sample = f"{args.steps} V(1,1) cycles of the full-size {WORKLOAD} problem (oracle.cycles, C, 1 thread)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "d": D, "N": N, "unknowns": UNKNOWNS},
        "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def reduce_over_ranks(ms: float, cycles: float, device) -> tuple[float, float]:
    """The job's timing across ranks: the slowest rank's time and the sum of
    the cycles every rank ran (each rank solves its own replica). One rank
    returns its own numbers. `device` is where the collective's tensor lives
    (the rank's GPU under NCCL; the CPU under gloo)."""
    import torch

    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(ms), float(cycles)
    if torch.distributed.get_world_size() == 1:
        return float(ms), float(cycles)
    t = torch.tensor([ms, cycles], dtype=torch.float64, device=device)
    tmax = t.clone()
    torch.distributed.all_reduce(tmax, op=torch.distributed.ReduceOp.MAX)
    tsum = t.clone()
    torch.distributed.all_reduce(tsum, op=torch.distributed.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[1])


def _cpu_baseline_sample(threads: int = 1):
    """The oracle timed on a bounded sample: one V(1,1) cycle of the full
    problem (a few seconds of single-threaded CPU work). threads > 1 spreads
    the oracle's grid loops over that many host cores (OpenMP)."""
    import numpy as np

    import oracle
    from oracle import coeffs
    from paper_2206_05543_gb300 import inputs

    b = inputs.uniform(D, N, SEED)
    u = np.zeros_like(b)
    used = oracle.set_threads(threads)
    try:
        t0 = time.perf_counter()
        oracle.cycles(b, u, coeffs.default(D), 1)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(1)
    return {"value": UNKNOWNS / dt, "unit": "DOF/s", "cores": used, "kind": "oracle",
            "sample": f"1 V(1,1) cycle of the full-size problem in {dt:.2f} s (C oracle, {used} thread"
                      f"{'' if used == 1 else 's'})"}


def make_workload(name, torch):
    """(step, unknowns, description, close) for one workload; step() runs one
    full solve (or adjoint) and returns the cycle count."""
    import numpy as np

    from paper_2206_05543_gb300 import inputs, smoothers
    from paper_2206_05543_gb300.binding import BatchedSolver, Solver

    # "-mixed": FP32 cycles in FP64 refinement, one cycle per refinement
    # iteration; "-mixed2": two cycles per iteration
    inner = 2 if name.endswith("-mixed2") else 1
    if name in ("2d8192", "2d8192-mixed", "2d8192-mixed2", "2d64"):
        n_ = 64 if name == "2d64" else N
        prec = "fp32_ir" if "-mixed" in name else "fp64"
        b = torch.from_numpy(inputs.sine(2, n_) if name == "2d64" else inputs.uniform(2, n_, SEED)).cuda()
        u = torch.zeros_like(b)
        s = Solver(2, n_, smoothers.M9, nu1=1, nu2=1, precision=prec)
        if inner > 1:
            s.set_refinement_cycles(inner)

        last = {}

        def step():  # V-cycles run
            info = s.solve(b, u, tol=TOL, max_cycles=100, zero_start=True)
            last.update(u=u, relres=info.relres)
            return info.cycles * inner
        step.last = last
        return step, (n_ - 1) ** 2, f"2D N={n_} {prec}{'' if inner == 1 else f' x{inner}'} V(1,1) M9 to 1e-10", s.close
    if name.startswith("3d") and name.endswith(("-fp64", "-mixed", "-mixed2")):
        # 3d512-*: the rows; smaller sizes (3d256-mixed, ...) serve profiling
        n_ = int(name[2:name.index("-")])
        prec = "fp32_ir" if "-mixed" in name else "fp64"
        b = torch.from_numpy(inputs.uniform(3, n_, SEED)).cuda()
        u = torch.zeros_like(b)
        s = Solver(3, n_, smoothers.M7, nu1=2, nu2=2, precision=prec)
        if inner > 1:
            s.set_refinement_cycles(inner)

        last = {}

        def step():  # V-cycles run
            info = s.solve(b, u, tol=TOL, max_cycles=100, zero_start=True)
            last.update(u=u, relres=info.relres)
            return info.cycles * inner
        step.last = last
        return step, (n_ - 1) ** 3, f"3D N={n_} {prec}{'' if inner == 1 else f' x{inner}'} V(2,2) M7 to 1e-10", s.close
    if name in ("batch256", "batch256-2"):
        Ns = [int(x) for x in inputs.batch_sizes(256, 0)]
        bs = [torch.from_numpy(b).cuda() for b in inputs.batch_rhs(Ns, 1)]
        # the 256 results are views of one buffer (each 256-byte aligned)
        offs, o = [], 0
        for b in bs:
            offs.append(o)
            o += (b.numel() + 31) // 32 * 32
        u_all = torch.zeros(o, dtype=torch.float64, device="cuda")
        us = [u_all[a:a + b.numel()].view(b.shape) for a, b in zip(offs, bs)]
        s = BatchedSolver(Ns, smoothers.M9, nu1=1, nu2=1)
        inner_b = 2 if name.endswith("-2") else 1
        if inner_b > 1:
            s.set_refinement_cycles(inner_b)
        tot = sum((n_ - 1) ** 2 for n_ in Ns)

        def step():  # V-cycles run, weighted by problem size; from u = 0 (the us are output only)
            _, st, cyc, _ = s.solve(bs, us, tol=TOL, max_cycles=100, zero_start=True)
            return inner_b * sum((n_ - 1) ** 2 * c for n_, c in zip(Ns, cyc)) / tot
        return step, tot, (f"256 2D problems, N in {{64..1024}}, FP32 V(1,1) in FP64 refinement to 1e-10"
                           f"{'' if inner_b == 1 else f', {inner_b} cycles per iteration'}"), s.close
    if name in ("2d8192-m5", "2d8192-jacobi", "3d512-jacobi"):
        # the smoother comparison on the full-size FP64 problems: the same
        # cycle with other SPAI coefficient sets (Sec. 3.1)
        d_ = 2 if name.startswith("2d") else 3
        n_ = N if d_ == 2 else 512
        w = smoothers.M5 if name.endswith("-m5") else smoothers.get(d_, "jacobi")
        nu = 1 if d_ == 2 else 2
        b = torch.from_numpy(inputs.uniform(d_, n_, SEED)).cuda()
        u = torch.zeros_like(b)
        s = Solver(d_, n_, w, nu1=nu, nu2=nu, precision="fp64")

        def step():
            info = s.solve(b, u, tol=TOL, max_cycles=200, zero_start=True)
            return info.cycles
        label = "M5" if name.endswith("-m5") else "weighted Jacobi"
        return step, (n_ - 1) ** d_, f"{d_}D N={n_} fp64 V({nu},{nu}) {label} to 1e-10", s.close
    if name in ("3d512-m27", "3d512-m27-v22"):
        # the LFA-optimal symmetric 27-point smoother (min-max over its
        # family, Sec. 3.2's wider stencils), FP64, V(1,1) and V(2,2)
        nu = 2 if name.endswith("-v22") else 1
        b = torch.from_numpy(inputs.uniform(3, 512, SEED)).cuda()
        u = torch.zeros_like(b)
        s = Solver(3, 512, smoothers.M27, nu1=nu, nu2=nu, precision="fp64")

        def step():
            info = s.solve(b, u, tol=TOL, max_cycles=100, zero_start=True)
            return info.cycles
        return step, 511 ** 3, f"3D N=512 fp64 V({nu},{nu}) 27-point LFA-optimal M to 1e-10", s.close
    if name == "adjoint128":
        b = torch.from_numpy(inputs.gaussian(3, 128, 0)).to("cuda", torch.float32)
        g = torch.from_numpy(np.random.default_rng(1).standard_normal(b.shape)).to("cuda", torch.float32)
        s = Solver(3, 128, smoothers.M7, nu1=1, nu2=1, precision="fp32")

        def step():
            s.vcycles_adjoint(b, g, 4)
            return 4
        return step, 127 ** 3, "adjoint of 4 FP32 V(1,1) cycles, 3D N=128 (forward replay + reverse)", s.close
    raise ValueError(name)


ROWS = ["2d64", "2d8192-mixed", "2d8192-mixed2", "3d512-fp64", "3d512-mixed", "3d512-mixed2", "batch256", "batch256-2",
        "adjoint128", "2d8192-m5", "2d8192-jacobi", "3d512-jacobi", "3d512-m27", "3d512-m27-v22"]


def time_workload(name, torch, warmup=2, steps=5, keep=None):
    """Median of `steps` timed runs (CUDA events) after `warmup` (the best run
    as ms_min); for solver workloads also the final relative residual (FP64,
    from the library) and, when `keep` is a dict, the last solution under
    keep[name] (compared after timing)."""
    step, unknowns, desc, close = make_workload(name, torch)
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    times, cycles = [], 0
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        cycles = step()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    r = {"workload": desc, "ms": ms, "ms_min": min(times), "cycles": cycles,
         "dof_per_s": unknowns * cycles / (ms * 1e-3)}
    last = getattr(step, "last", None)
    if last:
        r["final_relres"] = last["relres"]
        if keep is not None:
            keep[name] = last["u"].clone()
    close()
    return r


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2206_05543_gb300 import binding, inputs, smoothers
    from paper_2206_05543_gb300.binding import Solver

    if args.workload != "2d8192":
        # profiling entry: time --steps runs of another workload
        r = time_workload(args.workload, torch, args.warmup, args.steps)
        if rank == 0:
            print(json.dumps({"workload": args.workload, **r, "note": "single-workload run"}), flush=True)
        return
    peaks = _peaks()
    stream = torch.cuda.current_stream()
    b_host = torch.from_numpy(inputs.uniform(D, N, SEED)).pin_memory()
    b = b_host.to("cuda", non_blocking=False)
    u = torch.zeros_like(b)
    solver = Solver(D, N, smoothers.M9, nu1=NU1, nu2=NU2, precision="fp64")

    def one_solve():  # from u = 0 (u is output only: MG_SOLVE_ZERO_START)
        return solver.solve(b, u, tol=TOL, max_cycles=100, zero_start=True)

    for _ in range(args.warmup):
        info = one_solve()
        assert info.converged, info.status

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    launches0 = binding.kernel_launch_count()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cycles = 0
    for _ in range(args.steps):
        info = one_solve()
        cycles += info.cycles
    e1.record(stream)
    barrier()
    launches = binding.kernel_launch_count() - launches0
    ms = e0.elapsed_time(e1)
    if args.only_solve:
        clocks.stop()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": UNKNOWNS * cycles / (ms * 1e-3), "unit": "DOF/s",
                              "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                              "ms_per_step": ms / args.steps, "cycles": cycles, "gpu_launches": launches,
                              "note": "solve-only run"}), flush=True)
        solver.close()
        return
    ms, total_cycles = reduce_over_ranks(ms, cycles, "cuda")
    value = UNKNOWNS * total_cycles / (ms * 1e-3)

    # end to end through the public API, every step: its b from pinned host
    # memory to the device, the solve, its u back to pinned host memory, its
    # outcome (mg_solve_info) written by the device into pinned host memory.
    # Two device slots of (b, u) alternate: step k+1's input is copied in and
    # step k-1's result copied out, each direction on its own copy stream,
    # while step k solves (mg_solve_async: the solve, stop test included, is
    # queued without synchronising; the context keeps the graphs of both
    # slots).
    u_host = torch.empty_like(b_host).pin_memory()
    slots_b = [torch.empty_like(b) for _ in range(2)]
    slots_u = [torch.empty_like(b) for _ in range(2)]
    infos = [torch.zeros(24, dtype=torch.uint8, pin_memory=True) for _ in range(args.steps)]
    for sb, su in zip(slots_b, slots_u):  # record both slots' graphs before timing
        sb.copy_(b)
        solver.solve_async(sb, su, tol=TOL, max_cycles=100, zero_start=True, info_buf=infos[0]).result()
    cs_in, cs_out = torch.cuda.Stream(), torch.cuda.Stream()

    def copy_gbs(dst, src, cs):  # one copy alone, for the record (host links differ between machines)
        with torch.cuda.stream(cs):
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(cs)
            dst.copy_(src, non_blocking=True)
            z.record(cs)
        z.synchronize()
        return src.numel() * src.element_size() / (a.elapsed_time(z) * 1e-3) / 1e9

    h2d_gbs, d2h_gbs = copy_gbs(slots_b[0], b_host, cs_in), copy_gbs(u_host, slots_u[0], cs_out)
    in_ready = [torch.cuda.Event() for _ in range(2)]
    solved = [torch.cuda.Event() for _ in range(2)]
    out_done = [torch.cuda.Event() for _ in range(2)]
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    with torch.cuda.stream(cs_in):  # step 0's input
        cs_in.wait_event(f0)
        slots_b[0].copy_(b_host, non_blocking=True)
        in_ready[0].record(cs_in)
    pending = []
    for k in range(args.steps):
        sl = k % 2
        if k + 1 < args.steps:
            with torch.cuda.stream(cs_in):  # the next step's input, once step k-1 stopped reading its slot
                if k >= 1:
                    cs_in.wait_event(solved[1 - sl])
                slots_b[1 - sl].copy_(b_host, non_blocking=True)
                in_ready[1 - sl].record(cs_in)
        stream.wait_event(in_ready[sl])
        if k >= 2:
            stream.wait_event(out_done[sl])  # step k-2's result has left this slot
        pending.append(solver.solve_async(slots_b[sl], slots_u[sl], tol=TOL, max_cycles=100, zero_start=True,
                                          info_buf=infos[k]))
        solved[sl].record(stream)
        with torch.cuda.stream(cs_out):  # this step's result, during the next solve
            cs_out.wait_event(solved[sl])
            u_host.copy_(slots_u[sl], non_blocking=True)
            out_done[sl].record(cs_out)
    stream.wait_stream(cs_in)
    stream.wait_stream(cs_out)
    f1.record(stream)
    barrier()
    clocks.stop()
    e2e_ms = f0.elapsed_time(f1)
    e2e_cycles = 0
    for p in pending:
        r = p.result()
        assert r.converged, r.status
        e2e_cycles += r.cycles
    e2e_value = world * UNKNOWNS * e2e_cycles / (e2e_ms * 1e-3)

    # dominant kernel: the finest-level FP64 sweep, timed alone on the stream
    # it is launched on, same launch configuration as inside the cycle
    out = torch.empty_like(b)
    ur = torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, b.shape)).cuda()
    for _ in range(3):
        binding.op_sweep(ur, b, smoothers.M9, b_unscaled=True, stream=stream, out=out)
    reps = 20
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(reps):
        binding.op_sweep(ur, b, smoothers.M9, b_unscaled=True, stream=stream, out=out)
    k1.record(stream)
    torch.cuda.synchronize()
    sweep_s = k0.elapsed_time(k1) * 1e-3 / reps
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    clk_hz = peaks["sm_max_mhz"] * 1e6
    # nominal FP64 FLOP peak (FMA = 2 flops) and the measured DFMA issue rate
    peak_flops = 2 * FP64_OPS_PER_SM_CLK * sms * clk_hz
    rates = {k: binding.measure_fp64_rate(k) for k in binding.FP64_RATE_KINDS}
    measured_flops = 2 * rates["dfma_reg"][0] * sms * clk_hz
    achieved_flops = SWEEP_FLOPS_PER_POINT * UNKNOWNS / sweep_s
    issued_ops = SWEEP_DP_INSTR_PER_POINT * UNKNOWNS / sweep_s
    sweep_gbs = SWEEP_BYTES_PER_POINT * UNKNOWNS / sweep_s / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            traffic = json.load(f).get("sweep2d_fp64_n8191")

    solve_s = ms * 1e-3 / args.steps
    cyc_per_solve = cycles / args.steps
    eff_lo = WORDS_FUSED_LOWER * 8 * LEVEL_SUM * UNKNOWNS * cyc_per_solve / solve_s / 1e9
    eff_un = WORDS_UNFUSED * 8 * LEVEL_SUM * UNKNOWNS * cyc_per_solve / solve_s / 1e9

    rows = {}
    if not args.no_rows:
        sols = {}
        for w in ROWS:
            rows[w] = time_workload(w, torch, keep=sols if ("-mixed" in w or w == "3d512-fp64") else None)
            # mixed precision against the plain FP64 solution of the same grid:
            # ||u_mixed - u_fp64|| / ||u_fp64|| (after timing, on the device)
            ref = u if w.startswith("2d8192") else sols.get("3d512-fp64")
            if "-mixed" in w and ref is not None:
                rows[w]["diff_vs_fp64"] = float(torch.linalg.vector_norm(sols.pop(w) - ref) /
                                                torch.linalg.vector_norm(ref))
        sols.clear()
        rows["3d512_mixed_speedup_vs_fp64"] = rows["3d512-fp64"]["ms"] / rows["3d512-mixed"]["ms"]
        rows["3d512_mixed2_speedup_vs_fp64"] = rows["3d512-fp64"]["ms"] / rows["3d512-mixed2"]["ms"]
        # time to 1e-10 of the other smoothers over that of the paper's optimum
        # (M9 in 2D: this run's headline solve; M7 in 3D)
        rows["time_ratio_vs_optimal_smoother"] = {
            "2d_m5_vs_m9": rows["2d8192-m5"]["ms"] / (ms / args.steps),
            "2d_jacobi_vs_m9": rows["2d8192-jacobi"]["ms"] / (ms / args.steps),
            "3d_jacobi_vs_m7": rows["3d512-jacobi"]["ms"] / rows["3d512-fp64"]["ms"],
            "3d_m27_v11_vs_m7_v22": rows["3d512-m27"]["ms"] / rows["3d512-fp64"]["ms"],
            "3d_m27_v22_vs_m7_v22": rows["3d512-m27-v22"]["ms"] / rows["3d512-fp64"]["ms"]}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "d": D, "N": N, "unknowns": UNKNOWNS, "smoother": "M9",
                       "cycle": "V(1,1)", "levels": 12, "tol": TOL, "rhs": "U[-1,1] seed 0", "u0": "zero",
                       "l2": "no flush: every field (537 MB) is larger than L2",
                       "parallelism": f"replicas{world}"},
            "vcycles_per_s": total_cycles / (ms * 1e-3) / world,
            "cycles_per_solve": cycles / args.steps,
            "time_to_tol_ms": ms / args.steps,
            "mixed_fp32_ir": ({"time_to_tol_ms": rows["2d8192-mixed"]["ms"],
                               "iterations": rows["2d8192-mixed"]["cycles"],
                               "speedup_vs_fp64": (ms / args.steps) / rows["2d8192-mixed"]["ms"],
                               "two_cycles_per_iteration": {
                                   "time_to_tol_ms": rows["2d8192-mixed2"]["ms"],
                                   "vcycles": rows["2d8192-mixed2"]["cycles"],
                                   "speedup_vs_fp64": (ms / args.steps) / rows["2d8192-mixed2"]["ms"]}}
                              if rows else None),
            "roofline": {"bound": "alu", "achieved": achieved_flops / 1e9, "peak": peak_flops / 1e9,
                         "unit": "GFLOP/s FP64", "frac": achieved_flops / peak_flops, "traffic": traffic,
                         "kernel": "sweep2d_kernel<double> (finest level, n=8191)",
                         "achieved_basis": f"{SWEEP_FLOPS_PER_POINT} algorithmic flops/point x {UNKNOWNS} points"
                                           " / CUDA-event time per launch",
                         "peak_basis": f"nominal: {FP64_OPS_PER_SM_CLK} FP64 FMA/SM/clk x 2 flops x {sms} SMs x "
                                       f"{peaks['sm_max_mhz']:.0f} MHz (max SM clock, {peaks['source']})",
                         "flop_frac_nominal": achieved_flops / peak_flops,
                         "flop_frac_measured_dfma": achieved_flops / measured_flops,
                         "measured_dfma_gflops": measured_flops / 1e9,
                         "fp64_issue_occupancy": issued_ops / (FP64_OPS_PER_SM_CLK * sms * clk_hz),
                         "issue_basis": f"{SWEEP_DP_INSTR_PER_POINT} FP64 instructions/point issued by the kernel "
                                        f"against the nominal {FP64_OPS_PER_SM_CLK}/SM/clk",
                         "fp64_rates_ops_per_sm_clk": {k: round(v[0], 4) for k, v in rates.items()},
                         "fp64_rates_sm_mhz": {k: round(v[1], 1) for k, v in rates.items()},
                         "hbm_gbs": sweep_gbs, "hbm_frac": sweep_gbs / peaks["hbm_gbs"],
                         "hbm_frac_nominal_7900": sweep_gbs / 7900.0,
                         "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_peak_source": peaks["source"],
                         "ms_per_launch": sweep_s * 1e3},
            # the whole solve against the algorithmic bytes of its cycles
            "effective_bandwidth": {
                "fused_lower_bound_bytes_per_cycle": WORDS_FUSED_LOWER * 8 * LEVEL_SUM * UNKNOWNS,
                "unfused_bytes_per_cycle": WORDS_UNFUSED * 8 * LEVEL_SUM * UNKNOWNS,
                "gbs_fused_lower_bound": eff_lo, "gbs_unfused": eff_un,
                "frac_measured_hbm": eff_lo / peaks["hbm_gbs"], "frac_nominal_7900": eff_lo / NOMINAL_HBM_GBS,
                "note": "FP64 ALU-bound: the cycle's bytes are not its limit"},
            "e2e": {"value": e2e_value, "unit": "DOF/s", "h2d_bytes_per_step": b.numel() * 8,
                    "d2h_bytes_per_step": u.numel() * 8 + 24, "h2d_gbs": h2d_gbs, "d2h_gbs": d2h_gbs},
            "gpu_launches": launches,
            "clocks": clocks.summary(),
            "rows": rows,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = _cpu_baseline_sample()
            # the same oracle with its grid loops on every host core
            line["cpu_baseline_all_cores"] = _cpu_baseline_sample(_cpu_cores())
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing (debug runs)")
    ap.add_argument("--no-rows", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--workload", default="2d8192", choices=["2d8192"] + ROWS + ["3d256-mixed", "3d256-mixed2", "3d256-fp64"],
                    help="with --only-solve: which workload to time (profiling)")
    ap.add_argument("--only-solve", action="store_true",
                    help="time the solves only (no e2e, kernel, mixed or CPU legs); used for profiler launch lists")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
