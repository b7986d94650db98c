"""Benchmark of the blended D2Q5 vectorial LBM step on GB300.

Default workload: the 4096 x 4096 near-vacuum blast (rho = 1, p = 1e-6, total
energy 1 in the 2x2 centre cells, reflective walls), second order with the PP
limiter (eps = 1e-13), FP32 populations with FP64 theta_p solves, dynamic
kinetic speed. One "step" is one time step of the whole grid. The metric is
MLUPS (million cell updates per second), next to the fraction of the HBM
roofline of the step kernel (160 algorithmic bytes per cell update: 20 FP32
values read and 20 written).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank advances its own replica of
the grid (the single-grid step is not sharded: "replicas only"); value is the
sum of all ranks' cell updates over the slowest rank's time.

The reference arm (--impl reference) times the FP64 CPU oracle (test
infrastructure under oracle/) on this machine's host cores, on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("MLUPS & % HBM roofline, 2nd-order+PP FP32 at 4096^2; batched vs sequential; "
          "adjoint/forward")
BYTES_PER_LU = 160           # 20 FP32 values read + 20 written per cell update
N_SIDE = 4096
EPS = 1e-13
FALLBACK_HBM_GBS = 6800.0
SPONGE = 5                   # theta = 0 layer at zero-gradient sides, as the paper pairs them (Sec. 4.2)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


# The 1024^2 LMP quadrant run (FP32 populations, to t = 0.25) is held to the spread
# of the FP64 oracle itself under float-level noise, not to the stated 1e-3 L1 target:
# tests/test_gpu_fullsize.py and tests/golden/quadrant1024_lmp_jitter.txt.
ACCURACY_GAP_1024_LMP = (
    "1024^2 four-quadrant Riemann problem, LMP, FP32 populations, t = 0.25: the stated L1(rho) "
    "target of 1e-3 against FP64 is not met (measured about 4e-3); the FP64 oracle run under "
    "2^-24 relative noise per step spreads 5.4e-3 from its own clean run (discontinuous data "
    "amplifies rounding), and the test holds FP32 to 1.1 x that spread")


# The sources the FP32 step kernel is compiled from (its translation unit and
# headers): a committed ncu summary counts for the kernel while their code (comments
# aside) is unchanged.
STEP_KERNEL_SOURCES = ("common.cuh", "kernels_f32.cu", "kernels_impl.cuh", "physics.cuh", "step_fused.cuh",
                       "step_simple.cuh", "tma.cuh", "vlbm_internal.h")


def _code_only(text: str) -> str:
    """C++ source without comments, blank lines and trailing spaces (a comment edit does
    not change the kernel)."""
    out, i, n = [], 0, len(text)
    while i < n:
        if text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        elif text[i] == '"':                       # string literal: copied as is
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(text[i])
            i += 1
    lines = (line.rstrip() for line in "".join(out).splitlines())
    return "\n".join(line for line in lines if line)


def _kernel_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2411_15001_gb300", "csrc")
    for name in STEP_KERNEL_SOURCES:
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def _ncu_summary():
    """The committed ncu summary of the step kernel, if it was taken on the current
    kernel sources; else {}."""
    path = os.path.join(ROOT, "profiles", "step_fused_blast.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except OSError:
        return {}
    return d if d.get("kernel_hash") == _kernel_hash() else {}


def _ncu_traffic():
    """DRAM bytes per launch of the step kernel (full size), or None."""
    return _ncu_summary().get("dram_bytes_per_launch_full_size")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, device=None) -> float:
    """The maximum of x over all ranks (x itself without a process group)."""
    import torch

    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world: int, cells: int, steps: int, seconds: float) -> float:
    """Cell updates of all ranks (each advances its own replica) over the slowest rank's time."""
    return world * cells * steps / seconds / 1e6


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(n_side: int = N_SIDE, target_s: float = 15.0, max_steps: int = 50,
                 single_thread_s: float = 8.0):
    """The FP64 oracle on this host's cores, timed over whole time steps of the blast:
    all cores (OpenMP over rows), then one thread on the steps that follow."""
    from oracle import oracle as O
    from paper_2411_15001_gb300 import workloads as W

    cores = os.cpu_count() or 1
    mem_gb = None
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable"):
                    mem_gb = int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    n = n_side if (mem_gb is None or mem_gb > 40 or n_side <= 2048) else 2048
    p = W.blast(n)
    cfg = O.Config(n, n, p.bc, O.LIM_PP, p.gamma, 0.5, EPS)
    state = O.new_state(p.conserved())
    a = O.kinetic_speed(O.max_speed(cfg, state), 0.5)
    state = O.init_populations(cfg, state, a)

    def timed(threads, budget, limit):
        nonlocal state, a
        O.set_threads(threads)
        steps, t0 = 0, time.perf_counter()
        while True:
            state = O.step(cfg, state, a)
            a = O.kinetic_speed(O.max_speed(cfg, state), 0.5)
            steps += 1
            if time.perf_counter() - t0 > budget or steps >= limit:
                break
        return steps, time.perf_counter() - t0

    steps, dt = timed(cores, target_s, max_steps)
    steps1, dt1 = timed(1, single_thread_s, max(1, max_steps // 4))
    return {"value": n * n * steps / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "single_thread_value": n * n * steps1 / dt1 / 1e6, "cpu_model": _cpu_model(),
            "sample": f"first {steps} time steps of the {n}x{n} blast on {cores} threads (FP64 oracle, "
                      f"OpenMP over rows, per-step array allocation included), then {steps1} more on "
                      f"one thread"}


def cpu_baseline_batched(probs, steps: int = 50, budget_s: float = 10.0):
    """The FP64 oracle on this host's cores over the batched workload's grids, in index
    order, a fixed window of `steps` steps each, until `budget_s` seconds have passed."""
    from oracle import oracle as O

    cores = os.cpu_count() or 1
    O.set_threads(cores)
    lu, grids, t0 = 0, 0, time.perf_counter()
    for p in probs:
        cfg = O.Config(p.nx, p.ny, p.bc, O.LIM_PP, p.gamma, 0.5, EPS, SPONGE)
        O.run(cfg, p.conserved(), p.dx, nsteps=steps)
        lu += p.nx * p.ny * steps
        grids += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": lu / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"the first {grids} of the {len(probs)} grids, {steps} steps each from t = 0, on "
                      f"{cores} threads (FP64 oracle, OpenMP over rows)"}


def workload_config(n: int, world: int) -> dict:
    """The workload both arms time (the reference arm on a bounded sample of its steps)."""
    return {"workload": f"blast {n}x{n} near-vacuum (rho=1, p=1e-6, E=1 in 2x2 centre), reflective walls, "
                        "2nd order + PP limiter eps=1e-13, dynamic a^n",
            "nx": n, "ny": n, "limiter": "PP", "parallelism": f"replicas x{world}"}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    cb = cpu_baseline(args.n, target_s=min(120.0, 8.0 * max(1, args.steps)), max_steps=max(1, args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": dict(workload_config(args.n, args.gpus), precision="fp64 (FP64 oracle)"),
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2411_15001_gb300 import vlbm as V
    from paper_2411_15001_gb300 import workloads as W

    p = W.blast(args.n)
    cons = torch.tensor(p.conserved(), dtype=torch.float32)
    solver = V.VLBM(p.nx, p.ny, p.dx, bc=p.bc, gamma=p.gamma, limiter=V.LIM_PP, precision=V.FP32,
                    eps=EPS, device=dev)
    d = cons.to(dev)
    solver.set_conserved(d[0].contiguous(), d[1:3].contiguous(), d[3].contiguous())

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # ---------------------------------------------------------- device-resident timing
    solver.step(args.warmup)
    barrier()
    stream = solver.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    solver.profile(True)
    with ClockSampler(local) as clk:
        barrier()
        e0.record(stream)
        solver.step(args.steps)
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1)
    kernel_ms, launches = solver.profile_read()
    solver.profile(False)
    mon = solver.monitors()
    ms_max = max_over_ranks(ms, dev)
    cells = p.nx * p.ny
    value = whole_job_mlups(world, cells, args.steps, ms_max / 1e3)

    # ---------------------------------------------------------- end to end (host buffers)
    e2e = None
    if not args.no_e2e:
        host = cons.pin_memory()
        out_host = torch.empty((4, p.ny, p.nx), dtype=torch.float32).pin_memory()
        dbuf = torch.empty_like(d)
        barrier()
        t0 = time.perf_counter()
        dbuf.copy_(host, non_blocking=True)
        solver.set_conserved(dbuf[0].contiguous(), dbuf[1:3].contiguous(), dbuf[3].contiguous())
        # every step's monitors (positivity, lambda) are read back to the host and checked
        # there, one step behind: the copy of step k's record completes while step k + 1
        # runs, so the host never stalls the stream
        bufs = [solver.monitor_buffer() for _ in range(2)]
        evs = [torch.cuda.Event() for _ in range(2)]
        bad = 0

        def check(k):
            nonlocal bad
            evs[k & 1].synchronize()
            m = solver.decode_monitors(bufs[k & 1])
            if m["status"] != 0 or m["n"] != k + 1:
                raise RuntimeError(f"step {k}: status {m['status']}, n {m['n']}")
            bad += m["bad_cells"] + m["nonfinite_cells"]

        for k in range(args.steps):
            solver.step(1)
            solver.monitors_async(bufs[k & 1])
            evs[k & 1].record(solver.stream)
            if k > 0:
                check(k - 1)
        check(args.steps - 1)
        rho, mom, E = solver.moments()
        out_dev = torch.cat([rho[None], mom, E[None]])
        out_host.copy_(out_dev, non_blocking=True)
        torch.cuda.synchronize(dev)
        t_e2e = max_over_ranks(time.perf_counter() - t0, dev)
        e2e = {"value": whole_job_mlups(world, cells, args.steps, t_e2e), "unit": "MLUPS",
               "h2d_bytes_per_step": host.numel() * 4 / args.steps,
               "d2h_bytes_per_step": (out_host.numel() * 4) / args.steps + bufs[0].numel(),
               "positivity_violations": int(bad)}

    full = full_run(dev, args.n) if (not args.no_full_run and world == 1) else None

    peaks, peak_src = _peaks()
    achieved = BYTES_PER_LU * cells / (kernel_ms / launches / 1e3) / 1e9 if launches else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"] if achieved else None,
            "traffic": _ncu_traffic() if args.n == N_SIDE else None,
            "peak_source": f"hbm_gbs of MEASURED_PEAKS.json ({peak_src})",
            "kernel": "k_step_fused<float, PP>", "kernel_ms_avg": kernel_ms / launches if launches else None}
    nsum = _ncu_summary()
    if nsum and args.n == N_SIDE:   # ncu figures of the same kernel (profiles/): DRAM bytes per cell update, FP64 share
        roof["dram_bytes_per_lu"] = nsum["dram_bytes_per_launch_full_size"] / (N_SIDE * N_SIDE)
        roof["fp64_pipe_pct"] = nsum.get("fp64_pipe_pct")

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": dict(workload_config(p.nx, world),
                               precision="fp32 (FP32 populations; FP64 theta_p solve where the float "
                                         "bounds cannot settle a face; FP64 sums)",
                               l2="state 2x1.34 GB >> L2 129 MB; no flush",
                               steps_total=args.warmup + args.steps,
                               positivity_violations=mon["bad_cells"] + mon["nonfinite_cells"],
                               first_bad_step=mon["first_bad_step"], status=mon["status"]),
                "known_gaps": [ACCURACY_GAP_1024_LMP],
                "clocks": clk.summary(), "e2e": e2e, "gpu_launches": launches,
                "roofline": roof, "full_run": full}
        if not args.no_batched:
            line["batched"] = bench_batched(dev, cpu=world == 1 and not args.no_cpu_baseline)
        if not args.no_adjoint:
            line["adjoint"] = bench_adjoint(dev)
            line["adjoint_2048"] = bench_adjoint(dev, n=2048)   # state and cotangents far larger than L2
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.n)
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def full_run(dev, n: int = N_SIDE, steps: int = 2000, skip: int = 100):
    """The blast as specified: `steps` steps from t = 0 (graph replays), timed with CUDA
    events over steps skip..steps; the device's sticky first-bad-step record then says
    whether any step left G or produced a non-finite value."""
    import torch

    from paper_2411_15001_gb300 import vlbm as V
    from paper_2411_15001_gb300 import workloads as W

    p = W.blast(n)
    s = V.VLBM(p.nx, p.ny, p.dx, bc=p.bc, gamma=p.gamma, limiter=V.LIM_PP, precision=V.FP32, eps=EPS,
               device=dev)
    c = torch.tensor(p.conserved(), dtype=torch.float32, device=dev)
    s.set_conserved(c[0].contiguous(), c[1:3].contiguous(), c[3].contiguous())
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    s.step(skip)
    e[0].record(s.stream)
    s.step(steps - skip)
    e[1].record(s.stream)
    torch.cuda.synchronize(dev)
    ms = e[0].elapsed_time(e[1]) / (steps - skip)
    m = s.monitors()
    s.close()
    return {"workload": f"blast {n}x{n}, PP eps=1e-13, FP32, {steps} steps from t = 0",
            "ms_per_step": ms, "mlups": n * n / (ms / 1e3) / 1e6, "timed_steps": f"{skip}..{steps}",
            "hbm_frac": BYTES_PER_LU * n * n / (ms / 1e3) / 1e9 / _peaks()[0]["hbm_gbs"],
            "steps_done": m["n"], "t": m["t"], "status": m["status"], "first_bad_step": m["first_bad_step"],
            "theta_p_fp64_faces_last_step": m["theta_p_fp64_faces"], "min_rho": m["min_rho"]}


def bench_batched(dev, steps: int = 500, count: int = 256, cpu: bool = False):
    """256 seeded quadrant problems of uneven sides (multiples of 64 up to 1024), FP32 PP:
    one launch per step over all grids (graph-replayed, autotuned decomposition) against
    the same problems stepped one grid at a time with one launch per grid and step."""
    import torch

    from paper_2411_15001_gb300 import vlbm as V
    from paper_2411_15001_gb300 import workloads as W

    probs = W.batch_instances(count, seed=1)
    cells = sum(p.nx * p.ny for p in probs)
    conss = [torch.tensor(p.conserved(), dtype=torch.float32, device=dev) for p in probs]

    def load(setter):
        for i, c in enumerate(conss):
            setter(i, c[0].contiguous(), c[1:3].contiguous(), c[3].contiguous())

    b = V.VLBMBatch([(p.nx, p.ny, p.dx, p.bc) for p in probs], limiter=V.LIM_PP, precision=V.FP32,
                    eps=EPS, device=dev, sponge=SPONGE)
    load(b.set_conserved)
    tuning = b.autotune(trial_steps=3)
    load(b.set_conserved)                    # time from n = 0 like the sequential arm
    b.step(3)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.step(steps)
    e1.record(b.stream)
    torch.cuda.synchronize(dev)
    ms_b = e0.elapsed_time(e1)
    mons = [b.monitors(i) for i in range(count)]
    status = [m["status"] for m in mons]
    fp64_faces = sum(m["theta_p_fp64_faces"] for m in mons)
    b.close()
    del b
    def sequential(kernel):
        """The same problems one after another (500 steps each, graph replays), one
        solver per grid, on one stream."""
        solvers = [V.VLBM(p.nx, p.ny, p.dx, bc=p.bc, gamma=p.gamma, limiter=V.LIM_PP, precision=V.FP32,
                          eps=EPS, device=dev, sponge=SPONGE, kernel=kernel) for p in probs]
        load(lambda i, r, m, e: solvers[i].set_conserved(r, m, e))
        for s in solvers:
            s.step(3)
        torch.cuda.synchronize(dev)
        stream = solvers[0].stream
        e0.record(stream)
        for s in solvers:
            s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        for s in solvers:
            s.close()
        return e0.elapsed_time(e1)

    ms_s = sequential(V.KERNEL_FUSED)      # the row-marching kernel, as the batch uses
    ms_a = sequential(V.KERNEL_AUTO)       # each grid with the kernel that is faster for it
    return {"workload": f"{count} quadrant Riemann problems, sides in {{64..1024}} step 64 (seed 1), "
                        f"FP32 PP eps=1e-13, zero-gradient sides with a {SPONGE}-cell theta = 0 sponge "
                        f"(Sec. 4.2), {steps} steps each",
            "cells": cells, "steps": steps,
            "batched_mlups": cells * steps / (ms_b / 1e3) / 1e6,
            "sequential_mlups": cells * steps / (ms_a / 1e3) / 1e6,
            "ratio": ms_a / ms_b, "batched_ms_per_step": ms_b / steps,
            "sequential_ms_per_step": ms_a / steps,
            "sequential": "each grid alone with the kernel the library picks for its size (the "
                          "one-thread-per-cell kernel below 2^19 cells), CUDA graph replays of 64 steps",
            "batched_hbm_frac": BYTES_PER_LU * cells / (ms_b / steps / 1e3) / 1e9 / _peaks()[0]["hbm_gbs"],
            "sequential_row_marching_mlups": cells * steps / (ms_s / 1e3) / 1e6,
            "ratio_vs_row_marching": ms_s / ms_b,
            "sequential_row_marching": "each grid alone with the row-marching kernel the batch uses",
            "tuning": tuning,
            "statuses_nonzero": sum(1 for x in status if x),
            "fp64_theta_p_faces_last_step": fp64_faces,
            "cpu_baseline": cpu_baseline_batched(probs) if cpu else None}


def bench_adjoint(dev, n: int = 512, steps: int = 500, every: int = 50):
    """Gradient of an L2 loss of u^N with respect to u_0 for the 512^2 periodic vortex with
    8 density bumps, FP32, fixed a: forward step vs rollout (checkpoints) vs adjoint sweep
    (recomputation + adjoint kernels), per step."""
    import torch

    from paper_2411_15001_gb300 import vlbm as V
    from paper_2411_15001_gb300 import workloads as W

    p = W.vortex_with_bumps(n)
    u0 = torch.tensor(p.conserved(), dtype=torch.float32, device=dev)
    probe = V.VLBM(p.nx, p.ny, p.dx, bc=p.bc, limiter=V.LIM_PP, precision=V.FP32, device=dev)
    probe.set_conserved(u0[0].contiguous(), u0[1:3].contiguous(), u0[3].contiguous())
    lam = 1.05 * probe.monitors()["lambda"]
    probe.close()
    s = V.VLBM(p.nx, p.ny, p.dx, bc=p.bc, lam=lam, limiter=V.LIM_PP, precision=V.FP32, device=dev)
    scratch = s.adjoint_scratch(steps, every)
    # target: the unperturbed vortex advanced by the same scheme and speed
    base = torch.tensor(W.isentropic_vortex(n).conserved(), dtype=torch.float32, device=dev)
    s.set_conserved(base[0].contiguous(), base[1:3].contiguous(), base[3].contiguous())
    s.step(steps)
    r_, m_, E_ = s.moments()
    target = torch.cat([r_[None], m_, E_[None]])
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]

    def fwd():
        s.set_conserved(u0[0].contiguous(), u0[1:3].contiguous(), u0[3].contiguous())

    # untimed warm-up of every path (kernel loading, descriptors, clocks)
    fwd()
    s.step(5)
    wsteps = 2 * every
    wscratch = s.adjoint_scratch(wsteps, every)
    fwd()
    s.rollout(wsteps, every, wscratch)
    s.adjoint(torch.zeros((4, n, n), dtype=torch.float32, device=dev), wsteps, every, wscratch)
    torch.cuda.synchronize(dev)
    del wscratch
    fwd()
    ev[0].record(s.stream)
    s.step(steps)
    ev[1].record(s.stream)
    fwd()
    ev[2].record(s.stream)
    s.rollout(steps, every, scratch)
    ev[3].record(s.stream)
    rho, mom, E = s.moments()
    uN = torch.cat([rho[None], mom, E[None]])
    dL = (p.dx * p.dx * (uN - target)).contiguous()     # L = dx^2 / 2 sum |u^N - u_target|^2
    ev[4].record(s.stream)
    g = s.adjoint(dL, steps, every, scratch)
    ev[5].record(s.stream)
    torch.cuda.synchronize(dev)
    t_f = ev[0].elapsed_time(ev[1]) / steps
    t_r = ev[2].elapsed_time(ev[3]) / steps
    t_a = ev[4].elapsed_time(ev[5]) / steps
    finite = bool(torch.isfinite(g).all())
    s.close()
    return {"workload": f"{n}x{n} periodic isentropic vortex + 8 Gaussian density bumps (seed 2), FP32, "
                        f"PP, fixed a = 4 x 1.05 lambda_0 (about 14), {steps} steps, checkpoints every {every}, "
                        "L = dx^2/2 sum |u^N - u_target|^2, u_target = the unperturbed vortex after the "
                        "same steps",
            "forward_ms_per_step": t_f, "rollout_ms_per_step": t_r, "adjoint_ms_per_step": t_a,
            "adjoint_over_forward": t_a / t_f, "gradient_over_forward": (t_r + t_a) / t_f,
            "scratch_bytes": int(scratch.numel()), "gradient_finite": finite}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1900)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_SIDE, help="grid side (default 4096)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-full-run", action="store_true", help="skip the 2000-step run from t = 0")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
