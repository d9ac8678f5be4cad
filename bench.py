#!/usr/bin/env python
"""Benchmark of the implicit laplacianFoam time step on GB300.

Default workload: the 200^3 box graded 1.02x per cell in x (8,000,000 cells, 23,880,000
internal faces), T=373 K / 273 K fixedValue on x0 / x1, zeroGradient elsewhere, T0=273 K,
DT=4e-5, dt=0.005, diagonal PCG to tol 1e-6 (relTol 0), FP64, with the mixed-precision
form run side by side. One bench step = one implicit time step (assembly, initial residual
and normFactor, PCG to convergence). Inputs stay resident in HBM; the working set
(~2 GB) is far larger than the 129 MB L2, so no L2 flush is needed between steps.

Metric: PCG cell-iterations/s = sum over timed steps of n_cells * PCG iterations / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: every rank advances its own replica (the step does not shard
without a halo exchange; replicas are independent), time = max over ranks, value = all
ranks' cell-iterations / that time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lapcase  # noqa: E402

METRIC = "PCG cell-iterations/s and achieved HBM GB/s (FP64 vs mixed), p99 solve latency"
UNIT = "cell-iterations/s"
WORKLOAD = ("graded200: 200^3 unit box graded 1.02x per cell in x (8.0M cells, 23.88M internal "
            "faces), DT=4e-5, dt=0.005, x0=373 K / x1=273 K fixedValue, zeroGradient elsewhere, "
            "T0=273 K, diagonal PCG tol 1e-6 relTol 0")
# Sources of each step kernel's arithmetic and memory traffic: a stored ncu traffic ratio is
# used only while these are unchanged since the capture.
KERNEL_SOURCES = {
    "fp64": ["csrc/lfm_solve.cuh", "csrc/lfm_device.cuh"],
    "df64": ["csrc/lfm_solve_df.cuh", "csrc/lfm_df64.cuh", "csrc/lfm_solve.cuh", "csrc/lfm_device.cuh"],
    "mixed": ["csrc/lfm_solve_mixed_df.cuh", "csrc/lfm_solve_df.cuh", "csrc/lfm_df64.cuh", "csrc/lfm_solve.cuh",
              "csrc/lfm_device.cuh"],
}


def _code_tokens(text: str) -> str:
    """A source file without its comments and with whitespace collapsed: edits to comments
    or layout do not invalidate a stored capture, edits to code do."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_hash(family: str = "fp64") -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES[family]:
        with open(os.path.join(ROOT, "paper_2507_18268_gb300", p), encoding="utf-8") as f:
            h.update(_code_tokens(f.read()).encode())
    return h.hexdigest()[:16]


def algorithmic_bytes(N: int, F: int, iters: int, steps: int, precision: int) -> float:
    """Minimum DRAM bytes of `steps` steps with `iters` PCG iterations in total.

    Per PCG iteration (every array touched once per pass, int32 addressing):
      FP64  112 N + 16 F  (p update 32N; A p and p.q 24N + 16F; x, r updates and dots 56N)
      mixed  56 N + 12 F  (the same passes on 4-byte values)
    Per step: assembly 40 N + 16 F (reads V, T, the face coefficients and addressing; writes
    diag, source, 1/diag and the off-diagonals) and the initial residual 48 N + 16 F.
    """
    if precision == 0:
        per_iter = 112 * N + 16 * F
    else:
        per_iter = 56 * N + 12 * F
    per_step = (40 * N + 16 * F) + (48 * N + 16 * F)
    return float(iters) * per_iter + float(steps) * per_step


def algorithmic_flops(N: int, F: int, iters: int, steps: int) -> float:
    """Minimum FP64 floating-point operations (an FMA counts 2) of `steps` FP64 steps with
    `iters` PCG iterations: per iteration 13 N + 4 F (p update 2N; A p 1N + 4F and p.Ap 2N;
    x, r updates, w = rD r, w.r and sum|r| 8N); per step the assembly 5 N + 4 F and the
    initial residual / normFactor 11 N + 4 F."""
    return float(iters) * (13 * N + 4 * F) + float(steps) * (16 * N + 8 * F)


FP64_NOMINAL_TFLOPS = 1.25  # GB300 dense FP64, nominal
HBM_NOMINAL_GBS = 7900.0    # GB300 HBM3e, nominal (the roofline's peak is the measured copy bandwidth)


def solve_only(N: int, iters: int, steps: int, phases: dict) -> dict:
    """Cell-iterations/s of the PCG iteration passes alone (p update, A p with p.Ap, the
    updates with their dots; barrier waits included), from the kernel's phase clocks: the
    per-step assembly, initial residual and (mixed) correction passes excluded."""
    ms = phases["p_update"] + phases["amul_dot"] + phases["update_dots"]
    return {"value": float(N) * iters / steps / (ms * 1e-3) if ms > 0 else None, "unit": UNIT,
            "iteration_passes_ms_per_step": ms}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def load_traffic_ratio(name: str):
    """DRAM-traffic / algorithmic-bytes ratio from a committed ncu summary, if it was taken
    on the current kernel source."""
    p = os.path.join(ROOT, "profiles", f"traffic_{name}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    family = "mixed" if "mixed" in name else ("df64" if "df64" in name else "fp64")
    if d.get("kernel_hash") != kernel_hash(family):
        return None
    return float(d["dram_bytes"]) / float(d["algorithmic_bytes"])


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
            os.unlink(self.path)
        except OSError:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def reference_slab_case() -> lapcase.RawCase:
    """A 200 x 200 x 25 slab of the graded 200^3 box (same cell sizes, same x grading and
    boundary conditions, zeroGradient z faces): the same 1D-in-x physics per cell."""
    full = lapcase.graded_box(200)
    return full.with_(zs=lapcase.uniform_axis(200)[:26].copy(), name="graded200_slab25")


def run_cpu_oracle(case, n_steps: int, warmup: int = 0):
    import oracle
    mesh = oracle.mesh_of(case)
    T = oracle.initial_field(case)
    if warmup:
        T, _ = oracle.advance(case, n_steps=warmup, mesh=mesh, T=T)
    t0 = time.perf_counter()
    T, st = oracle.advance(case, n_steps=n_steps, mesh=mesh, T=T)
    dt = time.perf_counter() - t0
    iters = sum(s.iters for s in st)
    return mesh.n_cells * iters / dt, dt, iters


def _oracle_replica(queue, barrier, steps: int, warmup: int):
    """One serial oracle process on its own slab: warm-up, wait for the others, timed steps."""
    import oracle
    case = reference_slab_case()
    mesh = oracle.mesh_of(case)
    T = oracle.initial_field(case)
    if warmup:
        T, _ = oracle.advance(case, n_steps=warmup, mesh=mesh, T=T)
    barrier.wait()
    t0 = time.perf_counter()
    T, st = oracle.advance(case, n_steps=steps, mesh=mesh, T=T)
    secs = time.perf_counter() - t0
    iters = sum(s.iters for s in st)
    queue.put((mesh.n_cells * iters, secs, iters))


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_cpu_oracle_all_cores(n_proc: int, steps: int, warmup: int = 0):
    """The serial oracle on every host core at once, one independent slab per process (started
    with spawn). Returns (cell-iterations/s of all processes over the slowest one's time,
    that time, PCG iterations of one process)."""
    import multiprocessing as mp

    import oracle
    oracle.build()  # once, before the processes load it
    ctx = mp.get_context("spawn")
    queue, barrier = ctx.Queue(), ctx.Barrier(n_proc)
    procs = [ctx.Process(target=_oracle_replica, args=(queue, barrier, steps, warmup)) for _ in range(n_proc)]
    for pr in procs:
        pr.start()
    res = [queue.get() for _ in procs]
    for pr in procs:
        pr.join()
    secs = max(r[1] for r in res)
    return sum(r[0] for r in res) / secs, secs, res[0][2]


def main_reference(args, world, rank):
    if rank != 0:
        return
    case = reference_slab_case()
    cores = host_cores()
    value, secs, iters = run_cpu_oracle_all_cores(cores, args.steps, args.warmup)
    sample = (f"oracle (serial FP64 C, scatter face loops) in {cores} processes at once, one per host "
              f"core, each on its own 200x200x25 slab of graded200 ({case.n_cells} cells), "
              f"{args.warmup} warm-up + {args.steps} timed steps, {iters} PCG iterations each in "
              f"{secs:.2f} s (slowest process); a sample, not the 8 M-cell case: each slab's working "
              f"set (~0.1 GB) sits far closer to the host's caches than the full case's (~1 GB)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "200x200x25 slab"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_device_resident(solver, B, torch, stream, n_steps: int):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    B.lfm_advance_async(solver.ctx, n_steps)
    ev1.record(stream)
    stats = solver.finish(n_steps)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) * 1e-3, stats


def repeat_runs(solver, B, torch, stream, n_steps: int, N: int, T_start, first: float, runs: int) -> dict:
    """Spread of the timed region: `runs` regions of the same n_steps from the same starting
    field (the headline region first; each other one restarts from T_start, set outside the
    timed region), as cell-iterations/s of this rank."""
    vals = [first]
    for _ in range(max(0, runs - 1)):
        solver.set_field(T_start)
        secs, st = time_device_resident(solver, B, torch, stream, n_steps)
        vals.append(float(N) * sum(x["iters"] for x in st) / secs)
    return {"runs": len(vals), "median": statistics.median(vals),
            "std": statistics.pstdev(vals) if len(vals) > 1 else 0.0, "min": min(vals), "max": max(vals),
            "unit": UNIT, "note": "the headline region and its repeats from the same starting field"}


def run_workload(argv, timeout_s: float = 900.0):
    """Runs this script with argv in a subprocess and returns its JSON line (None on failure)."""
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__)] + argv, capture_output=True, text=True,
                           timeout=timeout_s, cwd=ROOT)
    except subprocess.TimeoutExpired:
        return None
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    if r.returncode != 0 or not lines:
        return None
    return json.loads(lines[-1])


def main_ours(args, world, rank, local):
    import torch

    from paper_2507_18268_gb300 import Solver
    from paper_2507_18268_gb300 import binding as B
    from paper_2507_18268_gb300.mesh import box_mesh, field_by_label

    torch.cuda.set_device(local)
    case = lapcase.graded_box(200)
    mesh = box_mesh(case)
    N, F = mesh.n_cells, mesh.n_faces
    stream = torch.cuda.Stream(device=local)
    hbm_peak, peak_kind = load_peaks()
    K, W = args.steps, args.warmup

    if args.only in ("mixed", "df64"):
        return main_only(args, world, rank, local, case, mesh, stream)

    # ---- FP64, device-resident --------------------------------------------------------
    s64 = Solver.from_case(case, mesh=mesh, device=local, stream=stream)
    s64.advance(W)
    T_start = s64.field().copy()
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    if rank == 0:
        clocks.start()
    secs, st = time_device_resident(s64, B, torch, stream, K)
    barrier(world)
    clk = clocks.stop() if rank == 0 else None
    iters = sum(x["iters"] for x in st)
    assert all(x["converged"] for x in st), "FP64 step did not converge"
    phases = {k: v / K for k, v in s64.phase_times().items()}
    secs_max = reduce_max(secs, world)
    cell_iters_all = reduce_sum(float(N) * iters, world)
    value = cell_iters_all / secs_max
    alg = algorithmic_bytes(N, F, iters, K, 0)
    achieved_gbs = alg / secs / 1e9
    ratio = load_traffic_ratio("graded200_fp64")
    T64 = s64.field()
    launch = s64.launch()
    spread = repeat_runs(s64, B, torch, stream, K, N, T_start, float(N) * iters / secs, args.repeats)

    # ---- df64 (double-float on the FP32 pipe), device-resident -----------------------
    df64 = None
    if not args.no_df64:
        sdf = Solver.from_case(case.with_(precision=B.LFM_DF64), mesh=mesh, device=local, stream=stream)
        sdf.advance(W)
        Td_start = sdf.field().copy()
        barrier(world)
        dsecs, dst = time_device_resident(sdf, B, torch, stream, K)
        barrier(world)
        diters = sum(x["iters"] for x in dst)
        dphases = {k: v / K for k, v in sdf.phase_times().items()}
        assert all(x["converged"] for x in dst), "df64 step did not converge"
        dsecs_max = reduce_max(dsecs, world)
        dvalue = reduce_sum(float(N) * diters, world) / dsecs_max
        dalg = algorithmic_bytes(N, F, diters, K, 0)
        Td = sdf.field()
        dspread = repeat_runs(sdf, B, torch, stream, K, N, Td_start, float(N) * diters / dsecs, args.repeats)
        dratio = load_traffic_ratio("graded200_df64")
        df64 = {"value": dvalue, "unit": UNIT, "ms_per_step": 1e3 * dsecs_max / K,
                "iters_per_step": diters / K,
                "iters_equal_fp64": [x["iters"] for x in dst] == [x["iters"] for x in st],
                "speedup_vs_fp64": secs_max / dsecs_max,
                "max_rel_diff_vs_fp64": float(np.max(np.abs(Td - T64) / np.abs(T64))),
                "dtype": "df64 (FP32 pairs, 48-bit significand; FP64 scalars)",
                "phases_ms_per_step": dphases,
                "solve_only": solve_only(N, diters, K, dphases),
                "spread": dspread,
                "roofline": {"bound": "hbm", "achieved": dalg / dsecs / 1e9, "peak": hbm_peak, "unit": "GB/s",
                             "frac": dalg / dsecs / 1e9 / hbm_peak,
                             "frac_of_nominal": dalg / dsecs / 1e9 / HBM_NOMINAL_GBS,
                             "traffic": (dratio * dalg / K) if dratio else None,
                             "peak_kind": peak_kind, "kernel": "step_kernel_df64",
                             "per": "one step (one launch runs all timed steps)"}}
        sdf.close()

    # ---- mixed precision, device-resident ------------------------------------------
    mixed = None
    if not args.no_mixed:
        smx = Solver.from_case(case.with_(precision=B.LFM_MIXED), mesh=mesh, device=local, stream=stream)
        smx.advance(W)
        Tm_start = smx.field().copy()
        barrier(world)
        msecs, mst = time_device_resident(smx, B, torch, stream, K)
        barrier(world)
        miters = sum(x["iters"] for x in mst)
        mphases = {k: v / K for k, v in smx.phase_times().items()}
        assert all(x["converged"] for x in mst), "mixed step did not converge"
        msecs_max = reduce_max(msecs, world)
        mvalue = reduce_sum(float(N) * miters, world) / msecs_max
        malg = algorithmic_bytes(N, F, miters, K, 1)
        Tm = smx.field()
        mspread = repeat_runs(smx, B, torch, stream, K, N, Tm_start, float(N) * miters / msecs, args.repeats)
        mratio = load_traffic_ratio("graded200_mixed")
        mixed = {"value": mvalue, "unit": UNIT, "ms_per_step": 1e3 * msecs_max / K,
                 "iters_per_step": miters / K, "sweeps_per_step": sum(x["sweeps"] for x in mst) / K,
                 "speedup_vs_fp64_cell_steps": (secs_max / msecs_max),
                 "max_rel_diff_vs_fp64": float(np.max(np.abs(Tm - T64) / np.abs(T64))),
                 "phases_ms_per_step": mphases,
                 "solve_only": solve_only(N, miters, K, mphases),
                 "spread": mspread,
                 "roofline": {"bound": "hbm", "achieved": malg / msecs / 1e9, "peak": hbm_peak, "unit": "GB/s",
                              "frac": malg / msecs / 1e9 / hbm_peak,
                              "frac_of_nominal": malg / msecs / 1e9 / HBM_NOMINAL_GBS,
                              "traffic": (mratio * malg / K) if mratio else None,
                              "peak_kind": peak_kind, "kernel": "step_kernel_mixed_df",
                              "per": "one step (one launch runs all timed steps)"}}
        smx.close()

    # ---- end to end through the public API with pinned host buffers ---------------
    e2e = None
    if not args.no_e2e:
        T_host = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
        T_host[:] = field_by_label(case, mesh)
        s64.set_field(T_host)
        s64.advance(W)
        T_host[:] = s64.field()
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eiters = 0
        for _ in range(K):
            B.lfm_set_field(s64.ctx, T_host)
            est = B.lfm_advance(s64.ctx, 1)
            B.lfm_get_field(s64.ctx, N, out=T_host)
            eiters += est[0].iters
        torch.cuda.synchronize()
        esecs = time.perf_counter() - t0
        barrier(world)
        esecs_max = reduce_max(esecs, world)
        e2e = {"value": reduce_sum(float(N) * eiters, world) / esecs_max, "unit": UNIT,
               "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N + 40 + 4,
               "ms_per_step": 1e3 * esecs_max / K}
    s64.close()

    # ---- CPU baseline: the oracle on a bounded sample -------------------------------
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cb_case = reference_slab_case()
        cb_steps = 20
        cores = host_cores()
        cval, csecs, citers = run_cpu_oracle_all_cores(cores, cb_steps)
        sval, ssecs, _ = run_cpu_oracle(cb_case, cb_steps)
        cpu = {"value": cval, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"serial FP64 oracle in {cores} processes at once (one per host core), each "
                         f"20 steps of its own 200x200x25 slab of graded200 ({cb_case.n_cells} cells, "
                         f"{citers} PCG iterations, {csecs:.1f} s for the slowest); a sample, not the "
                         f"8 M-cell case: each slab's working set (~0.1 GB) sits far closer to the host's "
                         f"caches than the full case's (~1 GB)",
               "single_core_value": sval}

    # ---- the FP64 issue rate this step is bound by, measured on this GPU -------------
    fclk = ClockSampler(local)
    if rank == 0:
        fclk.start()
    fma_rate = B.lfm_measure_fp64_fma_rate(local)
    fclk = fclk.stop() if rank == 0 else None
    fp64_peak_tflops = 2.0 * fma_rate / 1e12

    # ---- the batched and served forms beside the headline ---------------------------
    # each in a fresh process, exactly as `--workload batch512` / `--workload serve` run alone
    # (a served run's latency is host-bound and suffers from what earlier legs leave in the
    # process); under torchrun each workload is its own launch instead
    subs = {}
    if not args.no_sub and world == 1:
        subs["batch512"] = run_workload(["--workload", "batch512", "--warmup", str(args.warmup)])
        subs["serve1000"] = run_workload(["--workload", "serve", "--requests", "1000"])
        subs["serve100"] = run_workload(["--workload", "serve", "--requests", "100"])
        subs["large600"] = run_workload(["--workload", "large", "--warmup", str(args.warmup)])

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": 1e3 * secs_max / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": N, "internal_faces": F, "precision": "fp64",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (~2 GB working set vs 129 MB L2); no flush",
                   "launch": {"ctas": launch[0], "threads": launch[1]}},
        "iters_per_step": iters / K,
        "cell_steps_per_s": float(N) * K * world / secs_max,
        "phases_ms_per_step": phases,
        "per_step_passes_ms": phases["assembly_faces"] + phases["rows_initial_residual"],
        "iteration_passes_ms_per_step": phases["p_update"] + phases["amul_dot"] + phases["update_dots"],
        "solve_only": solve_only(N, iters, K, phases),
        "spread": spread,
        "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved_gbs / hbm_peak, "traffic": (ratio * alg / K) if ratio else None,
                     "frac_of_nominal": achieved_gbs / HBM_NOMINAL_GBS,
                     "peak_kind": peak_kind, "kernel": "step_kernel_f64",
                     "per": "one step (one launch runs all timed steps)"},
        "roofline_fp64_pipe": {"bound": "alu", "achieved": algorithmic_flops(N, F, iters, K) / secs / 1e12,
                               "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                               "frac": algorithmic_flops(N, F, iters, K) / secs / 1e12 / fp64_peak_tflops,
                               "peak_kind": "measured: lfm_measure_fp64_fma_rate (independent FMA chains on "
                                            "every SM, 2 flops per FMA)",
                               "fma_per_s": fma_rate, "clocks": fclk,
                               "frac_of_nominal": algorithmic_flops(N, F, iters, K) / secs / 1e12
                               / FP64_NOMINAL_TFLOPS,
                               "note": "ncu: FP64 pipe 75% busy, DRAM 64% (profiles/step_kernel_f64_graded200.md)"},
        "gpu_launches": 1,
        "clocks": clk,
        "df64": df64,
        "mixed": mixed,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    for k, v in subs.items():  # compact: the headline figures of each, with their clocks
        if v is None:
            continue
        if k == "batch512":
            line[k] = {"config": v["config"]["workload"], "clocks": v["clocks"],
                       "batched_fp64": v["batched_fp64"]["value"], "batched_df64": v["batched_df64"]["value"],
                       "batched_mixed": v["batched_mixed"]["value"],
                       "plain_fp64_sequential": v["plain_fp64_sequential"]["value"], "unit": UNIT,
                       "max_rel_diff_batched_vs_alone":
                           v["plain_fp64_sequential"]["max_rel_diff_batched_vs_alone"],
                       "mixed_max_rel_diff_vs_fp64_batch": v["batched_mixed"]["max_rel_diff_vs_fp64_batch"]}
        elif k == "large600":
            line[k] = {"config": v["config"]["workload"], "clocks": v["clocks"], "unit": UNIT,
                       **{f: {kk: v[f][kk] for kk in ("value", "ms_per_step", "iters_per_step", "device_GB",
                                                      "roofline")} for f in ("fp64", "mixed")}}
        else:
            line[k] = {"config": v["config"]["workload"], "clocks": v["clocks"], "served": v["served"],
                       "serial_plain_fp64": v["serial_plain_fp64"],
                       "p99_latency_ratio_serial_over_served": v["p99_latency_ratio_serial_over_served"]}
    print(json.dumps(line), flush=True)


SKEWED = ("skewed200: graded200 sheared by x' = x + 0.25 y + 0.15 z (8.0M parallelepiped cells, 23.88M "
          "internal faces, up to 16 degrees non-orthogonal), corrected laplacian with 1 non-orthogonal "
          "corrector per step (2 assemble-and-solve passes), DT, dt, BCs and PCG controls as graded200")


def algorithmic_bytes_corrected(N: int, F: int, iters: int, passes: int) -> float:
    """Minimum DRAM bytes of the corrected FP64 step: per PCG iteration as the orthogonal
    step (112 N + 16 F); per assemble-and-solve pass the orthogonal assembly and initial
    residual (88 N + 32 F) plus the Gauss gradient (T, Sf, w in; G out: 32 N + 32 F) and the
    correction flux (G, k, w, |Sf| in; flux out, read back by the rows: 24 N + 56 F)."""
    return float(iters) * (112 * N + 16 * F) + float(passes) * ((88 + 32 + 24) * N + (32 + 32 + 56) * F)


def main_decomp(args, world, rank, local):
    """One graded200 case decomposed into label-range parts (the paper's multi-GPU data flow
    emulated on one GPU: halo exchange of T per step and of p per PCG iteration, global sums
    over all parts) against the undecomposed FP64 step, from the same starting field."""
    import torch

    from paper_2507_18268_gb300 import Solver
    from paper_2507_18268_gb300 import binding as B
    from paper_2507_18268_gb300.decomp import Decomposed

    torch.cuda.set_device(local)
    K = args.steps if args.steps_given else 20
    W = args.warmup
    case = lapcase.graded_box(args.decomp_n, n_steps=K)
    stream = torch.cuda.Stream(device=local)
    s = Solver.from_case(case, device=local, stream=stream)
    N = s.mesh.n_cells
    T0 = s.field().copy()
    s.advance(W)
    s.set_field(T0)
    clocks = ClockSampler(local)
    barrier(world)
    if rank == 0:
        clocks.start()
    secs, st = time_device_resident(s, B, torch, stream, K)
    iters = sum(x["iters"] for x in st)
    Tref = s.field().copy()
    single = {"value": float(N) * iters / secs, "unit": UNIT, "ms_per_step": 1e3 * secs / K, "iters": iters}
    parts = {}
    for n_parts in args.decomp_parts:
        s.set_field(T0)
        with Decomposed(s, n_parts) as dd:
            dd.set_field(T0)
            dd.advance(W)
            dd.set_field(T0)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            sd = dd.advance(K)  # enqueued on the case's stream, waited for inside
            ev1.record(stream)
            torch.cuda.synchronize()
            dsecs = ev0.elapsed_time(ev1) * 1e-3
            diters = sum(x["iters"] for x in sd)
            Td = dd.field()
            halo = sum(c.n_ghost for c in dd.counts())
        parts[str(n_parts)] = {"value": float(N) * diters / dsecs, "unit": UNIT, "ms_per_step": 1e3 * dsecs / K,
                               "iters_equal_single": diters == iters, "ghost_cells": halo,
                               "time_vs_single": dsecs / secs,
                               "max_rel_diff_vs_single": float(np.max(np.abs(Td - Tref) / np.abs(Tref)))}
    clk = clocks.stop() if rank == 0 else None
    s.close()
    if rank != 0:
        return
    last = parts[str(args.decomp_parts[-1])]
    line = {"metric": METRIC, "value": last["value"], "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": last["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"decomp{args.decomp_n}: graded{args.decomp_n} ({N} cells) in label-range "
                                   f"parts, emulated on one GPU; value = {args.decomp_parts[-1]} parts",
                       "parallelism": "single GPU (the parts' data flow, not several GPUs)"},
            "clocks": clk, "single_fp64": single, "parts": parts}
    print(json.dumps(line))


def main_large(args, world, rank, local):
    """Capacity: an n^3 box with graded200's total grading (ratio 1.02^(200/n) per cell),
    built on the device, FP64 and mixed, with the device memory each case holds."""
    import torch

    from paper_2507_18268_gb300 import Solver
    from paper_2507_18268_gb300 import binding as B

    torch.cuda.set_device(local)
    K = args.steps if args.steps_given else 20
    W = args.warmup
    n = args.large_n
    stream = torch.cuda.Stream(device=local)
    forms = {}
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    for prec, name in ((B.LFM_FP64, "fp64"), (B.LFM_MIXED, "mixed")):
        case = lapcase.graded_box(n, ratio=1.02 ** (200.0 / n), n_steps=K, precision=prec)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info(local)
        s = Solver.from_box_case(case, device=local, stream=stream, layout=prec)
        free1, _ = torch.cuda.mem_get_info(local)
        s.advance(W)
        barrier(world)
        secs, st = time_device_resident(s, B, torch, stream, K)
        iters = sum(x["iters"] for x in st)
        N = n ** 3
        secs_max = reduce_max(secs, world)
        F = 3 * n * n * (n - 1)
        alg = algorithmic_bytes(N, F, iters, K, 0 if prec == B.LFM_FP64 else 1)
        hbm_peak, peak_kind = load_peaks()
        forms[name] = {"value": reduce_sum(float(N) * iters, world) / secs_max, "unit": UNIT,
                       "ms_per_step": 1e3 * secs_max / K, "iters_per_step": iters / K,
                       "converged": all(x["converged"] for x in st), "device_GB": (free0 - free1) / 1e9,
                       "bytes_per_cell": (free0 - free1) / N,
                       "roofline": {"bound": "hbm", "achieved": alg / secs_max / 1e9, "peak": hbm_peak, "unit": "GB/s",
                                    "frac": alg / secs_max / 1e9 / hbm_peak, "peak_kind": peak_kind,
                                    "traffic": None}}
        s.close()
        del s
        torch.cuda.synchronize()
    clk = clocks.stop() if rank == 0 else None
    if rank != 0:
        return
    line = {"metric": METRIC, "value": forms["fp64"]["value"], "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": forms["fp64"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"large{n}: {n}^3 box ({n ** 3} cells) graded {1.02 ** (200.0 / n):.6f}x per cell "
                                   f"in x (graded200's total grading), graded200's BCs and controls, built on the "
                                   f"device; value = FP64", "parallelism": "single GPU"},
            "clocks": clk, "fp64": forms["fp64"], "mixed": forms["mixed"]}
    print(json.dumps(line))


def main_skewed(args, world, rank, local):
    """The non-orthogonal workload: device-resident FP64 and mixed, the oracle on a slab."""
    import torch

    from paper_2507_18268_gb300 import Solver
    from paper_2507_18268_gb300 import binding as B
    from paper_2507_18268_gb300.mesh import hex_mesh

    torch.cuda.set_device(local)
    K = args.steps if args.steps_given else 20
    W = args.warmup
    case = lapcase.skewed_box(args.skewed_n)
    mesh, geo = hex_mesh(case)
    N, F = mesh.n_cells, mesh.n_faces
    stream = torch.cuda.Stream(device=local)
    hbm_peak, peak_kind = load_peaks()
    s64 = Solver.from_case(case, mesh=mesh, geometry=geo, device=local, stream=stream)
    s64.advance(W)
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    if rank == 0:
        clocks.start()
    secs, st = time_device_resident(s64, B, torch, stream, K)
    barrier(world)
    clk = clocks.stop() if rank == 0 else None
    assert all(x["converged"] for x in st), "corrected FP64 step did not converge"
    iters = sum(x["iters"] for x in st)
    passes = K * (1 + case.n_nonorth_corr)
    phases = {k: v / K for k, v in s64.phase_times().items()}
    secs_max = reduce_max(secs, world)
    value = reduce_sum(float(N) * iters, world) / secs_max
    alg = algorithmic_bytes_corrected(N, F, iters, passes)
    sratio = load_traffic_ratio("skewed_fp64")
    T64 = s64.field()
    launch = s64.launch()
    s64.close()
    mixed = None
    if not args.no_mixed:
        smx = Solver.from_case(case.with_(precision=B.LFM_MIXED), mesh=mesh, geometry=geo, device=local,
                               stream=stream)
        smx.advance(W)
        msecs, mst = time_device_resident(smx, B, torch, stream, K)
        miters = sum(x["iters"] for x in mst)
        Tm = smx.field()
        smx.close()
        msecs_max = reduce_max(msecs, world)
        mixed = {"value": reduce_sum(float(N) * miters, world) / msecs_max, "unit": UNIT,
                 "ms_per_step": 1e3 * msecs_max / K, "iters_per_step": miters / K,
                 "converged": all(x["converged"] for x in mst),
                 "max_rel_diff_vs_fp64": float(np.max(np.abs(Tm - T64) / np.abs(T64)))}
    df64 = None
    if not args.no_df64:
        sdf = Solver.from_case(case.with_(precision=B.LFM_DF64), mesh=mesh, geometry=geo, device=local,
                               stream=stream)
        sdf.advance(W)
        dsecs, dst = time_device_resident(sdf, B, torch, stream, K)
        diters = sum(x["iters"] for x in dst)
        dpasses = K * (1 + case.n_nonorth_corr)
        Td = sdf.field()
        dphases = {k: v / K for k, v in sdf.phase_times().items()}
        sdf.close()
        dsecs_max = reduce_max(dsecs, world)
        dalg = algorithmic_bytes_corrected(N, F, diters, dpasses)
        df64 = {"value": reduce_sum(float(N) * diters, world) / dsecs_max, "unit": UNIT,
                "ms_per_step": 1e3 * dsecs_max / K, "iters_per_step": diters / K,
                "converged": all(x["converged"] for x in dst),
                "max_rel_diff_vs_fp64": float(np.max(np.abs(Td - T64) / np.abs(T64))),
                "phases_ms_per_step": dphases,
                "solve_only": solve_only(N, diters, K, dphases),
                "roofline": {"bound": "hbm", "achieved": dalg / dsecs / 1e9, "peak": hbm_peak, "unit": "GB/s",
                             "frac": dalg / dsecs / 1e9 / hbm_peak,
                             "frac_of_nominal": dalg / dsecs / 1e9 / HBM_NOMINAL_GBS,
                             "traffic": None, "peak_kind": peak_kind, "kernel": "step_kernel_df64"}}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        slab = case.with_(zs=lapcase.uniform_axis(200)[:26].copy(),
                          points=np.ascontiguousarray(case.points[:26]), name="skewed200_slab25")
        cval, csecs, citers = run_cpu_oracle(slab, 10)
        cpu = {"value": cval, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"serial FP64 oracle, 10 steps (20 corrected passes) of a 200x200x25 slab of skewed200 "
                         f"({slab.n_cells} cells, {citers} PCG iterations, {csecs:.1f} s)"}
    if rank != 0:
        return
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": 1e3 * secs_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": SKEWED if args.skewed_n == 200 else SKEWED.replace("skewed200", f"skewed{args.skewed_n}"),
                   "cells": N, "internal_faces": F, "precision": "fp64",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2; no flush", "launch": {"ctas": launch[0], "threads": launch[1]}},
        "iters_per_step": iters / K, "passes_per_step": 1 + case.n_nonorth_corr,
        "phases_ms_per_step": phases,
        "roofline": {"bound": "hbm", "achieved": alg / secs / 1e9, "peak": hbm_peak, "unit": "GB/s",
                     "frac": alg / secs / 1e9 / hbm_peak, "traffic": (sratio * alg / K) if sratio else None,
                     "peak_kind": peak_kind,
                     "kernel": "step_kernel_f64", "per": "one step (one launch runs all timed steps)"},
        "gpu_launches": 1, "clocks": clk, "df64": df64, "mixed": mixed, "cpu_baseline": cpu,
        "e2e": None,
    }), flush=True)


def main_only(args, world, rank, local, case, mesh, stream):
    """Profiling mode: the mixed or the df64 form alone (one warm-up launch, one timed launch)."""
    import torch

    from paper_2507_18268_gb300 import Solver
    from paper_2507_18268_gb300 import binding as B

    K, W = args.steps, args.warmup
    prec = B.LFM_MIXED if args.only == "mixed" else B.LFM_DF64
    smx = Solver.from_case(case.with_(precision=prec), mesh=mesh, device=local, stream=stream)
    smx.advance(W)
    secs, st = time_device_resident(smx, B, torch, stream, K)
    iters = sum(x["iters"] for x in st)
    phases = {k: v / K for k, v in smx.phase_times().items()}
    smx.close()
    if rank == 0:
        print(json.dumps({"metric": METRIC, "value": mesh.n_cells * iters / secs, "unit": UNIT,
                          "mode": f"{args.only} only (profiling)", "steps": K, "warmup": W,
                          "ms_per_step": 1e3 * secs / K, "iters_per_step": iters / K,
                          "phases_ms_per_step": phases}), flush=True)


def _cases_with_meshes(cases):
    """Box meshes depend only on the edge length here (uniform DT): build each once."""
    from paper_2507_18268_gb300.mesh import box_mesh
    cache = {}
    out = []
    for c in cases:
        key = (c.nx, c.ny, c.nz)
        if key not in cache:
            cache[key] = box_mesh(c)
        out.append((c, cache[key]))
    return out


def batch_record(args, world, rank, local):
    """batch512: 512 independent cases (edge log-uniform 16..96), 10 steps each, in one
    persistent launch per step (graph replay), FP64, df64 and mixed, against the plain FP64
    single-case path run case after case. With N ranks the 512 cases are split over the
    GPUs by the longest-processing-time plan of shard.py (no collective on the data path;
    strong scaling: the batch is the same at every N); times are the maximum over ranks and
    the work the sum."""
    import torch

    from paper_2507_18268_gb300 import binding as B
    from paper_2507_18268_gb300 import shard
    from paper_2507_18268_gb300.batch import Batch

    torch.cuda.set_device(local)
    n_cases = args.batch_cases
    steps = args.steps if args.steps_given else 10
    all_cases = lapcase.batch_cases(n_cases=n_cases, seed=3, n_steps=steps)
    mine = shard.shard_of([shard.case_cost(c) for c in all_cases], world, rank)
    base_cases = [all_cases[i] for i in mine]
    total_cells = sum(c.n_cells for c in all_cases)
    stream = torch.cuda.Stream(device=local)
    results = {}
    fields = {}
    clocks, clk = ClockSampler(local), None
    for prec, name in ((B.LFM_FP64, "fp64"), (B.LFM_DF64, "df64"), (B.LFM_MIXED, "mixed")):
        cases = [c.with_(precision=prec) for c in base_cases]
        bt = Batch(device=local, stream=stream)
        ids = [bt.add_case(c, mesh=m) for c, m in _cases_with_meshes(cases)]
        tune = bt.autotune()
        T0 = {cid: bt.field(cid).copy() for cid in ids}
        # warm-up: W batch steps, then restore the initial fields
        bt.advance(args.warmup)
        for cid in ids:
            bt.cases[cid].set_field(T0[cid])
        torch.cuda.synchronize()
        mark = args.profile_range == name
        if prec == B.LFM_FP64 and rank == 0:  # clocks during the headline (FP64) timed region
            clocks.start()
        if mark:  # this form's timed region is the profiler range (ncu --profile-from-start off)
            torch.cuda.profiler.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        bt.advance_async(steps, use_graph=True)
        ev1.record(stream)
        rc = bt.finish()
        torch.cuda.synchronize()
        if mark:
            torch.cuda.profiler.stop()
        if prec == B.LFM_FP64 and rank == 0:
            clk = clocks.stop()
        assert rc == B.LFM_OK, B.lfm_batch_last_error(bt.handle)
        secs = reduce_max(ev0.elapsed_time(ev1) * 1e-3, world)
        cell_iters = 0
        conv = True
        for cid in ids:
            st = bt.stats(cid, steps)
            cell_iters += bt.cases[cid].mesh.n_cells * sum(x["iters"] for x in st)
            conv = conv and all(x["converged"] for x in st)
        cell_iters = reduce_sum(cell_iters, world)
        conv = reduce_sum(0.0 if conv else 1.0, world) == 0.0
        fields[name] = {cid: bt.field(cid) for cid in ids}
        results[name] = {"value": cell_iters / secs, "ms_total": 1e3 * secs, "converged": conv,
                         "cell_steps_per_s": total_cells * steps / secs,
                         "launch": {"threads": tune["threads"], "cells_per_thread": tune["cells_per_thread"],
                                    "ctas": B.lfm_batch_get_launch(bt.handle)[0]}}
        if prec == B.LFM_FP64:
            # plain FP64: the same cases, one after another, each with the single-case path
            for cid in ids:
                bt.cases[cid].set_field(T0[cid])
            solvers = [bt.remove(cid, close=False) for cid in ids]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plain_iters = 0
            for s in solvers:
                st = s.advance(steps)
                plain_iters += s.mesh.n_cells * sum(x["iters"] for x in st)
            torch.cuda.synchronize()
            psecs = reduce_max(time.perf_counter() - t0, world)
            plain_iters = reduce_sum(plain_iters, world)
            diff = reduce_max(max(float(np.max(np.abs(s.field() - fields["fp64"][cid]) / np.abs(fields["fp64"][cid])))
                                  for cid, s in zip(ids, solvers)), world)
            results["plain_fp64_sequential"] = {"value": plain_iters / psecs, "ms_total": 1e3 * psecs,
                                                "max_rel_diff_batched_vs_alone": diff}
            for s in solvers:
                s.close()
        else:
            ref = fields["fp64"]
            results[name]["max_rel_diff_vs_fp64_batch"] = reduce_max(max(
                float(np.max(np.abs(fields[name][cid] - ref[cid]) / np.abs(ref[cid]))) for cid in ids), world)
        bt.close()
    if rank != 0:
        return None
    line = {"metric": METRIC, "value": results["fp64"]["value"], "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": results["fp64"]["ms_total"] / steps, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"batch{n_cases}: {n_cases} cases, edge log-uniform 16..96 (seed 3), "
                                   f"{total_cells} cells in total, {steps} steps each, graph-replayed step",
                       "parallelism": "single GPU" if world == 1 else
                       f"{world} GPUs, cases split by the longest-processing-time plan (no collective)"},
            "clocks": clk,
            "batched_fp64": results["fp64"], "batched_df64": results["df64"], "batched_mixed": results["mixed"],
            "plain_fp64_sequential": results["plain_fp64_sequential"],
            "speedup_batched_fp64_vs_plain": results["fp64"]["value"] / results["plain_fp64_sequential"]["value"],
            "speedup_batched_df64_vs_plain": results["df64"]["value"] / results["plain_fp64_sequential"]["value"],
            "speedup_batched_mixed_vs_plain": results["mixed"]["value"] / results["plain_fp64_sequential"]["value"]}
    return line


def main_batch(args, world, rank, local):
    line = batch_record(args, world, rank, local)
    if line is not None:
        print(json.dumps(line), flush=True)


def serve_record(args, world, rank, local, n_requests: int):
    """serve: Poisson arrivals (200/s, seed 4) of requests with edge log-uniform 32..160,
    1..50 steps, FP64 or mixed with probability 1/2, under a 120 GB HBM budget; continuous
    batching (up to 8 steps per tick, each request capped at its own count) against the same
    requests solved alone one after another in FP64. With N ranks the stream is dispatched
    over the GPUs by shard.dispatch_stream (no collective on the data path); latencies are
    gathered over ranks."""
    import torch

    from paper_2507_18268_gb300 import shard
    from paper_2507_18268_gb300.serve import Server, serve_serial_fp64

    torch.cuda.set_device(local)
    reqs_all = lapcase.serving_stream(n_requests=n_requests, seed=4)
    if world > 1:
        # each GPU serves ~2e10 cost units per second (cells x (iterations + 2) x steps)
        dev = shard.dispatch_stream(reqs_all, world, rate=2e10)
        reqs = [r for r, d in zip(reqs_all, dev) if d == rank]
    else:
        reqs = reqs_all
    warm = lapcase.serving_stream(n_requests=8, seed=99, n_min=16, n_max=24, max_steps=2)
    srv = Server(device=local, budget_bytes=120e9)
    srv.run(warm)
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    rep = srv.run(reqs)
    clk = clocks.stop() if rank == 0 else None
    srv.close()
    serial = serve_serial_fp64(reqs, device=local)
    lat = [d.latency_s for d in rep["done"]]
    lat_serial = serial["latencies_s"]
    if world > 1:
        import torch.distributed as dist
        got, got_s = [None] * world, [None] * world
        dist.all_gather_object(got, lat)
        dist.all_gather_object(got_s, lat_serial)
        lat = [x for g in got for x in g]
        lat_serial = [x for g in got_s for x in g]
    makespan = reduce_max(rep["makespan_s"], world)
    smakespan = reduce_max(serial["makespan_s"], world)
    cell_iters = reduce_sum(rep["cell_iterations_per_s"] * rep["makespan_s"], world)
    if rank != 0:
        return None
    pct = lambda xs, q: float(np.percentile(np.asarray(xs), q))  # noqa: E731
    served = {"requests": len(lat), "makespan_s": makespan, "throughput_req_s": len(lat) / makespan,
              "cell_iterations_per_s": cell_iters / makespan, "p50_latency_s": pct(lat, 50),
              "p99_latency_s": pct(lat, 99), "mean_latency_s": float(np.mean(lat)), "ticks": rep["ticks"],
              "steps_per_tick": 8, "peak_hbm_bytes": rep["peak_hbm_bytes"], "failed": rep["failed"]}
    ser = {"requests": len(lat_serial), "makespan_s": smakespan, "throughput_req_s": len(lat_serial) / smakespan,
           "p50_latency_s": pct(lat_serial, 50), "p99_latency_s": pct(lat_serial, 99),
           "mean_latency_s": float(np.mean(lat_serial))}
    return {"metric": METRIC, "value": served["cell_iterations_per_s"], "unit": UNIT, "n_gpus": world,
            "steps": n_requests, "warmup": 1, "ms_per_step": 1e3 * makespan / max(n_requests, 1),
            "higher_is_better": True, "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
            "dtype": "f64+mixed", "data": "synthetic",
            "config": {"workload": f"serve: {n_requests} requests, Poisson 200/s (seed 4), edge log-uniform "
                                   "32..160, 1..50 steps, FP64/mixed 50/50, 120 GB HBM budget, up to 8 steps "
                                   "per tick"},
            "clocks": clk, "served": served, "serial_plain_fp64": ser,
            "p99_latency_ratio_serial_over_served": ser["p99_latency_s"] / served["p99_latency_s"],
            "throughput_ratio_served_over_serial": served["throughput_req_s"] / ser["throughput_req_s"]}


def main_serve(args, world, rank, local):
    line = serve_record(args, world, rank, local, args.requests)
    if line is not None:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--repeats", type=int, default=5,
                    help="graded200: timed regions per form for the median / spread (the first is the headline)")
    ap.add_argument("--no-df64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub", action="store_true",
                    help="graded200: leave out the batch512 / serve1000 / serve100 / large600 records")
    ap.add_argument("--workload", choices=["graded200", "batch512", "serve", "skewed200", "decomp", "large"],
                    default="graded200")
    ap.add_argument("--large-n", type=int, default=600, help="large: edge of the box")
    ap.add_argument("--decomp-n", type=int, default=200, help="decomp: edge of the graded box")
    ap.add_argument("--decomp-parts", type=int, nargs="+", default=[1, 2, 4, 8], help="decomp: part counts")
    ap.add_argument("--batch-cases", type=int, default=512)
    ap.add_argument("--profile-range", nargs="?", const="fp64", default=None, choices=["fp64", "df64", "mixed"],
                    help="batch512: make this form's timed region (default FP64) the CUDA profiler range "
                         "(ncu --profile-from-start off)")
    ap.add_argument("--skewed-n", type=int, default=200, help="edge of the skewed box (profiling: smaller)")
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--only", choices=["fp64", "mixed", "df64"], default=None,
                    help="profiling: run only this precision, device-resident, no e2e or CPU baseline")
    args = ap.parse_args()
    args.steps_given = any(a.startswith("--steps") for a in sys.argv[1:])
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.only:  # profiling: one timed launch per form
        args.no_e2e = args.no_cpu_baseline = args.no_sub = True
        args.no_mixed = args.no_df64 = args.only == "fp64"
        args.repeats = 1
    world, rank, local = dist_setup()
    try:
        if args.impl == "reference":
            main_reference(args, world, rank)
        elif args.workload == "batch512":
            main_batch(args, world, rank, local)
        elif args.workload == "serve":
            main_serve(args, world, rank, local)
        elif args.workload == "skewed200":
            main_skewed(args, world, rank, local)
        elif args.workload == "decomp":
            main_decomp(args, world, rank, local)
        elif args.workload == "large":
            main_large(args, world, rank, local)
        else:
            main_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
