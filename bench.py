#!/usr/bin/env python
"""Benchmark of the HB residual path on GB300.

Workload: the multi-block 2D laminar Navier-Stokes pitching-airfoil case --
an O-grid of 1280 x 192 cells (245,760) split into 8 uneven blocks with
T-junctions, N_H = 3 (7 snapshots), pitch +-3 deg at reduced frequency 0.1,
Re = 5e3, Mach 0.3 -- on seeded synthetic grids and states.

One step = one pass of the whole hot path: one 4-stage Runge-Kutta iteration
(halo/BC fill, fused residual + local time step + RK update, FP64 residual
norms) plus the FP64 force reduction (cl, cd, cm per snapshot, time-averaged
lift), through the C ABI of libhb.so.  Metric: HB cell-snapshot residual
updates per second = cells * snapshots * 4 stages / step time.

The state plus workspace (~110 MB in FP32) fits in the 129 MB L2, so an L2
flush (a 512 MB write) runs between timed steps, outside the timed events.

Other lines: ``--impl reference`` times the FP64 CPU oracle (the reference
arm).  Under torchrun every rank runs an independent replica (the path has no
cross-rank exchange on one GPU per case: "replicas only"), timing is the max
over ranks and the value is the sum of the units all ranks processed.
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

WORKLOAD = dict(workload="ns_ogrid8: 2D laminar NS pitching O-grid, 8 uneven blocks with "
                "T-junctions, 1280x192 = 245,760 cells, N_H=3 (7 snapshots), Re=5e3, M=0.3",
                cells=245760, blocks=8, n_harm=3, snapshots=7)
METRIC = "HB cell-snapshot residual updates/s"
UNIT = "cell-snapshot-stage updates/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 9:
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ------------------------------------------------------------ reference arm --
def _cpu_model():
    """Host CPU model (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def _oracle_threads():
    """The OpenMP build of the oracle and the host cores it may use."""
    from oracle.hb_oracle import build, build_openmp
    build()
    build_openmp()
    return _cpu_cores()


def run_reference(args):
    """FP64 CPU oracle as it stands, with its residual sweeps over (block,
    snapshot) rows on all host cores (OpenMP build, the same result bit for
    bit as one thread): each step is one RK iteration of the benchmark
    workload, the full 8-block 1280 x 192 NS O-grid when the whole run fits in
    about two minutes, else a smaller member of the same family, timed on the
    host clock."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle.hb_oracle import Oracle
    from paper_1304_7654_gb300 import cases as C
    cores = _oracle_threads()
    ni, nj = 1280, 192
    cs = C.ns_ogrid8(ni, nj)
    o = Oracle(cs, openmp=True)
    U = o.init_state(C.noise(cs), 0.01)
    t = time.perf_counter()
    U, _ = o.rk_smooth_threads(U, 1, cores)            # first warm-up step, timed to size the sample
    t1 = time.perf_counter() - t
    while ni > 80 and (args.steps + args.warmup) * t1 > 120:
        ni //= 2
        nj = max(24, nj // 2)
        t1 /= 4
    if ni != 1280:
        cs = C.ns_ogrid8(ni, nj)
        o = Oracle(cs, openmp=True)
        U = o.init_state(C.noise(cs), 0.01)
    for _ in range(args.warmup - (1 if ni == 1280 else 0)):
        U, _ = o.rk_smooth_threads(U, 1, cores)
    t = time.perf_counter()
    for _ in range(args.steps):
        U, _ = o.rk_smooth_threads(U, 1, cores)
    dt = time.perf_counter() - t
    units = cs.n_cells * cs.n_snap * 4 * args.steps
    val = units / dt
    sample = (f"one RK iteration per step of the ns_ogrid8 family at {ni}x{nj} cells ({cs.n_cells:,} cells, "
              f"N_H=3), FP64 oracle, residual sweeps on {cores} threads ({_cpu_model()})")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD, sample=sample, same_config=(ni == 1280)),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline():
    """The oracle on a bounded sample of the benchmark workload itself: one RK
    iteration (4 stages) of the full 8-block 1280 x 192 NS O-grid on all host
    cores (OpenMP build over (block, snapshot) rows; about 1-2 s on 16 cores)
    and on one thread (about 10 s)."""
    from oracle.hb_oracle import Oracle
    from paper_1304_7654_gb300 import cases as C
    cores = _oracle_threads()
    cs = C.ns_ogrid8()
    o = Oracle(cs, openmp=True)
    U = o.init_state(C.noise(cs), 0.01)
    units = cs.n_cells * cs.n_snap * 4
    t = time.perf_counter()
    o.rk_smooth_threads(U, 1, cores)
    dt_n = time.perf_counter() - t
    t = time.perf_counter()
    o.rk_smooth_threads(U, 1, 1)
    dt_1 = time.perf_counter() - t
    model = _cpu_model()
    return {"value": units / dt_n, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"1 RK iteration of the full ns_ogrid8 workload (1280x192, {cs.n_cells:,} cells, N_H=3), "
                      f"FP64, residual sweeps over (block, snapshot) rows on {cores} threads, {dt_n:.2f} s",
            "host_cores": cores, "cpu_model": model,
            "single_thread": {"value": units / dt_1, "unit": UNIT, "cores": 1, "seconds": dt_1}}


# --------------------------------------------------------------- our arm --
def max_over_ranks(values, dev):
    """Element-wise maximum of a list of floats over the ranks of the default
    process group (the values themselves on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def replica_throughput(world_size, units_per_rank_step, ms_per_step):
    """Whole-job throughput of independent replicas: every rank's units over
    the slowest rank's step time."""
    return world_size * units_per_rank_step / (ms_per_step * 1e-3)


def algorithmic_bytes_per_unit(nv, s, dim, ns):
    """Algorithmic bytes of one cell-snapshot-stage, averaged over the 4
    stages of a fused RK iteration: stage 1 reads U and writes U1 (2 nv s);
    stages 2-4 read U^(s-1) and U^(0) and write (3 nv s); the grid enters as
    its nodes (dim values per cell), read once per stage for all N_s
    snapshots.  FP32 2D, N_s = 7: 44 + 8/7 = 45.1 B."""
    state = (2 + 3 + 3 + 3) / 4.0 * nv * s
    return state + dim * s / ns


def _checked_status(ctx, what):
    """A run whose state went non-finite (or whose barrier timed out) is not
    a measurement: fail loudly instead of printing its time."""
    from paper_1304_7654_gb300 import hb
    st = ctx.sync_status()
    if st != hb.HB_OK:
        raise RuntimeError(f"{what} run ended with status {st}: not a valid measurement")
    return st


def _tuning_desc(mode, TI, TJ):
    return {"driver": "persistent" if mode & 1 else "per-phase launches", "tile": [TI, TJ],
            "ghost_fill": "halo passes" if mode & 2 else "fused into the stage"}


def roofline(peaks, src, bpu_stage, cells_snaps, mode, launch_ms, kernel, traffic):
    """Dominant kernel: the tile kernel (one RK stage per launch) or the
    persistent driver (one RK iteration = 4 stages per launch)."""
    stages = 4 if mode & 1 else 1
    units = cells_snaps * stages
    achieved = bpu_stage * units / (launch_ms * 1e-3) / 1e9 if launch_ms > 0 else 0.0
    return {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "frac_of_nominal_8TBs": achieved / 8000.0,
            "traffic": traffic, "kernel": kernel,
            "peak_source": src, "bytes_per_unit": bpu_stage, "unit_def": "cell-snapshot-stage",
            "units_per_launch": units, "launch_ms": launch_ms}


def run_ours(args):
    import numpy as np
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0:
        from paper_1304_7654_gb300 import build as hbuild
        hbuild.build()
    if ws > 1:
        dist.barrier()
    from paper_1304_7654_gb300 import cases as C
    from paper_1304_7654_gb300 import hb

    cs = C.ns_ogrid8()
    units_per_step = cs.n_cells * cs.n_snap * 4
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def run_prec(prec, steps, warmup, timing=True, tune=True):
        ctx = hb.HBContext(cs, prec)
        U = ctx.new_state(dev)
        noise = torch.as_tensor(C.noise(cs), device=dev)
        ctx.init_state(U, noise, 0.01)
        if tune and args.tuning:
            m, ti, tj = (int(x) for x in args.tuning.split(","))
            ctx.set_tuning(m, ti, tj)
        elif tune:
            ctx.autotune(U, iters=3)
        norms = torch.zeros((1, cs.nv), dtype=torch.float64, device=dev)
        coef = torch.zeros((cs.n_snap, cs.n_bodies, 3), dtype=torch.float64, device=dev)
        J = torch.zeros(1, dtype=torch.float64, device=dev)

        def step():
            ctx.rk_smooth_into(U, 1, norms)
            ctx.forces_into(U, coef, J)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        assert ctx.sync_status() == hb.HB_OK

        def timed(n, per_launch):
            # per_launch: events around every library launch (kernel times for
            # the roofline); off for the step time itself
            ctx.kernel_stats(0, reset=True)
            ctx.set_timing(per_launch)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
            if ws > 1:
                dist.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(n):
                flush.zero_()                     # evict L2 between timed steps (not timed)
                ev[k][0].record(stream)
                step()
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            if ws > 1:
                dist.barrier()
            ms = sum(a.elapsed_time(b) for a, b in ev)
            stats = (ctx.kernel_stats(0), ctx.kernel_stats(1), ctx.kernel_stats(2)[1])
            ctx.set_timing(False)
            return ms, wall, stats

        ms, wall, (_, _, launches) = timed(steps, False)
        # kernel times from a second, shorter pass with per-launch events
        kms, _, ((tile_ms, tile_n), (halo_ms, halo_n), _) = timed(max(3, min(steps, 100)), timing)
        st = ctx.sync_status()
        if st != hb.HB_OK:
            raise RuntimeError(f"{prec} run ended with status {st} (non-finite state): not a valid measurement")
        return dict(ms=ms, wall=wall, tile_ms=tile_ms, tile_n=tile_n, halo_ms=halo_ms, halo_n=halo_n,
                    kernel_pass_ms=kms, launches=launches, status=st, ctx=ctx, U=U, tuning=ctx.tuning())

    # FP32 flux path with FP64 norms and force sums (headline)
    clocks = ClockSampler(local)
    clocks.start()
    r32 = run_prec("fp32", args.steps, args.warmup)
    clk = clocks.stop()
    # FP64 plain path on the same workload, for comparison (one launch per phase)
    fp64_steps = args.fp64_steps or max(3, min(args.steps, 20))
    r64 = run_prec("fp64", fp64_steps, 2, tune=False)
    batch = run_batch(args, dev) if not args.no_batch else None
    adj = adjoint_ratio(dev) if not args.no_adjoint else None
    box = run_box3d(args, dev) if not args.no_batch else None
    shapes = run_paper_shapes(args, dev) if not args.no_batch else None

    # e2e: host buffers in pinned memory, H2D of the state and D2H of the
    # step's results (norms, force coefficients, J) inside the timed region
    ctx = r32["ctx"]
    U = r32["U"]
    host_U = U.cpu().pin_memory()
    host_out = torch.zeros(cs.nv + cs.n_snap * cs.n_bodies * 3 + 1, dtype=torch.float64).pin_memory()
    norms = torch.zeros((1, cs.nv), dtype=torch.float64, device=dev)
    coef = torch.zeros((cs.n_snap, cs.n_bodies, 3), dtype=torch.float64, device=dev)
    J = torch.zeros(1, dtype=torch.float64, device=dev)
    outdev = torch.zeros_like(host_out, device=dev)
    e2e_steps = max(3, args.steps // 2)

    def e2e_step():
        U.copy_(host_U, non_blocking=True)
        ctx.rk_smooth_into(U, 1, norms)
        ctx.forces_into(U, coef, J)
        outdev[:cs.nv].copy_(norms[0])
        outdev[cs.nv:-1].copy_(coef.reshape(-1))
        outdev[-1:].copy_(J)
        host_out.copy_(outdev, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    evs = []
    for _ in range(e2e_steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    e2e_ms = sum(a.elapsed_time(b) for a, b in evs) / e2e_steps

    # max over ranks; every rank ran its own replica of the workload
    ms32, e2e_ms = max_over_ranks([r32["ms"], e2e_ms], dev)
    ms_per_step = ms32 / args.steps
    value = replica_throughput(ws, units_per_step, ms_per_step)
    v64 = units_per_step / (r64["ms"] / fp64_steps * 1e-3)

    peaks, src = _peaks()
    bpu = algorithmic_bytes_per_unit(cs.nv, 4, cs.dim, cs.n_snap)
    mode, TI, TJ = r32["tuning"]
    launch_ms = r32["tile_ms"] / max(1, r32["tile_n"])
    kname = (f"persist_kernel<float,VISC,{TI},{TJ}>" if mode & 1 else f"tile2d_kernel<float,7,VISC,RK,{TI},{TJ}>")
    roof = roofline(peaks, src, bpu, cs.n_cells * cs.n_snap, mode, launch_ms, kname,
                    _traffic_record(f"{'persist' if mode & 1 else 'tile2d'}_f32_{TI}x{TJ}_ns_ogrid8"))
    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(WORKLOAD, precision="FP32 flux/source/update, FP64 norms and force sums",
                           parallelism="replicas only" if ws > 1 else "single GPU",
                           l2="flushed between timed steps (512 MB write, not timed)",
                           step="1 RK iteration (4 stages) + force reduction"),
            "roofline": roof,
            "roofline_alu": alu_roofline(f"{'persist' if mode & 1 else 'tile2d'}_f32_{TI}x{TJ}_ns_ogrid8",
                                         cs.n_cells * cs.n_snap * (4 if mode & 1 else 1), launch_ms),
            "e2e": {"value": ws * units_per_step / (e2e_ms * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": int(host_U.numel() * host_U.element_size()),
                    "d2h_bytes_per_step": int(host_out.numel() * host_out.element_size())},
            "gpu_launches": int(r32["launches"]),
            "clocks": clk,
            "useful_GBs": bpu * value / 1e9,
            "binding_roof": binding_roof(peaks, bpu, f"{'persist' if mode & 1 else 'tile2d'}_f32_{TI}x{TJ}_ns_ogrid8"),
            "fp64_plain": {"value": v64, "unit": UNIT, "ms_per_step": r64["ms"] / fp64_steps,
                           "steps": fp64_steps,
                           "tile_launch_ms": r64["tile_ms"] / max(1, r64["tile_n"]),
                           "roofline_fp64": fp64_roofline("tile2d_f64_32x8_ns_ogrid8", cs.n_cells * cs.n_snap,
                                                          r64["tile_ms"] / max(1, r64["tile_n"]))},
            "fp32_over_fp64": value / ws / v64,
            "tuning": _tuning_desc(mode, TI, TJ),
            "batched_fp32": batch,
            "adjoint": adj,
            "box3d_fp32": box,
            "paper_shapes_fp32": shapes,
            "kernel_share": {"tile_ms": r32["tile_ms"], "halo_ms": r32["halo_ms"],
                             "step_ms_total": r32["kernel_pass_ms"],
                             "pass": "a second pass of min(steps, 100) steps with per-launch CUDA events"},
            "status": [r32["status"], r64["status"]]}
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args, dev):
    """64 independent inviscid pitching O-grids (seeded sizes 32x16..512x256,
    N_H in 1..4): FP32, all cases advanced together by the library's driver
    (autotuned); the state (~150 MB) exceeds L2, so no flush is needed."""
    import numpy as np
    import torch
    from paper_1304_7654_gb300 import cases as C
    from paper_1304_7654_gb300 import hb
    cases = C.batch_cases()
    ctx = hb.HBContext(cases, "fp32")
    U = ctx.new_state(dev)
    ctx.init_state(U, torch.as_tensor(np.concatenate([C.noise(c) for c in cases]), device=dev), 0.01)
    mode, TI, TJ = ctx.autotune(U, iters=2)
    ctx.rk_smooth(U, 3, norms=False)
    K = max(4, args.steps)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ctx.kernel_stats(0, reset=True)
    a.record()
    ctx.rk_smooth(U, K, norms=False)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / K
    units = sum(c.n_cells * c.n_snap for c in cases) * 4
    cap, replays, persist_replays, direct = ctx.graph_info()
    # algorithmic bytes of one iteration of the mixed-N_s batch (4 stages per
    # cell-snapshot, each case with its own N_s) over the measured iteration
    it_bytes = sum(4 * algorithmic_bytes_per_unit(c.nv, 4, c.dim, c.n_snap) * c.n_cells * c.n_snap for c in cases)
    peaks, src = _peaks()
    achieved = it_bytes / (ms * 1e-3) / 1e9
    kname = f"persist_kernel<float,0,{TI},{TJ}>" if mode & 1 else f"tile2d_kernel<float,NS,0,RK,{TI},{TJ}>"
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "frac_of_nominal_8TBs": achieved / 8000.0,
            "traffic": _traffic_record(f"persist_f32_{TI}x{TJ}_batch64") if mode & 1 else None,
            "kernel": kname, "peak_source": src,
            "bytes_per_iteration": it_bytes, "units_per_iteration": units,
            "time_basis": "CUDA events around K iterations replayed from the captured persistent-launch graph"}
    return {"value": units / (ms * 1e-3), "unit": UNIT, "ms_per_iteration": ms, "iterations": K,
            "cases": len(cases), "cells": int(sum(c.n_cells for c in cases)),
            "cell_snapshots": int(sum(c.n_cells * c.n_snap for c in cases)),
            "roofline": roof,
            "l2": "not flushed: the batch state (~150 MB FP32 plus the RK buffers) exceeds the 129 MB L2",
            "graph": {"persistent_chunk_captured": cap, "graph_replays": replays,
                      "persistent_replays": persist_replays, "persistent_direct_launches": direct},
            **_tuning_desc(mode, TI, TJ),
            "status": _checked_status(ctx, "batched FP32")}


def run_paper_shapes(args, dev):
    """The shapes of the paper's two test cases (Sec. 4.1), FP32, one launch
    per phase (N_s above 9: HB source from its own launch): TC1-like, 512
    blocks of 32x16 = 262,144 cells, 31 snapshots, pitching; TC2-like, 2048
    blocks of 64x32 = 4,194,304 cells, 17 snapshots, yawing inflow.  Inputs
    (~0.7 and ~1.4 GB per state) exceed L2."""
    import numpy as np
    import torch
    from paper_1304_7654_gb300 import cases as C
    from paper_1304_7654_gb300 import hb
    out = {}
    for name, make in (("tc1_like", C.paper_tc1), ("tc2_like", C.paper_tc2)):
        cs = make()
        ctx = hb.HBContext(cs, "fp32")
        U = ctx.new_state(dev)
        ctx.init_state(U, torch.as_tensor(C.noise(cs), device=dev), 0.01)
        mode, TI, TJ = ctx.autotune(U, iters=1)
        ctx.rk_smooth(U, 3, norms=False)
        steps = max(3, min(args.steps, 20))
        torch.cuda.synchronize()
        ctx.kernel_stats(0, reset=True)
        ctx.set_timing(True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            ctx.rk_smooth(U, 1, norms=False)
        b.record()
        torch.cuda.synchronize()
        tile_ms, tile_n = ctx.kernel_stats(0)
        aux_ms, aux_n = ctx.kernel_stats(1)
        ctx.set_timing(False)
        ms = a.elapsed_time(b) / steps
        units = cs.n_cells * cs.n_snap * 4
        tl = tile_ms / max(1, tile_n)
        bpu = algorithmic_bytes_per_unit(cs.nv, 4, cs.dim, cs.n_snap)
        peaks, _ = _peaks()
        out[name] = {"value": units / (ms * 1e-3), "unit": UNIT, "ms_per_iteration": ms, "iterations": steps,
                     "cells": cs.n_cells, "blocks": len(cs.blocks), "n_snap": cs.n_snap,
                     **_tuning_desc(mode, TI, TJ),
                     "tile_kernel": {"launch_ms": tl,
                                     "algorithmic_GBs": bpu * cs.n_cells * cs.n_snap / (tl * 1e-3) / 1e9,
                                     "frac_of_measured_hbm": bpu * cs.n_cells * cs.n_snap / (tl * 1e-3) / 1e9
                                     / peaks["hbm_gbs"]},
                     "aux_launches_ms_per_iteration": aux_ms / steps,
                     "status": _checked_status(ctx, name)}
        del ctx, U
        torch.cuda.empty_cache()
    return out


def run_box3d(args, dev):
    """3D laminar HB NS box, 256x128x64 cells, N_H = 2, FP32 (state ~240 MB,
    larger than L2): per-kernel CUDA-event times and achieved algorithmic
    GB/s of the tile kernel (one RK stage per launch) and the halo kernel."""
    import torch
    from paper_1304_7654_gb300 import cases as C
    from paper_1304_7654_gb300 import hb
    cs = C.box3d()
    ctx = hb.HBContext(cs, "fp32")
    U = ctx.new_state(dev)
    ctx.init_state(U, torch.as_tensor(C.noise(cs), device=dev), 0.01)
    ctx.rk_smooth(U, 2, norms=False)
    steps = max(3, min(args.steps, 20))
    torch.cuda.synchronize()
    ctx.kernel_stats(0, reset=True)
    ctx.set_timing(True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        ctx.rk_smooth(U, 1, norms=False)
    b.record()
    torch.cuda.synchronize()
    tile_ms, tile_n = ctx.kernel_stats(0)
    halo_ms, halo_n = ctx.kernel_stats(1)
    ctx.set_timing(False)
    ms = a.elapsed_time(b) / steps
    cells_snaps = cs.n_cells * cs.n_snap
    nv, s = 5, 4
    tile_bytes = algorithmic_bytes_per_unit(nv, s, 3, cs.n_snap) * cells_snaps
    ghosts = sum((b_.n[0] + 4) * (b_.n[1] + 4) * (b_.n[2] + 4) - b_.n[0] * b_.n[1] * b_.n[2] for b_ in cs.blocks)
    halo_bytes = 2 * ghosts * nv * s * cs.n_snap / 3.0            # per pass, three passes per stage
    tl = tile_ms / max(1, tile_n)
    hl = halo_ms / max(1, halo_n)
    peaks, _ = _peaks()
    return {"value": cells_snaps * 4 / (ms * 1e-3), "unit": UNIT, "ms_per_iteration": ms,
            "workload": "ns_box3d: 256x128x64 cells, N_H=2, laminar, gust farfield, FP32",
            "tile_kernel": {"launch_ms": tl, "algorithmic_GBs": tile_bytes / (tl * 1e-3) / 1e9,
                            "frac_of_measured_hbm": tile_bytes / (tl * 1e-3) / 1e9 / peaks["hbm_gbs"]},
            "halo_kernel": {"launch_ms": hl, "algorithmic_GBs": halo_bytes / (hl * 1e-3) / 1e9,
                            "frac_of_measured_hbm": halo_bytes / (hl * 1e-3) / 1e9 / peaks["hbm_gbs"]},
            "status": _checked_status(ctx, "3D box")}


def adjoint_ratio(dev):
    """Adjoint/primal time on the 4-block 512x256 laminar N_H=4 case (FP64):
    hb_adjoint_residual (halo fill, reverse face sweep, gather, ghost
    transpose) over hb_residual (halo fill and residual)."""
    import torch
    from paper_1304_7654_gb300 import cases as C
    from paper_1304_7654_gb300 import hb
    cs = C.adjoint_ogrid4()
    cs.alpha0_deg = 2.0
    ctx = hb.HBContext(cs, "fp64")
    U = ctx.new_state(dev)
    ctx.init_state(U, torch.as_tensor(C.noise(cs), device=dev), 0.01)
    psi = torch.randn(ctx.size, dtype=torch.float64, device=dev)
    R = ctx.new_state(dev)
    r = ctx.new_state(dev)

    def timed(fn, n=5):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(n):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    tp = timed(lambda: ctx.residual(U, R))
    ta = timed(lambda: ctx.adjoint_residual(U, psi, 0.5, r))
    return {"primal_ms": tp, "adjoint_ms": ta, "ratio": ta / tp,
            "workload": "adjoint_ogrid4: 4 blocks, 512x256 cells, N_H=4, laminar, FP64"}


def kernel_source_hash(names):
    """SHA-1 of the kernel sources' code: comments removed and whitespace
    collapsed, so that an edited comment does not orphan a profile record."""
    import hashlib
    import re
    text = ""
    for n in names:
        with open(os.path.join(ROOT, "paper_1304_7654_gb300", "csrc", n)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        text += " ".join(src.split()) + "\n"
    return hashlib.sha1(text.encode()).hexdigest()


def _profile_record(name):
    """The committed ncu record of a kernel (profiles/traffic.json), if it was
    taken on the current kernel source, else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[name]
        ok = rec.get("kernel_sha1") == kernel_source_hash(rec.get("sources", ["hb_kernels.cuh"]))
        return rec if ok else None
    except Exception:
        return None


# FP32 FMA-pipe peak from the unit counts and clock: 152 SMs x 128 lanes x 2 flops x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def alu_roofline(name, units, launch_ms):
    """The tile kernel against the FP32 arithmetic roof: executed FP32 flops
    per cell-snapshot-stage from the committed ncu record, over the measured
    launch time."""
    rec = _profile_record(name)
    if not rec or "fp32_flops_per_unit" not in rec or launch_ms <= 0:
        return None
    achieved = rec["fp32_flops_per_unit"] * units / (launch_ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_TFLOPS, "flops_per_unit": rec["fp32_flops_per_unit"],
            "flops_source": "executed FP32 operations per cell-snapshot-stage from ncu per-opcode counts "
                            "(FFMA 2, FADD/FMUL 1, packed FFMA2 4, FADD2/FMUL2 2)",
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}


# FP64 pipe: about 2 DFMA lanes per clock per SM on this part (ncu pipe
# utilisation of the FP64 tile kernel), 152 SMs x 2 x 2 flops x 2.07 GHz,
# consistent with the nominal 1.25 TFLOP/s
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def fp64_roofline(name, units, launch_ms):
    """The FP64 tile kernel against the FP64 pipe: executed FP64 operations per
    cell-snapshot-stage from the committed ncu record over the launch time."""
    rec = _profile_record(name)
    if not rec or "fp64_flops_per_unit" not in rec or launch_ms <= 0:
        return None
    achieved = rec["fp64_flops_per_unit"] * units / (launch_ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "flops_per_unit": rec["fp64_flops_per_unit"],
            "flops_source": "executed FP64 operations per cell-snapshot-stage from ncu per-opcode counts "
                            "(DFMA 2, DADD/DMUL 1)",
            "peak_source": "derived: 152 SMs x 2 DFMA lanes x 2 x 2.07 GHz"}


def binding_roof(peaks, bpu, name):
    """Which roof caps the FP32 tile kernel: cell-snapshot-stages per second
    at the HBM roof (algorithmic bytes) and at the FP32 arithmetic roof
    (executed flops from the committed ncu record); the lower one binds."""
    hbm = peaks["hbm_gbs"] * 1e9 / bpu
    rec = _profile_record(name)
    if not rec or "fp32_flops_per_unit" not in rec:
        return {"bound": "hbm", "hbm_cap_units_per_s": hbm, "alu_cap_units_per_s": None}
    alu = FP32_PEAK_TFLOPS * 1e12 / rec["fp32_flops_per_unit"]
    return {"bound": "alu" if alu < hbm else "hbm", "hbm_cap_units_per_s": hbm, "alu_cap_units_per_s": alu}


def _traffic_record(name):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    rec = _profile_record(name)
    return rec["dram_bytes_per_launch"] if rec else None


def run_profile_adjoint(args):
    """ncu entry point for the adjoint: warmup + steps pairs of an FP64
    residual and an adjoint residual on the 4-block 512x256 laminar N_H=4
    case, nothing timed."""
    import torch
    from paper_1304_7654_gb300 import cases as C
    from paper_1304_7654_gb300 import hb
    if args.profile != "fp64":
        raise SystemExit("the adjoint is FP64: use --profile fp64")
    cs = C.adjoint_ogrid4()
    cs.alpha0_deg = 2.0
    ctx = hb.HBContext(cs, "fp64")
    U = ctx.new_state()
    ctx.init_state(U, torch.as_tensor(C.noise(cs), device="cuda"), 0.01)
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    psi = torch.randn(ctx.size, dtype=torch.float64, device="cuda", generator=g)
    R, r = ctx.new_state(), ctx.new_state()
    for _ in range(args.warmup + args.steps):
        ctx.residual(U, R)
        ctx.adjoint_residual(U, psi, 0.5, r)
    torch.cuda.synchronize()
    st = ctx.sync_status()
    print(json.dumps({"profile": "fp64 adjoint", "iterations": args.warmup + args.steps, "status": st,
                      "r_adj_norm": float(r.norm())}))
    return 0 if st == 0 else 1


def run_profile(args):
    """Small entry point for ncu captures: warmup + steps RK iterations (and
    force reductions) of the workload in one precision, nothing timed."""
    import torch
    from paper_1304_7654_gb300 import build as hbuild
    hbuild.build()
    from paper_1304_7654_gb300 import cases as C
    from paper_1304_7654_gb300 import hb
    if args.profile_shape == "adjoint":
        return run_profile_adjoint(args)
    if args.profile_shape:
        cs = {"tc1": C.paper_tc1, "tc2": C.paper_tc2, "box3d": C.box3d}[args.profile_shape]()
        ctx = hb.HBContext(cs, args.profile)
        U = ctx.new_state()
        ctx.init_state(U, torch.as_tensor(C.noise(cs), device="cuda"), 0.01)
    elif args.profile_batch:
        import numpy as np
        cases = C.batch_cases()
        ctx = hb.HBContext(cases, args.profile)
        U = ctx.new_state()
        ctx.init_state(U, torch.as_tensor(np.concatenate([C.noise(c) for c in cases]), device="cuda"), 0.01)
        cs = cases[0]
    else:
        cs = C.ns_ogrid8()
        ctx = hb.HBContext(cs, args.profile)
        U = ctx.new_state()
        ctx.init_state(U, torch.as_tensor(C.noise(cs), device="cuda"), 0.01)
    if args.tuning:
        mode, ti, tj = (int(x) for x in args.tuning.split(","))
        ctx.set_tuning(mode, ti, tj)
    norms = torch.zeros((1, cs.nv), dtype=torch.float64, device="cuda")
    for _ in range(args.warmup + args.steps):
        if args.profile_batch or args.profile_shape:
            ctx.rk_smooth_into(U, 1, None)
        else:
            ctx.rk_smooth_into(U, 1, norms)
            ctx.forces_into(U)
    torch.cuda.synchronize()
    st = ctx.sync_status()
    print(json.dumps({"profile": args.profile, "iterations": args.warmup + args.steps, "status": st,
                      "norms": norms.cpu().tolist()}))
    return 0 if st == 0 else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="timed steps of the FP64 plain path (default: min(steps, 20))")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--profile", choices=["fp32", "fp64"], default=None)
    ap.add_argument("--profile-batch", action="store_true")
    ap.add_argument("--profile-shape", default=None, choices=["tc1", "tc2", "box3d", "adjoint"],
                    help="with --profile: a paper-shaped workload, the 3D box or (fp64) the adjoint "
                         "case instead of the 8-block O-grid")
    ap.add_argument("--tuning", default=None,
                    help="mode,TI,TJ (0 per-phase, 1 persistent; +2 separate halo passes instead of the fused ghost fill)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.profile:
        return run_profile(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
