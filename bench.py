#!/usr/bin/env python
"""Benchmark of the SyMBA hot path (arXiv:2304.07325) on GB300.

Workload: the Sec. 3 planetesimal disk with N = 10,000 bodies, all massive, FP64, tau = 0.5 yr,
M = 4, shell ratio 2.08, l = 3 (seed 1002).  A step is one full SyMBA step (sun drifts, both
trapezoid kicks with the fused encounter check, grouping, Kepler drifts, group recursion).
Metric: trapezoid pair interactions per second, 2 P per step with P = N (N - 1) / 2.

Prints one JSON line.  `--impl reference` times the serial FP64 oracle (the CPU restatement the
tests check the GPU against) on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

FP64_PEAK_TFLOPS_NOMINAL = 1.25   # GB300 FP64 (no tensor cores for this path)
FLOPS_PER_PAIR_KICK = 26          # 3 sub, 5 r^2, 2 for 1/sqrt, 2 for r^-3, 2 mass scalings, 12 FMA flops
FLOPS_PER_PAIR_CHECK = 18
# The group recursion is a chain of dependent sub-steps per group; the longest chain sets the step
# time.  Its roofline is the FP64 issue rate of one warp: a GB300 warp completes one FP64
# instruction per DFMA_LATENCY_CYCLES, dependent or not (measured with 1 to 8 independent DFMA
# chains per warp; the limit is per warp, four warps per SM reach it at once), and a chain
# sub-step of the single-pair path executes FP64_INSTR_PER_CHAIN_SUBSTEP FP64 warp instructions
# (ncu smsp__inst_executed_pipe_fp64.sum over the sub-steps of the bound-pair group).
DFMA_LATENCY_CYCLES = 64.3
FP64_INSTR_PER_CHAIN_SUBSTEP = 34.0
# DRAM read + write per launch at N = 10,000, FP64 (one-pass ncu captures of one step): the
# trapezoid kick (mean of kick 1 and kick 2) and the group recursion (first step)
KICK_TRAFFIC_BYTES_N10000 = ((1.8944 + 13.7940) + (1.4029 + 11.9360)) / 2 * 1e6
# FP64 pipe of the kick kernels busy (ncu sm__pipe_fp64_cycles_active over active cycles, kick 1
# and kick 2 at N = 10,000, FP64): the issue-side fraction of the FP64 peak
KICK_FP64_PIPE_ACTIVE_N10000 = (0.8836 + 0.8883) / 2
RECURSION_TRAFFIC_BYTES_N10000 = 1.487872e6 + 18.432e3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=10000, help="massive bodies")
    ap.add_argument("--n-field", type=int, default=0, help="massless field particles")
    ap.add_argument("--seed", type=int, default=1002)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="end-to-end steps (default: the timed steps, replayed on a second context)")
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--mode", default="single", choices=["single", "batched", "serve", "field"],
                    help="single: the N=10k headline; batched: 64 disks in one pool vs one at a time; "
                         "serve: Poisson request stream through the continuous-batching server; "
                         "field: N_m massive + field particles, mixed vs FP64 (use --n 1000)")
    ap.add_argument("--systems", type=int, default=64)
    ap.add_argument("--n-lo", type=int, default=1000)
    ap.add_argument("--n-hi", type=int, default=10000)
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--steps-cap", type=int, default=40)
    ap.add_argument("--second-n", type=int, default=5000,
                    help="single mode: also time this disk size (0 = off), reported under 'second'")
    ap.add_argument("--second-seed", type=int, default=1001)
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched mode: keep the default launch schedule instead of autotuning it")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def reduce_max(value: float, device, world: int) -> float:
    """The maximum of a per-rank value over all ranks (the timing rule: max over ranks)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(args):
    from paper_2304_07325_gb300 import disk
    d = disk.planetesimal_disk(args.n, args.seed, n_field=args.n_field)
    P = args.n * (args.n - 1) // 2 + args.n * args.n_field
    return d, P


def host_cpu():
    """The host CPU as /proc/cpuinfo names it (x86: model name; Arm: implementer and part), the
    logical CPUs and those this process may run on."""
    model = None
    try:
        info = open("/proc/cpuinfo").read().splitlines()
        names = [ln.split(":", 1)[1].strip() for ln in info if ln.lower().startswith("model name")]
        if names:
            model = names[0]
        else:
            impl = [ln.split(":", 1)[1].strip() for ln in info if ln.startswith("CPU implementer")]
            part = [ln.split(":", 1)[1].strip() for ln in info if ln.startswith("CPU part")]
            if impl and part:
                known = {("0x41", "0xd4f"): "Arm Neoverse V2", ("0x41", "0xd40"): "Arm Neoverse V1",
                         ("0x41", "0xd0c"): "Arm Neoverse N1", ("0x41", "0xd49"): "Arm Neoverse N2"}
                model = known.get((impl[0], part[0]), f"implementer {impl[0]} part {part[0]}")
    except OSError:
        pass
    try:
        affinity = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        affinity = None
    import platform
    return {"model": model, "arch": platform.machine(), "nproc": os.cpu_count(), "affinity": affinity}


def cpu_baseline(args, d, P, budget_s):
    """The oracle, as it stands, on full steps of the same disk until the time budget is spent."""
    import oracle
    oracle.build()
    sim = oracle.OracleSim(d.x, d.v, d.m, d.radius, n_massive=d.n_massive)
    t0 = time.perf_counter()
    steps = 0
    while True:
        sim.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or steps >= max(1, args.steps):
            break
    value = 2.0 * P * steps / el
    cb = {"value": value, "unit": "pair-interactions/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
          "sample": f"{steps} full oracle steps of the N={args.n} disk (seed {args.seed}), "
                    f"{el:.1f} s on 1 host core, serial FP64 C"}
    cb["parallel_kick"] = parallel_kick(sim, P)
    return cb, steps, el


def parallel_kick(sim, P, budget_s=3.0):
    """The multi-core CPU reference point for the pair kick: the trapezoid accelerations of the
    oracle's current state and level-0 list, rows spread over every host thread (OpenMP)."""
    import oracle
    pairs, _, _ = sim.enc_groups()
    args = (sim.x, sim.m, sim.rhill, sim.alive, pairs, sim.n_massive, sim.params)
    oracle.trap_accel_omp(*args)                   # warm-up (threads, pages)
    t0 = time.perf_counter()
    reps, used = 0, 0
    while True:
        _, used = oracle.trap_accel_omp(*args)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= 50:
            break
    t = el / reps
    return {"pairs_per_s": P / t, "ms_per_kick": 1e3 * t, "threads": used,
            "kind": "OpenMP trapezoid kick (the oracle's pair arithmetic, rows over threads)",
            "sample": f"{reps} kicks of {P} pairs in {el:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    d, P = workload(args)
    cb, steps, el = cpu_baseline(args, d, P, budget_s=min(150.0, max(10.0, 2.0 * args.cpu_budget_s)))
    line = {"impl": "reference", "metric": "pair-interactions/s", "value": cb["value"],
            "unit": "pair-interactions/s", "n_gpus": args.gpus, "steps": steps, "warmup": 0,
            "ms_per_step": 1e3 * el / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"planetesimal disk N_m={args.n} + {args.n_field} field, FP64, dt=0.5 yr, "
                                   f"M=4, R_k/R_k+1=2.08, l=3 (seed {args.seed})"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "pair-interactions/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_second_disk(sy, disk, n, seed, steps, warmup, stream, flush):
    """The same device-timed measurement on a second disk size (the other benchmark size), one
    GPU: value and steps/s over `steps` steps after `warmup`, L2 flushed between steps."""
    import torch
    d = disk.planetesimal_disk(n, seed)
    P = n * (n - 1) // 2
    s = sy.System(d.x, d.v, d.m, d.radius, stream=stream)
    s.profile_step(max(1, warmup))
    if s.sync() < 0:
        raise RuntimeError("second disk: warm-up failed")
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    chain = []
    for k in range(steps):
        if flush is not None:
            flush.fill_(float(k))
        starts[k].record(stream)
        ph = s.profile_step(1)
        ends[k].record(stream)
        st = s.stats()
        if st.max_chain > 0:
            chain.append(1e3 * ph[5] / st.max_chain)
    torch.cuda.synchronize()
    if s.sync() < 0:
        raise RuntimeError("second disk: timed steps failed")
    ms = [starts[k].elapsed_time(ends[k]) for k in range(steps)]
    t = sum(ms) / 1e3
    s.close()
    return {"n": n, "seed": seed, "pairs_per_kick": P, "steps": steps, "warmup": warmup,
            "value": 2.0 * P * steps / t, "unit": "pair-interactions/s", "steps_per_s": steps / t,
            "ms_per_step": 1e3 * t / steps, "p50_step_ms": statistics.median(ms),
            "p99_step_ms": float(np.percentile(ms, 99)),
            "us_per_chain_substep_median": statistics.median(chain) if chain else None}


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2304_07325_gb300 as sy

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2304_07325_gb300 import build
    build.build()
    stream = torch.cuda.current_stream(dev)

    # every rank integrates its own replica (independent disks: replicas, no exchange)
    seed = args.seed + 1000 * rank
    from paper_2304_07325_gb300 import disk
    d = disk.planetesimal_disk(args.n, seed, n_field=args.n_field)
    P = args.n * (args.n - 1) // 2 + args.n * args.n_field
    prec = sy.SYMBA_PRECISION_MIXED if args.precision == "mixed" else sy.SYMBA_PRECISION_FP64
    params = sy.default_params(precision=prec)
    sysm = sy.System(d.x, d.v, d.m, d.radius, n_massive=d.n_massive, params=params, stream=stream)

    # warm-up
    sysm.profile_step(max(1, args.warmup))
    st = sysm.sync()
    if st < 0:
        raise RuntimeError(f"warm-up failed: {sy.status_string(st)}")

    # L2 flush buffer (larger than the 129 MB L2), written between timed steps
    flush = None if args.no_flush else torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    phase_tot = np.zeros(sy.SYMBA_NPHASES)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall0 = time.perf_counter()
    depth_max, substeps, pair_substeps = 0, 0, 0
    chain_us_list = []                         # recursion time per sub-step of the longest chain
    chain_max = 0
    for k in range(args.steps):
        if flush is not None:
            flush.fill_(float(k))
        starts[k].record(stream)
        ph = sysm.profile_step(1)              # events between the step's kernels, same stream
        ends[k].record(stream)
        phase_tot += ph
        s = sysm.stats()
        depth_max = max(depth_max, s.max_depth)
        substeps += s.substeps
        pair_substeps += s.pair_substeps
        chain_max = max(chain_max, s.max_chain)
        if s.max_chain > 0:
            chain_us_list.append(1e3 * ph[5] / s.max_chain)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    step_ms = [starts[k].elapsed_time(ends[k]) for k in range(args.steps)]
    t_local = sum(step_ms) / 1e3
    st = sysm.sync()
    if st < 0:
        raise RuntimeError(f"timed steps failed: {sy.status_string(st)}")
    t_max = reduce_max(t_local, dev, world)
    units = 2.0 * P * args.steps * world
    value = units / t_max

    # end to end through the C ABI with host buffers -- set state (H2D), one step, get state (D2H)
    # every step -- on a second context of the same disk after the same warm-up, so that it steps
    # through the same trajectory as the timed loop (the state round trip is exact: heliocentric
    # positions and barycentric velocities both ways)
    ne = args.steps if args.e2e_steps is None else max(1, min(args.e2e_steps, args.steps))
    s2 = sy.System(d.x, d.v, d.m, d.radius, n_massive=d.n_massive, params=params, stream=stream)
    s2.profile_step(max(1, args.warmup))
    if s2.sync() < 0:
        raise RuntimeError("end-to-end warm-up failed")
    ntot = d.n
    xh = torch.empty((ntot, 3), dtype=torch.float64, pin_memory=True)
    vh = torch.empty((ntot, 3), dtype=torch.float64, pin_memory=True)
    x0, v0, *_ = s2.get_state()
    xh.numpy()[...] = x0
    vh.numpy()[...] = v0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    for _ in range(ne):
        sy.lib().symba_set_state(s2._h, sy.c_void_p(xh.data_ptr()), sy.c_void_p(vh.data_ptr()))
        s2.step(1)
        sy.lib().symba_get_state(s2._h, sy.c_void_p(xh.data_ptr()), sy.c_void_p(vh.data_ptr()),
                                 None, None, None)
    te = time.perf_counter() - te0
    s2.close()
    e2e_value = 2.0 * P * ne * world / reduce_max(te, dev, world)

    if rank == 0:
        kick_ms = (phase_tot[1] + phase_tot[6]) / (2 * args.steps)
        kick_flops = FLOPS_PER_PAIR_KICK * P
        kick_achieved = kick_flops / (kick_ms * 1e-3) / 1e12
        rec_ms = phase_tot[5] / args.steps
        peak_note = "GB300 FP64 1.25 TFLOP/s (recipe's figure; a DFMA loop measured 1.19 here)"
        # the dominant kernel by time: the group recursion, bound by the FP64 latency of the warp
        # that runs the longest chain of dependent sub-steps
        sm_hz = 1e6 * (clk.get("sm_mhz") or 2070.0)
        chain_peak = sm_hz / DFMA_LATENCY_CYCLES / 1e6                    # M FP64 instr/s, one warp
        chain_us = statistics.median(chain_us_list) if chain_us_list else float("nan")
        chain_achieved = FP64_INSTR_PER_CHAIN_SUBSTEP / chain_us         # M FP64 instr/s
        roofline = {"kernel": "k_recursion (per-group recursive sub-stepping)", "bound": "alu",
                    "achieved": chain_achieved, "peak": chain_peak,
                    "unit": "M FP64 warp-instr/s on the longest group chain (one warp)",
                    "frac": chain_achieved / chain_peak,
                    "traffic": RECURSION_TRAFFIC_BYTES_N10000 if args.n == 10000 and args.n_field == 0 and prec == 0 else None,
                    "share_of_step": phase_tot[5] / phase_tot.sum(),
                    "peak_source": f"SM clock {sm_hz / 1e6:.0f} MHz / {DFMA_LATENCY_CYCLES} cycles per "
                                   "FP64 instruction of one warp, dependent or not (measured)",
                    "fp64_instr_per_chain_substep": FP64_INSTR_PER_CHAIN_SUBSTEP,
                    "us_per_chain_substep": chain_us,
                    "note": "latency-bound: one warp runs a group's dependent sub-steps; the longest "
                            "chain sets the step time; the rest of each sub-step is shuffles, branches "
                            "and issue"}
        roofline_kick = {"kernel": "k_trap_fp64 (trapezoid pair kick)", "bound": "alu", "achieved": kick_achieved,
                         "peak": FP64_PEAK_TFLOPS_NOMINAL, "unit": "TFLOP/s",
                         "frac": kick_achieved / FP64_PEAK_TFLOPS_NOMINAL,
                         "traffic": KICK_TRAFFIC_BYTES_N10000 if args.n == 10000 and args.n_field == 0 and prec == 0 else None,
                         "ms_per_launch": kick_ms, "peak_source": peak_note,
                         "fp64_pipe_active": KICK_FP64_PIPE_ACTIVE_N10000 if args.n == 10000 and args.n_field == 0 and prec == 0 else None,
                         "fp64_pipe_active_source": "ncu sm__pipe_fp64_cycles_active (kick 1, kick 2), "
                                                    "profiles/k_trap_fp64_disk_N10000.md"}
        phases = {name: phase_tot[i] / args.steps for i, name in enumerate(sy.PHASES)}
        second = None
        if args.second_n > 0 and world == 1 and args.n_field == 0 and prec == 0:
            second = time_second_disk(sy, disk, args.second_n, args.second_seed, min(args.steps, 50),
                                      args.warmup, stream, flush)
        cb = None
        if not args.no_cpu_baseline and world == 1:
            cb, _, _ = cpu_baseline(args, d, P, args.cpu_budget_s)
        line = {"metric": "pair-interactions/s", "value": value, "unit": "pair-interactions/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if prec == 0 else "f32-pair/f64-state", "data": "synthetic",
                "config": {"workload": f"planetesimal disk N_m={args.n} + {args.n_field} field, "
                                       f"{'FP64' if prec == 0 else 'FP32-pair/FP64-state'}, dt=0.5 yr, M=4, "
                                       f"R_k/R_k+1=2.08, l=3 (seed {args.seed}+1000*rank)",
                           "n": args.n, "pairs_per_kick": P, "l2": "flushed between steps (256 MB write)"
                           if flush is not None else "not flushed",
                           "parallelism": f"replicas x{world}"},
                "steps_per_s": args.steps * world / t_max,
                "p50_step_ms": statistics.median(step_ms), "p99_step_ms": float(np.percentile(step_ms, 99)),
                "phase_ms_per_step": phases, "max_depth": depth_max,
                "substeps_per_step": substeps / args.steps, "longest_chain_substeps": chain_max,
                "pair_path_share_of_substeps": pair_substeps / substeps if substeps else None,
                "us_per_chain_substep_median": statistics.median(chain_us_list) if chain_us_list else None,
                "roofline": roofline, "roofline_kick": roofline_kick, "cpu_baseline": cb,
                "e2e": {"value": e2e_value, "unit": "pair-interactions/s",
                        "h2d_bytes_per_step": 2 * 8 * 3 * ntot, "d2h_bytes_per_step": 2 * 8 * 3 * ntot,
                        "steps": ne, "trajectory": "the timed steps' (second context, same warm-up)"
                        if ne == args.steps else f"the first {ne} of the timed steps'"},
                # per timed step: the step's 12 kernels plus the per-call statistics reset (the
                # loop times each step as its own call; the launch list shows the same 13)
                "gpu_launches": args.steps * 13,
                "clocks": clk, "wall_s": wall, "second": second}
        print(json.dumps(line), flush=True)
    sysm.close()
    if world > 1:
        dist.destroy_process_group()


def run_batched(args):
    """Many independent disks (N log-uniform in [n_lo, n_hi], seeds 2000+k) stepped together in
    one pool, against the same disks stepped one context at a time (FP64 both, or mixed for the
    pool when --precision mixed).  Metric: simulation steps per second."""
    # more hardware work queues for the concurrently stepped contexts below (read when the CUDA
    # context is created, so before the first CUDA call of this process)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import torch

    import paper_2304_07325_gb300 as sy
    from paper_2304_07325_gb300 import build, disk
    from paper_2304_07325_gb300.serve import tiles_for
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    sizes = disk.batch_sizes(args.systems, 2000, args.n_lo, args.n_hi)
    disks = [disk.planetesimal_disk(n, 2000 + k) for k, n in enumerate(sizes)]
    prec = sy.SYMBA_PRECISION_MIXED if args.precision == "mixed" else sy.SYMBA_PRECISION_FP64
    tiles = sum(tiles_for(d.n, d.n_massive) for d in disks)
    pool = sy.Pool(len(disks), sum(d.n for d in disks) + 32 * len(disks), tiles, prec)
    slots = [pool.admit(d.x, d.v, d.m, d.radius) for d in disks]
    E0 = [pool.energy(s)[0] for s in slots]
    pool.step(args.warmup)
    pool.sync()
    # launch schedules timed on this pool (state left as it was), the fastest kept
    tune = None if args.no_autotune else pool.autotune(reps=3)
    schedule = pool.schedule
    clocks = ClockSampler(0)
    torch.cuda.synchronize()
    clocks.start()
    step_ms = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        pool.step(1)
        pool.sync()
        step_ms.append(1e3 * (time.perf_counter() - t0))
    clk = clocks.stop()
    t_pool = sum(step_ms) / 1e3
    # energy error per disk; mergers (inelastic) change the energy, so disks that had one are
    # reported apart from the integration error of the others
    dE = [abs((pool.energy(s)[0] - e0) / e0) for s, e0 in zip(slots, E0)]
    merged = [pool.stats(s).merges > 0 for s in slots]
    dE_clean = [e for e, mg in zip(dE, merged) if not mg]
    pool.close()
    # the same disks one context (one launch sequence) at a time, FP64
    serial_steps = max(1, min(args.steps, 5))
    t_serial = 0.0
    dE_serial = []
    for d in disks:
        s1 = sy.System(d.x, d.v, d.m, d.radius)
        e0 = s1.energy()[0]
        s1.step(1)
        s1.sync()
        t0 = time.perf_counter()
        s1.step(serial_steps)
        s1.sync()
        t_serial += time.perf_counter() - t0
        if s1.stats().merges == 0:
            dE_serial.append(abs((s1.energy()[0] - e0) / e0))
        s1.close()
    # the same disks as independent contexts, each on its own stream, stepped by the native
    # scheduler with one step in flight per system (no lock-step)
    ctxs = [sy.System(d.x, d.v, d.m, d.radius, params=sy.default_params(precision=prec)) for d in disks]
    sy.step_many(ctxs, max(1, args.warmup))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sy.step_many(ctxs, args.steps)
    t_conc = time.perf_counter() - t0
    for c in ctxs:
        c.close()
    conc_rate = len(disks) * args.steps / t_conc
    pool_rate = len(disks) * args.steps / t_pool
    serial_rate = len(disks) * serial_steps / t_serial
    line = {"metric": "batched sim-steps/s", "value": pool_rate, "unit": "sim-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_pool / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == 0 else "f32-pair/f64-state", "data": "synthetic",
            "config": {"workload": f"{len(disks)} planetesimal disks, N log-uniform {args.n_lo}-{args.n_hi} "
                                   f"(seeds 2000+k), all massive, dt=0.5 yr, M=4, one pool",
                       "sizes": sizes, "schedule": schedule},
            "autotune": tune,
            "p50_step_ms": statistics.median(step_ms), "p99_step_ms": float(np.percentile(step_ms, 99)),
            "energy_error": {"max_no_merger": max(dE_clean) if dE_clean else None,
                             "median_no_merger": statistics.median(dE_clean) if dE_clean else None,
                             "disks_no_merger": len(dE_clean), "max_all": max(dE),
                             "steps": args.warmup + args.steps,
                             "what": "|E - E0| / |E0| per disk after the pool's steps; disks with a "
                                     "merger (inelastic, energy not conserved) counted apart"},
            "serial_fp64_one_at_a_time": {"value": serial_rate, "unit": "sim-steps/s", "steps_each": serial_steps,
                                          "energy_error_max_no_merger": max(dE_serial) if dE_serial else None,
                                          "energy_steps": 1 + serial_steps},
            "speedup_vs_serial": pool_rate / serial_rate,
            "concurrent_contexts": {"value": conc_rate, "unit": "sim-steps/s", "steps": args.steps,
                                    "speedup_vs_serial": conc_rate / serial_rate,
                                    "how": "symba_step_many: one context per disk on its own stream, one step in "
                                           "flight each, CUDA_DEVICE_MAX_CONNECTIONS="
                                           + os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS", "")},
            "clocks": clk}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Poisson request stream (mean 20/s; N log-uniform, step budgets capped for a bounded run)
    through the continuous-batching server; mixed-precision kick, FP64 drifts."""
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")     # one stream per request slot
    import torch

    import paper_2304_07325_gb300 as sy
    from paper_2304_07325_gb300 import build
    from paper_2304_07325_gb300.serve import ConcurrentServer, Server, poisson_requests, tiles_for
    build.build()
    torch.cuda.set_device(0)
    prec = sy.SYMBA_PRECISION_FP64 if args.precision == "fp64" else sy.SYMBA_PRECISION_MIXED
    reqs = poisson_requests(args.requests, 20.0, 3000, args.n_lo, args.n_hi, 100, 5000,
                            steps_cap=args.steps_cap)
    max_n = max(len(r.m) for r in reqs)
    # the continuous-batching pool: every pool step advances all residents together
    srv = Server(max_systems=32, max_particles=32 * (max_n + 32), max_tiles=16 * tiles_for(max_n, max_n),
                 precision=prec, hbm_budget_bytes=64 << 30)
    results, stats = srv.run(reqs, keep_state=False)
    srv.close()
    summ = stats.summary()
    # the same stream served without lock-step: one resident single-system pool per slot
    csrv = ConcurrentServer(32, max_n, precision=prec, hbm_budget_bytes=64 << 30)
    cres, cstats = csrv.run(reqs, keep_state=False)
    csrv.close()
    csumm = cstats.summary()
    line = {"metric": "served sim-steps/s", "value": csumm["sim_steps_per_s"], "unit": "sim-steps/s",
            "n_gpus": 1, "steps": csumm["sim_steps"], "warmup": 0, "ms_per_step": csumm["p50_step_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32-pair/f64-state" if prec == 1 else "f64", "data": "synthetic",
            "config": {"workload": f"{args.requests} Poisson requests (20/s), N log-uniform {args.n_lo}-{args.n_hi}, "
                                   f"step budgets U[100,5000] capped at {args.steps_cap}",
                       "server": "concurrent: 32 resident single-system pools, one stream each, one step "
                                 "in flight per request"},
            "p50_step_ms": csumm["p50_step_ms"], "p99_step_ms": csumm["p99_step_ms"],
            "step_latency": "per request step, launch to observed completion",
            "max_resident": csumm["max_resident"], "completed": len(cres), "wall_s": csumm["wall_s"],
            "pool_server": {"value": summ["sim_steps_per_s"], "unit": "sim-steps/s",
                            "p50_step_ms": summ["p50_step_ms"], "p99_step_ms": summ["p99_step_ms"],
                            "step_latency": "per pool step (all residents)", "pool_steps": summ["pool_steps"],
                            "max_resident": summ["max_resident"], "completed": len(results),
                            "wall_s": summ["wall_s"]}}
    print(json.dumps(line), flush=True)


def run_field(args):
    """Field-particle-dominated disk (N_m massive + n_field massless; default 1,000 + 100,000):
    the mixed-precision path (FP32 pair math, FP64 state) timed per step, and its accuracy after
    the same number of steps against the FP64 path from the same input (energy error of each,
    largest relative position difference).  Metric: pair interactions per second."""
    import torch

    import paper_2304_07325_gb300 as sy
    from paper_2304_07325_gb300 import build, disk
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    nm, nf = args.n, args.n_field if args.n_field > 0 else 100000
    d = disk.planetesimal_disk(nm, 1003, n_field=nf)
    P = nm * (nm - 1) // 2 + nm * nf
    out = {}
    for name, prec in (("mixed", sy.SYMBA_PRECISION_MIXED), ("fp64", sy.SYMBA_PRECISION_FP64)):
        s = sy.System(d.x, d.v, d.m, d.radius, n_massive=nm, params=sy.default_params(precision=prec))
        E0, _ = s.energy()
        s.profile_step(max(1, args.warmup))
        clocks = ClockSampler(0)
        torch.cuda.synchronize()
        clocks.start()
        ph = np.zeros(sy.SYMBA_NPHASES)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ph += s.profile_step(1)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        clk = clocks.stop()
        st = s.sync()
        if st < 0:
            raise RuntimeError(f"{name}: {sy.status_string(st)}")
        E1, _ = s.energy()
        x, *_ = s.get_state()
        dev_ms = float(ph.sum())
        out[name] = {"ms_per_step": dev_ms / args.steps, "pairs_per_s": 2.0 * P * args.steps / (dev_ms * 1e-3),
                     "dE_rel": abs((E1 - E0) / E0), "x": x, "clocks": clk, "wall_s": wall,
                     "kick_ms": float(ph[1] + ph[6]) / (2 * args.steps)}
        s.close()
    xm, xd = out["mixed"].pop("x"), out["fp64"].pop("x")
    rel = np.linalg.norm(xm - xd, axis=1) / np.linalg.norm(xd, axis=1)
    dx = {"p50": float(np.percentile(rel, 50)), "p99": float(np.percentile(rel, 99)),
          "max": float(rel.max()), "frac_below_1e-10": float(np.mean(rel < 1e-10)),
          "note": "close encounters amplify rounding differences; the tail is chaotic divergence"}
    m = out["mixed"]
    line = {"metric": "pair-interactions/s", "value": m["pairs_per_s"], "unit": "pair-interactions/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32-pair/f64-state", "data": "synthetic",
            "config": {"workload": f"field-dominated disk N_m={nm} + {nf} massless (seed 1003), dt=0.5 yr, "
                                   "M=4, R_k/R_k+1=2.08, l=3", "pairs_per_kick": P, "l2": "inputs > L2"},
            "mixed": m, "fp64": out["fp64"],
            "rel_dx_mixed_vs_fp64": dx, "clocks": m["clocks"]}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "batched":
        run_batched(args)
    elif args.mode == "serve":
        run_serve(args)
    elif args.mode == "field":
        run_field(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
