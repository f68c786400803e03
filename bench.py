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

FLOPS_PER_PAIR_KICK = 26          # 3 sub, 5 r^2, 2 for 1/sqrt, 2 for r^-3, 2 mass scalings, 12 FMA flops
FLOPS_PER_PAIR_CHECK = 18
# FP64 warp instructions of the group recursion per sub-step, by path: least-squares fit of ncu's
# smsp__inst_executed_pipe_fp64.sum per k_recursion launch against the launches' per-path sub-step
# counts over four steps of the N = 10,000 disk (residuals <= 1.1 %; profiles/k_recursion_fp64_fit.md).
# A general sub-step of a large group covers every body and pair of the group.
FP64_PER_PAIR_SUBSTEP = 21.70
FP64_PER_GENERAL_SUBSTEP = 936.0
# The recursion of the bound-pair group the profiles use (bodies of the N = 10,000 disk, seed 1002)
BOUND_PAIR_GROUP = [1244, 3406, 4643, 5122, 9870]
# DRAM read + write per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum, N = 10,000, FP64)
# of the current kernels; None until a capture of the current kernel is on record
RECURSION_TRAFFIC_BYTES = 1987840 + 19968      # first step of the disk (profiles/k_recursion_fp64_fit.md)
KICK_TRAFFIC_BYTES = ((1148928 + 0) + (725248 + 256)) / 2        # kick 1, kick 2 (profiles/k_trap_fp64_disk_N10000.md)
# Step size at which the batched and served forms and the one-at-a-time form all keep the energy
# error of every merger-free disk below 1e-10 (measured on the 64 batched disks: 5.7e-11 after 20
# steps at 0.125 yr, 1.1e-10 at 0.2, 5.2e-10 at 0.5)
MATCHED_TAU = 0.125


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
    ap.add_argument("--no-batched", action="store_true",
                    help="single mode: skip the 64-disk batched comparison at matched accuracy")
    ap.add_argument("--no-served", action="store_true",
                    help="single mode: skip the served Poisson stream at matched accuracy")
    ap.add_argument("--no-field", action="store_true",
                    help="single mode: skip the field-dominated disk (1,000 + 100,000) against the oracle")
    ap.add_argument("--field-steps", type=int, default=3)
    ap.add_argument("--batched-steps", type=int, default=20)
    ap.add_argument("--served-requests", type=int, default=16)
    ap.add_argument("--served-steps-cap", type=int, default=10)
    ap.add_argument("--oracle-steps", type=int, default=50,
                    help="field mode: steps of the FP64 oracle (host, in parallel) the GPU paths are compared with")
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


def workload_name(args, seed=None):
    """The workload string both arms print (rank 0's seed; replicas add 1000 per rank)."""
    return (f"planetesimal disk N_m={args.n} + {args.n_field} field, "
            f"{'FP64' if args.precision == 'fp64' else 'FP32-pair/FP64-state'}, dt=0.5 yr, M=4, "
            f"R_k/R_k+1=2.08, l=3 (seed {args.seed if seed is None else seed})")


def cpu_baseline(args, d, P, budget_s):
    """The oracle, as it stands, on full steps of the same disk: the same warm-up steps as the GPU
    arm untimed, then timed steps until the time budget is spent (the GPU arm's first timed steps)."""
    import oracle
    oracle.build()
    sim = oracle.OracleSim(d.x, d.v, d.m, d.radius, n_massive=d.n_massive)
    sim.step(args.warmup)
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
          "sample": f"steps {args.warmup}..{args.warmup + steps - 1} of the N={args.n} disk (seed {args.seed}) "
                    f"after {args.warmup} untimed steps: {el:.1f} s on 1 host core, serial FP64 C"}
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
    """The oracle on the GPU arm's step window: `warmup` untimed steps, then exactly `steps`
    timed steps of the same disk (serial FP64 C on one host core)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    d, P = workload(args)
    sim = oracle.OracleSim(d.x, d.v, d.m, d.radius, n_massive=d.n_massive)
    if sim.step(args.warmup) < 0:
        raise RuntimeError("oracle warm-up failed")
    t0 = time.perf_counter()
    st = sim.step(args.steps)
    el = time.perf_counter() - t0
    if st < 0:
        raise RuntimeError("oracle steps failed")
    value = 2.0 * P * args.steps / el
    cb = {"value": value, "unit": "pair-interactions/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
          "sample": f"steps {args.warmup}..{args.warmup + args.steps - 1} of the workload after {args.warmup} "
                    f"untimed steps (the GPU arm's window): {el:.1f} s on 1 host core, serial FP64 C"}
    cb["parallel_kick"] = parallel_kick(sim, P)
    line = {"impl": "reference", "metric": "pair-interactions/s", "value": value,
            "unit": "pair-interactions/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args)},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "pair-interactions/s", "h2d_bytes_per_step": 0,
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


def _energy_errors(E0, E1, merges):
    """|E1 - E0| / |E0| per system; systems with a merger (inelastic: energy is not conserved)
    are counted apart from the integration error of the others."""
    dE = [abs((b - a) / a) for a, b in zip(E0, E1)]
    clean = [e for e, m in zip(dE, merges) if m == 0]
    return {"max_no_merger": max(clean) if clean else None,
            "median_no_merger": statistics.median(clean) if clean else None,
            "systems_no_merger": len(clean), "max_all": max(dE) if dE else None,
            "le_1e-10": bool(clean) and max(clean) <= 1e-10}


def bench_batched(sy, disk, steps, warmup, serial_steps):
    """Config-4 shape: 64 disks (N log-uniform 1,000-10,000, seeds 2000+k, all massive) at the
    matched-accuracy step size, as (a) independent contexts advanced by symba_step_many (FP64 and
    mixed), (b) one pool stepped by shared launches (mixed), (c) one simulation per launch sequence,
    FP64, one disk at a time.  Sim-steps/s of each, and each form's energy error per disk."""
    import torch
    from paper_2304_07325_gb300.serve import tiles_for
    sizes = disk.batch_sizes(64, 2000, 1000, 10000)
    disks = [disk.planetesimal_disk(n, 2000 + k) for k, n in enumerate(sizes)]
    out = {"workload": f"64 planetesimal disks, N log-uniform 1,000-10,000 (seeds 2000+k), all massive, "
                       f"dt={MATCHED_TAU} yr, M=4, R_k/R_k+1=2.08, l=3", "sizes": sizes, "dt": MATCHED_TAU,
           "steps": steps, "warmup": warmup}
    for name, prec in (("step_many_fp64", sy.SYMBA_PRECISION_FP64), ("step_many_mixed", sy.SYMBA_PRECISION_MIXED)):
        ctxs = [sy.System(d.x, d.v, d.m, d.radius, params=sy.default_params(dt=MATCHED_TAU, precision=prec))
                for d in disks]
        E0 = [c.energy()[0] for c in ctxs]
        sy.step_many(ctxs, warmup)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sy.step_many(ctxs, steps)
        t = time.perf_counter() - t0
        E1 = [c.energy()[0] for c in ctxs]
        merges = [c.stats().merges for c in ctxs]
        out[name] = {"value": len(disks) * steps / t, "unit": "sim-steps/s",
                     "energy_error": _energy_errors(E0, E1, merges)}
        for c in ctxs:
            c.close()
    prec = sy.SYMBA_PRECISION_MIXED
    pool = sy.Pool(len(disks), sum(d.n for d in disks) + 32 * len(disks), sum(tiles_for(d.n, d.n) for d in disks), prec)
    slots = [pool.admit(d.x, d.v, d.m, d.radius, params=sy.default_params(dt=MATCHED_TAU, precision=prec))
             for d in disks]
    E0 = [pool.energy(k)[0] for k in slots]
    pool.step(warmup)
    pool.sync()
    torch.cuda.synchronize()
    step_ms = []
    for _ in range(steps):
        t0 = time.perf_counter()
        pool.step(1)
        pool.sync()
        step_ms.append(1e3 * (time.perf_counter() - t0))
    E1 = [pool.energy(k)[0] for k in slots]
    merges = [pool.stats(k).merges for k in slots]
    out["pool_mixed"] = {"value": len(disks) * steps / (sum(step_ms) / 1e3), "unit": "sim-steps/s",
                         "p50_step_ms": statistics.median(step_ms), "p99_step_ms": float(np.percentile(step_ms, 99)),
                         "energy_error": _energy_errors(E0, E1, merges)}
    pool.close()
    # one simulation per launch sequence, one disk at a time (FP64): its trajectory is the
    # step_many FP64 one, bit for bit (tests/test_gpu_pool.py), hence the same energy error
    t_serial = 0.0
    for d in disks:
        s1 = sy.System(d.x, d.v, d.m, d.radius, params=sy.default_params(dt=MATCHED_TAU))
        s1.step(warmup)
        s1.sync()
        t0 = time.perf_counter()
        s1.step(serial_steps)
        s1.sync()
        t_serial += time.perf_counter() - t0
        s1.close()
    serial = len(disks) * serial_steps / t_serial
    out["one_at_a_time_fp64"] = {"value": serial, "unit": "sim-steps/s", "steps_each": serial_steps,
                                 "energy_error": "that of step_many_fp64 (the same trajectories, bit for bit)"}
    for k in ("step_many_fp64", "step_many_mixed", "pool_mixed"):
        out[k]["speedup_vs_one_at_a_time_fp64"] = out[k]["value"] / serial
    return out


def bench_served(sy, count, steps_cap):
    """Config-5 shape: Poisson arrivals (20/s), N log-uniform 500-20,000, step budgets U[100, 5000]
    capped for a bounded run, mixed-precision kick, served by the concurrent server (resident
    single-system pools, one stream each, one step in flight per request) at the matched-accuracy
    step size; against the same requests one at a time in FP64."""
    from paper_2304_07325_gb300.serve import ConcurrentServer, poisson_requests
    prec = sy.SYMBA_PRECISION_MIXED
    reqs = poisson_requests(count, 20.0, 3000, 500, 20000, 100, 5000, steps_cap=steps_cap,
                            params=sy.default_params(dt=MATCHED_TAU, precision=prec))
    max_n = max(len(r.m) for r in reqs)
    srv = ConcurrentServer(32, max_n, precision=prec, hbm_budget_bytes=64 << 30)
    results, stats = srv.run(reqs, keep_state=True)
    srv.close()
    summ = stats.summary()
    E0, E1, merges = [], [], []
    for res in results:
        r = reqs[res.rid]
        s0 = sy.System(r.x, r.v, r.m, r.radius, n_massive=r.n_massive, params=r.params)
        E0.append(s0.energy()[0])
        s0.close()
        E1.append(res.energy[0])
        merges.append(res.merges)
    # the same requests one at a time, FP64, each for its whole (capped) budget: the same work
    t_serial, n_serial = 0.0, 0
    for r in reqs:
        s1 = sy.System(r.x, r.v, r.m, r.radius, n_massive=r.n_massive, params=sy.default_params(dt=MATCHED_TAU))
        t0 = time.perf_counter()
        s1.step(r.steps)
        s1.sync()
        t_serial += time.perf_counter() - t0
        n_serial += r.steps
        s1.close()
    serial = n_serial / t_serial
    return {"workload": f"{count} Poisson requests (20/s), N log-uniform 500-20,000, step budgets U[100,5000] "
                        f"capped at {steps_cap}, dt={MATCHED_TAU} yr, FP32-pair kick, FP64 state",
            "server": "concurrent: resident single-system pools, one stream each, one step in flight per request",
            "value": summ["sim_steps_per_s"], "unit": "sim-steps/s", "completed": len(results),
            "p50_step_ms": summ["p50_step_ms"], "p99_step_ms": summ["p99_step_ms"],
            "step_latency": "per request step, launch to observed completion", "wall_s": summ["wall_s"],
            "max_resident": summ["max_resident"], "energy_error": _energy_errors(E0, E1, merges),
            "one_at_a_time_fp64": {"value": serial, "unit": "sim-steps/s",
                                   "sample": "every request alone for its whole capped budget, FP64, one after "
                                             "another (the same sim-steps as the served run)"},
            "speedup_vs_one_at_a_time_fp64": summ["sim_steps_per_s"] / serial}


def chain_vs_cpu(sy, disk):
    """The dominant kernel's chain against one host core: one step of the bound-pair group (five
    bodies of the N = 10,000 disk, one dependent chain of ~34,000 sub-steps), recursion time per
    sub-step on the GPU and the oracle's whole-step time per sub-step on this host."""
    import oracle
    d = disk.planetesimal_disk(10000, 1002)
    g = BOUND_PAIR_GROUP
    s = sy.System(d.x[g], d.v[g], d.m[g], d.radius[g])
    s.profile_step(1)
    s.close()
    s = sy.System(d.x[g], d.v[g], d.m[g], d.radius[g])
    ph = s.profile_step(1)
    st = s.stats()
    s.close()
    ref = oracle.OracleSim(d.x[g], d.v[g], d.m[g], d.radius[g])
    t0 = time.perf_counter()
    ref.step(1)
    t = time.perf_counter() - t0
    n_orc = sum(ref.level_calls)
    return {"case": "one step of bodies [1244, 3406, 4643, 5122, 9870] of the N=10,000 disk (seed 1002)",
            "gpu_substeps": int(st.substeps), "gpu_us_per_substep": 1e3 * ph[5] / max(1, st.substeps),
            "oracle_substeps": n_orc, "oracle_us_per_substep": 1e6 * t / max(1, n_orc),
            "oracle_host": host_cpu()["model"]}


def bench_field_small(sy, disk, steps, oracle_res):
    """Config-3 shape in the default line: N_m = 1,000 + 100,000 field particles (seed 1003),
    `steps` steps of the mixed and the FP64 path (the field rectangle does the kicks), each against
    the FP64 oracle's state after the same steps (computed meanwhile on the host)."""
    d = disk.planetesimal_disk(1000, 1003, n_field=100000)
    P = 1000 * 999 // 2 + 1000 * 100000
    out = {"workload": "field-dominated disk N_m=1000 + 100000 massless (seed 1003), dt=0.5 yr, M=4, "
                       "R_k/R_k+1=2.08, l=3", "steps": steps, "pairs_per_kick": P}
    for name, prec in (("mixed", sy.SYMBA_PRECISION_MIXED), ("fp64", sy.SYMBA_PRECISION_FP64)):
        s = sy.System(d.x, d.v, d.m, d.radius, n_massive=1000, params=sy.default_params(precision=prec))
        E0, _ = s.energy()
        ph = s.profile_step(steps)
        if s.sync() < 0:
            raise RuntimeError(f"field {name}: {sy.status_string(s.sync())}")
        x, *_ = s.get_state()
        E1, _ = s.energy()
        s.close()
        kick_ms = float(ph[1] + ph[6]) / (2 * steps)
        r = {"ms_per_step": float(ph.sum()) / steps, "kick_ms": kick_ms,
             "pairs_per_s": 2.0 * P * steps / (float(ph.sum()) * 1e-3), "dE_rel": abs((E1 - E0) / E0)}
        if oracle_res is not None and oracle_res.get("status", -1) >= 0:
            rel = np.linalg.norm(x - oracle_res["x"], axis=1) / np.linalg.norm(oracle_res["x"], axis=1)
            r["vs_oracle"] = {"position_p50": float(np.median(rel)), "position_p99": float(np.percentile(rel, 99)),
                              "position_max": float(rel.max()),
                              "dE_minus_oracle": abs((E1 - oracle_res["E1"]) / E0)}
        out[name] = r
    if oracle_res is not None:
        out["oracle_seconds"] = oracle_res.get("seconds")
    return out


def run_ours(args):
    # the oracle's run of the field-dominated disk, on a host core while the GPU works (spawned
    # before the first CUDA call)
    oracle_field = None
    rank0, world0, _ = dist_env()
    if rank0 == 0 and world0 == 1 and not args.no_field and not args.no_cpu_baseline:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        conn, child_conn = ctx.Pipe(duplex=False)
        proc = ctx.Process(target=_oracle_field_run, args=(1000, 100000, 1003, args.field_steps, child_conn))
        proc.start()
        oracle_field = (proc, conn)
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
    # the device rates the roofline divides by, measured now on this GPU (a few milliseconds)
    rates = sy.measure_rates()

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
        kick_tflops = FLOPS_PER_PAIR_KICK * P / (kick_ms * 1e-3) / 1e12
        fp64_tflops = rates["fp64_flops"] / 1e12
        rec_s = phase_tot[5] * 1e-3
        sm_hz = 1e6 * (clk.get("sm_mhz") or 2070.0)
        # the dominant kernel: the group recursion.  Its FP64 warp instructions per step are the
        # run's own per-path sub-step counts times the per-path counts ncu measured
        gen_substeps = substeps - pair_substeps
        fp64_instr = FP64_PER_PAIR_SUBSTEP * pair_substeps + FP64_PER_GENERAL_SUBSTEP * gen_substeps
        chip_peak = rates["fp64_flops"] / 64.0          # FP64 warp instructions/s (32 lanes x 2 flops)
        rec_achieved = fp64_instr / rec_s if rec_s > 0 else 0.0
        chain_us = statistics.median(chain_us_list) if chain_us_list else float("nan")
        chain_peak = sm_hz / rates["warp_dfma_dep_cycles"]                # one warp, FP64 instr/s
        chain_achieved = FP64_PER_PAIR_SUBSTEP / (chain_us * 1e-6)
        traffic_ok = args.n == 10000 and args.n_field == 0 and prec == 0
        roofline = {"kernel": "k_recursion (per-group recursive sub-stepping)", "bound": "alu",
                    "achieved": rec_achieved, "peak": chip_peak, "unit": "FP64 warp-instructions/s",
                    "frac": rec_achieved / chip_peak, "traffic": RECURSION_TRAFFIC_BYTES if traffic_ok else None,
                    "share_of_step": phase_tot[5] / phase_tot.sum(),
                    "peak_source": f"measured by symba_measure_rates in this run: {fp64_tflops:.4f} TFLOP/s FP64 "
                                   "(independent FMAs on every SM) / 64 flops per warp instruction",
                    "fp64_instr_per_step": fp64_instr / args.steps,
                    "fp64_instr_model": f"{FP64_PER_PAIR_SUBSTEP} per single-pair sub-step x {pair_substeps} + "
                                        f"{FP64_PER_GENERAL_SUBSTEP} per general sub-step x {gen_substeps} "
                                        "(this run's counts; per-path figures from ncu, "
                                        "profiles/k_recursion_fp64_fit.md)",
                    "chain": {"what": "the longest group's dependent chain on one warp against one warp's FP64 "
                                      "issue (one instruction per warp_dfma_dep_cycles, measured)",
                              "achieved": chain_achieved, "peak": chain_peak, "unit": "FP64 instr/s, one warp",
                              "frac": chain_achieved / chain_peak, "us_per_chain_substep": chain_us,
                              "warp_dfma_dep_cycles": rates["warp_dfma_dep_cycles"]},
                    "note": "latency-bound: each group's sub-steps are one dependent chain on one warp, and the "
                            "longest chain sets the step time, so most of the chip's FP64 lanes idle"}
        roofline_kick = {"kernel": "k_trap_fp64 (trapezoid pair kick)", "bound": "alu", "achieved": kick_tflops,
                         "peak": fp64_tflops, "unit": "TFLOP/s", "frac": kick_tflops / fp64_tflops,
                         "traffic": KICK_TRAFFIC_BYTES if traffic_ok else None,
                         "algorithmic_bytes": 32 * args.n + 48 * args.n,
                         "ms_per_launch": kick_ms, "flops_per_pair": FLOPS_PER_PAIR_KICK,
                         "peak_source": "measured by symba_measure_rates in this run (FP64 FMAs on every SM)"}
        phases = {name: phase_tot[i] / args.steps for i, name in enumerate(sy.PHASES)}
        second = None
        if args.second_n > 0 and world == 1 and args.n_field == 0 and prec == 0:
            second = time_second_disk(sy, disk, args.second_n, args.second_seed, min(args.steps, 50),
                                      args.warmup, stream, flush)
        cb = None
        if not args.no_cpu_baseline and world == 1:
            cb, _, _ = cpu_baseline(args, d, P, args.cpu_budget_s)
        chain = chain_vs_cpu(sy, disk) if world == 1 and not args.no_cpu_baseline else None
        # the batched and served forms against one simulation per launch sequence, FP64, at a
        # step size where every form keeps the energy error <= 1e-10
        batched = None if args.no_batched or world > 1 else bench_batched(sy, disk, args.batched_steps, 1, 2)
        served = None if args.no_served or world > 1 else bench_served(sy, args.served_requests,
                                                                          args.served_steps_cap)
        field = None
        if not args.no_field and world == 1:
            ores = None
            if oracle_field is not None:
                ores = oracle_field[1].recv()
                oracle_field[0].join()
            field = bench_field_small(sy, disk, args.field_steps, ores)
        line = {"metric": "pair-interactions/s", "value": value, "unit": "pair-interactions/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if prec == 0 else "f32-pair/f64-state", "data": "synthetic",
                "config": {"workload": workload_name(args),
                           "seeds": f"{args.seed} + 1000 * rank (replicas)" if world > 1 else str(args.seed),
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
                "clocks": clk, "wall_s": wall, "second": second, "rates": rates,
                "chain_vs_cpu": chain, "batched": batched, "served": served, "field": field}
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


def _oracle_field_run(nm, nf, seed, steps, conn):
    """Child process (spawned): the oracle on the field-dominated disk for `steps` steps."""
    import oracle
    from paper_2304_07325_gb300 import disk
    d = disk.planetesimal_disk(nm, seed, n_field=nf)
    sim = oracle.OracleSim(d.x, d.v, d.m, d.radius, n_massive=nm)
    E0, _ = sim.energy()
    t0 = time.perf_counter()
    st = sim.step(steps)
    el = time.perf_counter() - t0
    E1, _ = sim.energy()
    conn.send({"status": st, "x": sim.x.copy(), "E0": E0, "E1": E1, "seconds": el, "alive": sim.alive.copy()})
    conn.close()


def run_field(args):
    """Field-particle-dominated disk (N_m massive + n_field massless; default 1,000 + 100,000,
    seed 1003): the mixed-precision path (FP32 pair math, FP64 state) and the FP64 path timed per
    step over `steps` steps, the error of both against the FP64 oracle after `--oracle-steps`
    steps (the oracle runs meanwhile in a spawned process on the host), and mixed against FP64
    after all steps.  Metric: pair interactions per second of the mixed path."""
    import multiprocessing as mp
    nm, nf = args.n, args.n_field if args.n_field > 0 else 100000
    ko = max(0, args.oracle_steps)
    child, conn = None, None
    if ko > 0:
        ctx = mp.get_context("spawn")          # started before the first CUDA call
        conn, child_conn = ctx.Pipe(duplex=False)
        child = ctx.Process(target=_oracle_field_run, args=(nm, nf, 1003, ko, child_conn))
        child.start()
    import torch

    import paper_2304_07325_gb300 as sy
    from paper_2304_07325_gb300 import build, disk
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rates = sy.measure_rates()
    d = disk.planetesimal_disk(nm, 1003, n_field=nf)
    P = nm * (nm - 1) // 2 + nm * nf
    out, snap = {}, {}
    for name, prec in (("mixed", sy.SYMBA_PRECISION_MIXED), ("fp64", sy.SYMBA_PRECISION_FP64)):
        s = sy.System(d.x, d.v, d.m, d.radius, n_massive=nm, params=sy.default_params(precision=prec))
        E0, _ = s.energy()
        clocks = ClockSampler(0)
        torch.cuda.synchronize()
        clocks.start()
        ph = np.zeros(sy.SYMBA_NPHASES)
        t0 = time.perf_counter()
        for k in range(args.steps):
            if k == ko and ko > 0:
                xk, *_ = s.get_state()
                snap[name] = (xk, s.energy()[0])
            ph += s.profile_step(1)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        clk = clocks.stop()
        st = s.sync()
        if st < 0:
            raise RuntimeError(f"{name}: {sy.status_string(st)}")
        E1, _ = s.energy()
        x, *_ = s.get_state()
        if ko > 0 and name not in snap:
            snap[name] = (x, E1)
        dev_ms = float(ph.sum())
        kick_ms = float(ph[1] + ph[6]) / (2 * args.steps)
        out[name] = {"ms_per_step": dev_ms / args.steps, "pairs_per_s": 2.0 * P * args.steps / (dev_ms * 1e-3),
                     "dE_rel": abs((E1 - E0) / E0), "x": x, "E0": E0, "clocks": clk, "wall_s": wall,
                     "kick_ms": kick_ms, "recursion_ms_per_step": float(ph[5]) / args.steps,
                     "kick_tflops": FLOPS_PER_PAIR_KICK * P / (kick_ms * 1e-3) / 1e12}
        s.close()
    xm, xd = out["mixed"].pop("x"), out["fp64"].pop("x")

    def rel_err(a, b):
        r = np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
        return {"p50": float(np.percentile(r, 50)), "p99": float(np.percentile(r, 99)), "max": float(r.max()),
                "frac_below_1e-12": float(np.mean(r < 1e-12))}

    vs_oracle = None
    if child is not None:
        res = conn.recv()
        child.join()
        vs_oracle = {"steps": ko, "oracle_seconds": res["seconds"], "oracle_status": res["status"],
                     "oracle_dE_rel": abs((res["E1"] - res["E0"]) / res["E0"])}
        for name in ("mixed", "fp64"):
            xk, Ek = snap[name]
            E0 = out[name]["E0"]
            vs_oracle[name] = {"dE_rel": abs((Ek - E0) / E0), "dE_minus_oracle": abs((Ek - res["E1"]) / E0),
                               "position_rel_err": rel_err(xk, res["x"])}
    for name in ("mixed", "fp64"):
        out[name].pop("E0")
    m = out["mixed"]
    line = {"metric": "pair-interactions/s", "value": m["pairs_per_s"], "unit": "pair-interactions/s",
            "n_gpus": 1, "steps": args.steps, "warmup": 0, "ms_per_step": m["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32-pair/f64-state", "data": "synthetic",
            "config": {"workload": f"field-dominated disk N_m={nm} + {nf} massless (seed 1003), dt=0.5 yr, "
                                   "M=4, R_k/R_k+1=2.08, l=3", "pairs_per_kick": P, "l2": "inputs > L2"},
            "mixed": m, "fp64": out["fp64"], "rates": rates,
            "rel_dx_mixed_vs_fp64": dict(rel_err(xm, xd), after_steps=args.steps,
                                         note="close encounters amplify rounding differences; the tail "
                                              "is chaotic divergence"),
            "vs_oracle": vs_oracle, "clocks": m["clocks"]}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    # one hardware work queue per stream for the concurrently stepped contexts of the batched and
    # served forms (read when the CUDA context is created, so before the first CUDA call)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
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
