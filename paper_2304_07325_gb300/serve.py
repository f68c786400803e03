"""Continuous batching of independent SyMBA simulations on one GPU.

The paper motivates SyMBAp by parameter scans -- many simulations sharing fixed computing
resources (Sec. 1).  A Server keeps one pool (C ABI symba_pool_*) resident on the device and runs
a request loop: requests that have arrived are admitted as soon as a slot and enough device
memory (bodies, trapezoid tiles, pair lists, within an HBM budget) are free; every loop turn
advances all admitted simulations by one step with the same kernel launches; a simulation that
has used its step budget is read back and evicted, which frees room for the next arrivals.
Results do not depend on the mix: every kernel works per system with a fixed summation order.

A ConcurrentServer serves the same requests without lock-step: each admitted simulation sits in
a resident single-system pool of its own, on its own stream, and advances as soon as its previous
step has completed, so no simulation waits for another's longest chain of recursion sub-steps.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import Pool, SymbaError, default_params, SYMBA_PRECISION_FP64


@dataclass
class Request:
    rid: int
    arrival_s: float
    x: np.ndarray
    v: np.ndarray
    m: np.ndarray
    radius: np.ndarray
    n_massive: int
    steps: int
    params: object = None


@dataclass
class Result:
    rid: int
    n: int
    steps: int
    admitted_s: float
    finished_s: float
    x: np.ndarray = None
    v: np.ndarray = None
    alive: np.ndarray = None
    energy: tuple = None
    status: int = 0
    merges: int = 0


@dataclass
class ServeStats:
    step_ms: list = field(default_factory=list)        # per pool step (all resident systems)
    sim_steps: int = 0                                   # system-steps completed
    wall_s: float = 0.0
    max_resident: int = 0

    def summary(self):
        s = np.array(self.step_ms) if self.step_ms else np.zeros(1)
        return {"sim_steps": self.sim_steps, "wall_s": self.wall_s,
                "sim_steps_per_s": self.sim_steps / self.wall_s if self.wall_s > 0 else 0.0,
                "p50_step_ms": float(np.percentile(s, 50)), "p99_step_ms": float(np.percentile(s, 99)),
                "pool_steps": len(self.step_ms), "max_resident": self.max_resident}


def tiles_for(n: int, n_massive: int) -> int:
    """Trapezoid tiles of a system: 32 x 32 blocks (I, J), I <= J, over the column blocks that
    hold massive bodies (blocks of field particles only form the field rectangle instead)."""
    nbm = (n_massive + 31) // 32
    return nbm * (nbm + 1) // 2


class Server:
    """A pool plus the admission and eviction loop."""

    def __init__(self, max_systems: int, max_particles: int, max_tiles: int,
                 precision: int = SYMBA_PRECISION_FP64, hbm_budget_bytes: int | None = None,
                 stream=None, clock=time.perf_counter, pool=None, footprint=None):
        self.pool = pool if pool is not None else Pool(max_systems, max_particles, max_tiles, precision, stream)
        self._footprint = footprint
        self.precision = precision
        self.max_systems, self.max_particles, self.max_tiles = max_systems, max_particles, max_tiles
        self.hbm_budget = hbm_budget_bytes
        self.clock = clock
        self.resident = {}          # slot -> [request, steps done, admitted_s]
        self.used_particles = 0
        self.used_tiles = 0
        self.used_bytes = 0

    def footprint(self, req: Request) -> int:
        if self._footprint is not None:
            return self._footprint(req)
        return Pool.footprint(len(req.m), req.n_massive, req.params or default_params(precision=self.precision))

    def fits(self, req: Request) -> bool:
        n = len(req.m)
        if len(self.resident) >= self.max_systems:
            return False
        if self.used_particles + 32 * ((n + 31) // 32) > self.max_particles:
            return False
        if self.used_tiles + tiles_for(n, req.n_massive) > self.max_tiles:
            return False
        if self.hbm_budget is not None and self.used_bytes + self.footprint(req) > self.hbm_budget:
            return False
        return True

    def admit(self, req: Request, now: float) -> bool:
        if not self.fits(req):
            return False
        p = req.params
        try:
            slot = self.pool.admit(req.x, req.v, req.m, req.radius, n_massive=req.n_massive, params=p)
        except SymbaError:
            return False
        n = len(req.m)
        self.resident[slot] = [req, 0, now]
        self.used_particles += 32 * ((n + 31) // 32)
        self.used_tiles += tiles_for(n, req.n_massive)
        self.used_bytes += self.footprint(req)
        return True

    def _retire(self, slot: int, now: float, keep_state: bool) -> Result:
        req, done, t_adm = self.resident.pop(slot)
        res = Result(rid=req.rid, n=len(req.m), steps=done, admitted_s=t_adm, finished_s=now)
        if keep_state:
            res.x, res.v, _, _, res.alive = self.pool.get_state(slot)
            res.energy = self.pool.energy(slot)
        st = self.pool.stats(slot)
        res.status, res.merges = st.status, int(st.merges)
        self.pool.evict(slot)
        n = len(req.m)
        self.used_particles -= 32 * ((n + 31) // 32)
        self.used_tiles -= tiles_for(n, req.n_massive)
        self.used_bytes -= self.footprint(req)
        return res

    def run(self, requests, keep_state: bool = True, time_scale: float = 1.0, max_wall_s: float | None = None):
        """Serve `requests` (arrival_s on the wall clock, scaled by time_scale).  Returns the
        results in completion order and the loop statistics."""
        pending = sorted(requests, key=lambda r: r.arrival_s)
        results, stats = [], ServeStats()
        t0 = self.clock()
        qi = 0
        while qi < len(pending) or self.resident:
            now = self.clock() - t0
            if max_wall_s is not None and now > max_wall_s:
                break
            # admit everything that has arrived and fits (first come, first served)
            while qi < len(pending) and pending[qi].arrival_s * time_scale <= now:
                if not self.admit(pending[qi], now):
                    break
                qi += 1
            if not self.resident:
                if qi < len(pending):
                    time.sleep(min(0.001, max(0.0, pending[qi].arrival_s * time_scale - now)))
                    continue
                break
            stats.max_resident = max(stats.max_resident, len(self.resident))
            ts = self.clock()
            self.pool.step(1)
            self.pool.sync()
            stats.step_ms.append(1e3 * (self.clock() - ts))
            stats.sim_steps += len(self.resident)
            now = self.clock() - t0
            for slot in list(self.resident):
                self.resident[slot][1] += 1
                if self.resident[slot][1] >= self.resident[slot][0].steps:
                    results.append(self._retire(slot, now, keep_state))
        stats.wall_s = self.clock() - t0
        return results, stats

    def close(self):
        self.pool.close()


class ConcurrentServer:
    """Requests served without lock-step.  `slots` single-system pools stay resident on the
    device, each with its own stream and each sized for the largest request, so admitting and
    evicting allocate nothing.  An arrived request takes a free slot; the loop keeps exactly one
    step in flight per admitted request and launches its next step as soon as that step's
    completion event has fired, so a request never waits for another's chain of recursion
    sub-steps (in a Server every pool step waits for the slowest resident).  Each result is that
    of the request alone: its slot is a pool of one.  Step latencies are taken on the host from a
    step's launch to the loop turn that sees it complete."""

    def __init__(self, slots: int, max_n: int, precision: int = SYMBA_PRECISION_FP64,
                 hbm_budget_bytes: int | None = None, pools=None, streams=None, events=None,
                 clock=time.perf_counter, idle_s: float = 5e-5):
        if pools is None:
            if hbm_budget_bytes is not None:
                # as many resident slots as the device-memory budget holds at the largest request
                per_slot = Pool.footprint(max_n, max_n, default_params(precision=precision))
                slots = max(1, min(slots, hbm_budget_bytes // max(1, per_slot)))
            import torch
            streams = [torch.cuda.Stream() for _ in range(slots)]
            events = [torch.cuda.Event() for _ in range(slots)]
            pools = [Pool(1, max_n + 64, tiles_for(max_n, max_n), precision, stream=st) for st in streams]
        self.pools, self.streams, self.events = pools, streams, events
        self.precision = precision
        self.clock = clock
        self.idle_s = idle_s
        self.free = list(range(len(pools)))[::-1]
        self.active = {}            # slot -> [request, steps done, admitted_s, in flight, launched_s, pool slot]

    def admit(self, req: Request, now: float) -> bool:
        if not self.free:
            return False
        k = self.free[-1]
        try:
            ps = self.pools[k].admit(req.x, req.v, req.m, req.radius, n_massive=req.n_massive, params=req.params)
        except SymbaError:
            return False
        self.free.pop()
        self.active[k] = [req, 0, now, False, 0.0, ps]
        return True

    def _retire(self, k: int, now: float, keep_state: bool) -> Result:
        req, done, t_adm, _, _, ps = self.active.pop(k)
        pool = self.pools[k]
        res = Result(rid=req.rid, n=len(req.m), steps=done, admitted_s=t_adm, finished_s=now)
        if keep_state:
            res.x, res.v, _, _, res.alive = pool.get_state(ps)
            res.energy = pool.energy(ps)
        st = pool.stats(ps)
        res.status, res.merges = st.status, int(st.merges)
        pool.evict(ps)
        self.free.append(k)
        return res

    def run(self, requests, keep_state: bool = True, time_scale: float = 1.0, max_wall_s: float | None = None):
        """Serve `requests` (arrival_s on the wall clock, scaled by time_scale).  Returns the
        results in completion order and the loop statistics (step_ms: one entry per request
        step)."""
        pending = sorted(requests, key=lambda r: r.arrival_s)
        results, stats = [], ServeStats()
        t0 = self.clock()
        qi = 0
        while qi < len(pending) or self.active:
            now = self.clock() - t0
            if max_wall_s is not None and now > max_wall_s:
                break
            while qi < len(pending) and pending[qi].arrival_s * time_scale <= now:
                if not self.admit(pending[qi], now):
                    break
                qi += 1
            stats.max_resident = max(stats.max_resident, len(self.active))
            progressed = False
            for k in list(self.active):
                st = self.active[k]
                if st[3]:
                    if not self.events[k].query():
                        continue
                    t = self.clock() - t0
                    stats.step_ms.append(1e3 * (t - st[4]))
                    stats.sim_steps += 1
                    st[1] += 1
                    st[3] = False
                    progressed = True
                    if st[1] >= st[0].steps:
                        results.append(self._retire(k, t, keep_state))
                        continue
                self.pools[k].step(1)
                self.events[k].record(self.streams[k])
                st[3] = True
                st[4] = self.clock() - t0
                progressed = True
            if not progressed:
                if not self.active and qi < len(pending):
                    time.sleep(min(0.001, max(0.0, pending[qi].arrival_s * time_scale - now)))
                else:
                    time.sleep(self.idle_s)
        stats.wall_s = self.clock() - t0
        return results, stats

    def close(self):
        for p in self.pools:
            p.close()


def poisson_requests(count: int, rate_per_s: float = 20.0, seed: int = 3000, n_lo: int = 500,
                     n_hi: int = 20000, steps_lo: int = 100, steps_hi: int = 5000, n_cap: int | None = None,
                     steps_cap: int | None = None, params=None):
    """The served workload: Poisson arrivals, N log-uniform, step budgets uniform (optionally
    capped for a bounded run); `params` (a symba_params, e.g. a step size and precision) applies
    to every request (None: the defaults)."""
    from . import disk
    out = []
    for k, (t, n, steps, s) in enumerate(disk.request_stream(count, rate_per_s, seed, n_lo, n_hi, steps_lo, steps_hi)):
        if n_cap is not None:
            n = min(n, n_cap)
        if steps_cap is not None:
            steps = min(steps, steps_cap)
        d = disk.planetesimal_disk(n, s)
        out.append(Request(rid=k, arrival_s=t, x=d.x, v=d.v, m=d.m, radius=d.radius, n_massive=d.n_massive, steps=steps,
                           params=params))
    return out
