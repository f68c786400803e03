"""Host logic of the serving loop (admission, eviction, capacity accounting) against a fake pool
(CPU only)."""
import numpy as np

from paper_2304_07325_gb300.serve import Request, Server


class FakeStats:
    status = 0


class FakePool:
    """Records calls; every admitted system advances one step per pool step."""

    def __init__(self, max_slots):
        self.free = list(range(max_slots))
        self.live = {}
        self.log = []

    def admit(self, x, v, m, radius, n_massive=None, params=None):
        slot = self.free.pop(0)
        self.live[slot] = len(m)
        self.log.append(("admit", slot, len(m)))
        return slot

    def step(self, n):
        self.log.append(("step", tuple(sorted(self.live))))

    def sync(self):
        return 0

    def get_state(self, slot):
        n = self.live[slot]
        return np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n), np.zeros(n), np.ones(n, dtype=np.int32)

    def energy(self, slot):
        return -1.0, np.zeros(3)

    def stats(self, slot):
        return FakeStats()

    def evict(self, slot):
        self.live.pop(slot)
        self.free.append(slot)
        self.free.sort()
        self.log.append(("evict", slot))

    def close(self):
        pass


def _req(rid, t, n, steps):
    z = np.zeros((n, 3))
    return Request(rid=rid, arrival_s=t, x=z, v=z, m=np.ones(n), radius=np.zeros(n), n_massive=n, steps=steps)


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001
        return self.t


def test_admission_respects_every_capacity_and_evicts_on_budget():
    pool = FakePool(3)
    srv = Server(max_systems=3, max_particles=3 * 64, max_tiles=10_000, pool=pool,
                 footprint=lambda r: 100, hbm_budget_bytes=250, clock=FakeClock())
    reqs = [_req(0, 0.0, 64, 3), _req(1, 0.0, 64, 1), _req(2, 0.0, 64, 2), _req(3, 0.0, 32, 1)]
    results, stats = srv.run(reqs)
    assert sorted(r.rid for r in results) == [0, 1, 2, 3]
    # the HBM budget (250 B at 100 B each) allows two residents at a time, never three
    resident = set()
    peak = 0
    for ev in pool.log:
        if ev[0] == "admit":
            resident.add(ev[1])
        elif ev[0] == "evict":
            resident.discard(ev[1])
        peak = max(peak, len(resident))
    assert peak == 2 and stats.max_resident == 2
    # every request ran exactly its budget
    assert {r.rid: r.steps for r in results} == {0: 3, 1: 1, 2: 2, 3: 1}
    assert stats.sim_steps == 7
    assert srv.used_particles == 0 and srv.used_tiles == 0 and srv.used_bytes == 0


def test_first_come_first_served_and_late_arrivals_wait():
    pool = FakePool(1)
    clock = FakeClock()
    srv = Server(max_systems=1, max_particles=1024, max_tiles=10_000, pool=pool, clock=clock,
                 footprint=lambda r: 1)
    reqs = [_req(0, 0.0, 32, 2), _req(1, 0.0005, 32, 1), _req(2, 0.5, 32, 1)]
    results, stats = srv.run(reqs)
    assert [r.rid for r in results] == [0, 1, 2]
    admits = [ev[1] for ev in pool.log if ev[0] == "admit"]
    assert admits == [0, 0, 0]                  # one slot, reused in arrival order
    assert results[2].admitted_s >= 0.5
