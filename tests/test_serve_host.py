"""Host logic of the serving loop (admission, eviction, capacity accounting) against a fake pool
(CPU only)."""
import numpy as np

from paper_2304_07325_gb300.serve import Request, Server


class FakeStats:
    status = 0
    merges = 0


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


# --------------------------------------------------------------------------------------------
# the concurrent server: one step in flight per request, no lock-step
# --------------------------------------------------------------------------------------------
class FakeOnePool:
    """A single-system pool; logs its steps with the shared log."""

    def __init__(self, k, log):
        self.k, self.log, self.n = k, log, None

    def admit(self, x, v, m, radius, n_massive=None, params=None):
        assert self.n is None
        self.n = len(m)
        self.log.append(("admit", self.k))
        return 0

    def step(self, n):
        assert n == 1 and self.n is not None
        self.log.append(("step", self.k))

    def get_state(self, slot):
        return np.zeros((self.n, 3)), np.zeros((self.n, 3)), np.zeros(self.n), np.zeros(self.n), np.ones(self.n, dtype=np.int32)

    def energy(self, slot):
        return -1.0, np.zeros(3)

    def stats(self, slot):
        return FakeStats()

    def evict(self, slot):
        self.n = None
        self.log.append(("evict", self.k))

    def close(self):
        pass


class FakeEvent:
    """Completes `lag` queries after it was recorded; checks that a step is never launched on a
    slot whose previous step is still in flight."""

    def __init__(self, lag):
        self.lag, self.left, self.recorded = lag, 0, False

    def record(self, stream):
        assert not self.recorded or self.left == 0, "a second step launched while one is in flight"
        self.recorded, self.left = True, self.lag

    def query(self):
        if self.left > 0:
            self.left -= 1
            return False
        return True


def _conc(lags):
    from paper_2304_07325_gb300.serve import ConcurrentServer
    log = []
    pools = [FakeOnePool(k, log) for k in range(len(lags))]
    events = [FakeEvent(l) for l in lags]
    srv = ConcurrentServer(len(lags), 64, pools=pools, streams=[None] * len(lags), events=events,
                           clock=FakeClock(), idle_s=0.0)
    return srv, log


def test_concurrent_server_runs_every_budget_with_one_step_in_flight():
    srv, log = _conc([0, 2, 5])
    reqs = [_req(0, 0.0, 32, 3), _req(1, 0.0, 32, 1), _req(2, 0.0, 32, 4), _req(3, 0.0, 32, 2),
            _req(4, 0.01, 32, 2)]
    results, stats = srv.run(reqs)
    assert {r.rid: r.steps for r in results} == {0: 3, 1: 1, 2: 4, 3: 2, 4: 2}
    assert stats.sim_steps == 12 and len(stats.step_ms) == 12 and stats.max_resident == 3
    # every slot is admitted, stepped and evicted in turn, never holding two requests
    for k in range(3):
        seq = [e[0] for e in log if e[1] == k]
        held = 0
        for e in seq:
            held += {"admit": 1, "evict": -1}.get(e, 0)
            assert 0 <= held <= 1
        assert held == 0
    assert sorted(srv.free) == [0, 1, 2] and not srv.active


def test_concurrent_server_a_slow_request_does_not_hold_back_a_fast_one():
    srv, log = _conc([40, 0])                   # slot 0's steps take 40 polls, slot 1's none
    reqs = [_req(0, 0.0, 32, 2), _req(1, 0.0, 32, 5)]
    results, stats = srv.run(reqs)
    assert [r.rid for r in results] == [1, 0]   # the fast request finishes first
    steps = [e[1] for e in log if e[0] == "step"]
    first_slow_done = steps.index(0, 1)         # the slow slot's second launch
    assert steps[:first_slow_done].count(1) == 5  # all five fast steps ran meanwhile


def test_concurrent_server_slots_follow_the_memory_budget(monkeypatch):
    """With a device-memory budget the server keeps as many resident slots as the budget holds
    at the largest request's footprint (no device needed: the pools are replaced)."""
    import paper_2304_07325_gb300.serve as serve
    made = []

    class P:
        def __init__(self, *a, **k):
            made.append(a)

        @staticmethod
        def footprint(n, nm, params=None):
            return 1000

    class FakeTorch:
        class cuda:
            Stream = object
            Event = object

    monkeypatch.setattr(serve, "Pool", P)
    monkeypatch.setitem(__import__("sys").modules, "torch", FakeTorch)
    srv = serve.ConcurrentServer(32, 5000, hbm_budget_bytes=4500)
    assert len(srv.pools) == 4 and len(made) == 4
