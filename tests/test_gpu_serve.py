"""The serving loop on the GPU: requests arriving while others run are admitted as room frees
up, overlap on the device, and each result equals the same simulation run alone, bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone():
    import paper_2304_07325_gb300 as sy
    from paper_2304_07325_gb300 import build
    from paper_2304_07325_gb300.serve import Server, poisson_requests

    build.build()
    reqs = poisson_requests(6, rate_per_s=200.0, seed=3100, n_lo=200, n_hi=1500, steps_lo=2, steps_hi=6)
    # room for three systems at a time: later arrivals wait for evictions
    srv = Server(max_systems=3, max_particles=3 * 1536, max_tiles=3 * 48 * 49 // 2)
    results, stats = srv.run(reqs)
    srv.close()
    assert sorted(r.rid for r in results) == list(range(6))
    assert stats.max_resident >= 2
    for res in results:
        req = reqs[res.rid]
        assert res.steps == req.steps and res.status == 0
        alone = sy.System(req.x, req.v, req.m, req.radius, n_massive=req.n_massive)
        alone.step(req.steps)
        assert alone.sync() >= 0
        x, v, m, r, a = alone.get_state()
        assert np.array_equal(x, res.x) and np.array_equal(v, res.v) and np.array_equal(a, res.alive)
        assert alone.energy()[0] == res.energy[0]
        alone.close()


def test_concurrent_server_results_equal_alone():
    """The concurrent server (a resident single-system pool per slot, one step in flight per
    request): every result equals the same simulation run alone, bit for bit."""
    import paper_2304_07325_gb300 as sy
    from paper_2304_07325_gb300 import build
    from paper_2304_07325_gb300.serve import ConcurrentServer, poisson_requests

    build.build()
    reqs = poisson_requests(6, rate_per_s=200.0, seed=3200, n_lo=200, n_hi=1500, steps_lo=2, steps_hi=6)
    srv = ConcurrentServer(3, max(len(r.m) for r in reqs))
    results, stats = srv.run(reqs)
    srv.close()
    assert sorted(r.rid for r in results) == list(range(6))
    assert stats.max_resident >= 2 and stats.sim_steps == sum(r.steps for r in reqs)
    for res in results:
        req = reqs[res.rid]
        assert res.steps == req.steps and res.status == 0
        alone = sy.System(req.x, req.v, req.m, req.radius, n_massive=req.n_massive)
        alone.step(req.steps)
        assert alone.sync() >= 0
        x, v, m, r, a = alone.get_state()
        assert np.array_equal(x, res.x) and np.array_equal(v, res.v) and np.array_equal(a, res.alive)
        assert alone.energy()[0] == res.energy[0]
        alone.close()
