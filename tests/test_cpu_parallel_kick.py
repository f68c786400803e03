"""The multi-core CPU trapezoid kick (the benchmark's multi-core CPU reference point) against the
oracle's trapezoid accelerations (no GPU).

It sums in another order than the oracle (per-thread arrays added in thread order), so the bar is
rounding: every acceleration component within 1e-12 of the largest component's magnitude for its
body, whatever the thread count, on disks with massless field bodies, flagged pairs and dead
bodies.
"""
import numpy as np
import pytest

import oracle as orc_mod
from paper_2304_07325_gb300 import disk


@pytest.fixture(scope="module")
def omp():
    orc_mod.build_omp()
    return orc_mod


def _case(n, n_field, seed, dead=()):
    d = disk.planetesimal_disk(n, seed, n_field=n_field)
    sim = orc_mod.OracleSim(d.x, d.v, d.m, d.radius, n_massive=d.n_massive)
    for i in dead:
        sim.alive[i] = 0
    # flagged pairs: the disk's level-0 encounters, plus every 97th trapezoid pair with a Hill
    # sum large enough that its shell weight lies strictly between 0 and 1 for some pairs
    rng = np.random.default_rng(seed)
    nm = d.n_massive
    extra = set()
    for _ in range(200):
        i = int(rng.integers(0, nm))
        j = int(rng.integers(i + 1, sim.n)) if i + 1 < sim.n else None
        if j is not None:
            extra.add((i, j))
    sim.step(1)
    p, _, _ = sim.enc_groups()
    flagged = sorted(set(map(tuple, np.asarray(p).reshape(-1, 2).tolist())) | extra)
    return sim, np.array(flagged, dtype=np.int32).reshape(-1, 2)


@pytest.mark.parametrize("n,n_field,threads", [(300, 0, 1), (300, 0, 4), (200, 500, 3), (64, 0, 0)])
def test_parallel_kick_equals_oracle(omp, n, n_field, threads):
    sim, flagged = _case(n, n_field, 7000 + n + n_field, dead=(3, 17) if n > 20 else ())
    ref = sim.accel_trapezoid(flagged)
    a, used = omp.trap_accel_omp(sim.x, sim.m, sim.rhill, sim.alive, flagged, sim.n_massive, sim.params,
                                 threads=threads)
    assert used >= 1 and (threads == 0 or used == threads)
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    assert np.all(np.abs(a - ref) <= 1e-12 * np.maximum(scale, 1e-300))
    # dead bodies feel and exert nothing
    for i in (3, 17) if n > 20 else ():
        assert np.all(a[i] == 0.0) and np.all(ref[i] == 0.0)


def test_weights_between_zero_and_one_are_exercised(omp):
    """Some flagged pairs of the test disks sit inside the changeover shell: there the weight,
    and so the force, differs from the unweighted one (a weight dropped from the parallel kick
    would fail the comparison above)."""
    sim, flagged = _case(300, 0, 7300)
    a_w, _ = omp.trap_accel_omp(sim.x, sim.m, sim.rhill, sim.alive, flagged, sim.n_massive, sim.params)
    a_1, _ = omp.trap_accel_omp(sim.x, sim.m, sim.rhill, sim.alive, np.zeros((0, 2), np.int32),
                                sim.n_massive, sim.params)
    assert np.max(np.abs(a_w - a_1)) > 0.0
