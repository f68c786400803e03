"""Pools (many systems stepped by the same kernel launches) on the GPU.

Every kernel works per tile, per group or per body with a fixed summation order, so a system's
trajectory cannot depend on the other systems in the pool: the results must equal the system
integrated alone, bit for bit, including across evictions and admissions.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from paper_2304_07325_gb300 import disk  # noqa: E402


@pytest.fixture(scope="module")
def sy():
    import paper_2304_07325_gb300 as m
    from paper_2304_07325_gb300 import build
    build.build()
    return m


def _alone(sy, d, steps):
    s = sy.System(d.x, d.v, d.m, d.radius, n_massive=d.n_massive)
    s.step(steps)
    assert s.sync() >= 0
    out = s.get_state()
    E = s.energy()
    s.close()
    return out, E


def test_pool_results_equal_alone_bit_for_bit(sy):
    disks = [disk.planetesimal_disk(n, 2000 + k, n_field=nf)
             for k, (n, nf) in enumerate([(1000, 0), (333, 0), (2049, 0), (200, 800)])]
    tiles = sum(((d.n + 31) // 32) * ((d.n_massive + 31) // 32) for d in disks)
    pool = sy.Pool(8, sum(d.n for d in disks) + 1024, tiles)
    slots = [pool.admit(d.x, d.v, d.m, d.radius, n_massive=d.n_massive) for d in disks]
    pool.step(6)
    assert pool.sync() >= 0
    for d, s in zip(disks, slots):
        (xa, va, ma, ra, aa), Ea = _alone(sy, d, 6)
        x, v, m, r, a = pool.get_state(s)
        assert np.array_equal(x, xa) and np.array_equal(v, va) and np.array_equal(a, aa)
        E = pool.energy(s)
        assert E[0] == Ea[0] and np.array_equal(E[1], Ea[1])
    pool.close()


def test_pool_evict_and_admit_keep_the_others_unchanged(sy):
    a = disk.planetesimal_disk(700, 3001)
    b = disk.planetesimal_disk(500, 3002)
    c = disk.planetesimal_disk(900, 3003)
    tiles = 3 * ((900 + 31) // 32) ** 2
    pool = sy.Pool(4, 4000, tiles)
    sa = pool.admit(a.x, a.v, a.m, a.radius)
    sb = pool.admit(b.x, b.v, b.m, b.radius)
    pool.step(3)
    pool.evict(sb)
    sc = pool.admit(c.x, c.v, c.m, c.radius)
    pool.step(4)
    assert pool.sync() >= 0
    (xa, va, _, _, _), _ = _alone(sy, a, 7)
    (xc, vc, _, _, _), _ = _alone(sy, c, 4)
    x, v, *_ = pool.get_state(sa)
    assert np.array_equal(x, xa) and np.array_equal(v, va)
    x, v, *_ = pool.get_state(sc)
    assert np.array_equal(x, xc) and np.array_equal(v, vc)
    pool.close()


def test_pool_rejects_what_does_not_fit(sy):
    d = disk.planetesimal_disk(2000, 3004)
    pool = sy.Pool(2, 2100, 100)          # far too few tiles for 2,000 bodies
    with pytest.raises(sy.SymbaError):
        pool.admit(d.x, d.v, d.m, d.radius)
    small = disk.planetesimal_disk(64, 3005)
    s1 = pool.admit(small.x, small.v, small.m, small.radius)
    s2 = pool.admit(small.x, small.v, small.m, small.radius)
    with pytest.raises(sy.SymbaError):
        pool.admit(small.x, small.v, small.m, small.radius)   # no slot left
    pool.evict(s1)
    s3 = pool.admit(small.x, small.v, small.m, small.radius)
    assert s3 == s1 and s2 != s1
    pool.close()


def test_step_many_equals_each_system_alone(sy):
    """Independent contexts advanced together by symba_step_many (each on its own stream, one step
    in flight) end bit for bit where each ends alone."""
    disks = [disk.planetesimal_disk(n, 5100 + k) for k, n in enumerate([1200, 400, 2500])]
    systems = [sy.System(d.x, d.v, d.m, d.radius) for d in disks]
    assert sy.step_many(systems, 5) >= 0
    for d, s in zip(disks, systems):
        (xa, va, ma, ra, aa), Ea = _alone(sy, d, 5)
        x, v, m, r, a = s.get_state()
        assert np.array_equal(x, xa) and np.array_equal(v, va) and np.array_equal(a, aa)
        s.close()
