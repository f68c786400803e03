"""Launch schedules and their autotuner on the GPU.

The pair kick is a queue of 32 x 32 tiles and the group recursion a queue of encounter groups,
both drained by persistent warps; how the queues are cut and ordered (CTAs per SM, tiles per
grab, recursion CTAs per SM, group order) must change no bit of any result, and the autotuner
must leave every system as it found it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from paper_2304_07325_gb300 import disk  # noqa: E402

DISKS = [(1000, 4101), (1500, 4102), (700, 4103)]


@pytest.fixture(scope="module")
def sy():
    import paper_2304_07325_gb300 as m
    from paper_2304_07325_gb300 import build
    build.build()
    return m


def _pool(sy, precision):
    ds = [disk.planetesimal_disk(n, seed) for n, seed in DISKS]
    tiles = sum(((d.n + 31) // 32) ** 2 for d in ds)
    pool = sy.Pool(4, sum(d.n for d in ds) + 1024, tiles, precision=precision)
    slots = [pool.admit(d.x, d.v, d.m, d.radius) for d in ds]
    return pool, slots


def _states(pool, slots):
    return [pool.get_state(s) for s in slots]


def _same(a, b):
    return all(all(np.array_equal(u, v) for u, v in zip(sa, sb)) for sa, sb in zip(a, b))


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_every_schedule_gives_the_same_steps(sy, precision):
    ref, slots = _pool(sy, precision)
    ref.step(4)
    assert ref.sync() >= 0
    want = _states(ref, slots)
    subs = [ref.stats(s).substeps for s in slots]
    for sched in (dict(kick_blocks_per_sm=1, kick_tiles_per_item=1, rec_blocks_per_sm=2, group_order=1),
                  dict(kick_blocks_per_sm=2, kick_tiles_per_item=16, rec_blocks_per_sm=1, group_order=1),
                  dict(kick_blocks_per_sm=1, kick_tiles_per_item=64, rec_blocks_per_sm=2, group_order=0)):
        pool, sl = _pool(sy, precision)
        pool.schedule = sched
        assert pool.schedule == sched
        pool.step(4)
        assert pool.sync() >= 0
        assert _same(_states(pool, sl), want), sched
        assert [pool.stats(s).substeps for s in sl] == subs
        pool.close()
    ref.close()


def test_autotune_leaves_the_pool_as_it_was(sy):
    pool, slots = _pool(sy, 0)
    twin, tslots = _pool(sy, 0)
    pool.step(2)
    twin.step(2)
    assert pool.sync() >= 0 and twin.sync() >= 0
    before = _states(pool, slots)
    st_before = [(pool.stats(s).substeps, pool.stats(s).n_pairs, pool.stats(s).status) for s in slots]
    r = pool.autotune(reps=2)
    assert r["identical"] == 1
    assert r["kick_candidates"] >= 5 and r["recursion_candidates"] == 4
    assert r["kick_ms"] <= r["kick_ms_before"] and r["recursion_ms"] <= r["recursion_ms_before"]
    assert pool.schedule == r["chosen"]
    assert _same(_states(pool, slots), before)
    assert [(pool.stats(s).substeps, pool.stats(s).n_pairs, pool.stats(s).status) for s in slots] == st_before
    # the tuned pool keeps stepping exactly like an untuned one
    pool.step(3)
    twin.step(3)
    assert pool.sync() >= 0 and twin.sync() >= 0
    assert _same(_states(pool, slots), _states(twin, tslots))
    pool.close()
    twin.close()


def test_autotune_through_a_context(sy):
    d = disk.planetesimal_disk(2000, 4104)
    s = sy.System(d.x, d.v, d.m, d.radius)
    s.step(1)
    assert s.sync() >= 0
    x0 = s.get_state()
    r = s.autotune(reps=1)
    assert r["identical"] == 1 and r["recursion_candidates"] == 4
    assert all(np.array_equal(u, v) for u, v in zip(s.get_state(), x0))
    s.close()


def test_empty_pool_and_bad_schedules(sy):
    pool = sy.Pool(2, 2048, 64)
    r = pool.autotune(reps=1)
    assert r["kick_candidates"] == 0 and r["recursion_candidates"] == 0 and r["identical"] == 1
    sched = pool.schedule
    for bad in (dict(rec_blocks_per_sm=3), dict(rec_blocks_per_sm=0), dict(kick_blocks_per_sm=0),
                dict(kick_blocks_per_sm=64), dict(kick_tiles_per_item=0), dict(kick_tiles_per_item=65),
                dict(group_order=2)):
        with pytest.raises(sy.SymbaError) as e:
            pool.schedule = bad
        assert e.value.code == sy.SYMBA_E_INVAL
    assert pool.schedule == sched
    with pytest.raises(sy.SymbaError):
        pool.autotune(reps=0)
    pool.close()
