"""Removal of bodies by heliocentric distance (rmin: the star, rmax: ejection) against the oracle,
through the C ABI (needs a GB300).

A 300-body disk (5-20 AU) with two massive bodies and one field particle beyond rmax = 30 AU and a
field particle inside rmin = 2 AU: the four leave at the end of the first step on both sides, the
massive ones taking their momentum out of the closing sun drift.  Bars: alive flags and masses
bit-exact, removal counts equal, positions to 1e-12 relative or within 100x the spread of the
oracle's rounding-level sensitivity twin, each step from the same input.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from paper_2304_07325_gb300 import disk  # noqa: E402

G = 4.0 * math.pi ** 2
LIMITS = dict(rmin=2.0, rmax=30.0)


@pytest.fixture(scope="module")
def sy():
    import paper_2304_07325_gb300 as m
    from paper_2304_07325_gb300 import build
    build.build()
    return m


def _system():
    d = disk.planetesimal_disk(300, 4201)

    def circ(r, phase):
        c, s = math.cos(phase), math.sin(phase)
        return [r * c, r * s, 0.0], [-math.sqrt(G / r) * s, math.sqrt(G / r) * c, 0.0]

    extra_m = [circ(35.0, 0.3), circ(41.0, 2.1)]
    extra_f = [circ(50.0, 4.0), circ(1.0, 1.0)]
    x = np.vstack([d.x] + [[p] for p, _ in extra_m] + [[p] for p, _ in extra_f])
    v = np.vstack([d.v] + [[q] for _, q in extra_m] + [[q] for _, q in extra_f])
    m = np.concatenate([d.m, [1e-8, 2e-8], [0.0, 0.0]])
    rad = np.concatenate([d.radius, [1e-6, 1e-6], [0.0, 0.0]])
    return x, v, m, rad, 302


def test_removal_matches_the_oracle(orc, sy):
    x, v, m, rad, nm = _system()
    ref = orc.OracleSim(x, v, m, rad, n_massive=nm, params=orc.make_params(**LIMITS))
    gpu = sy.System(x, v, m, rad, n_massive=nm, params=sy.default_params(**LIMITS))
    assert np.array_equal(gpu.rhill(), ref.rhill)
    removed = 0
    for step in range(3):
        twin = orc.OracleSim(x, v, m, rad, n_massive=nm, rhill=ref.rhill,
                             params=orc.make_params(noise=1, **LIMITS))
        twin.set_state(ref.x, ref.v)
        for a in ("alive", "m", "radius", "rhill"):
            getattr(twin, a)[...] = getattr(ref, a)
        gpu.set_state(ref.x, ref.v)
        assert ref.step(1) >= 0 and twin.step(1) >= 0
        removed += ref.removals
        gpu.step(1)
        assert gpu.sync() >= 0
        xg, vg, mg, rg, ag = gpu.get_state()
        assert np.array_equal(ag, ref.alive) and np.array_equal(mg, ref.m)
        assert gpu.stats().removals == removed
        norm = np.linalg.norm(ref.x, axis=1)
        rel = np.linalg.norm(xg - ref.x, axis=1) / norm
        spread = np.linalg.norm(twin.x - ref.x, axis=1) / norm
        bad = np.where(rel > np.maximum(1e-12, 100.0 * spread))[0]
        assert len(bad) == 0, [(int(i), rel[i], spread[i]) for i in bad[:5]]
    assert removed == 4
    assert list(np.where(ref.alive == 0)[0]) == [300, 301, 302, 303]
    # the removed bodies no longer count: energies agree
    E_ref, L_ref = ref.energy()
    E_gpu, L_gpu = gpu.energy()
    assert abs(E_gpu - E_ref) <= 1e-12 * abs(E_ref)
    gpu.close()


def test_removal_limits_are_validated(sy):
    x, v, m, rad, nm = _system()
    for bad in (dict(rmin=-1.0), dict(rmax=-2.0), dict(rmin=5.0, rmax=4.0), dict(rmax=float("inf"))):
        with pytest.raises(sy.SymbaError) as e:
            sy.System(x, v, m, rad, n_massive=nm, params=sy.default_params(**bad))
        assert e.value.code == sy.SYMBA_E_INVAL


def test_without_limits_no_body_leaves(sy):
    x, v, m, rad, nm = _system()
    s = sy.System(x, v, m, rad, n_massive=nm)
    s.step(2)
    assert s.sync() >= 0
    assert s.stats().removals == 0 and s.get_state()[4].all()
    s.close()


def test_removal_limits_are_per_system_in_a_pool(sy):
    """Two systems in one pool with different limits (and one without): each removes exactly what
    it removes alone, bit for bit, so the limits travel with the system."""
    x, v, m, rad, nm = _system()
    specs = [dict(rmin=2.0, rmax=30.0), dict(rmax=45.0), dict()]
    alone = []
    for lim in specs:
        s = sy.System(x, v, m, rad, n_massive=nm, params=sy.default_params(**lim))
        s.step(2)
        assert s.sync() >= 0
        alone.append((s.get_state(), s.stats().removals))
        s.close()
    pool = sy.Pool(4, 4 * (len(m) + 64), 4 * ((len(m) + 31) // 32) ** 2)
    slots = [pool.admit(x, v, m, rad, n_massive=nm, params=sy.default_params(**lim)) for lim in specs]
    pool.step(2)
    assert pool.sync() >= 0
    for slot, ((xa, va, ma, ra, aa), removed) in zip(slots, alone):
        xp, vp, mp, rp, ap = pool.get_state(slot)
        assert np.array_equal(xp, xa) and np.array_equal(vp, va) and np.array_equal(ap, aa)
        assert pool.stats(slot).removals == removed
    assert [r for _, r in alone] == [4, 1, 0]
    pool.close()
