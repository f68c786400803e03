"""The single-pair path of the group recursion (a lone pair below some level runs packed across
the warp) against the oracle, through the C ABI (needs a GB300).

The path takes every sub-step of a group whose F_{k-1} holds one pair, so these cases spend
nearly all their sub-steps in it: a bound pair inside a 5-body group of the 10,000-body disk
(depth 12), an isolated tight binary, and a pair on a collision course (the path hands the
contact check back to the general path, which merges the bodies).  Bars: the recursion takes the
same sub-steps as the oracle (same decisions at every level), positions agree to 1e-12
relative or within 100x the spread of the oracle's rounding-level sensitivity twin.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from paper_2304_07325_gb300 import disk  # noqa: E402

BOUND_PAIR_GROUP = [1244, 3406, 4643, 5122, 9870]    # 10,000-body disk, seed 1002


@pytest.fixture(scope="module")
def sy():
    import paper_2304_07325_gb300 as m
    from paper_2304_07325_gb300 import build
    build.build()
    return m


def _twin(orc, x, v, m, radius, rhill, ref):
    tw = orc.OracleSim(x, v, m, radius, rhill=rhill, params=orc.make_params(noise=1))
    tw.set_state(ref.x, ref.v)
    return tw


def _close(x, ref, twin, tol=1e-12, factor=100.0):
    norm = np.linalg.norm(ref.x, axis=1)
    rel = np.linalg.norm(x - ref.x, axis=1) / norm
    spread = np.linalg.norm(twin.x - ref.x, axis=1) / norm
    bad = np.where(rel > np.maximum(tol, factor * spread))[0]
    assert len(bad) == 0, [(int(i), rel[i], spread[i]) for i in bad]
    return rel


def _run(orc, sy, x, v, m, radius, steps):
    ref = orc.OracleSim(x, v, m, radius)
    gpu = sy.System(x, v, m, radius)
    assert np.array_equal(gpu.rhill(), ref.rhill)
    out = []
    for _ in range(steps):
        twin = _twin(orc, x, v, m, radius, ref.rhill, ref)
        twin.alive[...] = ref.alive
        twin.m[...] = ref.m
        twin.radius[...] = ref.radius
        twin.rhill[...] = ref.rhill
        gpu.set_state(ref.x, ref.v)
        assert ref.step(1) >= 0 and twin.step(1) >= 0
        gpu.step(1)
        assert gpu.sync() >= 0
        st = gpu.stats()
        xg, vg, mg, rg, ag = gpu.get_state()
        assert np.array_equal(ag, ref.alive)
        out.append((st, sum(ref.level_calls[1:]), ref.max_depth_seen, _close(xg, ref, twin)))
    return ref, gpu, out


def _binary():
    m = np.array([3e-9, 2e-9])
    G = 4.0 * np.pi ** 2
    sep = 1e-4
    vrel = np.sqrt(G * m.sum() / sep)
    x = np.array([[1.0, 0.0, 0.0], [1.0 + sep, 0.0, 0.0]])
    vc = np.array([0.0, 2.0 * np.pi, 0.0])
    v = np.array([vc - [0.0, vrel * m[1] / m.sum(), 0.0], vc + [0.0, vrel * m[0] / m.sum(), 0.0]])
    return x, v, m, np.array([2e-7, 2e-7])


def test_bound_pair_group(orc, sy):
    d = disk.planetesimal_disk(10000, 1002)
    g = BOUND_PAIR_GROUP
    ref, gpu, out = _run(orc, sy, d.x[g], d.v[g], d.m[g], d.radius[g], 2)
    st, calls, depth, rel = out[0]
    assert depth >= 10 and st.max_depth == depth
    assert st.substeps == calls > 10000
    assert st.pair_substeps > 0.9 * st.substeps      # below level 2 the pair is alone
    E_ref, _ = ref.energy()
    E_gpu, _ = gpu.energy()
    assert abs(E_gpu - E_ref) <= 1e-12 * abs(E_ref)


def test_isolated_tight_binary(orc, sy):
    """Two planetesimals 1e-4 AU apart on a mutual orbit at 1 AU: deep recursion every step."""
    x, v, m, radius = _binary()
    ref, gpu, out = _run(orc, sy, x, v, m, radius, 3)
    for st, calls, depth, rel in out:
        assert depth >= 6 and st.max_depth == depth and st.substeps == calls
    assert gpu.stats().merges == 0 and ref.mergers == 0


def test_pair_on_collision_course_merges(orc, sy):
    """Two bodies falling onto each other: the contact happens deep in the recursion; the bodies
    merge in the same sub-step as in the oracle (one survivor, same mass and momentum)."""
    m = np.array([3e-9, 2e-9])
    x = np.array([[1.0, 0.0, 0.0], [1.0 + 2e-4, 1e-9, 0.0]])
    vc = np.array([0.0, 2.0 * np.pi, 0.0])
    v = np.array([vc + [0.02, 0.0, 0.0], vc - [0.02, 0.0, 0.0]])
    radius = np.array([1e-5, 1e-5])
    ref = orc.OracleSim(x, v, m, radius)
    gpu = sy.System(x, v, m, radius)
    assert np.array_equal(gpu.rhill(), ref.rhill)
    assert ref.step(1) >= 0
    gpu.step(1)
    assert gpu.sync() >= 0
    assert ref.mergers == 1 and gpu.stats().merges == 1
    xg, vg, mg, rg, ag = gpu.get_state()
    assert np.array_equal(ag, ref.alive)
    assert np.array_equal(mg, ref.m)
    k = int(np.argmax(ag))
    assert np.linalg.norm(xg[k] - ref.x[k]) <= 1e-12 * np.linalg.norm(ref.x[k])
    assert np.linalg.norm(vg[k] - ref.v[k]) <= 1e-10 * np.linalg.norm(ref.v[k])


def test_depth_limit_inside_the_pair_path(orc, sy):
    """The binary needs depth 7; with max_depth = 4 the path reports SYMBA_E_DEPTH and, like the
    oracle, drifts the pair at the deepest allowed level: same sub-steps, same positions."""
    x, v, m, radius = _binary()
    ref = orc.OracleSim(x, v, m, radius, params=orc.make_params(max_depth=4))
    gpu = sy.System(x, v, m, radius, params=sy.default_params(max_depth=4))
    twin = orc.OracleSim(x, v, m, radius, rhill=ref.rhill, params=orc.make_params(max_depth=4, noise=1))
    assert ref.step(1) == orc.E_DEPTH
    twin.step(1)
    gpu.step(1)
    with pytest.raises(sy.SymbaError) as e:
        gpu.sync()
    assert e.value.code == sy.SYMBA_E_DEPTH
    # the sticky status makes the synchronising calls report the error; the data is still copied
    st = gpu.stats()
    assert st.status == sy.SYMBA_E_DEPTH
    assert st.max_depth == ref.max_depth_seen == 4
    assert st.substeps == sum(ref.level_calls[1:])
    xg, vg = np.zeros((2, 3)), np.zeros((2, 3))
    assert sy.lib().symba_get_state(gpu._h, sy._ptr(xg), sy._ptr(vg), None, None, None) == sy.SYMBA_E_DEPTH
    _close(xg, ref, twin)


def test_substep_budget_inside_the_pair_path(sy):
    """A sub-step budget far below the binary's 21,844 sub-steps per step: SYMBA_E_DEPTH, and the
    context is usable again once a state is set."""
    x, v, m, radius = _binary()
    s = sy.System(x, v, m, radius, params=sy.default_params(max_substeps=100))
    s.step(1)
    with pytest.raises(sy.SymbaError) as e:
        s.sync()
    assert e.value.code == sy.SYMBA_E_DEPTH
    assert s.stats().substeps == 101
    s.set_state(x, v)
    assert s.sync() == sy.SYMBA_OK
    s.close()
