"""GPU path vs the oracle, element by element, through the C ABI (needs a GB300).

Bars: bit-exact for the encounter pair lists, their groups and every exactly-rounded quantity
(initial barycentric velocities, energy and angular momentum of identical states); positions to
1e-12 relative after 100 FP64 steps on the 1,000-body disk; one step of the 10,000-body disk
(the benchmark size) from the same input.
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


def _pair(orc, sy, d, params=None, oparams=None, **kw):
    """The oracle and the GPU path on the same input, each computing its own Hill radii (the
    product's default set-up), which must agree bit for bit."""
    ref = orc.OracleSim(d.x, d.v, d.m, d.radius, n_massive=d.n_massive, params=oparams, **kw)
    gpu = sy.System(d.x, d.v, d.m, d.radius, n_massive=d.n_massive, params=params)
    assert np.array_equal(gpu.rhill(), ref.rhill)
    return ref, gpu


def _same_groups(ref, gpu):
    p_ref, g_ref, ng_ref = ref.enc_groups()
    p_gpu, g_gpu, ng_gpu = gpu.enc_groups()
    assert ng_ref == ng_gpu
    assert np.array_equal(p_ref, p_gpu)
    assert np.array_equal(g_ref, g_gpu)
    return len(p_ref)


def test_init_is_bit_exact(orc, sy):
    d = disk.planetesimal_disk(1000, 1000)
    ref = orc.OracleSim(d.x, d.v, d.m, d.radius)
    gpu = sy.System(d.x, d.v, d.m, d.radius)
    x, v, m, r, a = gpu.get_state()
    assert np.array_equal(x, ref.x) and np.array_equal(v, ref.v)
    assert np.array_equal(m, ref.m) and np.all(a == 1)
    # Hill radii a (m / 3 m0)^{1/3}: both sides take the correctly rounded cube root, so they
    # agree bit for bit (the library cube roots differ in the last bit for about half the masses)
    assert np.array_equal(gpu.rhill(), ref.rhill)
    assert np.all(ref.rhill > 0.0)


def test_energy_and_momentum_bit_exact_on_identical_state(orc, sy):
    for n, nf, seed in ((1000, 0, 1000), (300, 700, 5), (1, 0, 9)):
        d = disk.planetesimal_disk(n, seed, n_field=nf)
        ref, gpu = _pair(orc, sy, d)
        E_ref, L_ref = ref.energy()
        E_gpu, L_gpu = gpu.energy()
        assert E_gpu == E_ref and np.array_equal(L_gpu, L_ref), (E_gpu, E_ref)


def test_one_step_encounters_bit_exact_and_positions(orc, sy):
    d = disk.planetesimal_disk(1000, 1000)
    ref, gpu = _pair(orc, sy, d)
    assert ref.step(1) >= 0
    gpu.step(1)
    assert gpu.sync() >= 0
    npairs = _same_groups(ref, gpu)
    assert npairs > 50
    x, v, m, r, a = gpu.get_state()
    assert np.abs(x - ref.x).max() <= 1e-13 * np.abs(ref.x).max()
    assert np.abs(v - ref.v).max() <= 1e-12 * np.abs(ref.v).max()


@pytest.mark.parametrize("k", [3, 17, 41])
def test_encounters_bit_exact_from_oracle_snapshots(orc, sy, k):
    """The oracle runs k steps; the GPU starts from that state; both take one step."""
    d = disk.planetesimal_disk(1000, 1000)
    ref, gpu = _pair(orc, sy, d)
    assert ref.step(k) >= 0
    gpu.set_state(ref.x, ref.v)
    assert ref.step(1) >= 0
    gpu.step(1)
    assert gpu.sync() >= 0
    _same_groups(ref, gpu)


def _twin(orc, d, ref):
    """The sensitivity twin: the oracle with rounding-level perturbations at every recursion
    sub-step (test hook), started from the same state."""
    tw = orc.OracleSim(d.x, d.v, d.m, d.radius, n_massive=d.n_massive, rhill=ref.rhill,
                       params=orc.make_params(noise=1))
    tw.set_state(ref.x, ref.v)
    return tw


def _check_positions(x, ref, twin, tol=1e-12, factor=100.0):
    """Every body within tol relative, or -- for the bodies whose close encounters amplify
    rounding-level differences -- within factor x the spread the sensitivity twin shows."""
    norm = np.linalg.norm(ref.x, axis=1)
    rel = np.linalg.norm(x - ref.x, axis=1) / norm
    spread = np.linalg.norm(twin.x - ref.x, axis=1) / norm
    bound = np.maximum(tol, factor * spread)
    bad = np.where(rel > bound)[0]
    assert len(bad) == 0, [(int(i), rel[i], spread[i]) for i in bad[:5]]
    return rel, spread


def test_100_steps_positions_1e12(orc, sy):
    """100 FP64 steps of the 1,000-body disk: 1e-12 relative for every body except those whose
    deep encounters amplify rounding differences, which must stay within 100x the spread of the
    sensitivity twin (the oracle perturbed at the rounding level at every recursion sub-step)."""
    d = disk.planetesimal_disk(1000, 1000)
    ref, gpu = _pair(orc, sy, d)
    twin = _twin(orc, d, ref)
    for s in range(100):
        assert ref.step(1) >= 0
        assert twin.step(1) >= 0
    gpu.step(100)
    assert gpu.sync() >= 0
    x, v, m, r, a = gpu.get_state()
    assert np.array_equal(a, ref.alive)
    rel, spread = _check_positions(x, ref, twin)
    # printed so that a regression shows before it fails: the share of bodies at 1e-12, and how
    # far the others are from the twin's spread
    frac = float(np.mean(rel <= 1e-12))
    over = rel > 1e-12
    worst = float(np.max(rel[over] / np.maximum(spread[over], 1e-300))) if over.any() else 0.0
    print(f"100 steps, N = 1,000: {100 * frac:.1f} % of bodies within 1e-12; the other {int(over.sum())} "
          f"within {worst:.2f}x the twin's spread (bound 100x); median {np.median(rel):.2e}, max {rel.max():.2e}")
    assert frac > 0.9
    E_ref, _ = ref.energy()
    E_gpu, _ = gpu.energy()
    assert abs(E_gpu - E_ref) <= 1e-12 * abs(E_ref)


def test_single_steps_from_oracle_states_positions(orc, sy):
    """Each GPU step starts from the oracle's state: one step agrees to 1e-12 (chaos-aware)."""
    d = disk.planetesimal_disk(1000, 1000)
    ref, gpu = _pair(orc, sy, d)
    for s in range(30):
        gpu.set_state(ref.x, ref.v)
        twin = _twin(orc, d, ref)
        twin.alive[...] = ref.alive
        twin.m[...] = ref.m
        twin.radius[...] = ref.radius
        twin.rhill[...] = ref.rhill
        assert ref.step(1) >= 0
        assert twin.step(1) >= 0
        gpu.step(1)
        assert gpu.sync() >= 0
        x, v, m, r, a = gpu.get_state()
        assert np.array_equal(a, ref.alive)
        _check_positions(x, ref, twin)


@pytest.mark.parametrize("n,nf", [(1, 0), (2, 0), (33, 0), (97, 31), (0, 64), (64, 0), (200, 1000)])
def test_edge_sizes(orc, sy, n, nf):
    """Ragged tails, a single body, no massive body, mostly field particles."""
    if n == 0:
        d = disk.planetesimal_disk(1, 3, n_field=nf)
        d.x, d.v, d.m, d.radius, d.n_massive = d.x[1:], d.v[1:], d.m[1:], d.radius[1:], 0
    else:
        d = disk.planetesimal_disk(n, 3 + n, n_field=nf)
    ref, gpu = _pair(orc, sy, d)
    for _ in range(5):
        assert ref.step(1) >= 0
        gpu.step(1)
        assert gpu.sync() >= 0
        _same_groups(ref, gpu)
    x, v, m, r, a = gpu.get_state()
    assert np.abs(x - ref.x).max() <= 1e-12 * max(1.0, np.abs(ref.x).max())


def test_dense_cluster_many_encounters(orc, sy):
    """A compact clump: most pairs flagged, large groups, deep recursion and mergers."""
    rng = np.random.default_rng(12)
    n = 48
    d = disk.planetesimal_disk(n, 77)
    d.x = np.array([10.0, 0.0, 0.0]) + rng.normal(scale=0.05, size=(n, 3)) * [1, 1, 0.01]
    vc = np.array([0.0, 2.0 * np.pi / np.sqrt(10.0), 0.0])
    d.v = vc + rng.normal(scale=0.01, size=(n, 3)) * [1, 1, 0.01]
    d.radius = d.radius * 50.0
    ref, gpu = _pair(orc, sy, d)
    # one step from the same input: identical level-0 encounters, depth and mergers
    assert ref.step(1) >= 0
    gpu.step(1)
    assert gpu.sync() >= 0
    _same_groups(ref, gpu)
    st = gpu.stats()
    assert st.max_depth == ref.max_depth_seen and st.merges == ref.mergers
    x, v, m, r, a = gpu.get_state()
    assert np.array_equal(a, ref.alive)
    # then each step from the oracle's state
    for _ in range(3):
        gpu.set_state(ref.x, ref.v)
        assert ref.step(1) >= 0
        gpu.step(1)
        assert gpu.sync() >= 0
        _same_groups(ref, gpu)


def test_benchmark_size_one_step(orc, sy):
    """The 10,000-body disk the benchmark times: one step from the same input."""
    d = disk.planetesimal_disk(10000, 1002)
    ref, gpu = _pair(orc, sy, d)
    assert ref.step(1) >= 0
    gpu.step(1)
    assert gpu.sync() >= 0
    npairs = _same_groups(ref, gpu)
    assert npairs > 5000
    x, v, m, r, a = gpu.get_state()
    assert np.array_equal(a, ref.alive)
    twin = _twin(orc, d, ref)
    twin.set_state(d.x, orc.OracleSim(d.x, d.v, d.m, d.radius, rhill=ref.rhill).v)
    assert twin.step(1) >= 0
    rel, spread = _check_positions(x, ref, twin)
    assert np.mean(rel <= 1e-12) > 0.99
    st = gpu.stats()
    assert st.max_depth == ref.max_depth_seen


@pytest.mark.parametrize("n,seed", [(5000, 1001), (10000, 1002)])
def test_benchmark_sizes_steps_from_oracle_states(orc, sy, n, seed):
    """Both benchmark sizes (N = 5,000 and 10,000): two steps, each started from the oracle's
    state, through the graph-replayed step the benchmark times; encounters bit-exact, positions
    1e-12 relative (chaos-aware), same mergers."""
    d = disk.planetesimal_disk(n, seed)
    ref, gpu = _pair(orc, sy, d)
    for _ in range(2):
        gpu.set_state(ref.x, ref.v)
        twin = _twin(orc, d, ref)
        twin.alive[...] = ref.alive
        twin.m[...] = ref.m
        twin.radius[...] = ref.radius
        twin.rhill[...] = ref.rhill
        assert ref.step(1) >= 0 and twin.step(1) >= 0
        gpu.step(1)
        assert gpu.sync() >= 0
        _same_groups(ref, gpu)
        x, v, m, r, a = gpu.get_state()
        assert np.array_equal(a, ref.alive) and np.array_equal(m, ref.m)
        rel, spread = _check_positions(x, ref, twin)
        assert np.mean(rel <= 1e-12) > 0.99
