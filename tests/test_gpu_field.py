"""The field rectangle (Sec. 2: field particles interact only with massive bodies) on the GPU,
against the oracle (needs a GB300).

Blocks of field particles beyond the last block holding a massive body are rows of the
rectangle N_m x N_field, kicked by k_field_* (the trapezoid's tiles cover the massive column
blocks only).  Each step starts the GPU from the oracle's state: the level-0 encounter pairs
and groups must be bit-exact (the fused check of kick 1 runs in the rectangle too), positions
within 1e-12 relative (chaos-aware), and field particles' velocities, which the rectangle alone
kicks, within 1e-12 of each body's speed in FP64 and within the mixed path's stated bound in
mixed precision.  Sizes: the benchmark's 300 + 3,000 shape, a ragged boundary block (301 + 2,999),
N_m a multiple of 32 (320 + 700) and no massive body at all (0 + 96).
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


def _twin(orc, d, ref):
    tw = orc.OracleSim(d.x, d.v, d.m, d.radius, n_massive=d.n_massive, rhill=ref.rhill,
                       params=orc.make_params(noise=1))
    tw.set_state(ref.x, ref.v)
    for a in ("alive", "m", "radius", "rhill"):
        getattr(tw, a)[...] = getattr(ref, a)
    return tw


@pytest.mark.parametrize("nm,nf,prec", [(300, 3000, 0), (301, 2999, 0), (320, 700, 0), (0, 96, 0),
                                        (300, 3000, 1), (301, 2999, 1)])
def test_field_rectangle_steps_from_oracle_states(orc, sy, nm, nf, prec):
    d = disk.planetesimal_disk(nm, 1003, n_field=nf)
    ref = orc.OracleSim(d.x, d.v, d.m, d.radius, n_massive=nm)
    gpu = sy.System(d.x, d.v, d.m, d.radius, n_massive=nm, params=sy.default_params(precision=prec))
    assert np.array_equal(gpu.rhill(), ref.rhill)
    field = np.arange(nm, nm + nf)
    pairs_total, worst_v = 0, 0.0
    for step in range(3):
        tw = _twin(orc, d, ref)
        gpu.set_state(ref.x, ref.v)
        assert ref.step(1) >= 0 and tw.step(1) >= 0
        gpu.step(1)
        assert gpu.sync() >= 0
        p_ref, g_ref, ng_ref = ref.enc_groups()
        p_gpu, g_gpu, ng_gpu = gpu.enc_groups()
        assert ng_gpu == ng_ref and np.array_equal(p_gpu, p_ref) and np.array_equal(g_gpu, g_ref), step
        pairs_total += len(p_ref)
        x, v, m, r, a = gpu.get_state()
        assert np.array_equal(a, ref.alive)
        norm = np.linalg.norm(ref.x, axis=1)
        rel = np.linalg.norm(x - ref.x, axis=1) / norm
        spread = np.linalg.norm(tw.x - ref.x, axis=1) / norm
        tol = 1e-12 if prec == 0 else 1e-10
        bad = np.where(rel > np.maximum(tol, 100.0 * spread))[0]
        assert len(bad) == 0, [(int(i), rel[i], spread[i]) for i in bad[:5]]
        # field particles in no encounter: their velocity change is the two rectangle kicks and
        # the Kepler drift
        quiet = np.setdiff1d(field, p_ref.reshape(-1)) if len(p_ref) else field
        vrel = np.linalg.norm(v[quiet] - ref.v[quiet], axis=1) / np.linalg.norm(ref.v[quiet], axis=1)
        worst_v = max(worst_v, float(vrel.max()) if len(vrel) else 0.0)
    print(f"N_m={nm} + {nf} field, precision {prec}: {pairs_total} level-0 pairs over 3 steps; "
          f"field particles' velocities within {worst_v:.2e} relative")
    assert worst_v < (1e-14 if prec == 0 else 1e-11)
    if nm >= 300:
        assert pairs_total > 0
