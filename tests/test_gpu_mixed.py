"""Mixed precision: FP32 pair kick (two-float displacements, Kahan accumulation into FP64), with
FP64 state, drifts, encounter decisions and energy.  Encounter pairs and groups are FP64
decisions and stay bit-exact; positions and energy differ from the FP64 oracle by the FP32
rounding of the pair forces, at the bounds stated here."""
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


def _mixed(sy, d):
    p = sy.default_params(precision=sy.SYMBA_PRECISION_MIXED)
    return sy.System(d.x, d.v, d.m, d.radius, n_massive=d.n_massive, params=p)


def test_mixed_one_step_encounters_exact_positions_close(orc, sy):
    d = disk.planetesimal_disk(1000, 1000)
    ref = orc.OracleSim(d.x, d.v, d.m, d.radius)
    gpu = _mixed(sy, d)
    assert ref.step(1) >= 0
    gpu.step(1)
    assert gpu.sync() >= 0
    p_ref, g_ref, ng_ref = ref.enc_groups()
    p_gpu, g_gpu, ng_gpu = gpu.enc_groups()
    assert np.array_equal(p_ref, p_gpu) and np.array_equal(g_ref, g_gpu) and ng_ref == ng_gpu
    x, v, *_ = gpu.get_state()
    rel = np.linalg.norm(x - ref.x, axis=1) / np.linalg.norm(ref.x, axis=1)
    assert np.median(rel) < 1e-13 and np.percentile(rel, 99) < 1e-10, (np.median(rel), rel.max())


def test_mixed_field_particles_against_fp64(orc, sy):
    """Massive/field split (N_m = 300 + 3,000 field particles): 20 steps in mixed precision vs the
    FP64 oracle; every encounter decision of the first step is identical, energy and positions
    agree to the stated bounds."""
    d = disk.planetesimal_disk(300, 1003, n_field=3000)
    ref = orc.OracleSim(d.x, d.v, d.m, d.radius, n_massive=300)
    gpu = _mixed(sy, d)
    E0, _ = ref.energy()
    assert ref.step(1) >= 0
    gpu.step(1)
    assert gpu.sync() >= 0
    p_ref, _, _ = ref.enc_groups()
    p_gpu, _, _ = gpu.enc_groups()
    assert np.array_equal(p_ref, p_gpu)
    assert ref.step(19) >= 0
    gpu.step(19)
    assert gpu.sync() >= 0
    x, *_ = gpu.get_state()
    rel = np.linalg.norm(x - ref.x, axis=1) / np.linalg.norm(ref.x, axis=1)
    assert np.median(rel) < 1e-12, np.median(rel)
    E_ref, _ = ref.energy()
    E_gpu, _ = gpu.energy()
    assert abs(E_gpu - E_ref) <= 1e-10 * abs(E0)


def test_mixed_energy_error_bounded(sy):
    """Sec. 3 accuracy disk (100 bodies, no mergers), tau = 0.1 yr, 2,000 steps: the energy error
    of the mixed-precision path stays below 1e-10 and within 1e-11 of the FP64 path's."""
    d = disk.hill_spaced_disk()
    out = {}
    for prec in (sy.SYMBA_PRECISION_FP64, sy.SYMBA_PRECISION_MIXED):
        p = sy.default_params(precision=prec, dt=0.1)
        s = sy.System(d.x, d.v, d.m, d.radius, params=p)
        E0, _ = s.energy()
        s.step(2000)
        assert s.sync() >= 0
        E1, _ = s.energy()
        out[prec] = (E1 - E0) / abs(E0)
        s.close()
    assert abs(out[sy.SYMBA_PRECISION_MIXED]) < 1e-10
    assert abs(out[sy.SYMBA_PRECISION_MIXED] - out[sy.SYMBA_PRECISION_FP64]) < 1e-11
