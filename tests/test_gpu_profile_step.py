"""symba_profile_step runs the same kernels as symba_step (without the graph, with events between
them), so the two give the same bits; the benchmark's end-to-end figure relies on it (a second
context stepped with symba_step replays the trajectory the timed loop stepped with
symba_profile_step).  Needs a GB300."""
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


@pytest.mark.parametrize("n,seed,precision", [(2000, 4201, 0), (1500, 4202, 1)])
def test_profile_step_equals_step(sy, n, seed, precision):
    d = disk.planetesimal_disk(n, seed)
    params = sy.default_params(precision=precision)
    a = sy.System(d.x, d.v, d.m, d.radius, params=params)
    b = sy.System(d.x, d.v, d.m, d.radius, params=params)
    for _ in range(3):
        a.step(1)
        ph = b.profile_step(1)
        assert a.sync() >= 0 and b.sync() >= 0
        assert len(ph) == sy.SYMBA_NPHASES and all(t >= 0.0 for t in ph)
        sa, sb = a.stats(), b.stats()
        assert (sa.substeps, sa.n_pairs, sa.n_groups, sa.max_depth, sa.merges) == \
               (sb.substeps, sb.n_pairs, sb.n_groups, sb.max_depth, sb.merges)
    for u, w in zip(a.get_state(), b.get_state()):
        assert np.array_equal(u, w)
    a.close()
    b.close()
