"""Failure reporting and checkpoint/resume on the GPU.  Every failure is a status code the device
writes and the host reads at the next synchronising call -- no trap, no fault -- and the context
stays usable after set_state."""
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


def test_pair_capacity_overflow_is_reported(sy):
    d = disk.planetesimal_disk(1000, 1000)
    p = sy.default_params(pair_capacity=8)          # ~100 level-0 pairs will be flagged
    s = sy.System(d.x, d.v, d.m, d.radius, params=p)
    x0, v0, *_ = s.get_state()
    s.step(1)
    with pytest.raises(sy.SymbaError) as e:
        s.sync()
    assert e.value.code == sy.SYMBA_E_CAPACITY
    npairs = s.stats().n_pairs
    assert npairs > 8
    # the context is usable again after the state is restored
    s.set_state(x0, v0)
    assert s.sync() == sy.SYMBA_OK


def test_depth_limit_and_substep_budget_are_reported(sy):
    d = disk.planetesimal_disk(1000, 1000)
    for kw in (dict(max_depth=2), dict(max_substeps=50)):
        s = sy.System(d.x, d.v, d.m, d.radius, params=sy.default_params(**kw))
        s.step(1)
        with pytest.raises(sy.SymbaError) as e:
            s.sync()
        assert e.value.code == sy.SYMBA_E_DEPTH, kw
        s.close()


def test_resume_from_checkpoint_is_bit_identical(sy):
    d = disk.hill_spaced_disk()
    p = sy.default_params(dt=0.1)
    a = sy.System(d.x, d.v, d.m, d.radius, params=p)
    a.step(40)
    assert a.sync() == sy.SYMBA_OK
    xa, va, *_ = a.get_state()
    b = sy.System(d.x, d.v, d.m, d.radius, params=p)
    b.step(25)
    xc, vc, *_ = b.get_state()
    b.close()
    c = sy.System(d.x, d.v, d.m, d.radius, params=p)     # same inputs -> same Hill radii
    c.set_state(xc, vc)
    c.step(15)
    assert c.sync() == sy.SYMBA_OK
    x, v, *_ = c.get_state()
    assert np.array_equal(x, xa) and np.array_equal(v, va)


def test_device_pointers_are_accepted(sy):
    import torch
    d = disk.planetesimal_disk(300, 31)
    dev = torch.device("cuda", 0)
    t = {k: torch.from_numpy(getattr(d, k)).to(dev) for k in ("x", "v", "m", "radius")}
    a = sy.System(t["x"], t["v"], t["m"], t["radius"])
    b = sy.System(d.x, d.v, d.m, d.radius)
    a.step(3)
    b.step(3)
    xa, *_ = a.get_state()
    xb, *_ = b.get_state()
    assert np.array_equal(xa, xb)
