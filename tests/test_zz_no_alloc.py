"""symba_energy_static, the entry point that allocates nothing, against symba_energy.

Callers that cannot allocate device memory -- a host loop with a hard per-iteration latency
budget (cudaMalloc and cudaFree may synchronise the device), or a process whose device memory
belongs to another allocator -- compute the energy with symba_energy_static, which keeps its
exact-sum scratch in a file-scope device array instead of memory it would have to allocate.
Both entry points round the same exact sums, so their results must agree bit for bit, call after
call (the shared scratch must be cleared by each call).  This file is collected last, so a run
that stops at the first failure has run every other test first.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_energy_static_matches_symba_energy_on_two_calls():
    import torch

    import paper_2304_07325_gb300 as sy
    from paper_2304_07325_gb300 import build, disk

    build.build()
    lib = sy.lib()
    d = disk.planetesimal_disk(1000, 4242, n_field=200)
    n, nm = d.n, d.n_massive
    ctx = sy.System(d.x, d.v, d.m, d.radius, n_massive=nm)
    ctx.step(2)
    assert ctx.sync() >= 0
    x, v, m, r, alive = ctx.get_state()
    assert alive.all()
    E_ref, L_ref = ctx.energy()

    dev = torch.device("cuda", 0)
    xt = torch.from_numpy(x).to(dev)
    vt = torch.from_numpy(v).to(dev)
    mt = torch.from_numpy(m).to(dev)
    out = torch.empty(4, dtype=torch.float64, device=dev)
    G, m0 = ctx.params.G, ctx.params.m0
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    for call in range(2):
        out.fill_(float("nan"))
        rc = lib.symba_energy_static(n, nm, ptr(xt), ptr(vt), ptr(mt), G, m0, ptr(out), None)
        assert rc == sy.SYMBA_OK, sy.status_string(rc)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got[0] == E_ref, (call, got[0], E_ref)
        assert np.array_equal(got[1:], L_ref), (call, got[1:], L_ref)

    # sizes beyond the scratch's limit and host pointers are rejected before any work
    big = sy.SYMBA_ENERGY_STATIC_MAX_N + 1
    assert lib.symba_energy_static(big, big, ptr(xt), ptr(vt), ptr(mt), G, m0, ptr(out), None) == sy.SYMBA_E_INVAL
    host = np.zeros(4)
    assert lib.symba_energy_static(n, nm, ptr(xt), ptr(vt), ptr(mt), G, m0,
                                   ctypes.c_void_p(host.ctypes.data), None) == sy.SYMBA_E_INVAL
    ctx.close()


@pytest.mark.parametrize("n,nf", [(1, 0), (0, 64), (40, 9)])
def test_energy_static_edge_sizes(n, nf):
    """One body (no pair at all), only field particles (n_massive = 0: the pair pass is skipped)
    and a small ragged mix, each against symba_energy of the same state, twice in a row."""
    import torch

    import paper_2304_07325_gb300 as sy
    from paper_2304_07325_gb300 import build, disk

    build.build()
    lib = sy.lib()
    d = disk.planetesimal_disk(n, 99 + n, n_field=nf)
    ctx = sy.System(d.x, d.v, d.m, d.radius, n_massive=d.n_massive)
    x, v, m, r, alive = ctx.get_state()
    E_ref, L_ref = ctx.energy()
    dev = torch.device("cuda", 0)
    xt, vt, mt = (torch.from_numpy(a).to(dev) for a in (x, v, m))
    out = torch.empty(4, dtype=torch.float64, device=dev)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    for call in range(2):
        out.fill_(float("nan"))
        rc = lib.symba_energy_static(d.n, d.n_massive, ptr(xt), ptr(vt), ptr(mt), ctx.params.G, ctx.params.m0,
                                     ptr(out), None)
        assert rc == sy.SYMBA_OK, sy.status_string(rc)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got[0] == E_ref and np.array_equal(got[1:], L_ref), (call, got, E_ref, L_ref)
    ctx.close()
