"""The C-ABI library builds, loads without a GPU and exports every entry point include/symba.h
declares; the binding mirrors the header's structs (CPU only, no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "symba.h")).read()
    return sorted(set(re.findall(r"\b(symba_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2304_07325_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(built_lib):
    import paper_2304_07325_gb300 as sy
    assert sorted(sy.EXPORTED) == _declared()
    sy.lib()  # loads without a GPU


def test_param_struct_layout_matches_header(built_lib):
    import paper_2304_07325_gb300 as sy
    p = sy.default_params()
    assert (p.dt, p.M, p.shell_ratio, p.l, p.hill_scale, p.max_depth) == (0.5, 4, 2.08, 3, 6.5, 20)
    assert abs(p.G - 39.47841760435743) < 1e-14 and p.m0 == 1.0 and p.precision == 0
    assert p.rmin == 0.0 and p.rmax == 0.0
    assert ctypes.sizeof(sy.symba_params) == 5 * 8 + 6 * 4 + 2 * 8
    assert ctypes.sizeof(sy.symba_stats) == 4 * 4 + 6 * 8
    assert ctypes.sizeof(sy.symba_schedule) == 4 * 4
    assert ctypes.sizeof(sy.symba_tune_result) == 4 * 4 + 4 * 8 + 4 * 4


def test_status_strings(built_lib):
    import paper_2304_07325_gb300 as sy
    assert sy.status_string(sy.SYMBA_E_CAPACITY) == "encounter pair list overflow"
    assert sy.status_string(0) == "ok"


def test_footprint_grows_with_size(built_lib):
    import paper_2304_07325_gb300 as sy
    a, b = sy.Pool.footprint(1000, 1000), sy.Pool.footprint(10000, 10000)
    # N = 10,000: 313 massive blocks, ~6,300 macro-tiles of 4 x 2 tiles, 4.5 KiB of partials each
    assert 0 < a < b and 20e6 < b < 60e6


def test_macro_tile_capacity_bound():
    """The pool allocates partials for T / (4 C) + sqrt(2T) + 2 macro-tiles per system of T tiles
    (C column blocks per macro-tile): that must cover the macro-tiles of every block count."""
    import math
    for C in (2, 4):
        for nbm in range(1, 20001):
            T = nbm * (nbm + 1) // 2
            nq, ng = (nbm + 3) // 4, (nbm + C - 1) // C
            M = nq * ng - (4 // C) * nq * (nq - 1) // 2
            assert M <= T // (4 * C) + math.ceil(math.sqrt(2 * T)) + 2, (C, nbm)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2304_07325_gb300 as sy
    monkeypatch.setattr(sy, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(sy, "_lib", None)
    with pytest.raises(RuntimeError):
        sy.lib()


def test_invalid_arguments_are_rejected_before_any_device_call(built_lib):
    import ctypes as C

    import numpy as np

    import paper_2304_07325_gb300 as sy
    lib = sy.lib()
    p = sy.default_params()
    h = C.c_void_p()
    x = np.zeros((4, 3))
    ptr = lambda a: C.c_void_p(a.ctypes.data)
    m = np.zeros(4)
    # n < 1, n_massive > n, NULL params
    assert lib.symba_init(C.byref(h), C.byref(p), 0, 0, ptr(x), ptr(x), ptr(m), ptr(m), None, None) == sy.SYMBA_E_INVAL
    assert lib.symba_init(C.byref(h), C.byref(p), 4, 5, ptr(x), ptr(x), ptr(m), ptr(m), None, None) == sy.SYMBA_E_INVAL
    assert lib.symba_init(C.byref(h), None, 4, 4, ptr(x), ptr(x), ptr(m), ptr(m), None, None) == sy.SYMBA_E_INVAL
    assert lib.symba_step(None, 1) == sy.SYMBA_E_INVAL
    assert lib.symba_energy_static(0, 0, None, None, None, 1.0, 1.0, None, None) == sy.SYMBA_E_INVAL
    assert lib.symba_pool_create(C.byref(h), 0, 10, 10, 0, None) == sy.SYMBA_E_INVAL
    assert lib.symba_pool_create(C.byref(h), 1, 10, 10, 7, None) == sy.SYMBA_E_INVAL
    sched, res = sy.symba_schedule(), sy.symba_tune_result()
    assert lib.symba_pool_get_schedule(None, C.byref(sched)) == sy.SYMBA_E_INVAL
    assert lib.symba_pool_set_schedule(None, C.byref(sched)) == sy.SYMBA_E_INVAL
    assert lib.symba_pool_autotune(None, 1, C.byref(res)) == sy.SYMBA_E_INVAL
    assert lib.symba_autotune(None, 1, C.byref(res)) == sy.SYMBA_E_INVAL
    nulls = (C.c_void_p * 2)(None, None)
    assert lib.symba_step_many(None, 1, 1) == sy.SYMBA_E_INVAL
    assert lib.symba_step_many(nulls, 2, 1) == sy.SYMBA_E_INVAL
    assert lib.symba_step_many(nulls, 0, 1) == sy.SYMBA_OK
    assert lib.symba_step_many(nulls, -1, 1) == sy.SYMBA_E_INVAL
