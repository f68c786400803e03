"""SyMBA hot path on GB300 (arXiv:2304.07325, SyMBAp) -- Python binding of libsymba.so.

Argument marshalling only: every step runs in the library's CUDA kernels.  The functions keep
the C names (symba_init, symba_step, symba_energy, symba_enc_groups, ...); `System` and `Pool`
wrap them for convenience.  Arrays may be numpy arrays (host) or torch CUDA tensors (device);
vectors are (n, 3) float64, row-major.  Importing this package does not need a GPU; calling it
does, and a missing library raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import math
import os
from ctypes import POINTER, byref, c_double, c_int, c_longlong, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsymba.so")

SYMBA_OK = 0
SYMBA_E_INVAL = -1
SYMBA_E_NOMEM = -2
SYMBA_E_CUDA = -3
SYMBA_E_KEPLER = -4
SYMBA_E_DEPTH = -5
SYMBA_E_CAPACITY = -6
SYMBA_E_NONFINITE = -7
SYMBA_COLLISION = 1
SYMBA_PRECISION_FP64 = 0
SYMBA_PRECISION_MIXED = 1
SYMBA_ENERGY_STATIC_MAX_N = 65534

EXPORTED = ["symba_default_params", "symba_init", "symba_step", "symba_sync", "symba_energy",
            "symba_enc_groups", "symba_get_state", "symba_set_state", "symba_get_stats",
            "symba_free", "symba_pool_create", "symba_pool_footprint", "symba_pool_admit",
            "symba_pool_step", "symba_pool_sync", "symba_pool_get_state", "symba_pool_energy",
            "symba_pool_get_stats", "symba_pool_evict", "symba_pool_free", "symba_status_string",
            "symba_profile_step", "symba_energy_static", "symba_pool_get_schedule",
            "symba_pool_set_schedule", "symba_pool_autotune", "symba_autotune", "symba_step_many",
            "symba_get_rhill", "symba_pool_get_rhill", "symba_measure_rates", "symba_pool_enc_groups",
            "symba_pool_set_state"]
SYMBA_NPHASES = 10
PHASES = ["sun drift + prologue", "kick 1 + encounter check", "kick-1 reduction", "grouping",
          "Kepler drift", "group recursion", "kick 2", "kick-2 reduction", "total momentum",
          "closing sun drift"]


class symba_params(ctypes.Structure):
    _fields_ = [("dt", c_double), ("shell_ratio", c_double), ("hill_scale", c_double),
                ("G", c_double), ("m0", c_double), ("M", c_int), ("l", c_int),
                ("max_depth", c_int), ("precision", c_int), ("pair_capacity", c_int),
                ("max_substeps", c_int), ("rmin", c_double), ("rmax", c_double)]


class symba_stats(ctypes.Structure):
    _fields_ = [("n_pairs", c_int), ("n_groups", c_int), ("max_depth", c_int), ("status", c_int),
                ("merges", c_longlong), ("substeps", c_longlong), ("steps", c_longlong),
                ("max_chain", c_longlong), ("removals", c_longlong), ("pair_substeps", c_longlong)]


class symba_schedule(ctypes.Structure):
    _fields_ = [("kick_blocks_per_sm", c_int), ("kick_tiles_per_item", c_int),
                ("rec_blocks_per_sm", c_int), ("group_order", c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class symba_tune_result(ctypes.Structure):
    _fields_ = [("chosen", symba_schedule), ("kick_ms", c_double), ("recursion_ms", c_double),
                ("kick_ms_before", c_double), ("recursion_ms_before", c_double),
                ("kick_candidates", c_int), ("recursion_candidates", c_int), ("identical", c_int),
                ("pad", c_int)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("chosen", "pad")}
        d["chosen"] = self.chosen.as_dict()
        return d


class SymbaError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code})")


_lib = None


def lib():
    """The loaded libsymba.so.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2304_07325_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, dp = c_void_p, POINTER(c_int), POINTER(c_double)
        sig = {
            "symba_default_params": (None, [POINTER(symba_params)]),
            "symba_init": (c_int, [POINTER(c_void_p), POINTER(symba_params), c_int, c_int, vp, vp, vp, vp, vp, vp]),
            "symba_step": (c_int, [vp, c_int]),
            "symba_sync": (c_int, [vp]),
            "symba_energy": (c_int, [vp, dp, dp]),
            "symba_enc_groups": (c_int, [vp, vp, vp, c_int, ip, ip]),
            "symba_get_state": (c_int, [vp, vp, vp, vp, vp, vp]),
            "symba_set_state": (c_int, [vp, vp, vp]),
            "symba_get_stats": (c_int, [vp, POINTER(symba_stats)]),
            "symba_free": (None, [vp]),
            "symba_pool_create": (c_int, [POINTER(c_void_p), c_int, c_longlong, c_longlong, c_int, vp]),
            "symba_pool_footprint": (c_longlong, [c_int, c_int, POINTER(symba_params)]),
            "symba_pool_admit": (c_int, [vp, POINTER(symba_params), c_int, c_int, vp, vp, vp, vp, vp, ip]),
            "symba_pool_step": (c_int, [vp, c_int]),
            "symba_pool_sync": (c_int, [vp]),
            "symba_pool_get_state": (c_int, [vp, c_int, vp, vp, vp, vp, vp]),
            "symba_pool_energy": (c_int, [vp, c_int, dp, dp]),
            "symba_pool_get_stats": (c_int, [vp, c_int, POINTER(symba_stats)]),
            "symba_pool_evict": (c_int, [vp, c_int]),
            "symba_pool_free": (None, [vp]),
            "symba_status_string": (ctypes.c_char_p, [c_int]),
            "symba_profile_step": (c_int, [vp, c_int, dp]),
            "symba_energy_static": (c_int, [c_int, c_int, vp, vp, vp, c_double, c_double, vp, vp]),
            "symba_pool_get_schedule": (c_int, [vp, POINTER(symba_schedule)]),
            "symba_pool_set_schedule": (c_int, [vp, POINTER(symba_schedule)]),
            "symba_pool_autotune": (c_int, [vp, c_int, POINTER(symba_tune_result)]),
            "symba_autotune": (c_int, [vp, c_int, POINTER(symba_tune_result)]),
            "symba_step_many": (c_int, [POINTER(c_void_p), c_int, c_int]),
            "symba_get_rhill": (c_int, [vp, vp]),
            "symba_pool_get_rhill": (c_int, [vp, c_int, vp]),
            "symba_measure_rates": (c_int, [dp]),
            "symba_pool_enc_groups": (c_int, [vp, c_int, vp, vp, c_int, ip, ip]),
            "symba_pool_set_state": (c_int, [vp, c_int, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_string(code: int) -> str:
    try:
        return lib().symba_status_string(int(code)).decode()
    except RuntimeError:
        return str(code)


def default_params(**kw) -> symba_params:
    p = symba_params()
    lib().symba_default_params(byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _ptr(a):
    """Device pointer of a torch tensor, or host pointer of a numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return c_void_p(a.data_ptr())
    return c_void_p(a.ctypes.data)


def _host(a, dtype, shape=None):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.contiguous()
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.reshape(shape) if shape is not None else arr


def _check(code: int, what: str) -> int:
    if code < 0:
        raise SymbaError(code, what)
    return code


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return c_void_p(stream.cuda_stream)
    return c_void_p(int(stream))


class System:
    """One system integrated on the GPU (a context of the C ABI)."""

    def __init__(self, x, v_helio, m, radius, n_massive=None, params: symba_params | None = None,
                 rhill=None, stream=None):
        self._keep = [_host(x, np.float64, (-1, 3)), _host(v_helio, np.float64, (-1, 3)),
                      _host(m, np.float64), _host(radius, np.float64), _host(rhill, np.float64)]
        xs, vs, ms, rs, hs = self._keep
        n = int(xs.shape[0])
        self.n = n
        self.n_massive = n if n_massive is None else int(n_massive)
        self.params = params if params is not None else default_params()
        h = c_void_p()
        _check(lib().symba_init(byref(h), byref(self.params), n, self.n_massive, _ptr(xs), _ptr(vs),
                                _ptr(ms), _ptr(rs), _ptr(hs), _stream_handle(stream)), "symba_init")
        self._h = h
        self._keep = None

    def step(self, nsteps: int = 1) -> None:
        _check(lib().symba_step(self._h, int(nsteps)), "symba_step")

    def sync(self) -> int:
        return _check(lib().symba_sync(self._h), "symba_sync")

    def energy(self):
        E = c_double()
        L = (c_double * 3)()
        _check(lib().symba_energy(self._h, byref(E), L), "symba_energy")
        return E.value, np.array(L[:])

    def enc_groups(self, cap: int | None = None):
        npairs, ngroups = c_int(), c_int()
        _check(lib().symba_enc_groups(self._h, None, None, 0, byref(npairs), byref(ngroups)), "symba_enc_groups")
        cap = npairs.value if cap is None else cap
        pairs = np.zeros((max(cap, 1), 2), dtype=np.int32)
        gop = np.zeros(max(cap, 1), dtype=np.int32)
        _check(lib().symba_enc_groups(self._h, _ptr(pairs), _ptr(gop), cap, byref(npairs), byref(ngroups)),
               "symba_enc_groups")
        k = min(cap, npairs.value)
        return pairs[:k].copy(), gop[:k].copy(), ngroups.value

    def get_state(self):
        """(x heliocentric, v barycentric, m, radius, alive) as numpy arrays."""
        x = np.zeros((self.n, 3)); v = np.zeros((self.n, 3))
        m = np.zeros(self.n); r = np.zeros(self.n); a = np.zeros(self.n, dtype=np.int32)
        _check(lib().symba_get_state(self._h, _ptr(x), _ptr(v), _ptr(m), _ptr(r), _ptr(a)), "symba_get_state")
        return x, v, m, r, a

    def rhill(self) -> np.ndarray:
        """The Hill radii the context uses (symba_get_rhill)."""
        rh = np.zeros(self.n)
        _check(lib().symba_get_rhill(self._h, _ptr(rh)), "symba_get_rhill")
        return rh

    def set_state(self, x, v_bary):
        xs, vs = _host(x, np.float64, (-1, 3)), _host(v_bary, np.float64, (-1, 3))
        _check(lib().symba_set_state(self._h, _ptr(xs), _ptr(vs)), "symba_set_state")

    def stats(self) -> symba_stats:
        s = symba_stats()
        _check(lib().symba_get_stats(self._h, byref(s)), "symba_get_stats")
        return s

    def autotune(self, reps: int = 3) -> dict:
        """Times the launch schedules on this system and keeps the fastest (symba_autotune);
        the system's state is left as it was."""
        r = symba_tune_result()
        _check(lib().symba_autotune(self._h, int(reps), byref(r)), "symba_autotune")
        return r.as_dict()

    def profile_step(self, nsteps: int = 1) -> np.ndarray:
        """Device milliseconds per phase (see PHASES), summed over nsteps steps."""
        out = (c_double * SYMBA_NPHASES)()
        _check(lib().symba_profile_step(self._h, int(nsteps), out), "symba_profile_step")
        return np.array(out[:])

    def close(self):
        if getattr(self, "_h", None):
            lib().symba_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pool:
    """Many independent systems stepped together (C ABI symba_pool_*)."""

    def __init__(self, max_systems: int, max_particles: int, max_tiles: int,
                 precision: int = SYMBA_PRECISION_FP64, stream=None):
        h = c_void_p()
        _check(lib().symba_pool_create(byref(h), int(max_systems), int(max_particles), int(max_tiles),
                                       int(precision), _stream_handle(stream)), "symba_pool_create")
        self._h = h
        self.precision = precision
        self.n = {}

    @staticmethod
    def footprint(n: int, n_massive: int, params: symba_params | None = None) -> int:
        p = params if params is not None else default_params()
        return int(lib().symba_pool_footprint(int(n), int(n_massive), byref(p)))

    def admit(self, x, v_helio, m, radius, n_massive=None, params: symba_params | None = None, rhill=None) -> int:
        xs, vs = _host(x, np.float64, (-1, 3)), _host(v_helio, np.float64, (-1, 3))
        ms, rs, hs = _host(m, np.float64), _host(radius, np.float64), _host(rhill, np.float64)
        n = int(xs.shape[0])
        p = params if params is not None else default_params(precision=self.precision)
        slot = c_int(-1)
        _check(lib().symba_pool_admit(self._h, byref(p), n, n if n_massive is None else int(n_massive),
                                      _ptr(xs), _ptr(vs), _ptr(ms), _ptr(rs), _ptr(hs), byref(slot)),
               "symba_pool_admit")
        self.n[slot.value] = n
        return slot.value

    def step(self, nsteps: int = 1) -> None:
        _check(lib().symba_pool_step(self._h, int(nsteps)), "symba_pool_step")

    def sync(self) -> int:
        return _check(lib().symba_pool_sync(self._h), "symba_pool_sync")

    def get_state(self, slot: int):
        n = self.n[slot]
        x = np.zeros((n, 3)); v = np.zeros((n, 3))
        m = np.zeros(n); r = np.zeros(n); a = np.zeros(n, dtype=np.int32)
        _check(lib().symba_pool_get_state(self._h, int(slot), _ptr(x), _ptr(v), _ptr(m), _ptr(r), _ptr(a)),
               "symba_pool_get_state")
        return x, v, m, r, a

    def energy(self, slot: int):
        E = c_double()
        L = (c_double * 3)()
        _check(lib().symba_pool_energy(self._h, int(slot), byref(E), L), "symba_pool_energy")
        return E.value, np.array(L[:])

    def stats(self, slot: int) -> symba_stats:
        s = symba_stats()
        _check(lib().symba_pool_get_stats(self._h, int(slot), byref(s)), "symba_pool_get_stats")
        return s

    def set_state(self, slot: int, x, v_bary) -> None:
        """Replaces one system's positions (heliocentric) and barycentric velocities."""
        xs, vs = _host(x, np.float64, (-1, 3)), _host(v_bary, np.float64, (-1, 3))
        _check(lib().symba_pool_set_state(self._h, int(slot), _ptr(xs), _ptr(vs)), "symba_pool_set_state")

    def enc_groups(self, slot: int, cap: int | None = None):
        """Level-0 pairs of the system's last step, their groups and the group count."""
        npairs, ngroups = c_int(), c_int()
        _check(lib().symba_pool_enc_groups(self._h, int(slot), None, None, 0, byref(npairs), byref(ngroups)),
               "symba_pool_enc_groups")
        cap = npairs.value if cap is None else cap
        pairs = np.zeros((max(cap, 1), 2), dtype=np.int32)
        gop = np.zeros(max(cap, 1), dtype=np.int32)
        _check(lib().symba_pool_enc_groups(self._h, int(slot), _ptr(pairs), _ptr(gop), cap, byref(npairs),
                                           byref(ngroups)), "symba_pool_enc_groups")
        k = min(cap, npairs.value)
        return pairs[:k].copy(), gop[:k].copy(), ngroups.value

    def rhill(self, slot: int) -> np.ndarray:
        rh = np.zeros(self.n[slot])
        _check(lib().symba_pool_get_rhill(self._h, int(slot), _ptr(rh)), "symba_pool_get_rhill")
        return rh

    def autotune(self, reps: int = 3) -> dict:
        """Times the launch schedules on the admitted systems and keeps the fastest
        (symba_pool_autotune); every system's state is left as it was."""
        r = symba_tune_result()
        _check(lib().symba_pool_autotune(self._h, int(reps), byref(r)), "symba_pool_autotune")
        return r.as_dict()

    @property
    def schedule(self) -> dict:
        s = symba_schedule()
        _check(lib().symba_pool_get_schedule(self._h, byref(s)), "symba_pool_get_schedule")
        return s.as_dict()

    @schedule.setter
    def schedule(self, d: dict) -> None:
        s = symba_schedule()
        _check(lib().symba_pool_get_schedule(self._h, byref(s)), "symba_pool_get_schedule")
        for k, v in d.items():
            setattr(s, k, int(v))
        _check(lib().symba_pool_set_schedule(self._h, byref(s)), "symba_pool_set_schedule")

    def evict(self, slot: int) -> None:
        _check(lib().symba_pool_evict(self._h, int(slot)), "symba_pool_evict")
        self.n.pop(slot, None)

    def close(self):
        if getattr(self, "_h", None):
            lib().symba_pool_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def step_many(systems, nsteps: int = 1) -> int:
    """Advances independent systems by nsteps each, every one on its own stream with one step in
    flight, so that none waits for a slower one (symba_step_many); waits for all."""
    arr = (c_void_p * len(systems))(*[s._h for s in systems])
    return _check(lib().symba_step_many(arr, len(systems), int(nsteps)), "symba_step_many")


SYMBA_NRATES = 6


def measure_rates() -> dict:
    """The device rates that bound this path, measured now (symba_measure_rates)."""
    out = (c_double * SYMBA_NRATES)()
    _check(lib().symba_measure_rates(out), "symba_measure_rates")
    v = list(out)
    return {"fp64_flops": v[0], "warp_dfma_dep_cycles": v[1], "warp_dfma_4chain_cycles": v[2],
            "named_barrier_round_trip_cycles": v[3], "sms": int(v[4]), "sm_clock_hz_nominal": v[5]}


def G_default() -> float:
    return 4.0 * math.pi ** 2
