"""Python access to the SyMBA oracle -- TEST INFRASTRUCTURE ONLY.

The oracle (symba_oracle.c) is a plain, serial FP64 CPU restatement of the SyMBA step with the
SyMBAp structure of arXiv:2304.07325 (Sec. 2 trapezoid loop and encounter grouping; Sec. 3
parameters M, R_k/R_{k+1}, l).  Only tests/, the package smoke check and the benchmark's CPU
baseline may import this package; the library path never does.

trap_omp.c is the benchmark's multi-core CPU reference point for the kick (the same trapezoid
accelerations with the rows spread over OpenMP threads); it is not the oracle and no parity claim
rests on it.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from ctypes import POINTER, c_double, c_int, c_long, c_longlong

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "symba_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_OMP_SRC = os.path.join(_HERE, "trap_omp.c")
_OMP_LIB = os.path.join(_HERE, "liboracle_omp.so")

OK, E_INVAL, E_NOMEM, E_KEPLER, E_DEPTH, E_NONFINITE = 0, -1, -2, -4, -5, -7
MAX_LEVELS = 64


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE FP64: no contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def build_omp(force: bool = False) -> str:
    """Compile the multi-core trapezoid kick (OpenMP; a serial build if the compiler has none)."""
    if force or not os.path.exists(_OMP_LIB) or os.path.getmtime(_OMP_LIB) < os.path.getmtime(_OMP_SRC):
        tmp = _OMP_LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O3", "-std=gnu11", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _OMP_SRC, "-lm"]
        try:
            subprocess.check_call(cmd[:1] + ["-fopenmp"] + cmd[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(cmd)
        os.replace(tmp, _OMP_LIB)
    return _OMP_LIB


_omp_lib = None


def trap_accel_omp(x, m, rhill, alive, pairs, n_massive: int, params: "Params", threads: int = 0):
    """Accelerations of the level-0 trapezoid (flagged pairs weighted by g_0, all others 1) on
    `threads` host threads (0: all OpenMP offers).  Returns (a [n, 3], threads used)."""
    global _omp_lib
    if _omp_lib is None:
        L = ctypes.CDLL(build_omp())
        dp, ip = POINTER(c_double), POINTER(c_int)
        L.trap_omp_accel.restype = c_int
        L.trap_omp_accel.argtypes = [c_int, c_int, dp, dp, dp, ip, ip, c_int, c_double, c_double, c_double,
                                     c_int, c_int, dp]
        _omp_lib = L
    xs = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    n = xs.shape[0]
    ms = np.ascontiguousarray(m, dtype=np.float64)
    rh = np.ascontiguousarray(rhill, dtype=np.float64)
    al = np.ascontiguousarray(alive, dtype=np.int32)
    pl = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    a = np.zeros((n, 3))
    t = _omp_lib.trap_omp_accel(n, int(n_massive), _dp(xs), _dp(ms), _dp(rh), _ip(al), _ip(pl), int(pl.shape[0]),
                                params.G, params.hill_scale, params.shell_ratio, params.l, int(threads), _dp(a))
    if t < 1:
        raise MemoryError("trap_omp_accel: scratch allocation failed")
    return a, t


class Params(ctypes.Structure):
    _fields_ = [("dt", c_double), ("shell_ratio", c_double), ("hill_scale", c_double),
                ("G", c_double), ("m0", c_double), ("M", c_int), ("l", c_int),
                ("max_depth", c_int), ("noise", c_int), ("rmin", c_double), ("rmax", c_double)]


class _Sim(ctypes.Structure):
    _fields_ = [("n", c_int), ("n_massive", c_int),
                ("x", POINTER(c_double)), ("v", POINTER(c_double)), ("m", POINTER(c_double)),
                ("radius", POINTER(c_double)), ("rhill", POINTER(c_double)),
                ("alive", POINTER(c_int)),
                ("cap", c_int), ("npairs", c_int), ("ngroups", c_int),
                ("pairs", POINTER(c_int)), ("group_of_pair", POINTER(c_int)),
                ("status", c_int), ("max_depth_seen", c_int),
                ("collisions", c_longlong), ("removals", c_longlong),
                ("level_flags", c_longlong * MAX_LEVELS),
                ("level_calls", c_longlong * MAX_LEVELS)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp, ip = POINTER(c_double), POINTER(c_int)
        L.orc_fsum.restype = c_double
        L.orc_fsum.argtypes = [dp, c_long]
        L.orc_partition.restype = c_double
        L.orc_partition.argtypes = [c_double, c_int]
        L.orc_weight.restype = c_double
        L.orc_weight.argtypes = [POINTER(Params), c_double, c_int, c_double]
        L.orc_encounter.restype = c_int
        L.orc_encounter.argtypes = [dp, dp, dp, dp, c_double, c_double, c_double, ip]
        L.orc_kepler_drift.restype = c_int
        L.orc_kepler_drift.argtypes = [c_double, c_double, dp, dp]
        L.orc_union_find.restype = None
        L.orc_union_find.argtypes = [c_int, ip, c_int, ip]
        L.orc_init.restype = None
        L.orc_init.argtypes = [POINTER(Params), POINTER(_Sim), dp, c_int]
        L.orc_step.restype = c_int
        L.orc_step.argtypes = [POINTER(Params), POINTER(_Sim)]
        L.orc_energy.restype = None
        L.orc_energy.argtypes = [POINTER(Params), POINTER(_Sim), dp, dp]
        L.orc_velocity_helio.restype = None
        L.orc_velocity_helio.argtypes = [POINTER(Params), POINTER(_Sim), dp]
        L.orc_cbrt_rn.restype = c_double
        L.orc_cbrt_rn.argtypes = [c_double]
        L.orc_accel_trapezoid.restype = None
        L.orc_accel_trapezoid.argtypes = [POINTER(Params), POINTER(_Sim), ip, c_int, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(POINTER(c_double))


def _ip(a):
    return a.ctypes.data_as(POINTER(c_int))


def make_params(dt=0.5, M=4, shell_ratio=2.08, hill_scale=6.5, l=3, G=4.0 * math.pi ** 2, m0=1.0,
                max_depth=20, noise=0, rmin=0.0, rmax=0.0) -> Params:
    return Params(dt=dt, shell_ratio=shell_ratio, hill_scale=hill_scale, G=G, m0=m0, M=M, l=l,
                  max_depth=max_depth, noise=noise, rmin=rmin, rmax=rmax)


def fsum(a) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return lib().orc_fsum(_dp(a), a.size)


def cbrt_rn(x: float) -> float:
    """The correctly rounded cube root (the double nearest the real cube root of x)."""
    return lib().orc_cbrt_rn(float(x))


def partition(x: float, l: int = 3) -> float:
    return lib().orc_partition(float(x), int(l))


def weight(params: Params, R0: float, k: int, r: float) -> float:
    return lib().orc_weight(ctypes.byref(params), float(R0), int(k), float(r))


def encounter(xi, xj, vi, vj, R, Rc, h):
    """(flag, contact) of the close-encounter predicate."""
    arrs = [np.ascontiguousarray(t, dtype=np.float64) for t in (xi, xj, vi, vj)]
    c = c_int(0)
    f = lib().orc_encounter(*[_dp(t) for t in arrs], float(R), float(Rc), float(h), ctypes.byref(c))
    return int(f), int(c.value)


def kepler_drift(mu, dt, x, v):
    """Kepler drift of one body; returns (status, x', v')."""
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    st = lib().orc_kepler_drift(float(mu), float(dt), _dp(x), _dp(v))
    return st, x, v


def union_find(n, pairs):
    p = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    lab = np.zeros(n, dtype=np.int32)
    lib().orc_union_find(int(n), _ip(p), int(p.shape[0]), _ip(lab))
    return lab


class OracleSim:
    """One system integrated by the oracle.  State: heliocentric x, barycentric v."""

    def __init__(self, x, v_helio, m, radius, n_massive=None, params: Params | None = None,
                 rhill=None, cap: int = 1 << 16):
        self.params = params if params is not None else make_params()
        self.x = np.array(x, dtype=np.float64).reshape(-1, 3).copy()
        n = self.x.shape[0]
        self.v = np.zeros((n, 3))
        self.m = np.ascontiguousarray(m, dtype=np.float64).copy()
        self.radius = np.ascontiguousarray(radius, dtype=np.float64).copy()
        self.rhill = np.zeros(n) if rhill is None else np.ascontiguousarray(rhill, dtype=np.float64).copy()
        self.alive = np.ones(n, dtype=np.int32)
        self.cap = cap
        self.pairs = np.zeros((cap, 2), dtype=np.int32)
        self.gop = np.zeros(cap, dtype=np.int32)
        self.n_massive = n if n_massive is None else int(n_massive)
        s = _Sim()
        s.n, s.n_massive = n, self.n_massive
        s.x, s.v, s.m, s.radius, s.rhill = _dp(self.x), _dp(self.v), _dp(self.m), _dp(self.radius), _dp(self.rhill)
        s.alive = _ip(self.alive)
        s.cap = cap
        s.pairs, s.group_of_pair = _ip(self.pairs), _ip(self.gop)
        self._s = s
        vh = np.ascontiguousarray(v_helio, dtype=np.float64).reshape(-1, 3)
        lib().orc_init(ctypes.byref(self.params), ctypes.byref(s), _dp(vh), int(rhill is None))

    @property
    def n(self):
        return self.x.shape[0]

    def step(self, nsteps: int = 1) -> int:
        st = 0
        for _ in range(nsteps):
            st = lib().orc_step(ctypes.byref(self.params), ctypes.byref(self._s))
            if st < 0:
                return st
        return st

    def energy(self):
        E = c_double(0.0)
        L = np.zeros(3)
        lib().orc_energy(ctypes.byref(self.params), ctypes.byref(self._s), ctypes.byref(E), _dp(L))
        return E.value, L

    def velocity_helio(self):
        vh = np.zeros((self.n, 3))
        lib().orc_velocity_helio(ctypes.byref(self.params), ctypes.byref(self._s), _dp(vh))
        return vh

    def set_state(self, x, v_bary):
        self.x[...] = np.asarray(x, dtype=np.float64).reshape(-1, 3)
        self.v[...] = np.asarray(v_bary, dtype=np.float64).reshape(-1, 3)

    def enc_groups(self):
        """Level-0 pairs of the last step (sorted (i, j)), their group index and the group count."""
        npairs = self._s.npairs
        k = min(npairs, self.cap)
        return self.pairs[:k].copy(), self.gop[:k].copy(), int(self._s.ngroups)

    @property
    def npairs(self):
        return int(self._s.npairs)

    @property
    def max_depth_seen(self):
        return int(self._s.max_depth_seen)

    @property
    def mergers(self):
        return int(self._s.collisions)

    @property
    def collisions(self):
        return int(self._s.collisions)

    @property
    def removals(self):
        return int(self._s.removals)

    @property
    def level_flags(self):
        return [int(t) for t in self._s.level_flags]

    @property
    def level_calls(self):
        return [int(t) for t in self._s.level_calls]

    def accel_trapezoid(self, pairs):
        p = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        a = np.zeros((self.n, 3))
        lib().orc_accel_trapezoid(ctypes.byref(self.params), ctypes.byref(self._s), _ip(p), int(p.shape[0]), _dp(a))
        return a
