"""Seeded synthetic inputs: the planetesimal disks of Sec. 3 and the request streams built on them.

This module holds input generation only -- random numbers, the mass law, orbital elements and
their conversion to heliocentric Cartesian state.  It contains none of the integrator's
arithmetic, so the CUDA path, the oracle, the tests and the benchmark can all draw their inputs
from it.

Units: AU, yr, solar masses, so G = 4 pi^2 and the central mass m0 = 1.

Disk recipe (Sec. 3, benchmark paragraph; unstated parts are readings):
  * mass m from the cumulative law N(>m) = C m^-0.3 exp(-m/m0), m0 = 1e-2 Earth masses,
    m_min = 1e-3 Earth masses (inverse CDF of F(m) = (m/m_min)^-0.3 exp(-(m - m_min)/m0));
  * radius from a bulk density of 2 g/cm^3;
  * semi-major axis uniform in 5-20 AU (reading: uniform in a);
  * eccentricity Rayleigh(1e-6), inclination Rayleigh(5e-7) radians;
  * node, argument of pericentre and mean anomaly uniform in [0, 2 pi).
Accuracy-test disk (Sec. 3, last paragraph): 100 bodies of 1e-2 Earth masses spaced by 5 mutual
Hill radii from 5 AU (reading: mutual Hill radius ((m_i + m_{i+1}) / 3)^{1/3} (a_i + a_{i+1}) / 2).

Random numbers: SplitMix64 (Steele, Lea & Flood 2014), one counter-based stream per (seed,
quantity), mapped to doubles in (0, 1] -- identical on every machine.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

G_AU_YR_MSUN = 4.0 * math.pi ** 2
M_EARTH_MSUN = 3.0034896e-6
AU_CM = 1.495978707e13
MSUN_G = 1.98841e33
RHO_2GCC_MSUN_AU3 = 2.0 * AU_CM ** 3 / MSUN_G

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n outputs of SplitMix64 started from state seed*2^16 + stream (wrapping uint64)."""
    base = np.uint64((int(seed) * 65536 + int(stream)) & 0xFFFFFFFFFFFFFFFF)
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = base + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, stream: int) -> np.ndarray:
    """Doubles in (0, 1]: (top 53 bits + 1) * 2^-53."""
    z = splitmix64(seed, n, stream)
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def mass_inverse_cdf(u: np.ndarray, m0: float = 1e-2, m_min: float = 1e-3) -> np.ndarray:
    """Solve (m/m_min)^-0.3 exp(-(m - m_min)/m0) = u for m >= m_min (Earth masses), by bisection
    on log m to the last bit.  F decreases from 1 at m_min to 0, so every u in (0, 1] has one root."""
    u = np.asarray(u, dtype=np.float64)
    lo = np.full(u.shape, math.log(m_min))
    hi = np.full(u.shape, math.log(m_min) + 80.0)

    def F(logm):
        m = np.exp(logm)
        return np.exp(-0.3 * (logm - math.log(m_min)) - (m - m_min) / m0)

    for _ in range(200):
        mid = 0.5 * (lo + hi)
        above = F(mid) > u  # still above the target: the root is further out
        lo = np.where(above, mid, lo)
        hi = np.where(above, hi, mid)
    return np.exp(0.5 * (lo + hi))


def elements_to_state(a, e, inc, node, peri, mean_anom, mu):
    """Heliocentric position and velocity of elliptic orbits (vectorised)."""
    a, e, inc, node, peri, M, mu = (np.asarray(t, dtype=np.float64) for t in
                                    (a, e, inc, node, peri, mean_anom, mu))
    E = M.copy()
    for _ in range(60):
        E = E - (E - e * np.sin(E) - M) / (1.0 - e * np.cos(E))
    cE, sE = np.cos(E), np.sin(E)
    b = np.sqrt(1.0 - e * e)
    xp = a * (cE - e)
    yp = a * b * sE
    n = np.sqrt(mu / a ** 3)
    rdot = n * a / (1.0 - e * cE)
    vxp = -rdot * sE
    vyp = rdot * b * cE
    cO, sO = np.cos(node), np.sin(node)
    cw, sw = np.cos(peri), np.sin(peri)
    ci, si = np.cos(inc), np.sin(inc)
    r11 = cO * cw - sO * sw * ci
    r12 = -cO * sw - sO * cw * ci
    r21 = sO * cw + cO * sw * ci
    r22 = -sO * sw + cO * cw * ci
    r31 = sw * si
    r32 = cw * si
    x = np.stack([r11 * xp + r12 * yp, r21 * xp + r22 * yp, r31 * xp + r32 * yp], axis=-1)
    v = np.stack([r11 * vxp + r12 * vyp, r21 * vxp + r22 * vyp, r31 * vxp + r32 * vyp], axis=-1)
    return x, v


@dataclass
class Disk:
    """One synthetic system: heliocentric state, masses, radii; massive bodies come first."""
    x: np.ndarray        # [n, 3] heliocentric positions (AU)
    v: np.ndarray        # [n, 3] heliocentric velocities (AU/yr)
    m: np.ndarray        # [n] masses (Msun), 0 for field particles
    radius: np.ndarray   # [n] physical radii (AU)
    n_massive: int
    seed: int
    label: str

    @property
    def n(self) -> int:
        return int(self.m.shape[0])


def planetesimal_disk(n: int, seed: int, n_field: int = 0, a_range=(5.0, 20.0),
                      e_scale: float = 1e-6, i_scale: float = 5e-7,
                      G: float = G_AU_YR_MSUN, m_central: float = 1.0) -> Disk:
    """The Sec. 3 benchmark disk: n massive planetesimals plus n_field massless field particles
    drawn from the same orbital distributions."""
    nt = n + n_field
    u = [uniform01(seed, nt, s) for s in range(7)]
    m_earth = mass_inverse_cdf(u[0][:n])
    m = np.concatenate([m_earth * M_EARTH_MSUN, np.zeros(n_field)])
    radius = np.cbrt(3.0 * m / (4.0 * math.pi * RHO_2GCC_MSUN_AU3))
    a = a_range[0] + (a_range[1] - a_range[0]) * u[1]
    e = e_scale * np.sqrt(-2.0 * np.log(u[2]))
    inc = i_scale * np.sqrt(-2.0 * np.log(u[3]))
    node = 2.0 * math.pi * (1.0 - u[4])
    peri = 2.0 * math.pi * (1.0 - u[5])
    mean = 2.0 * math.pi * (1.0 - u[6])
    x, v = elements_to_state(a, e, inc, node, peri, mean, G * (m_central + m))
    return Disk(x=np.ascontiguousarray(x), v=np.ascontiguousarray(v), m=m, radius=radius,
                n_massive=n, seed=seed, label=f"disk N_m={n} N_field={n_field} seed={seed}")


def hill_spaced_disk(n: int = 100, m_earth: float = 1e-2, a1: float = 5.0, spacing: float = 5.0,
                     seed: int = 7, G: float = G_AU_YR_MSUN, m_central: float = 1.0) -> Disk:
    """The Sec. 3 accuracy-test disk: equal masses, a_{i+1} = a_i + spacing * R_H,mut."""
    m = np.full(n, m_earth * M_EARTH_MSUN)
    K = spacing * ((2.0 * m[0]) / (3.0 * m_central)) ** (1.0 / 3.0)
    a = a1 * ((1.0 + 0.5 * K) / (1.0 - 0.5 * K)) ** np.arange(n)
    u = [uniform01(seed, n, s) for s in range(6)]
    e = 1e-6 * np.sqrt(-2.0 * np.log(u[0]))
    inc = 5e-7 * np.sqrt(-2.0 * np.log(u[1]))
    node = 2.0 * math.pi * (1.0 - u[2])
    peri = 2.0 * math.pi * (1.0 - u[3])
    mean = 2.0 * math.pi * (1.0 - u[4])
    x, v = elements_to_state(a, e, inc, node, peri, mean, G * (m_central + m))
    radius = np.cbrt(3.0 * m / (4.0 * math.pi * RHO_2GCC_MSUN_AU3))
    return Disk(x=np.ascontiguousarray(x), v=np.ascontiguousarray(v), m=m, radius=radius,
                n_massive=n, seed=seed, label=f"hill-spaced N={n}")


def batch_sizes(count: int = 64, seed: int = 2000, n_lo: int = 1000, n_hi: int = 10000):
    """Sizes of a batch of disks, log-uniform in [n_lo, n_hi]; disk k uses seed + k."""
    u = uniform01(seed, count, 99)
    return [int(round(math.exp(math.log(n_lo) + (math.log(n_hi) - math.log(n_lo)) * (1.0 - t))))
            for t in u]


def request_stream(count: int, rate_per_s: float = 20.0, seed: int = 3000, n_lo: int = 500,
                   n_hi: int = 20000, steps_lo: int = 100, steps_hi: int = 5000):
    """A Poisson stream of disk-simulation requests: (arrival time s, N, step budget, seed)."""
    u = [uniform01(seed, count, s) for s in range(3)]
    gaps = -np.log(u[0]) / rate_per_s
    t = np.cumsum(gaps) - gaps[0]
    n = np.exp(math.log(n_lo) + (math.log(n_hi) - math.log(n_lo)) * (1.0 - u[1]))
    steps = steps_lo + np.floor((steps_hi - steps_lo + 1) * (1.0 - u[2]))
    return [(float(t[k]), int(round(n[k])), int(min(steps[k], steps_hi)), seed + 1 + k)
            for k in range(count)]
