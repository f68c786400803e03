"""The synthetic disks against the paper's description of them (CPU only).

Sec. 3 (benchmark paragraph) draws masses from the cumulative law N(>m) = C m^-0.3 exp(-m/m0)
with m0 = 1e-2 and m_min = 1e-3 Earth masses, radii from a bulk density of 2 g/cm^3, semi-major
axes in 5-20 AU, eccentricities Rayleigh(1e-6) and inclinations Rayleigh(5e-7); the accuracy test
(last paragraph) spaces 100 bodies of 1e-2 Earth masses by 5 mutual Hill radii from 5 AU.  Every
workload and every timed number rests on this generator, so each ingredient is checked here
against the law it implements: quantiles of the mass law and a sample's survival fractions, the
density-to-radius conversion from CGS constants, the Hill spacing pair by pair, and the orbital
elements recovered from the Cartesian states.
"""
import math

import numpy as np

from paper_2304_07325_gb300 import disk

M0_E, MMIN_E = 1e-2, 1e-3


def _survival(m):
    """N(>m) / N(>m_min) of the mass law (Earth masses)."""
    return (m / MMIN_E) ** -0.3 * np.exp(-(m - MMIN_E) / M0_E)


def test_mass_law_quantiles_and_sample():
    u = np.array([1.0, 0.9, 0.5, 0.1, 1e-2, 1e-4, 1e-8])
    m = disk.mass_inverse_cdf(u)
    assert m[0] == MMIN_E or abs(m[0] / MMIN_E - 1.0) < 1e-14
    assert np.all(np.diff(m) > 0.0)
    assert np.max(np.abs(_survival(m) / u - 1.0)) < 1e-12
    # a sample of the generator's own draws: survival fractions within 5 binomial sigmas
    d = disk.planetesimal_disk(200000, 4321)
    me = d.m / disk.M_EARTH_MSUN
    assert me.min() >= MMIN_E * (1 - 1e-12)
    for q in (1.5e-3, 3e-3, 1e-2, 3e-2, 6e-2):
        p = float(_survival(q))
        frac = float(np.mean(me > q))
        assert abs(frac - p) < 5.0 * math.sqrt(p * (1 - p) / me.size), (q, frac, p)
    # well below m0 the law is the power law: N(>m1) / N(>m2) -> (m1 / m2)^-0.3
    a, b = 1.0e-3, 1.1e-3
    assert abs(_survival(b) / _survival(a) - (b / a) ** -0.3 * math.exp(-(b - a) / M0_E)) < 1e-15


def test_radius_from_density_two_g_per_cc():
    """R = (3 m / (4 pi rho))^{1/3}, rho = 2 g/cm^3, computed here in CGS from the IAU au and
    nominal solar and Earth masses: an Earth-mass body of that density has R = 8,932 km."""
    au_cm, msun_g, mearth_g = 1.495978707e13, 1.98841e33, 5.9722e27
    R_earthmass_cm = (3.0 * mearth_g / (4.0 * math.pi * 2.0)) ** (1.0 / 3.0)
    assert abs(R_earthmass_cm / 8.932e8 - 1.0) < 1e-3
    d = disk.planetesimal_disk(500, 77)
    m_g = d.m * msun_g
    R_cm = (3.0 * m_g / (4.0 * math.pi * 2.0)) ** (1.0 / 3.0)
    assert np.max(np.abs(d.radius * au_cm / R_cm - 1.0)) < 1e-12
    assert abs(disk.M_EARTH_MSUN * msun_g / mearth_g - 1.0) < 2e-5


def test_hill_spaced_disk_five_mutual_hill_radii():
    d = disk.hill_spaced_disk()
    G = 4.0 * math.pi ** 2
    r = np.linalg.norm(d.x, axis=1)
    v2 = np.sum(d.v * d.v, axis=1)
    a = 1.0 / (2.0 / r - v2 / (G * (1.0 + d.m)))
    assert d.n == 100 and np.all(d.m == 1e-2 * disk.M_EARTH_MSUN)
    assert abs(a[0] - 5.0) < 1e-9
    rh_mut = ((d.m[:-1] + d.m[1:]) / 3.0) ** (1.0 / 3.0) * 0.5 * (a[:-1] + a[1:])
    assert np.max(np.abs((a[1:] - a[:-1]) / rh_mut - 5.0)) < 1e-6
    assert 18.0 < a[-1] < 20.0            # "from 5 AU": 100 bodies reach ~19 AU


def test_orbital_elements_of_the_benchmark_disk():
    d = disk.planetesimal_disk(20000, 1002)
    G = 4.0 * math.pi ** 2
    mu = G * (1.0 + d.m)
    r = np.linalg.norm(d.x, axis=1)
    v2 = np.sum(d.v * d.v, axis=1)
    a = 1.0 / (2.0 / r - v2 / mu)
    h = np.cross(d.x, d.v)
    evec = ((v2 - mu / r)[:, None] * d.x - np.sum(d.x * d.v, axis=1)[:, None] * d.v) / mu[:, None]
    e = np.linalg.norm(evec, axis=1)
    inc = np.arccos(np.clip(h[:, 2] / np.linalg.norm(h, axis=1), -1.0, 1.0))
    assert a.min() > 5.0 - 1e-9 and a.max() < 20.0 + 1e-9
    # uniform in a: mean 12.5, standard deviation 15 / sqrt(12)
    assert abs(a.mean() - 12.5) < 5 * (15 / math.sqrt(12)) / math.sqrt(a.size)
    # Rayleigh(s): mean s sqrt(pi / 2), second moment 2 s^2
    for vals, s in ((e, 1e-6), (inc, 5e-7)):
        assert abs(vals.mean() / (s * math.sqrt(math.pi / 2)) - 1.0) < 0.03
        assert abs(np.mean(vals ** 2) / (2 * s * s) - 1.0) < 0.05
