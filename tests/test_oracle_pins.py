"""Pins of the oracle against things other than itself (CPU only).

Each test checks an oracle function against what the paper or the mathematics fixes: a library
routine (math.fsum), closed forms (two-body orbits from orbital elements, two-body energy and
angular momentum), brute force on tiny inputs (all ordered pairs, dense time sampling, BFS), an
independent route to the same quantity (barycentric-frame energy), convergence order, and a
hand-worked encounter whose shell crossings follow from straight-line geometry.
"""
import math

import numpy as np
import pytest

from paper_2304_07325_gb300 import disk

G = 4.0 * math.pi ** 2


# --------------------------------------------------------------------------------------------
# exact summation: the correctly rounded sum, pinned to Python's math.fsum
# --------------------------------------------------------------------------------------------
def test_fsum_matches_math_fsum(orc):
    rng = np.random.default_rng(1)
    cases = [
        rng.standard_normal(1000),
        rng.standard_normal(1000) * 10.0 ** rng.integers(-30, 30, 1000),
        np.array([1e100, 1.0, -1e100, 1e-100]),
        np.array([1.0, 2.0 ** -53, 2.0 ** -106]),          # half-way tie broken by a lower partial
        np.array([1.0, 2.0 ** -53]),                        # exact tie: round to even
        np.array([1.0, -2.0 ** -54, -2.0 ** -107]),
        np.array([]),
        np.array([0.1] * 10 + [-1.0]),
    ]
    big = rng.standard_normal(5000) * 1e8
    cases.append(np.concatenate([big, -big, [3.5e-9, 1e-30]]))
    for a in cases:
        assert orc.fsum(a) == math.fsum(a.tolist())


# --------------------------------------------------------------------------------------------
# partition function f_l (Sec. 3: l = 3) and the level weights
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("l", [1, 2, 3, 4])
def test_partition_polynomial_properties(orc, l):
    assert orc.partition(0.0, l) == 0.0 and orc.partition(1.0, l) == 1.0
    assert orc.partition(-0.3, l) == 0.0 and orc.partition(1.7, l) == 1.0
    xs = np.linspace(0.0, 1.0, 201)
    f = np.array([orc.partition(x, l) for x in xs])
    assert np.all(np.diff(f) >= 0.0)                                   # monotone
    # f(x) + f(1 - x) = 1, up to the rounding of a polynomial whose coefficients sum to < 2^(2l+2)
    assert np.max(np.abs(f + f[::-1] - 1.0)) < 4.0 ** (l + 1) * 2.0 ** -53
    # recover the polynomial from 2l+2 interior samples (exact for degree 2l+1) and check that its
    # first l derivatives vanish at 0 and 1
    nodes = 0.5 - 0.5 * np.cos(np.pi * (np.arange(2 * l + 2) + 0.5) / (2 * l + 2))
    coef = np.polynomial.polynomial.polyfit(nodes, [orc.partition(t, l) for t in nodes], 2 * l + 1)
    p = np.polynomial.Polynomial(coef)
    for d in range(1, l + 1):
        tol = 1e-11 * np.abs(p.deriv(d).coef).max()      # the fit's own conditioning
        assert abs(p.deriv(d)(0.0)) < tol and abs(p.deriv(d)(1.0)) < tol
    assert abs(p.deriv(l + 1)(0.0)) > 1e-3      # and no more than l


def test_partition_l1_is_textbook_smoothstep(orc):
    for x in np.linspace(0.0, 1.0, 101):
        assert abs(orc.partition(x, 1) - (3 * x * x - 2 * x ** 3)) < 4e-16


def test_level_weights_telescope(orc):
    P = orc.make_params(shell_ratio=2.08, l=3)
    R0 = 0.37
    for r in np.linspace(1e-4, 0.6, 997):
        w = [orc.weight(P, R0, k, r) for k in range(12)]
        assert all(-1e-15 <= t <= 1.0 + 1e-15 for t in w)
        Rk = [R0 / 2.08 ** k for k in range(13)]
        # w_0 + ... + w_K = g_K, which is 1 once r >= R_K
        for K in range(12):
            if r >= Rk[K] * (1 + 1e-12):
                assert abs(sum(w[:K + 1]) - 1.0) < 1e-14
        # at most two neighbouring levels share the force at any r
        nz = [k for k, t in enumerate(w) if t > 0.0]
        assert len(nz) <= 2 and (len(nz) < 2 or nz[1] == nz[0] + 1)


# --------------------------------------------------------------------------------------------
# Kepler drift vs closed-form propagation through orbital elements
# --------------------------------------------------------------------------------------------
def _ell_elements(x, v, mu):
    r = math.sqrt(x @ x)
    v2 = v @ v
    a = 1.0 / (2.0 / r - v2 / mu)
    h = np.cross(x, v)
    evec = ((v2 - mu / r) * x - (x @ v) * v) / mu
    e = math.sqrt(evec @ evec)
    P = evec / e
    Q = np.cross(h, P) / math.sqrt(h @ h)
    E0 = math.atan2((x @ v) / math.sqrt(mu * a), 1.0 - r / a)
    return a, e, P, Q, E0 - e * math.sin(E0)


def _bisect(f, lo, hi):
    for _ in range(300):
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        if f(mid) > 0.0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def closed_form_elliptic(x, v, mu, dt):
    a, e, P, Q, M0 = _ell_elements(x, v, mu)
    n = math.sqrt(mu / a ** 3)
    M = M0 + n * dt
    E = _bisect(lambda E: E - e * math.sin(E) - M, M - 1.0, M + 1.0)
    b = math.sqrt(1.0 - e * e)
    r = a * (1.0 - e * math.cos(E))
    pos = a * (math.cos(E) - e) * P + a * b * math.sin(E) * Q
    vel = math.sqrt(mu * a) / r * (-math.sin(E) * P + b * math.cos(E) * Q)
    return pos, vel


def closed_form_hyperbolic(x, v, mu, dt):
    r = math.sqrt(x @ x)
    v2 = v @ v
    aa = -1.0 / (2.0 / r - v2 / mu)          # |a|
    h = np.cross(x, v)
    evec = ((v2 - mu / r) * x - (x @ v) * v) / mu
    e = math.sqrt(evec @ evec)
    P = evec / e
    Q = np.cross(h, P) / math.sqrt(h @ h)
    H0 = math.asinh((x @ v) / (e * math.sqrt(mu * aa)))
    n = math.sqrt(mu / aa ** 3)
    M = e * math.sinh(H0) - H0 + n * dt
    H = _bisect(lambda H: e * math.sinh(H) - H - M, -50.0, 50.0)
    b = math.sqrt(e * e - 1.0)
    rr = aa * (e * math.cosh(H) - 1.0)
    pos = aa * (e - math.cosh(H)) * P + aa * b * math.sinh(H) * Q
    vel = n * aa * aa / rr * (-math.sinh(H) * P + b * math.cosh(H) * Q)
    return pos, vel


def _random_orbit(rng, e, mu, a):
    inc, node, peri, M = rng.uniform(0, math.pi), *rng.uniform(0, 2 * math.pi, 3)
    x, v = disk.elements_to_state(a, e, inc, node, peri, M, mu)
    return np.asarray(x, dtype=float), np.asarray(v, dtype=float)


@pytest.mark.parametrize("e", [0.02, 0.3, 0.7, 0.9])
def test_kepler_drift_elliptic_closed_form(orc, e):
    rng = np.random.default_rng(int(e * 100))
    mu = G
    for trial in range(20):
        a = rng.uniform(0.5, 30.0)
        x, v = _random_orbit(rng, e, mu, a)
        period = 2 * math.pi * math.sqrt(a ** 3 / mu)
        for dt in (1e-6 * period, 0.013 * period, 0.49 * period, 3.7 * period):
            st, x1, v1 = orc.kepler_drift(mu, dt, x, v)
            assert st == 0
            xr, vr = closed_form_elliptic(x, v, mu, dt)
            assert np.linalg.norm(x1 - xr) <= 5e-13 * a * max(1.0, dt / period)
            assert np.linalg.norm(v1 - vr) <= 5e-13 * math.sqrt(mu / a) / max(1e-2, 1 - e) * max(1.0, dt / period)


def test_kepler_drift_hyperbolic_closed_form(orc):
    rng = np.random.default_rng(5)
    mu = G
    for e in (1.05, 1.5, 3.0):
        for trial in range(10):
            q = rng.uniform(0.5, 5.0)
            aa = q / (e - 1.0)
            # state at pericentre, rotated, then drifted to a random time on either side
            x0 = np.array([q, 0.0, 0.0])
            v0 = np.array([0.0, math.sqrt(mu * (e + 1.0) / q), 0.0])
            Rm = np.linalg.qr(rng.standard_normal((3, 3)))[0]
            x0, v0 = Rm @ x0, Rm @ v0
            n = math.sqrt(mu / aa ** 3)
            t_start = rng.uniform(-3.0, 3.0) / n
            xs, vs = closed_form_hyperbolic(x0, v0, mu, t_start)
            for dt in (1e-5 / n, 0.3 / n, 2.0 / n):
                st, x1, v1 = orc.kepler_drift(mu, dt, xs, vs)
                assert st == 0
                xr, vr = closed_form_hyperbolic(x0, v0, mu, t_start + dt)
                scale = math.sqrt(xr @ xr)
                assert np.linalg.norm(x1 - xr) <= 2e-11 * scale
                assert np.linalg.norm(v1 - vr) <= 2e-11 * math.sqrt(vr @ vr)


def test_kepler_drift_many_orbits_phase(orc):
    """1,000 orbits in steps of 1/25 period: position error stays at the rounding level."""
    mu = G
    rng = np.random.default_rng(11)
    x, v = _random_orbit(rng, 0.1, mu, 10.0)
    period = 2 * math.pi * math.sqrt(1000.0 / mu)
    dt = period / 25.0
    xc, vc = x.copy(), v.copy()
    for _ in range(25 * 1000):
        st, xc, vc = orc.kepler_drift(mu, dt, xc, vc)
        assert st == 0
    xr, _ = closed_form_elliptic(x, v, mu, 25 * 1000 * dt)
    assert np.linalg.norm(xc - xr) / 10.0 < 1e-9


@pytest.mark.parametrize("h,steps", [(0.5 / 4 ** 12, 200000), (0.5 / 4 ** 6, 20000)])
def test_kepler_drift_short_intervals_unbiased(orc, h, steps):
    """Many drifts over the intervals of deep recursion levels (tau / M^k at 10 AU).  There
    f - 1 and g' - 1 (about -mu h^2 / (2 r^3), down to 2e-17 here) lie below half an ulp of 1:
    a drift that rounds f or g' to 1 loses them at every call, an error of one sign that adds up
    (3.5e-12 of the radius after 200,000 calls).  The exact motion on a circular orbit is a
    rotation by n t; the error must stay at the level of uncorrelated rounding."""
    mu = G
    R = 10.0
    x = np.array([R, 0.0, 0.0])
    v = np.array([0.0, math.sqrt(mu / R), 0.0])
    for _ in range(steps):
        st, x, v = orc.kepler_drift(mu, h, x, v)
        assert st == 0
    th = math.sqrt(mu / R ** 3) * h * steps
    xr = np.array([R * math.cos(th), R * math.sin(th), 0.0])
    assert np.linalg.norm(x - xr) / R < 1e-13


@pytest.mark.parametrize("direction", ["outbound", "inbound"])
def test_removal_at_the_closed_form_crossing_step(orc, direction):
    """A lone massless particle on a hyperbolic orbit (e = 1.5, q = 2 AU) moves on the exact
    two-body flow.  With rmax halfway between its closed-form distances at the ends of steps 4
    and 5 on the way out (rmin likewise on the way in), it must stay through step 4 and leave
    the system at the end of step 5, and stay removed."""
    mu, tau, e, q = G, 0.5, 1.5, 2.0
    xp = np.array([q, 0.0, 0.0])
    vp = np.array([0.0, math.sqrt(mu * (e + 1.0) / q), 0.0])
    t0 = 0.1 if direction == "outbound" else -6.0
    x0, v0 = closed_form_hyperbolic(xp, vp, mu, t0)
    r = [math.sqrt(p @ p) for p in (closed_form_hyperbolic(xp, vp, mu, t0 + k * tau)[0] for k in range(7))]
    lim = 0.5 * (r[4] + r[5])
    if direction == "outbound":
        assert r[4] < lim < r[5]
        params = orc.make_params(rmax=lim)
    else:
        assert r[4] > lim > r[5] and min(r[:5]) > lim
        params = orc.make_params(rmin=lim)
    sim = orc.OracleSim([x0], [v0], [0.0], [0.0], n_massive=0, params=params)
    for _ in range(4):
        sim.step(1)
        assert sim.alive[0] == 1 and sim.removals == 0
    sim.step(1)
    assert sim.alive[0] == 0 and sim.removals == 1
    x_removed = sim.x.copy()
    sim.step(2)
    assert sim.alive[0] == 0 and sim.removals == 0 and np.array_equal(sim.x, x_removed)


def test_removing_a_massless_particle_changes_no_other_body(orc):
    """A field particle on a circular orbit at 150 AU with rmax = 100 AU leaves at the end of the
    first step; having no mass, it never acted on the 40 bodies of the disk, whose states must
    equal, bit for bit, those of the same disk integrated without it."""
    d = disk.planetesimal_disk(40, 77)
    x = np.vstack([d.x, [[150.0, 0.0, 0.0]]])
    v = np.vstack([d.v, [[0.0, math.sqrt(G / 150.0), 0.0]]])
    m, rad = np.append(d.m, 0.0), np.append(d.radius, 0.0)
    a = orc.OracleSim(x, v, m, rad, n_massive=40, params=orc.make_params(rmax=100.0))
    b = orc.OracleSim(d.x, d.v, d.m, d.radius, params=orc.make_params(rmax=100.0), rhill=a.rhill[:40])
    a.step(1)
    b.step(1)
    assert a.alive[40] == 0 and a.removals == 1 and a.alive[:40].all() and b.removals == 0
    a.step(2)
    b.step(2)
    assert np.array_equal(a.x[:40], b.x) and np.array_equal(a.v[:40], b.v)


def test_kepler_drift_zero_dt_is_identity(orc):
    rng = np.random.default_rng(2)
    x, v = _random_orbit(rng, 0.2, G, 3.0)
    st, x1, v1 = orc.kepler_drift(G, 0.0, x, v)
    assert st == 0 and np.allclose(x1, x, rtol=0, atol=1e-15 * 3) and np.allclose(v1, v, rtol=0, atol=1e-14)


# --------------------------------------------------------------------------------------------
# close-encounter predicate vs dense sampling of the straight-line motion
# --------------------------------------------------------------------------------------------
def test_encounter_predicate_dense_sampling(orc):
    rng = np.random.default_rng(3)
    ts = np.linspace(0.0, 1.0, 20001)
    checked = 0
    for trial in range(3000):
        h = rng.uniform(0.05, 2.0)
        d = rng.standard_normal(3) * rng.uniform(0.01, 2.0)
        dv = rng.standard_normal(3) * rng.uniform(0.0, 3.0)
        R = rng.uniform(0.01, 1.5)
        dist = np.linalg.norm(d[None, :] + (ts * h)[:, None] * dv[None, :], axis=1)
        dmin = dist.min()
        grid_err = 0.5 * h * np.linalg.norm(dv) / (len(ts) - 1)
        if abs(dmin - R) <= grid_err + 1e-9:
            continue
        xi, vi = rng.standard_normal(3), rng.standard_normal(3)
        flag, contact = orc.encounter(xi, xi + d, vi, vi + dv, R, 1e-6, h)
        assert flag == int(dmin < R), (d, dv, R, h, dmin)
        checked += 1
    assert checked > 2500


def test_encounter_predicate_analytic_cases(orc):
    z = np.zeros(3)
    # head-on: closest approach 0 at t = 1; flagged over h = 2 (with contact), not over h = 0.5
    d, dv = np.array([2.0, 0, 0]), np.array([-2.0, 0, 0])
    assert orc.encounter(z, d, z, dv, 0.5, 0.1, 2.0) == (1, 1)
    assert orc.encounter(z, d, z, dv, 0.5, 0.1, 0.5)[0] == 0
    # receding pair outside R: never flagged
    assert orc.encounter(z, d, z, -dv, 1.9, 0.1, 100.0)[0] == 0
    # inside R at the start: flagged whatever the motion
    assert orc.encounter(z, d, z, -dv, 2.1, 0.1, 1e-9)[0] == 1
    # fly-by with impact parameter 0.3: flagged iff R > 0.3 and the approach happens within h
    d, dv = np.array([-1.0, 0.3, 0.0]), np.array([1.0, 0.0, 0.0])
    assert orc.encounter(z, d, z, dv, 0.31, 0.0, 1.5)[0] == 1
    assert orc.encounter(z, d, z, dv, 0.29, 0.0, 1.5)[0] == 0
    assert orc.encounter(z, d, z, dv, 0.31, 0.0, 0.9)[0] == 0       # closest point not reached
    # identical velocities (v2 = 0) outside R: not flagged, no division by zero
    assert orc.encounter(z, d, z, z, 0.5, 0.0, 1.0)[0] == 0


# --------------------------------------------------------------------------------------------
# union-find vs breadth-first search
# --------------------------------------------------------------------------------------------
def _bfs_labels(n, edges):
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    lab = [-1] * n
    for s in range(n):
        if lab[s] >= 0:
            continue
        comp, queue = [s], [s]
        lab[s] = s
        while queue:
            u = queue.pop()
            for w in adj[u]:
                if lab[w] < 0:
                    lab[w] = s
                    comp.append(w)
                    queue.append(w)
        m = min(comp)
        for u in comp:
            lab[u] = m
    return lab


def test_union_find_matches_bfs(orc):
    rng = np.random.default_rng(4)
    for trial in range(200):
        n = int(rng.integers(1, 80))
        ne = int(rng.integers(0, 2 * n))
        edges = []
        for _ in range(ne):
            a, b = sorted(rng.integers(0, n, 2))
            if a != b:
                edges.append((int(a), int(b)))
        edges = sorted(set(edges))
        lab = orc.union_find(n, edges if edges else np.zeros((0, 2), dtype=np.int32))
        assert list(lab) == _bfs_labels(n, edges)


# --------------------------------------------------------------------------------------------
# trapezoid kick vs brute force over all ordered pairs
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n,nm", [(2, 2), (3, 1), (7, 7), (17, 5), (40, 40), (64, 9)])
def test_trapezoid_equals_brute_force(orc, n, nm):
    rng = np.random.default_rng(n * 100 + nm)
    x = rng.standard_normal((n, 3))
    m = np.concatenate([rng.uniform(1e-6, 1e-3, nm), np.zeros(n - nm)])
    rhill = np.concatenate([rng.uniform(0.05, 0.3, nm), np.zeros(n - nm)])
    P = orc.make_params(hill_scale=2.0)
    sim = orc.OracleSim(x, np.zeros((n, 3)), m, np.zeros(n), n_massive=nm, params=P, rhill=rhill)
    trap = [(i, j) for i in range(nm) for j in range(i + 1, n)]
    flagged = sorted(p for p in trap if rng.random() < 0.4)
    a = sim.accel_trapezoid(np.array(flagged, dtype=np.int32).reshape(-1, 2))
    fset = set(flagged)
    for i in range(n):
        terms = [[], [], []]
        for j in range(n):
            if j == i:
                continue
            p = (min(i, j), max(i, j))
            if p[0] >= nm:
                continue            # field-field pairs do not interact
            d = x[j] - x[i]
            r = math.sqrt(d @ d)
            w = 1.0
            if p in fset:
                w = orc.weight(P, P.hill_scale * (rhill[i] + rhill[j]), 0, r)
            for c in range(3):
                terms[c].append(G * m[j] * w * d[c] / r ** 3)
        for c in range(3):
            ref = math.fsum(terms[c])
            scale = math.fsum(abs(t) for t in terms[c]) + 1e-300
            assert abs(a[i, c] - ref) <= 1e-14 * scale


# --------------------------------------------------------------------------------------------
# energy and angular momentum: closed forms and the barycentric route
# --------------------------------------------------------------------------------------------
def test_two_body_energy_and_momentum_closed_form(orc):
    rng = np.random.default_rng(6)
    for trial in range(20):
        m = 10.0 ** rng.uniform(-9, -3)
        a, e = rng.uniform(1, 30), rng.uniform(0.0, 0.8)
        mu = G * (1.0 + m)
        x, v = disk.elements_to_state(a, e, rng.uniform(0, 3), *rng.uniform(0, 6, 3), mu)
        sim = orc.OracleSim(x.reshape(1, 3), v.reshape(1, 3), [m], [0.0])
        E, L = sim.energy()
        mred = m / (1.0 + m)
        assert abs(E - (-G * m / (2.0 * a))) <= 1e-13 * abs(E)
        assert abs(np.linalg.norm(L) - mred * math.sqrt(mu * a * (1 - e * e))) <= 1e-13 * np.linalg.norm(L)


def test_energy_equals_barycentric_frame(orc):
    rng = np.random.default_rng(7)
    n = 6
    x = rng.standard_normal((n, 3)) * 5.0
    vh = rng.standard_normal((n, 3))
    m = 10.0 ** rng.uniform(-6, -2, n)
    sim = orc.OracleSim(x, vh, m, np.zeros(n))
    E, L = sim.energy()
    # barycentric positions and velocities of all n+1 bodies (sun = body 0)
    Mt = 1.0 + m.sum()
    X0 = -(m[:, None] * x).sum(0) / Mt
    V0 = -(m[:, None] * vh).sum(0) / Mt
    X = x + X0
    V = vh + V0
    ke = 0.5 * 1.0 * V0 @ V0 + 0.5 * (m * (V * V).sum(1)).sum()
    pe = -(G * m / np.linalg.norm(X - X0, axis=1)).sum()
    for i in range(n):
        for j in range(i + 1, n):
            pe -= G * m[i] * m[j] / np.linalg.norm(X[i] - X[j])
    Lb = np.cross(X0, V0) * 1.0 + (m[:, None] * np.cross(X, V)).sum(0)
    assert abs(E - (ke + pe)) <= 1e-13 * abs(ke) + 1e-13 * abs(pe)
    assert np.allclose(L, Lb, rtol=1e-12, atol=1e-14 * np.linalg.norm(Lb))


def test_democratic_heliocentric_round_trip(orc):
    d = disk.planetesimal_disk(200, 5)
    sim = orc.OracleSim(d.x, d.v, d.m, d.radius)
    # barycentric momentum of the planets plus the sun's is zero, and v_hel = v_bary + P / m0
    vb = sim.v
    V0 = -(d.m[:, None] * vb).sum(0) / 1.0
    assert np.allclose(vb - V0, d.v, rtol=0, atol=1e-15 * np.abs(d.v).max() * 4)
    assert np.allclose(sim.velocity_helio(), d.v, rtol=0, atol=1e-15 * np.abs(d.v).max() * 4)


# --------------------------------------------------------------------------------------------
# whole steps
# --------------------------------------------------------------------------------------------
def test_massless_test_particle_follows_exact_orbit(orc):
    """One field particle and no massive body: P = 0 and no pairs, so the step is a pure Kepler
    drift with mu = G m0 and the trajectory is the exact two-body orbit."""
    rng = np.random.default_rng(8)
    x, v = _random_orbit(rng, 0.4, G, 7.0)
    sim = orc.OracleSim(x.reshape(1, 3), v.reshape(1, 3), [0.0], [0.0], n_massive=0,
                        params=orc.make_params(dt=0.37))
    assert sim.step(200) == 0
    xr, vr = closed_form_elliptic(x, v, G, 200 * 0.37)
    assert np.linalg.norm(sim.x[0] - xr) < 1e-11 * 7.0
    assert np.linalg.norm(sim.v[0] - vr) < 1e-11 * math.sqrt(G / 7.0) * 3


def _planets():
    rng = np.random.default_rng(9)
    a = np.array([5.2, 9.5, 19.2])
    m = np.array([9.5e-4, 2.9e-4, 4.4e-5])
    x, v = disk.elements_to_state(a, [0.05, 0.06, 0.05], [0.02, 0.04, 0.01],
                                  rng.uniform(0, 6, 3), rng.uniform(0, 6, 3), rng.uniform(0, 6, 3),
                                  G * (1.0 + m))
    return x, v, m


def test_second_order_convergence(orc):
    """Global error of the split shrinks as tau^2 (no encounters: planets far apart)."""
    x, v, m = _planets()
    T = 24.0

    def run(tau):
        P = orc.make_params(dt=tau, hill_scale=0.5)
        s = orc.OracleSim(x, v, m, np.zeros(3), params=P)
        assert s.step(int(round(T / tau))) == 0
        assert s.npairs == 0
        return s.x.copy()

    ref = run(0.0125)
    errs = [np.abs(run(t) - ref).max() for t in (0.4, 0.2, 0.1)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.8 and 3.3 < r2 < 4.8, errs


def test_symplectic_energy_bounded_hill_spaced_disk(orc):
    """Sec. 3 accuracy disk: 100 bodies of 1e-2 Earth masses 5 mutual Hill radii apart, tau = 0.1
    yr, 10^4 steps: the energy error stays bounded and shows no secular drift, angular momentum
    is kept to rounding, and no contact happens."""
    d = disk.hill_spaced_disk()
    P = orc.make_params(dt=0.1)
    sim = orc.OracleSim(d.x, d.v, d.m, d.radius, params=P)
    E0, L0 = sim.energy()
    errs, ts = [], []
    coll = 0
    for k in range(100):
        assert sim.step(100) >= 0
        coll += sim.collisions
        E, L = sim.energy()
        errs.append((E - E0) / abs(E0))
        ts.append((k + 1) * 100 * 0.1)
        assert np.linalg.norm(L - L0) / np.linalg.norm(L0) < 1e-12
    errs = np.array(errs)
    assert np.abs(errs).max() < 1e-7
    slope = np.polyfit(ts, errs, 1)[0]
    assert abs(slope * ts[-1]) < 0.5 * np.abs(errs).max() + 1e-12
    assert coll == 0


def test_hand_worked_three_body_encounter(orc):
    """Sun plus two small bodies far out (1e4 AU, where solar tides are negligible) on crossing
    straight lines with impact parameter b.  With R_0 = 1 AU and shell ratio 2.08, b = 0.05 lies
    between R_5 and R_4, so the pair is flagged down to level 4 and level 5 is entered but never
    flagged.  The flagged sub-steps per level follow from the straight-line geometry alone."""
    lam, ratio, M, tau = 6.5, 2.08, 4, 0.5
    b, tc, u = 0.05, 1.3, 1.0
    m = 1e-9
    rh = 1.0 / (2.0 * lam)
    R0 = lam * (rh + rh)
    x = np.array([[1e4, -tc * u, 0.0], [1e4 + b, tc * u, 0.0]])
    v = np.array([[0.0, u, 0.0], [0.0, -u, 0.0]])
    P = orc.make_params(dt=tau, M=M, shell_ratio=ratio, hill_scale=lam)
    sim = orc.OracleSim(x, v, [m, m], [1e-6, 1e-6], params=P, rhill=[rh, rh])
    E0, _ = sim.energy()

    Rk = [R0]
    for k in range(1, 30):
        Rk.append(Rk[-1] / ratio)

    def dmin(ta, tb):
        t = min(max(tc, ta), tb)
        return math.hypot(b, 2.0 * u * (t - tc))

    def expect_step(s):
        flags, deepest = [0] * 30, [0]

        def E(k, ta, h):
            deepest[0] = max(deepest[0], k)
            dm = dmin(ta, ta + h)
            assert abs(dm - Rk[k]) > 1e-6 * Rk[k]
            if dm < Rk[k]:
                flags[k] += 1
                for r in range(M):
                    E(k + 1, ta + r * h / M, h / M)

        ta = s * tau
        dm = dmin(ta, ta + tau)
        if dm < R0:
            flags[0] = 1
            for r in range(M):
                E(1, ta + r * tau / M, tau / M)
        return flags, deepest[0]

    saw_depth = 0
    for s in range(7):
        assert sim.step(1) == 0
        flags, deepest = expect_step(s)
        assert sim.level_flags[:30] == flags, (s, sim.level_flags[:8], flags[:8])
        assert sim.max_depth_seen == deepest
        saw_depth = max(saw_depth, deepest)
    assert saw_depth == 5


@pytest.mark.parametrize("tc", [200.0, 200.3, 200.77])
def test_encounter_energy_recovery(orc, tc):
    """The same fly-by, slow enough (relative speed 0.1 AU/yr) that every shell transition is
    crossed over several sub-steps.  The pair starts 20 AU apart and is integrated until it is 20 AU
    apart again: the energy error is then a tiny fraction of the interaction energy G m^2 / b
    reached at closest approach."""
    lam, ratio, M, tau = 6.5, 2.08, 4, 0.5
    b, u, m = 0.05, 0.05, 1e-9
    rh = 1.0 / (2.0 * lam)
    x = np.array([[1e4, -tc * u, 0.0], [1e4 + b, tc * u, 0.0]])
    v = np.array([[0.0, u, 0.0], [0.0, -u, 0.0]])
    P = orc.make_params(dt=tau, M=M, shell_ratio=ratio, hill_scale=lam)
    sim = orc.OracleSim(x, v, [m, m], [1e-6, 1e-6], params=P, rhill=[rh, rh])
    E0, _ = sim.energy()
    depth = 0
    for _ in range(int(2.0 * tc / tau)):
        assert sim.step(1) == 0
        depth = max(depth, sim.max_depth_seen)
    assert depth == 5
    assert np.linalg.norm(sim.x[1] - sim.x[0]) > 19.0
    E1, _ = sim.energy()
    assert abs(E1 - E0) <= 1e-6 * G * m * m / b


def test_field_particles_do_not_interact(orc):
    """Sec. 2: field particles feel only massive ones.  A second field particle placed next to the
    first changes nothing in the first's trajectory, bit for bit."""
    d = disk.planetesimal_disk(1, 21, n_field=1)
    x = np.vstack([d.x, d.x[1] + [1e-3, 0, 0]])
    v = np.vstack([d.v, d.v[1]])
    m = np.array([d.m[0], 0.0, 0.0])
    r = np.array([d.radius[0], 0.0, 0.0])
    a = orc.OracleSim(x, v, m, r, n_massive=1)
    bsim = orc.OracleSim(x[:2], v[:2], m[:2], r[:2], n_massive=1)
    for _ in range(50):
        a.step()
        bsim.step()
        assert a.npairs == bsim.npairs
    assert np.array_equal(a.x[:2], bsim.x) and np.array_equal(a.v[:2], bsim.v)


def test_head_on_collision_merges_conserving_mass_and_momentum(orc):
    """Two bodies on a head-on course far from the sun: they merge at contact into one body with
    the summed mass and the volume-additive radius, the other index leaves the system, and the
    merged body moves on with the pair's centre of mass (the trajectory of a test particle
    started at the centre of mass, up to the tiny solar tide across the pair)."""
    m1, m2, R = 2e-9, 1e-9, 1e-3
    x = np.array([[1e4, -0.6, 0.0], [1e4, 0.6, 0.0]])
    v = np.array([[0.0, 0.3, 0.0], [0.0, -0.3, 0.0]])
    P = orc.make_params(dt=0.5, hill_scale=6.5)
    sim = orc.OracleSim(x, v, [m1, m2], [R, R], params=P, rhill=[0.05, 0.05])
    xc = (m1 * x[0] + m2 * x[1]) / (m1 + m2)
    vc = (m1 * v[0] + m2 * v[1]) / (m1 + m2)
    com = orc.OracleSim(xc.reshape(1, 3), vc.reshape(1, 3), [0.0], [0.0], n_massive=0, params=P)
    merges = 0
    for _ in range(6):
        assert sim.step(1) == 0
        merges += sim.mergers
        com.step(1)
    assert merges == 1 and list(sim.alive) == [1, 0]
    assert sim.m[0] == m1 + m2 and sim.m[1] == 0.0
    assert abs(sim.radius[0] - R * 2.0 ** (1.0 / 3.0)) < 1e-15
    assert abs(sim.rhill[0] - 0.05 * ((m1 + m2) / m1) ** (1.0 / 3.0)) < 1e-15
    vh = sim.velocity_helio()
    assert np.linalg.norm(vh[0] - com.v[0]) < 1e-9
    assert np.linalg.norm(sim.x[0] - com.x[0]) < 1e-8
    E, L = sim.energy()
    assert np.isfinite(E) and np.all(np.isfinite(L))


# --------------------------------------------------------------------------------------------
# correctly rounded cube root (Hill radii and merged radii), pinned by exact rational arithmetic
# --------------------------------------------------------------------------------------------
def _is_nearest_cbrt(x: float, y: float) -> bool:
    """y is the double nearest the real cube root of x > 0: x lies strictly between the cubes of
    the midpoints from y to its neighbours (exact rationals; the cube is increasing)."""
    from fractions import Fraction
    X, Y = Fraction(x), Fraction(y)
    hi = (Y + Fraction(math.nextafter(y, math.inf))) / 2
    lo = (Y + Fraction(math.nextafter(y, 0.0))) / 2
    return lo ** 3 < X < hi ** 3


def test_cbrt_rn_is_the_nearest_double(orc):
    from fractions import Fraction
    rng = np.random.default_rng(12)
    xs = [float(t) * 2.0 ** int(e) for t, e in zip(rng.uniform(0.5, 1.0, 3000), rng.integers(-1074, 1024, 3000))]
    xs = [x for x in xs if 0.0 < x < math.inf]
    xs += [5e-324, 2.2250738585072014e-308, 2.225073858507201e-308, 1.7976931348623157e308]
    # the hardest inputs: x = RN(b^3) for midpoints b between neighbouring doubles, whose cube roots
    # sit within a hair of a rounding boundary
    for y in rng.uniform(1.0, 2.0, 3000) * 2.0 ** rng.integers(-300, 300, 3000):
        b = (Fraction(float(y)) + Fraction(math.nextafter(float(y), math.inf))) / 2
        xs.append(float(b ** 3))
    # the disk's mass ratios m / 3 m0 and merged-radius sums
    d = disk.planetesimal_disk(2000, 77)
    xs += [float(t) for t in d.m / 3.0] + [float(t) for t in d.radius[:-1] ** 3 + d.radius[1:] ** 3]
    for x in xs:
        y = orc.cbrt_rn(x)
        assert _is_nearest_cbrt(x, y), x
        assert orc.cbrt_rn(-x) == -y
    # exact cubes have exact roots; zero and non-finite values pass through
    for k in range(-40, 41):
        assert orc.cbrt_rn(float(k) ** 3) == float(k)
        assert orc.cbrt_rn(8.0 ** k) == 2.0 ** k
    assert orc.cbrt_rn(0.0) == 0.0 and math.copysign(1.0, orc.cbrt_rn(-0.0)) == -1.0
    assert orc.cbrt_rn(math.inf) == math.inf and math.isnan(orc.cbrt_rn(math.nan))


def test_hill_radius_from_the_osculating_orbit(orc):
    """rH_i = a_i (m_i / 3 m0)^{1/3}, a_i the heliocentric semi-major axis of the two-body orbit
    with mu = G (m0 + m_i): bodies placed on orbits of known a (circular and eccentric, from
    orbital elements with that mu) give it to rounding; an unbound body uses its distance; a field
    particle has none.  A heavy body and m0 != 1 make each ingredient visible: mu = G m0 moves a
    by ~m/m0, m/m0 instead of m/3m0 moves rH by 3^{1/3}."""
    rng = np.random.default_rng(3)
    for m0 in (1.0, 2.5):
        P = orc.make_params(m0=m0)
        xs, vs, ms, want = [], [], [], []
        for m in (1e-3 * m0, 3e-8 * m0, 0.02 * m0):
            mu = G * (m0 + m)
            for a, e in ((5.0, 0.0), (12.5, 0.0), (7.0, 0.3), (19.0, 0.8)):
                inc, node, peri, M = rng.uniform(0, 1.0), *rng.uniform(0, 2 * math.pi, 3)
                x, v = disk.elements_to_state(a, e, inc, node, peri, M, mu)
                xs.append(x); vs.append(v); ms.append(m)
                want.append(a * (m / (3.0 * m0)) ** (1.0 / 3.0))
            # unbound: 1.5x the escape speed at r = 8
            r = 8.0
            xs.append([0.0, r, 0.0]); vs.append([1.5 * math.sqrt(2.0 * mu / r), 0.0, 0.0]); ms.append(m)
            want.append(r * (m / (3.0 * m0)) ** (1.0 / 3.0))
        xs.append([9.0, 0.0, 0.0]); vs.append([0.0, math.sqrt(G * m0 / 9.0), 0.0]); ms.append(0.0)
        want.append(0.0)
        n = len(ms)
        sim = orc.OracleSim(np.array(xs), np.array(vs), np.array(ms), np.zeros(n), n_massive=n, params=P)
        rel = np.abs(sim.rhill - np.array(want)) / np.maximum(np.array(want), 1e-300)
        assert rel.max() < 2e-15, rel
        assert sim.rhill[-1] == 0.0
