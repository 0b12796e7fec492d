"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the
mathematics, independent of the oracle's own code.

Each test below would fail on a plausible transcription mistake in the oracle
(a dropped term, a wrong sign, index or coefficient):

* Newtonian brute force at N = 3 and exact pair antisymmetry;
* the c -> infinity limit and exact linearity of the result in 1/c^2;
* the 1PN circular-orbit frequency and periastron advance of a test star
  (closed forms of the harmonic-gauge test-body equation, Eq. 5);
* the limited equations (Eq. 1-6) differ from the general EIH equations only
  by terms of fixed degree in the star mass (Section 2: the star-star 1PN
  interaction is dropped), checked by exact polynomial-degree ratios;
* the EIH evaluator itself reproduces the textbook two-body 1PN relative
  acceleration (Kidder 1995) and two-body 1PN energy (Blanchet 2014), and
  conserves its energy and momentum through 1PN order;
* Eq. 7 and Eq. 8 are conserved by Eq. 1-6 through 1PN order (along the
  flow dE/dt and dP/dt start at O(1/c^4));
* the integrator's convergence order in each velocity mode;
* rotation and translation invariance, thread-count independence.
"""
import math

import numpy as np
import pytest

from paper_1801_07986_b300.inputs import make_cluster


def _rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


def _random_state(n, seed, m_bh=1.0, m_star=1e-3, vscale=0.3, spread=1.0):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, 3)) * spread
    x[0] = 0.0
    v = rng.normal(size=(n, 3)) * vscale
    m = np.full(n, m_star)
    m[0] = m_bh
    return x, v, m


# ------------------------------------------------------------ Newtonian --

def test_newton_three_bodies_by_hand(orc):
    """Hole + 2 stars: Newton's law written out pair by pair (c = inf)."""
    G, eps = 1.3, 0.05
    x = np.array([[0.1, -0.2, 0.3], [1.0, 0.5, -0.25], [-0.7, 0.9, 0.4]])
    v = np.array([[0.0, 0.0, 0.0], [0.1, 0.2, 0.3], [-0.3, 0.1, 0.2]])
    m = np.array([2.0, 0.3, 0.7])

    def pull(i, j, soft):
        d = x[j] - x[i]
        r2 = d @ d + (eps * eps if soft else 0.0)
        return G * m[j] * d / r2 ** 1.5

    want = np.array([pull(0, 1, False) + pull(0, 2, False),
                     pull(1, 0, False) + pull(1, 2, True),
                     pull(2, 0, False) + pull(2, 1, True)])
    got = orc.accel(x, v, m, G=G, c=np.inf, eps=eps)
    assert np.all(_rel(got, want) < 1e-15)


def test_newton_momentum_conserved_exactly(orc):
    """sum_a m_a a_a = 0 for the Newtonian part (pair antisymmetry)."""
    x, v, m = make_cluster(200, 0.1, 11)
    a = orc.accel(x, v, m, c=np.inf, eps=1e-3)
    f = (m[:, None] * a).sum(0)
    scale = (m[:, None] * np.abs(a)).sum(0)
    assert np.all(np.abs(f) < 1e-14 * scale)


def test_c_infinity_is_newtonian_and_pn_is_linear_in_inv_c2(orc):
    x, v, m = make_cluster(96, 0.2, 12)
    eps = 1e-3
    a_inf = orc.accel(x, v, m, c=np.inf, eps=eps)
    a_newt = orc.newton_accel(x, m, eps=eps)
    assert np.all(_rel(a_inf, a_newt) < 1e-14)
    d1 = (orc.accel(x, v, m, c=20.0, eps=eps) - a_inf) * 20.0 ** 2
    d2 = (orc.accel(x, v, m, c=7.0, eps=eps) - a_inf) * 7.0 ** 2
    assert np.all(_rel(d1, d2) < 1e-9)
    assert np.all(np.linalg.norm(d1, axis=1) > 0)


# ------------------------------------------------------ test-body closed forms --

def test_circular_orbit_frequency(orc):
    """Eq. 5 on a circular orbit: omega^2 = GM/r^3 (1 - 3 GM/(c^2 r)) + O(c^-4)."""
    G, M, c = 1.0, 1.0, 40.0
    for r in (0.5, 1.0, 3.0):
        om2 = G * M / r ** 3 * (1.0 - 3.0 * G * M / (c * c * r))
        vt = math.sqrt(om2) * r
        x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
        v = np.array([[0.0, 0.0, 0.0], [0.0, vt, 0.0]])
        m = np.array([M, 0.0])
        a = orc.accel(x, v, m, G=G, c=c)[1]
        want = -om2 * r
        beta = G * M / (c * c * r)
        assert abs(a[0] - want) <= 5 * beta ** 2 * abs(want)
        assert abs(a[1]) < 1e-15 and abs(a[2]) < 1e-15
        # a wrong 1PN coefficient would show up at O(beta), not O(beta^2)
        assert abs(a[0] - (-G * M / r ** 2)) > 2.5 * beta * G * M / r ** 2


def _periapsis_angles(orc, c, a_orb, e, steps_per_orbit, n_orbits):
    G, M = 1.0, 1.0
    rp = a_orb * (1 - e)
    vp = math.sqrt(G * M * (1 + e) / rp)
    x = np.array([[0.0, 0.0, 0.0], [rp, 0.0, 0.0]])
    v = np.array([[0.0, 0.0, 0.0], [0.0, vp, 0.0]])
    m = np.array([M, 0.0])
    period = 2 * math.pi * math.sqrt(a_orb ** 3 / (G * M))
    dt = period / steps_per_orbit
    a = orc.accel(x, v, m, c=c)
    angles = []
    prev = None
    for _ in range(int(steps_per_orbit * (n_orbits + 0.5))):
        xn, vn, an = orc.step(x, v, m, a, dt, 1, c=c)
        s_old = x[1] @ v[1]
        s_new = xn[1] @ vn[1]
        if s_old < 0.0 <= s_new:
            # x.v crosses zero upward at periapsis: interpolate the angle
            f = -s_old / (s_new - s_old)
            th0 = math.atan2(x[1, 1], x[1, 0])
            th1 = math.atan2(xn[1, 1], xn[1, 0])
            dth = (th1 - th0 + math.pi) % (2 * math.pi) - math.pi
            th = th0 + f * dth
            if prev is not None:
                while th < prev - math.pi:
                    th += 2 * math.pi
            angles.append(th)
            prev = th
        x, v, a = xn, vn, an
    return np.array(angles)


def test_periastron_advance(orc):
    """Test star (m = 0) about the hole: the periapsis advances by
    6 pi G M / (c^2 a (1 - e^2)) per orbit (Eq. 5); the same run at c = inf
    removes the integrator's own precession."""
    a_orb, e, c = 1.0, 0.5, 100.0
    th_pn = _periapsis_angles(orc, c, a_orb, e, 2000, 8)
    th_n = _periapsis_angles(orc, np.inf, a_orb, e, 2000, 8)
    k = min(len(th_pn), len(th_n))
    assert k >= 7
    rate_pn = np.polyfit(np.arange(k), th_pn[:k], 1)[0]
    rate_n = np.polyfit(np.arange(k), th_n[:k], 1)[0]
    want = 6 * math.pi / (c * c * a_orb * (1 - e * e))
    got = rate_pn - rate_n
    assert abs(got - want) < 2e-3 * want, (got, want)


# ------------------------------------------------------------ EIH cross-check --

def _zero_momentum(v, m):
    v = v.copy()
    v[0] = -(m[1:, None] * v[1:]).sum(0) / m[0]
    return v


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_limited_equals_eih_up_to_dropped_orders(orc, seed):
    """Section 2: the limited equations keep every EIH term of the hole-star
    interaction.  With the hole's velocity set by zero momentum, the
    difference limited - EIH is a homogeneous polynomial of degree 2 in the
    star masses for a star and of degree 3 for the hole, so halving every
    star mass divides it by exactly 4 and 8.  A wrong or missing retained term
    would leave a degree-0 or degree-1 part and break the ratios."""
    x, v, m = _random_state(7, seed, m_bh=1.0, m_star=0.05, vscale=0.4)
    c = 6.0

    def diff(scale):
        mm = m.copy()
        mm[1:] *= scale
        vv = _zero_momentum(v, mm)
        return orc.accel(x, vv, mm, c=c) - orc.eih_accel(x, vv, mm, c=c)

    d1, d2, d3 = diff(1.0), diff(0.5), diff(0.25)
    np.testing.assert_allclose(d1[1:] / d2[1:], 4.0, rtol=1e-6)
    np.testing.assert_allclose(d2[1:] / d3[1:], 4.0, rtol=1e-6)
    np.testing.assert_allclose(d1[0] / d2[0], 8.0, rtol=1e-6)
    np.testing.assert_allclose(d2[0] / d3[0], 8.0, rtol=1e-6)


def test_eih_two_body_matches_kidder(orc):
    """Two-body EIH relative acceleration in the centre-of-mass frame equals
    the harmonic-gauge 1PN relative acceleration a = -(Gm/r^2)[(1+A) n + B v],
    A = [(1+3nu) v^2 - 3/2 nu rdot^2 - 2(2+nu) Gm/r]/c^2,
    B = -2(2-nu) rdot/c^2 (Kidder, PRD 52, 821 (1995), Eq. 2.2)."""
    G, c = 1.0, 5.0
    m1, m2 = 0.7, 0.45
    mt = m1 + m2
    nu = m1 * m2 / mt ** 2
    xr = np.array([1.1, -0.4, 0.3])
    vr = np.array([0.2, 0.6, -0.1])
    x = np.array([m2 / mt * xr, -m1 / mt * xr])
    v = np.array([m2 / mt * vr, -m1 / mt * vr])
    m = np.array([m1, m2])
    a = orc.eih_accel(x, v, m, G=G, c=c)
    r = np.linalg.norm(xr)
    nvec = xr / r
    rdot = nvec @ vr
    v2 = vr @ vr
    A = ((1 + 3 * nu) * v2 - 1.5 * nu * rdot ** 2 - 2 * (2 + nu) * G * mt / r) / c ** 2
    B = -2 * (2 - nu) * rdot / c ** 2
    want = -(G * mt / r ** 2) * ((1 + A) * nvec + B * vr)
    np.testing.assert_allclose(a[0] - a[1], want, rtol=1e-13, atol=1e-15)


def test_eih_two_body_energy_matches_textbook(orc):
    """E_1PN of a two-body system in the centre-of-mass frame:
    3/8 (1-3nu) mu v^4 + 1/2 (G m mu/r)[(3+nu) v^2 + nu rdot^2 + G m/r]
    (Blanchet, Living Rev. Rel. 17, 2 (2014), two-body 1PN energy)."""
    G, c = 1.0, 3.0
    m1, m2 = 0.8, 0.3
    mt = m1 + m2
    mu = m1 * m2 / mt
    nu = mu / mt
    xr = np.array([0.9, 0.2, -0.5])
    vr = np.array([-0.3, 0.7, 0.25])
    x = np.array([m2 / mt * xr, -m1 / mt * xr])
    v = np.array([m2 / mt * vr, -m1 / mt * vr])
    e = orc.eih_energy(x, v, np.array([m1, m2]), G=G, c=c)
    r = np.linalg.norm(xr)
    rdot = xr @ vr / r
    v2 = vr @ vr
    e1 = (0.375 * (1 - 3 * nu) * mu * v2 ** 2
          + 0.5 * G * mt * mu / r * ((3 + nu) * v2 + nu * rdot ** 2 + G * mt / r)) / c ** 2
    e0 = 0.5 * mu * v2 - G * mt * mu / r
    assert abs(e["E_N"] - e0) < 1e-14
    assert abs(e["E_PN"] - e1) < 1e-14 * abs(e1) + 1e-16


def _balance(E, A, x, v, m, c, key, h=1e-4):
    """d(key)/dt along the flow (xdot = v, vdot = A), by a 4th-order central
    difference of the conserved quantity along (v, a)."""
    a = A(x, v, m, c)
    f = lambda s: E(x + s * v, v + s * a, m, c)[key]
    return (8 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12 * h)


def _triple():
    m = np.array([1.0, 0.3, 0.2])
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.05], [0.0, -2.0, 0.3]])
    v = np.array([[0.0, 0.0, 0.0], [0.1, 1.08, 0.0], [0.87, 0.2, 0.02]])
    v -= (m[:, None] * v).sum(0) / m.sum()
    return x, v, m


def test_eih_energy_and_momentum_balance(orc):
    """The EIH equations conserve the EIH energy and momentum through 1PN
    order: along the flow dE/dt and dP/dt vanish at O(1/c^2) and start at
    O(1/c^4), so doubling c divides them by 16 (an error in any 1PN term of
    the equations or of E, P would leave an O(1/c^2) part, ratio 4).  Three
    bodies of comparable mass exercise the three-body terms."""
    x, v, m = _triple()
    E = lambda xx, vv, mm, c: orc.eih_energy(xx, vv, mm, c=c)
    A = lambda xx, vv, mm, c: orc.eih_accel(xx, vv, mm, c=c)
    for key in ("E", "P"):
        r = [_balance(E, A, x, v, m, c, key) for c in (10.0, 20.0, 40.0)]
        np.testing.assert_allclose(np.asarray(r[0]) / r[1], 16.0, rtol=5e-3)
        np.testing.assert_allclose(np.asarray(r[1]) / r[2], 16.0, rtol=5e-3)


@pytest.mark.parametrize("m_star,rtol", [(1e-9, 1e-5), (1e-3, 2e-2)])
def test_limited_energy_and_momentum_balance(orc, m_star, rtol):
    """Eq. 7 and Eq. 8 are conserved by Eq. 1-6 through 1PN order, up to the
    dropped terms of degree >= 3 in the star masses: dE/dt and dP/dt scale
    as 1/c^4 (ratio 16 when c doubles) once the star masses are small."""
    rng = np.random.default_rng(0)
    n = 6
    x = rng.normal(size=(n, 3))
    x[0] = 0.0
    v = rng.normal(size=(n, 3)) * 0.4
    m = np.full(n, m_star)
    m[0] = 1.0
    v = _zero_momentum(v, m)
    E = lambda xx, vv, mm, c: orc.energy(xx, vv, mm, c=c)
    A = lambda xx, vv, mm, c: orc.accel(xx, vv, mm, c=c)
    for key in ("E", "P"):
        r = [_balance(E, A, x, v, m, c, key) for c in (10.0, 20.0)]
        np.testing.assert_allclose(np.asarray(r[0]) / r[1], 16.0, rtol=rtol)


def test_limited_energy_and_momentum_equal_eih_up_to_dropped_orders(orc):
    """Eq. 7 and Eq. 8 keep every EIH energy and momentum term that is of
    degree <= 2 in the star masses; the dropped part is of degree >= 3, so
    the differences shrink by 8 (or 16) when the star masses halve."""
    x, v, m = _random_state(6, 5, m_bh=1.0, m_star=0.02, vscale=0.4)
    c = 5.0

    def diff(scale):
        mm = m.copy()
        mm[1:] *= scale
        vv = _zero_momentum(v, mm)
        lim = orc.energy(x, vv, mm, c=c)
        eih = orc.eih_energy(x, vv, mm, c=c)
        return lim["E"] - eih["E"], lim["P"] - eih["P"]

    (e1, p1), (e2, p2), (e3, p3) = diff(1.0), diff(0.5), diff(0.25)
    for r in (e1 / e2, e2 / e3):
        assert 7.9 < r < 16.1
    for r in (p1 / p2, p2 / p3):
        assert np.all((7.9 < r) & (r < 16.1)), r


# ------------------------------------------------------- conservation laws --

def _orbiting_stars(n_stars, m_star, M=1.0, seed=0):
    """Stars on near-circular orbits at well-separated radii."""
    rng = np.random.default_rng(seed)
    x = np.zeros((n_stars + 1, 3))
    v = np.zeros((n_stars + 1, 3))
    for k in range(n_stars):
        r = 1.0 + 0.7 * k
        h = rng.normal(size=3)
        h /= np.linalg.norm(h)
        p = np.cross(h, rng.normal(size=3))
        p /= np.linalg.norm(p)
        q = np.cross(h, p)
        x[k + 1] = r * p
        v[k + 1] = math.sqrt(M / r) * 1.1 * q
    m = np.full(n_stars + 1, m_star)
    m[0] = M
    v[0] = -(m[1:, None] * v[1:]).sum(0) / M
    return x, v, m


def _self_convergence(orc, vel_mode, c):
    x, v, m = _orbiting_stars(2, 1e-3, seed=4)
    a = orc.accel(x, v, m, c=c)
    T = 2.0
    xs = []
    for nst in (200, 400, 800):
        xx, vv, aa = orc.step(x, v, m, a, T / nst, nst, c=c, vel_mode=vel_mode)
        xs.append(xx)
    return np.linalg.norm(xs[0] - xs[1]) / np.linalg.norm(xs[1] - xs[2])


def test_integrator_order(orc):
    """KDK with the force taken at the predicted end-of-step velocity is
    second order (self-convergence ratio 4); taking it at the half-step
    velocity is only first order in the velocity-dependent 1PN part."""
    r_end = _self_convergence(orc, 0, 4.0)
    r_half = _self_convergence(orc, 1, 4.0)
    assert 3.6 < r_end < 4.4, r_end
    assert r_half < 3.0, r_half
    assert 3.6 < _self_convergence(orc, 1, np.inf) < 4.4


def test_softening_acts_only_between_stars(orc):
    """Eq. 10 softens star-star separations only.  Hole, a star at 0.01 and a
    star at 10 on one line: the only softened separation is ~10 long, so a
    softening of 1e-3 may move the far star's acceleration by ~eps^2/(2 r r')
    of its 1PN cross terms and the others by roundoff only.  Softening a
    hole-star separation instead would change them by ~eps^2/0.01^2.  Two
    stars 0.01 apart do feel the softening."""
    x = np.array([[0.0, 0.0, 0.0], [0.01, 0.0, 0.0], [10.0, 0.0, 0.0]])
    rng = np.random.default_rng(1)
    v = rng.normal(size=(3, 3)) * 0.3
    m = np.array([1.0, 1e-2, 1e-2])
    v = _zero_momentum(v, m)
    c, eps = 3.0, 1e-3
    a0 = orc.accel(x, v, m, c=c, eps=0.0)
    a1 = orc.accel(x, v, m, c=c, eps=eps)
    r = _rel(a1, a0)
    assert r[0] < 1e-12 and r[1] < 1e-12 and r[2] < 2e-5, r
    e0 = orc.energy(x, v, m, c=c, eps=0.0)
    e1 = orc.energy(x, v, m, c=c, eps=eps)
    assert abs(e1["E"] - e0["E"]) < 1e-10 * abs(e0["E"])
    assert np.linalg.norm(e1["P"] - e0["P"]) < 1e-10 * np.linalg.norm(m[:, None] * v)
    x2 = np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 0.0], [3.0, 0.01, 0.0]])
    b0 = orc.accel(x2, v, m, c=c, eps=0.0)
    b1 = orc.accel(x2, v, m, c=c, eps=0.01)
    assert np.min(_rel(b1[1:], b0[1:])) > 0.1


def test_rk4_is_fourth_order(orc):
    """The paper's integrator (Section 4): self-convergence ratio 2^4 = 16."""
    x, v, m = _orbiting_stars(2, 1e-3, seed=4)
    c = 4.0
    a = orc.accel(x, v, m, c=c)
    T = 2.0
    xs = []
    for nst in (50, 100, 200):
        xx, vv, aa = orc.rk4_step(x, v, m, a, T / nst, nst, c=c)
        xs.append(xx)
    r = np.linalg.norm(xs[0] - xs[1]) / np.linalg.norm(xs[1] - xs[2])
    assert 14.0 < r < 18.0, r
    # and its final acceleration is the force at the final state
    np.testing.assert_allclose(aa, orc.accel(xx, vv, m, c=c), rtol=0, atol=0)


# -------------------------------------------------------- jerk, Hermite --

def test_jerk_is_the_time_derivative_along_the_trajectory(orc):
    """Appendix A: j = dA/dt along x' = v, v' = A.  Checked against a
    Richardson-extrapolated central difference of A(x + h v, v + h a)."""
    x, v, m = _random_state(24, 31, m_star=1e-2)
    c, eps = 8.0, 1e-3
    a = orc.accel(x, v, m, c=c, eps=eps)
    j = orc.jerk(x, v, m, a, c=c, eps=eps)

    def cd(h):
        return (orc.accel(x + h * v, v + h * a, m, c=c, eps=eps)
                - orc.accel(x - h * v, v - h * a, m, c=c, eps=eps)) / (2 * h)

    fd = (4.0 * cd(5e-5) - cd(1e-4)) / 3.0
    assert np.max(_rel(j, fd)) < 1e-9
    # the 1PN part matters at this c: the jerk is not the Newtonian one
    jn = orc.jerk(x, v, m, orc.accel(x, v, m, eps=eps), eps=eps)
    assert np.median(_rel(j, jn)) > 1e-3


def test_jerk_newtonian_closed_form(orc):
    """c -> inf: d/dt of -G m_k x_ik / r^3 is -G m_k [v_ik/r^3 - 3 (x_ik.v_ik) x_ik/r^5]
    (the first terms of Appendix A), r softened between stars only."""
    x, v, m = _random_state(20, 32, m_star=1e-2)
    G, eps = 1.3, 1e-2
    j = orc.jerk(x, v, m, G=G, eps=eps)
    n = len(m)
    want = np.zeros_like(x)
    for i in range(n):
        for k in range(n):
            if k == i:
                continue
            d, u = x[i] - x[k], v[i] - v[k]
            r2 = d @ d + (eps * eps if (i and k) else 0.0)
            want[i] += -G * m[k] * (u / r2 ** 1.5 - 3.0 * (d @ u) * d / r2 ** 2.5)
    assert np.max(_rel(j, want)) < 1e-11


@pytest.mark.parametrize("c", [4.0, math.inf])
def test_hermite_is_fourth_order_and_matches_rk4(orc, c):
    """The Hermite scheme (Section 5) with the jerk: self-convergence ratio
    2^4 = 16 with the velocity-dependent 1PN force, and the same trajectory
    as the paper's RK4 at small steps."""
    x, v, m = _orbiting_stars(2, 1e-3, seed=4)
    a = orc.accel(x, v, m, c=c)
    T = 2.0
    xs = []
    for nst in (50, 100, 200):
        xx, vv, aa = orc.hermite_step(x, v, m, a, T / nst, nst, c=c)
        xs.append(xx)
    r = np.linalg.norm(xs[0] - xs[1]) / np.linalg.norm(xs[1] - xs[2])
    assert 14.0 < r < 18.0, r
    np.testing.assert_allclose(aa, orc.accel(xx, vv, m, c=c), rtol=0, atol=0)
    xr, _, _ = orc.rk4_step(x, v, m, a, T / 400, 400, c=c)
    assert np.linalg.norm(xs[2] - xr) < 0.2 * np.linalg.norm(xs[1] - xs[2])


# ------------------------------------------------------------ adjoint --

def test_accel_directional_derivative_matches_central_differences(orc):
    """The oracle's exact directional derivative of A (complex step), along a
    direction that moves positions, velocities, the hole mass and 1/c^2."""
    x, v, m = _random_state(16, 43, m_bh=0.4, m_star=1e-2)
    c, eps = 7.0, 1e-2
    rng = np.random.default_rng(5)
    dx, dv, dM, dic2 = rng.normal(size=x.shape), rng.normal(size=v.shape), 0.3, 1e-3
    jv = orc.accel_jvp(x, v, m, dx, dv, dM, dic2, c=c, eps=eps)

    def A(h):
        mm = m.copy()
        mm[0] += h * dM
        return orc.accel(x + h * dx, v + h * dv, mm, c=1.0 / math.sqrt(1.0 / c ** 2 + h * dic2),
                         eps=eps)

    def cd(h):
        return (A(h) - A(-h)) / (2 * h)

    fd = (4 * cd(5e-6) - cd(1e-5)) / 3
    assert np.abs(jv - fd).max() < 1e-8 * np.abs(fd).max()


def test_trajectory_derivative_matches_central_differences(orc):
    """The oracle's exact trajectory derivative (complex step through the KDK
    steps) against a Richardson central difference of the double-precision
    stepper, along a direction that moves positions, velocities, the hole
    mass and 1/c^2 at once."""
    x, v, m = _random_state(12, 41, m_bh=0.3, m_star=1e-2)
    c, eps, dt, nst = 10.0, 1e-2, 1.0 / 256, 20
    rng = np.random.default_rng(3)
    dx, dv = rng.normal(size=x.shape), rng.normal(size=v.shape)
    dM, dic2 = 0.7, -2e-3
    xt, vt, jx, jv = orc.traj_jvp(x, v, m, dt, nst, dx, dv, dM, dic2, c=c, eps=eps)
    x_ref, v_ref, _ = orc.step(x, v, m, orc.accel(x, v, m, c=c, eps=eps), dt, nst, c=c, eps=eps)
    assert np.abs(xt - x_ref).max() < 1e-13 and np.abs(vt - v_ref).max() < 1e-12

    def run(h):
        mm = m.copy()
        mm[0] += h * dM
        ic2 = 1.0 / c ** 2 + h * dic2
        cc = 1.0 / math.sqrt(ic2)
        xx, vv = x + h * dx, v + h * dv
        a = orc.accel(xx, vv, mm, c=cc, eps=eps)
        return orc.step(xx, vv, mm, a, dt, nst, c=cc, eps=eps)[:2]

    def cd(h):
        (xp, vp), (xm, vm) = run(h), run(-h)
        return (xp - xm) / (2 * h), (vp - vm) / (2 * h)

    (fx1, fv1), (fx2, fv2) = cd(2e-5), cd(1e-5)
    fx, fv = (4 * fx2 - fx1) / 3, (4 * fv2 - fv1) / 3
    assert np.abs(jx - fx).max() < 1e-7 * np.abs(fx).max()
    assert np.abs(jv - fv).max() < 1e-7 * np.abs(fv).max()


# ------------------------------------------------------------ invariances --

def test_rotation_and_translation_invariance(orc):
    x, v, m = make_cluster(128, 0.1, 21)
    c, eps = 15.0, 1e-3
    a = orc.accel(x, v, m, c=c, eps=eps)
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0],
                  [0.0, 0.0, 1.0]])
    R = R @ np.array([[1.0, 0.0, 0.0], [0.0, math.cos(0.3), -math.sin(0.3)],
                      [0.0, math.sin(0.3), math.cos(0.3)]])
    ar = orc.accel(x @ R.T, v @ R.T, m, c=c, eps=eps)
    assert np.max(_rel(ar, a @ R.T)) < 1e-12
    at = orc.accel(x + np.array([3.0, -2.0, 5.0]), v, m, c=c, eps=eps)
    assert np.max(_rel(at, a)) < 1e-11


def test_thread_count_does_not_change_results(orc):
    x, v, m = make_cluster(150, 0.1, 22)
    orc.set_threads(1)
    a1 = orc.accel(x, v, m, c=10.0, eps=1e-3)
    e1 = orc.energy(x, v, m, c=10.0, eps=1e-3)["E"]
    orc.set_threads(0)
    a2 = orc.accel(x, v, m, c=10.0, eps=1e-3)
    e2 = orc.energy(x, v, m, c=10.0, eps=1e-3)["E"]
    assert np.array_equal(a1, a2) and e1 == e2


def test_hole_partial_sums_partition_the_hole_acceleration(orc):
    """The hole's sums of Eq. 1-3 over a range of outer stars: over every star
    they are exactly the hole's acceleration (same operations), disjoint
    ranges add up to it within rounding, and a range's Newtonian part equals
    the Newtonian pull of those stars written out directly (Eq. 1)."""
    n, c, eps = 400, 9.0, 1e-3
    x, v, m = make_cluster(n, 0.1, 31)
    a_hole = orc.accel(x, v, m, c=c, eps=eps)[0]
    newt, pn = orc.bh_partial(x, v, m, 1, n, eps=eps)
    inv_c2 = 1.0 / (c * c)
    assert np.array_equal(newt + inv_c2 * pn, a_hole)
    cuts = [1, 97, 250, 251, n]
    parts = [orc.bh_partial(x, v, m, a, b, eps=eps) for a, b in zip(cuts[:-1], cuts[1:])]
    nsum = sum(p[0] for p in parts)
    psum = sum(p[1] for p in parts)
    scale = sum(np.abs(p[0]) + inv_c2 * np.abs(p[1]) for p in parts)
    assert np.all(np.abs(nsum + inv_c2 * psum - a_hole) <= 1e-14 * scale)
    d = x[97:250] - x[0]
    direct = (m[97:250, None] * d / np.linalg.norm(d, axis=1)[:, None] ** 3).sum(axis=0)
    assert np.allclose(orc.bh_partial(x, v, m, 97, 250, eps=eps)[0], direct, rtol=1e-13,
                       atol=0)
    empty = orc.bh_partial(x, v, m, 5, 5, eps=eps)
    assert not np.any(empty[0]) and not np.any(empty[1])


def test_eih_step_is_second_order_and_follows_the_limited_trajectory(orc):
    """The KDK integrator driven by the general EIH accelerations (the
    cross-check's integrator): second-order self-convergence, and over a few
    steps its trajectory departs from the limited equations' one by the
    dropped orders only (halving the star masses divides the position
    difference by 4, the degree of the star terms that Section 2 drops)."""
    x, v, m = _orbiting_stars(2, 1e-3, seed=4)
    c = 4.0
    v = _zero_momentum(v, m)
    a = orc.eih_accel(x, v, m, c=c)
    T = 2.0
    xs = []
    for nst in (200, 400, 800):
        xx, _, _ = orc.eih_step(x, v, m, a, T / nst, nst, c=c)
        xs.append(xx)
    r = np.linalg.norm(xs[0] - xs[1]) / np.linalg.norm(xs[1] - xs[2])
    assert 3.6 < r < 4.4, r

    xr, vr, mr = _random_state(6, 11, m_bh=1.0, m_star=0.02, vscale=0.3)

    def gap(scale):
        mm = mr.copy()
        mm[1:] *= scale
        vv = _zero_momentum(vr, mm)
        a_l = orc.accel(xr, vv, mm, c=c)
        a_e = orc.eih_accel(xr, vv, mm, c=c)
        x_l, _, _ = orc.step(xr, vv, mm, a_l, 1e-3, 5, c=c)
        x_e, _, _ = orc.eih_step(xr, vv, mm, a_e, 1e-3, 5, c=c)
        return np.linalg.norm(x_l[1:] - x_e[1:])

    g1, g2, g3 = gap(1.0), gap(0.5), gap(0.25)
    assert 3.5 < g1 / g2 < 4.5 and 3.5 < g2 / g3 < 4.5, (g1 / g2, g2 / g3)
