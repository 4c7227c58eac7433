"""Pins of the FP64 CPU oracle against results fixed by the mathematics.

None of these re-types the oracle's formula: each compares it with a closed
form (point mass, symmetric polyhedra, Kepler's equation, Plummer's potential
energy), an invariant (Newton's third law, time reversibility, energy
conservation), a convergence order, or a 40-digit brute force.
"""
import decimal
import math

import numpy as np
import pytest

import nbody_ics
import oracle as _oracle_mod
from tests import kepler

U = 2.0 ** -53


@pytest.fixture
def oracle():
    """The oracle under test (a planted-mistake copy in test_oracle_mutants)."""
    return _oracle_mod.default()


# ---------------------------------------------------------------- force, Eq. 1-2
@pytest.mark.parametrize("eps", [0.0, 0.1, 0.7])
def test_point_mass_and_test_particles(oracle, eps):
    """Massless test particles around a point mass M feel
    a = -G M r / (r^2 + eps^2)^{3/2}, pot = -G M / sqrt(r^2 + eps^2);
    the point mass itself feels nothing (the force carries m_j, not m_i)."""
    g = nbody_ics.rng(1)
    k = 50
    r = np.exp(g.uniform(-3, 3, k))
    d = g.standard_normal((k, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    M, G = 2.5, 0.7
    pos = np.vstack([[0.0, 0.0, 0.0], r[:, None] * d])   # d_ij is then exactly r d
    mass = np.concatenate([[M], np.zeros(k)])
    acc, pot, smag = oracle.accel(pos, mass, eps, G)
    w = (pos[1:] ** 2).sum(1) + eps * eps
    want = -G * M * pos[1:] / w[:, None] ** 1.5
    np.testing.assert_allclose(acc[1:], want, rtol=4e-15, atol=0)
    np.testing.assert_allclose(pot[1:], -G * M / np.sqrt(w), rtol=4e-15, atol=0)
    # the magnitude sum of a single term is that term's magnitude, G M r / (r^2 + eps^2)^{3/2}
    np.testing.assert_allclose(smag[1:], G * M * r / w ** 1.5, rtol=4e-15, atol=0)
    assert np.all(acc[0] == 0.0) and pot[0] == 0.0 and smag[0] == 0.0


@pytest.mark.parametrize("eps", [0.0, 0.05])
def test_octahedron_closed_form(oracle, eps):
    """Six equal masses at +-R on the axes: each is pulled radially inward with
    |a| = G m [4 R / (2R^2+eps^2)^{3/2} + 2R / (4R^2+eps^2)^{3/2}] and has
    pot = -G m [4 / sqrt(2R^2+eps^2) + 1 / sqrt(4R^2+eps^2)]."""
    R, m, G = 1.7, 0.3, 1.3
    pos = np.array([[R, 0, 0], [-R, 0, 0], [0, R, 0], [0, -R, 0], [0, 0, R], [0, 0, -R]], float)
    acc, pot, _ = oracle.accel(pos, np.full(6, m), eps, G)
    amag = G * m * (4 * R / (2 * R * R + eps * eps) ** 1.5 + 2 * R / (4 * R * R + eps * eps) ** 1.5)
    np.testing.assert_allclose(acc, -amag * pos / R, rtol=1e-15, atol=1e-15 * amag)
    p = -G * m * (4 / math.sqrt(2 * R * R + eps * eps) + 1 / math.sqrt(4 * R * R + eps * eps))
    np.testing.assert_allclose(pot, p, rtol=1e-15)


def test_tetrahedron_centre_is_force_free(oracle):
    """A test particle at the centre of a regular tetrahedron of equal masses
    feels zero net force and pot = -4 G m / sqrt(R^2 + eps^2)."""
    v = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float)
    pos = np.vstack([v, [[0, 0, 0]]])
    mass = np.array([1.0, 1.0, 1.0, 1.0, 0.0])
    acc, pot, smag = oracle.accel(pos, mass, 0.2, 1.0)
    assert np.all(np.abs(acc[4]) <= 4 * U * smag[4])
    assert pot[4] == pytest.approx(-4 / math.sqrt(3 + 0.04), rel=1e-15)


def _decimal_brute(pos, mass, eps, G):
    decimal.getcontext().prec = 40
    D = decimal.Decimal
    n = len(mass)
    P = [[D(float(c)) for c in p] for p in pos]
    Mm = [D(float(x)) for x in mass]
    e2 = D(float(eps)) ** 2
    Gd = D(float(G))
    acc = np.zeros((n, 3))
    pot = np.zeros(n)
    mag = np.zeros(n)
    for i in range(n):
        a = [D(0)] * 3
        p = D(0)
        sm = D(0)
        for j in range(n):
            if j == i:
                continue
            d = [P[i][c] - P[j][c] for c in range(3)]
            r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2]
            s2 = r2 + e2
            s = s2.sqrt()
            for c in range(3):
                a[c] -= Gd * Mm[j] * d[c] / (s2 * s)
            p -= Gd * Mm[j] / s
            sm += Gd * Mm[j] * r2.sqrt() / (s2 * s)   # |term|: the length of the pair's force
        acc[i] = [float(x) for x in a]
        pot[i] = float(p)
        mag[i] = float(sm)
    return acc, pot, mag


@pytest.mark.parametrize("n,eps", [(2, 0.0), (7, 0.01), (33, 0.3), (64, 1e-3)])
def test_brute_force_40_digits(oracle, n, eps):
    """Against a 40-digit decimal evaluation of the same sums on tiny inputs
    (lognormal masses, Plummer positions): |error| <= 4u * S_i per component."""
    pos = nbody_ics.plummer(n, 100 + n)[0]
    mass = nbody_ics.lognormal_masses(n, 200 + n)
    acc, pot, smag = oracle.accel(pos, mass, eps, 1.1)
    ea, ep, es = _decimal_brute(pos, mass, eps, 1.1)
    # smag is pinned first (terms of one sign: a few roundings each), because it
    # then sets the scale of the acceleration bound below
    assert np.all(np.abs(smag - es) <= 8 * U * es)
    assert np.all(np.abs(acc - ea) <= 4 * U * es[:, None] + 1e-300)
    assert np.all(np.abs(pot - ep) <= 4 * U * np.abs(ep))


def test_rows_subset_matches_full(oracle):
    w = nbody_ics.workload("plummer", n=300)
    full = oracle.accel(w["pos"], w["mass"], w["eps"])
    rows = np.array([299, 0, 17, 17, 150])
    sub = oracle.accel(w["pos"], w["mass"], w["eps"], rows=rows)
    for a, b in zip(full, sub):
        assert np.array_equal(a[rows], b)


def test_thread_count_does_not_change_result(oracle):
    w = nbody_ics.workload("sweep_uniform", n=700)
    a1 = oracle.accel(w["pos"], w["mass"], w["eps"], threads=1)
    a4 = oracle.accel(w["pos"], w["mass"], w["eps"], threads=4)
    for x, y in zip(a1, a4):
        assert np.array_equal(x, y)


def test_newtons_third_law(oracle):
    """sum_i m_i a_i = 0 (pairwise antisymmetry) to round-off."""
    w = nbody_ics.workload("sweep_uniform", n=1000)
    acc, _, smag = oracle.accel(w["pos"], w["mass"], 1e-3)
    tot = (w["mass"][:, None] * acc).sum(0)
    scale = (w["mass"] * smag).sum()
    assert np.all(np.abs(tot) <= 1e-14 * scale)


@pytest.mark.slow
def test_plummer_potential_energy(oracle):
    """Plummer sphere, eps = 0: E[W_N] = -(1 - 1/N) 3 pi G M^2 / (32 a).
    Sixteen seeds of N = 4096; the mean must lie within 3 standard errors,
    and the virial ratio 2K/|W| within 3 standard errors of 1."""
    n = 4096
    Ws, Qs = [], []
    for s in range(16):
        pos, vel, mass = nbody_ics.plummer(n, 5000 + s)
        d = oracle.diag(pos, vel, mass, 0.0, 1.0)
        Ws.append(d["W"])
        Qs.append(2 * d["K"] / -d["W"])
    Ws, Qs = np.array(Ws), np.array(Qs)
    want = -(1 - 1 / n) * 3 * np.pi / 32
    se = Ws.std(ddof=1) / 4
    assert abs(Ws.mean() - want) < 3 * se + 1e-3 * abs(want)
    assert 0.005 < Ws.std(ddof=1) / abs(want) < 0.05          # scatter is ~1%, not zero
    assert abs(Qs.mean() - 1) < 3 * Qs.std(ddof=1) / 4 + 5e-3


# ---------------------------------------------------------------- KDK, Eq. 5-7
def _kdk_error(oracle, e, steps_per_orbit, orbits=1.0):
    pos, vel, mass = kepler.two_body(0.0, e=e)
    T = kepler.period()
    nst = int(round(steps_per_orbit * orbits))
    p, v, _, _ = oracle.kdk(pos, vel, mass, 0.0, 1.0, T / steps_per_orbit, nst)
    pw, vw, _ = kepler.two_body(T * orbits, e=e)
    return np.abs(p - pw).max(), p, v, mass


@pytest.mark.parametrize("e", [0.0, 0.5])
def test_kdk_second_order_on_kepler_orbits(oracle, e):
    """Against Kepler's equation after one orbit: the error falls by ~4 per
    halving of dt (second order) and is small."""
    errs = [_kdk_error(oracle, e, s)[0] for s in (400, 800, 1600)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4, (errs, r1, r2)
    assert errs[-1] < (1e-4 if e == 0 else 2e-3)


def test_kdk_energy_bounded_and_second_order(oracle):
    """Energy error of the symplectic KDK scheme, sampled 32 times per orbit
    over 5 orbits of an e = 0.3 Kepler orbit, stays bounded and its maximum
    scales as dt^2."""
    pos, vel, mass = kepler.two_body(0.0, e=0.3)
    E0 = oracle.diag(pos, vel, mass, 0.0)["E"]
    T = kepler.period()
    maxerr = []
    for spo in (256, 512):
        p, v = pos, vel
        errs = []
        for _ in range(5 * 32):
            p, v, _, _ = oracle.kdk(p, v, mass, 0.0, 1.0, T / spo, spo // 32)
            errs.append(abs(oracle.diag(p, v, mass, 0.0)["E"] / E0 - 1))
        errs = np.array(errs)
        # bounded: the last orbit is no worse than the first (no secular drift)
        assert errs[-32:].max() < 1.05 * errs[:32].max()
        maxerr.append(errs.max())
    assert maxerr[1] < 1e-4
    assert 3.5 < maxerr[0] / maxerr[1] < 4.5, maxerr


def test_kdk_time_reversible(oracle):
    """n steps forward, reverse velocities, n steps, reverse again: back to
    the start to round-off (KDK is time symmetric)."""
    w = nbody_ics.workload("plummer", n=64)
    p, v, m = w["pos"], w["vel"], w["mass"]
    p1, v1, _, _ = oracle.kdk(p, v, m, 0.05, 1.0, 1e-3, 50)
    p2, v2, _, _ = oracle.kdk(p1, -v1, m, 0.05, 1.0, 1e-3, 50)
    assert np.abs(p2 - p).max() < 1e-12
    assert np.abs(-v2 - v).max() < 1e-11


def test_kdk_momentum_conserved(oracle):
    w = nbody_ics.workload("plummer", n=200)
    m = nbody_ics.lognormal_masses(200, 3)
    p, v, _, _ = oracle.kdk(w["pos"], w["vel"], m, 0.01, 1.0, 1e-3, 20)
    P0 = (m[:, None] * w["vel"]).sum(0)
    P1 = (m[:, None] * v).sum(0)
    assert np.abs(P1 - P0).max() < 1e-14


# ---------------------------------------------------------------- RK4
def test_rk4_fourth_order_on_kepler_orbit(oracle):
    pos, vel, mass = kepler.two_body(0.0, e=0.5)
    T = kepler.period()
    errs = []
    for spo in (200, 400, 800):
        p, v, _ = oracle.rk4(pos, vel, mass, 0.0, 1.0, T / spo, spo)
        pw, _, _ = kepler.two_body(T, e=0.5)
        errs.append(np.abs(p - pw).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 13 < r1 < 19 and 13 < r2 < 19, (errs, r1, r2)
    assert errs[-1] < 1e-6


# ---------------------------------------------------------------- FR4 (KDK composition)
def test_fr4_fourth_order_on_kepler_orbit(oracle):
    """Against Kepler's equation after one orbit of e = 0.5: the error falls by
    ~16 per halving of dt (fourth order)."""
    pos, vel, mass = kepler.two_body(0.0, e=0.5)
    T = kepler.period()
    pw, _, _ = kepler.two_body(T, e=0.5)
    errs = []
    for spo in (200, 400, 800):
        p, v, _, _ = oracle.fr4(pos, vel, mass, 0.0, 1.0, T / spo, spo)
        errs.append(np.abs(p - pw).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 13 < r1 < 19 and 13 < r2 < 19, (errs, r1, r2)
    assert errs[-1] < 1e-5


def test_fr4_energy_bounded_and_fourth_order(oracle):
    """The composition is symplectic: the energy error of an e = 0.3 Kepler
    orbit, sampled 32 times per orbit over 5 orbits, shows no secular growth,
    and its maximum scales as dt^4."""
    pos, vel, mass = kepler.two_body(0.0, e=0.3)
    E0 = oracle.diag(pos, vel, mass, 0.0)["E"]
    T = kepler.period()
    maxerr = []
    for spo in (128, 256):
        p, v = pos, vel
        errs = []
        for _ in range(5 * 32):
            p, v, _, _ = oracle.fr4(p, v, mass, 0.0, 1.0, T / spo, spo // 32)
            errs.append(abs(oracle.diag(p, v, mass, 0.0)["E"] / E0 - 1))
        errs = np.array(errs)
        assert errs[-32:].max() < 1.05 * errs[:32].max()
        maxerr.append(errs.max())
    assert 12 < maxerr[0] / maxerr[1] < 20, maxerr


def test_fr4_time_reversible(oracle):
    """n steps forward, reverse velocities, n steps, reverse again: back to
    the start to round-off (the composition is time symmetric)."""
    w = nbody_ics.workload("plummer", n=64)
    p, v, m = w["pos"], w["vel"], w["mass"]
    p1, v1, _, _ = oracle.fr4(p, v, m, 0.05, 1.0, 1e-3, 20)
    p2, v2, _, _ = oracle.fr4(p1, -v1, m, 0.05, 1.0, 1e-3, 20)
    assert np.abs(p2 - p).max() < 1e-12
    assert np.abs(-v2 - v).max() < 1e-11


# ---------------------------------------------------------------- diagnostics, Eq. 8-10
def test_diag_two_body_circular(oracle):
    """m = 1/2 each, separation 1, circular: E = -G m1 m2 / (2 d) = -1/8,
    L_z = mu d v_rel = 1/4, P = 0.  With softening W = -G m1 m2 / sqrt(d^2+eps^2)."""
    pos, vel, mass = kepler.two_body(0.0)
    d = oracle.diag(pos, vel, mass, 0.0)
    assert d["E"] == pytest.approx(-0.125, abs=1e-15)
    assert d["K"] == pytest.approx(0.125, abs=1e-15)
    assert d["L"][2] == pytest.approx(0.25, abs=1e-15)
    assert np.abs(d["P"]).max() < 1e-16 and np.abs(d["L"][:2]).max() == 0
    d = oracle.diag(pos, vel, mass, 0.5)
    assert d["W"] == pytest.approx(-0.25 / math.sqrt(1.25), rel=1e-15)


def test_diag_three_bodies_by_hand(oracle):
    """Values worked by hand: masses 1, 2, 3 at (0,0,0), (3,0,0), (0,4,0) with
    velocities (1,0,0), (0,1,0), (0,0,1), G = 1, eps = 0.
    K = (1 + 2 + 3)/2 = 3;  W = -(1*2/3 + 1*3/4 + 2*3/5) = -2.6166...;
    P = (1, 2, 3);  L = r x v summed = (12, 0, 6)."""
    pos = np.array([[0, 0, 0], [3, 0, 0], [0, 4, 0]], float)
    vel = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    mass = np.array([1.0, 2.0, 3.0])
    d = oracle.diag(pos, vel, mass, 0.0)
    assert d["K"] == 3.0
    assert d["W"] == pytest.approx(-(2 / 3 + 3 / 4 + 6 / 5), rel=1e-15)
    assert d["E"] == pytest.approx(3.0 - (2 / 3 + 3 / 4 + 6 / 5), rel=1e-15)
    np.testing.assert_array_equal(d["P"], [1.0, 2.0, 3.0])
    np.testing.assert_array_equal(d["L"], [12.0, 0.0, 6.0])


# ---------------------------------------------------------------- golden fixture
def load_golden():
    """tests/golden/plummer64.txt, written by tests/golden/make_golden.py from the oracle."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "plummer64.txt")
    with open(path) as f:
        diag_line = [ln for ln in f if ln.startswith("# diag")][0]
    diag = np.array([float(x) for x in diag_line.split(":")[1].split()])
    t = np.loadtxt(path)
    return dict(pos=t[:, 0:3], vel=t[:, 3:6], mass=t[:, 6], acc=t[:, 7:10], pot=t[:, 10],
                kdk_pos=t[:, 11:14], kdk_vel=t[:, 14:17], rk4_pos=t[:, 17:20], rk4_vel=t[:, 20:23],
                fr4_pos=t[:, 23:26], fr4_vel=t[:, 26:29],
                diag=diag, eps=0.05, G=1.0, dt=1e-3)


def test_golden_fixture_reproduced(oracle):
    """The oracle still reproduces its committed fixture bit for bit."""
    g = load_golden()
    acc, pot, _ = oracle.accel(g["pos"], g["mass"], g["eps"], g["G"])
    assert np.array_equal(acc, g["acc"]) and np.array_equal(pot, g["pot"])
    p, v, _, _ = oracle.kdk(g["pos"], g["vel"], g["mass"], g["eps"], g["G"], g["dt"], 10)
    assert np.array_equal(p, g["kdk_pos"]) and np.array_equal(v, g["kdk_vel"])
    p, v, _ = oracle.rk4(g["pos"], g["vel"], g["mass"], g["eps"], g["G"], g["dt"], 3)
    assert np.array_equal(p, g["rk4_pos"]) and np.array_equal(v, g["rk4_vel"])
    p, v, _, _ = oracle.fr4(g["pos"], g["vel"], g["mass"], g["eps"], g["G"], g["dt"], 3)
    assert np.array_equal(p, g["fr4_pos"]) and np.array_equal(v, g["fr4_vel"])
    d = oracle.diag(g["pos"], g["vel"], g["mass"], g["eps"], g["G"])
    assert np.array_equal(np.array([d["E"], d["K"], d["W"], *d["P"], *d["L"]]), g["diag"])
