"""Textbook two-body (Kepler) solution used to pin the integrators.

The relative orbit r = r2 - r1 of two point masses with G (m1 + m2) = mu is a
conic; starting at pericentre with semi-major axis a and eccentricity e, the
eccentric anomaly E solves Kepler's equation  n t = E - e sin E  with mean
motion n = sqrt(mu / a^3); then x = a (cos E - e), y = a sqrt(1 - e^2) sin E.
"""
import numpy as np


def solve_kepler(M, e):
    E = M if e < 0.8 else np.pi
    for _ in range(100):
        f = E - e * np.sin(E) - M
        E = E - f / (1.0 - e * np.cos(E))
        if abs(f) < 1e-16:
            break
    return E


def relative_state(t, a, e, mu):
    n = np.sqrt(mu / a ** 3)
    E = solve_kepler(n * t, e)
    c, s = np.cos(E), np.sin(E)
    den = 1.0 - e * c
    r = np.array([a * (c - e), a * np.sqrt(1 - e * e) * s, 0.0])
    v = np.array([-a * n * s / den, a * n * np.sqrt(1 - e * e) * c / den, 0.0])
    return r, v


def two_body(t, a=1.0, e=0.0, m1=0.5, m2=0.5, G=1.0):
    """Positions (2,3), velocities (2,3), masses (2,) at time t; centre of mass at rest at 0."""
    M = m1 + m2
    r, v = relative_state(t, a, e, G * M)
    pos = np.stack([-m2 / M * r, m1 / M * r])
    vel = np.stack([-m2 / M * v, m1 / M * v])
    return pos, vel, np.array([m1, m2])


def period(a=1.0, m1=0.5, m2=0.5, G=1.0):
    return 2 * np.pi * np.sqrt(a ** 3 / (G * (m1 + m2)))
