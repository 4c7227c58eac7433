"""Integrators at the benchmark sizes, checked on sampled particles.

One KDK step (Eq. 5-7) and one RK4 step on the disk + halo model at
N = 2^17, and the positions after one KDK step at N = 2^20.  The expected
values use only oracle force evaluations: Eq. 5-6 give
r(t+dt) = r + dt v + dt^2/2 a(r), which needs a(r) on the sampled particles
only; the velocity (Eq. 7) needs a at the new positions of the sampled
particles, hence a(r) of every particle first.  RK4 likewise needs the
stage-1 and stage-2 forces of every particle and the stage-3 and stage-4
forces of the sampled ones."""
import numpy as np
import pytest

import nbody_ics
import oracle
from tests.gates import fp64_accel_gate

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def nb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_1803_01190_gb300 as m
    return m


def _rows(n, k=48, seed=5):
    return np.sort(np.random.default_rng(seed).choice(n, k, replace=False))


@pytest.mark.parametrize("mode", ["fp64", "f64e"])
def test_kdk_one_step_2_17(nb, mode):
    n, dt = 2 ** 17, 5e-4
    w = nbody_ics.workload("disk_halo", n=n)
    r0, v0, m, eps = w["pos"], w["vel"], w["mass"], w["eps"]
    rows = _rows(n)
    with nb.Simulation(n, mode, eps=eps) as sim:
        sim.set_state(r0, v0, m)
        sim.step(dt, 1)
        p, v, _, _ = sim.get_state()
        acc, _ = sim.get_accel()
    a0 = oracle.accel(r0, m, eps)[0]                      # every particle (Eq. 5)
    vt = v0 + dt * a0
    r1 = r0 + (dt / 2) * (vt + v0)                         # Eq. 6
    a1, _, smag = oracle.accel(r1, m, eps, rows=rows)      # sampled (after Eq. 6)
    v1 = (v0[rows] + vt[rows]) / 2 + (dt / 2) * a1         # Eq. 7
    assert np.abs(p - r1).max() <= 1e-12 * np.abs(r1).max()
    assert np.abs(v[rows] - v1).max() <= 1e-12 * np.abs(v1).max()
    assert fp64_accel_gate(acc[rows], a1, smag, n)[0].all()


def test_rk4_one_step_2_17(nb):
    n, dt = 2 ** 17, 5e-4
    w = nbody_ics.workload("disk_halo", n=n)
    r0, v0, m, eps = w["pos"], w["vel"], w["mass"], w["eps"]
    rows = _rows(n, seed=6)
    with nb.Simulation(n, "fp64", eps=eps) as sim:
        sim.set_state(r0, v0, m)
        sim.step(dt, 1, scheme="rk4")
        p, v, _, _ = sim.get_state()
    a1 = oracle.accel(r0, m, eps)[0]
    v2 = v0 + (dt / 2) * a1
    a2 = oracle.accel(r0 + (dt / 2) * v0, m, eps)[0]
    v3 = v0 + (dt / 2) * a2
    a3 = oracle.accel(r0 + (dt / 2) * v2, m, eps, rows=rows)[0]
    v4 = v0[rows] + dt * a3
    a4 = oracle.accel(r0 + dt * v3, m, eps, rows=rows)[0]
    r_exp = r0[rows] + (dt / 6) * (v0[rows] + 2 * v2[rows] + 2 * v3[rows] + v4)
    v_exp = v0[rows] + (dt / 6) * (a1[rows] + 2 * a2[rows] + 2 * a3 + a4)
    assert np.abs(p[rows] - r_exp).max() <= 1e-12 * np.abs(r_exp).max()
    assert np.abs(v[rows] - v_exp).max() <= 1e-12 * np.abs(v_exp).max()
    P0 = (m[:, None] * v0).sum(0)
    assert np.abs((m[:, None] * v).sum(0) - P0).max() <= 1e-15


def test_kdk_positions_one_step_2_20(nb):
    """N = 2^20 (the benchmark workload), F64E: positions after one step on
    sampled particles (they need only a(r0) of those particles) and momentum."""
    n, dt = 2 ** 20, 5e-4
    w = nbody_ics.workload("disk_halo", n=n)
    r0, v0, m, eps = w["pos"], w["vel"], w["mass"], w["eps"]
    rows = _rows(n, 32, seed=7)
    with nb.Simulation(n, "f64e", eps=eps) as sim:
        sim.set_state(r0, v0, m)
        sim.step(dt, 1)
        p, v, _, _ = sim.get_state()
    a0 = oracle.accel(r0, m, eps, rows=rows)[0]
    r1 = r0[rows] + (dt / 2) * ((v0[rows] + dt * a0) + v0[rows])
    assert np.abs(p[rows] - r1).max() <= 1e-12 * np.abs(r1).max()
    P0 = (m[:, None] * v0).sum(0)
    assert np.abs((m[:, None] * v).sum(0) - P0).max() <= 1e-14
