"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

FP64: element-wise within the gate of tests/gates.py (1e-12 relative plus
the rounding floor of a reordered binary64 sum).  MIXED and FP32: the error
against the oracle is measured and bounded (no exact pin exists for reduced
precision).  Sizes span several tiles and ragged tails; the full-size
workloads are checked on sampled particles.
"""
import numpy as np
import pytest

import nbody_ics
import oracle
from tests.gates import U, fp64_accel_gate, rel_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_1803_01190_gb300 as m
    return m


def _check_fp64(acc, pot, pos, mass, eps, G=1.0, rows=None):
    acc_o, pot_o, smag = oracle.accel(pos, mass, eps, G, rows=rows)
    a = acc if rows is None else acc[rows]
    p = pot if rows is None else pot[rows]
    ok, err, amag = fp64_accel_gate(a, acc_o, smag, len(mass))
    assert ok.all(), (err[~ok][:5], amag[~ok][:5])
    assert np.all(np.abs(p - pot_o) <= 1e-12 * np.abs(pot_o) + 1e-300)
    return err / np.maximum(amag, 1e-300)


# ------------------------------------------------------------------ FP64 force, Eq. 1-2
@pytest.mark.parametrize("n", [1, 2, 3, 31, 127, 128, 129, 513, 1000, 4096, 5003])
@pytest.mark.parametrize("eps", [0.01, 0.0])
def test_fp64_accel_sizes(nb, n, eps):
    pos, _, _ = nbody_ics.plummer(n, 11 + n)
    mass = nbody_ics.lognormal_masses(n, 12 + n)
    with nb.Simulation(n, "fp64", eps=eps, G=1.3) as sim:
        acc, pot = sim.accel(pos, mass)
    if n == 1:
        assert np.all(acc == 0) and np.all(pot == 0)
        return
    _check_fp64(acc, pot, pos, mass, eps, 1.3)


@pytest.mark.parametrize("ipt", [1, 2, 4, 8])
@pytest.mark.parametrize("jsplit", [1, 3, 7, 64])
def test_fp64_launch_shapes(nb, ipt, jsplit):
    n = 3001
    w = nbody_ics.workload("plummer", n=n)
    with nb.Simulation(n, "fp64", eps=w["eps"]) as sim:
        sim.set_launch(ipt, jsplit)
        sh = sim.get_launch()
        assert sh["ipt"] == ipt and 1 <= sh["jsplit"] <= jsplit
        acc, pot = sim.accel(w["pos"], w["mass"])
    _check_fp64(acc, pot, w["pos"], w["mass"], w["eps"])


def test_fp64_device_pointers(nb):
    import torch
    n = 2000
    w = nbody_ics.workload("plummer", n=n)
    pos = torch.tensor(w["pos"], device="cuda")
    mass = torch.tensor(w["mass"], device="cuda")
    with nb.Simulation(n, "fp64", eps=w["eps"]) as sim:
        acc, pot = sim.accel(pos, mass)
    assert acc.is_cuda and pot.is_cuda
    _check_fp64(acc.cpu().numpy(), pot.cpu().numpy(), w["pos"], w["mass"], w["eps"])


def test_fp64_newton_third_law(nb):
    n = 4096
    w = nbody_ics.workload("sweep_uniform", n=n)
    with nb.Simulation(n, "fp64", eps=1e-3) as sim:
        acc, _ = sim.accel(w["pos"], w["mass"])
    _, _, smag = oracle.accel(w["pos"], w["mass"], 1e-3)
    tot = (w["mass"][:, None] * acc).sum(0)
    assert np.all(np.abs(tot) <= 64 * U * np.sqrt(n) * (w["mass"] * smag).sum())


def test_fp64_deterministic(nb):
    n = 5000
    w = nbody_ics.workload("plummer", n=n)
    with nb.Simulation(n, "fp64", eps=w["eps"]) as sim:
        a1, p1 = sim.accel(w["pos"], w["mass"])
        a2, p2 = sim.accel(w["pos"], w["mass"])
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2)


def test_golden_fixture(nb):
    from tests.test_oracle_pins import load_golden
    g = load_golden()
    n = len(g["mass"])
    with nb.Simulation(n, "fp64", eps=g["eps"], G=g["G"]) as sim:
        sim.set_state(g["pos"], g["vel"], g["mass"])
        acc, pot = sim.get_accel()
        d = sim.diagnostics()
        sim.step(g["dt"], 10, "kdk")
        kp, kv, _, _ = sim.get_state()
        sim.set_state(g["pos"], g["vel"], g["mass"])
        sim.step(g["dt"], 3, "rk4")
        rp, rv, _, _ = sim.get_state()
        sim.set_state(g["pos"], g["vel"], g["mass"])
        sim.step(g["dt"], 3, "fr4")
        fp, fv, _, _ = sim.get_state()
    _, _, smag = oracle.accel(g["pos"], g["mass"], g["eps"])
    assert fp64_accel_gate(acc, g["acc"], smag, n)[0].all()
    assert np.allclose(pot, g["pot"], rtol=1e-12, atol=0)
    scale = np.abs(g["pos"]).max()
    vscale = np.abs(g["vel"]).max()
    assert np.abs(kp - g["kdk_pos"]).max() <= 1e-12 * scale
    assert np.abs(kv - g["kdk_vel"]).max() <= 1e-12 * vscale
    assert np.abs(rp - g["rk4_pos"]).max() <= 1e-12 * scale
    assert np.abs(rv - g["rk4_vel"]).max() <= 1e-12 * vscale
    assert np.abs(fp - g["fr4_pos"]).max() <= 1e-12 * scale
    assert np.abs(fv - g["fr4_vel"]).max() <= 1e-12 * vscale
    assert abs(d["E"] - g["diag"][0]) <= 1e-13 * abs(g["diag"][0])


# ------------------------------------------------------------------ FP64, each pair once
# 384-particle blocks: n = 385 and 768 (M = 2: the half diagonal d = M/2; a tail of one, two full
# blocks), 1100 (M = 3), 1537 (M = 5, tail of one), 2559 (M = 7), 4099 (M = 11, ragged tail of 259)
@pytest.mark.parametrize("n", [385, 768, 1100, 1537, 2559, 4099])
@pytest.mark.parametrize("eps", [0.01, 0.0])
def test_fp64_symmetric_accel_sizes(nb, n, eps):
    pos, _, _ = nbody_ics.plummer(n, 31 + n)
    mass = nbody_ics.lognormal_masses(n, 32 + n)
    with nb.Simulation(n, "fp64", eps=eps, G=1.3) as sim:
        sim.set_symmetric(1)
        assert sim.get_symmetric() == (1, True)
        acc, pot = sim.accel(pos, mass)
    _check_fp64(acc, pot, pos, mass, eps, 1.3)


# F64E: 256-particle blocks (one float-float tile each): n = 257, 512 (M = 2), 700 (M = 3),
# 1025 (M = 5, tail of 1), 2303 (M = 9, odd tail)
@pytest.mark.parametrize("n", [257, 512, 700, 1025, 2303])
@pytest.mark.parametrize("eps", [0.01, 0.0])
def test_f64e_symmetric_accel_sizes(nb, n, eps):
    pos, _, _ = nbody_ics.plummer(n, 41 + n)
    mass = nbody_ics.lognormal_masses(n, 42 + n)
    with nb.Simulation(n, "f64e", eps=eps, G=0.7) as sim:
        sim.set_symmetric(1)
        assert sim.get_symmetric() == (1, True)
        acc, pot = sim.accel(pos, mass)
    _check_fp64(acc, pot, pos, mass, eps, 0.7)


def test_f64e_symmetric_against_one_sided_and_kdk(nb):
    n = 6000
    w = nbody_ics.workload("disk_halo", n=n)
    mass = w["mass"].copy()
    mass[::9] = 0.0
    with nb.Simulation(n, "f64e", eps=w["eps"]) as sim:
        sim.set_symmetric(1)
        acc_s, pot_s = sim.accel(w["pos"], mass)
        acc_s2, _ = sim.accel(w["pos"], mass)
        sim.set_symmetric(0)
        acc_o, pot_o = sim.accel(w["pos"], mass)
        sim.set_symmetric(1)
        sim.set_state(w["pos"], w["vel"], mass)
        sim.step(5e-4, 3)
        p, v, _, _ = sim.get_state()
    assert np.array_equal(acc_s, acc_s2)
    rows = np.arange(0, n, 37)
    _check_fp64(acc_s, pot_s, w["pos"], mass, w["eps"], rows=rows)
    _check_fp64(acc_o, pot_o, w["pos"], mass, w["eps"], rows=rows)
    op, ov, _, _ = oracle.kdk(w["pos"], w["vel"], mass, w["eps"], 1.0, 5e-4, 3)
    assert np.abs(p - op).max() <= 1e-12 * np.abs(op).max()
    assert np.abs(v - ov).max() <= 1e-11 * np.abs(ov).max()


@pytest.mark.parametrize("mode", ["fp64", "f64e"])
def test_symmetric_many_blocks_sampled(nb, mode):
    """N = 2^18 + 77: 683 FP64 blocks (1025 F64E tiles), several launch groups
    of block diagonals, diagonal blocks split into parts, ragged tail; sampled
    particles from every block against the oracle."""
    n = 2 ** 18 + 77
    pos, _, _ = nbody_ics.uniform_sphere(n, 51)
    mass = nbody_ics.lognormal_masses(n, 52)
    with nb.Simulation(n, mode, eps=1e-3) as sim:
        assert sim.get_symmetric() == (-1, True)
        acc, pot = sim.accel(pos, mass)
    rows = np.unique(np.concatenate([np.arange(0, n, 509), np.arange(n - 600, n)]))
    _check_fp64(acc, pot, pos, mass, 1e-3, rows=rows)


def test_fp64_symmetric_auto_and_off(nb):
    w = nbody_ics.workload("disk_halo", n=40000)
    with nb.Simulation(40000, "fp64", eps=w["eps"]) as sim:
        assert sim.get_symmetric() == (-1, True)      # 105 blocks: automatic choice takes it
        acc_s, pot_s = sim.accel(w["pos"], w["mass"])
        acc_s2, pot_s2 = sim.accel(w["pos"], w["mass"])
        sim.set_symmetric(0)
        assert sim.get_symmetric() == (0, False)
        acc_o, pot_o = sim.accel(w["pos"], w["mass"])
    assert np.array_equal(acc_s, acc_s2) and np.array_equal(pot_s, pot_s2)   # deterministic
    assert not np.array_equal(acc_s, acc_o)                                  # a different order
    _check_fp64(acc_s, pot_s, w["pos"], w["mass"], w["eps"], rows=np.arange(0, 40000, 97))
    _check_fp64(acc_o, pot_o, w["pos"], w["mass"], w["eps"], rows=np.arange(0, 40000, 97))
    with nb.Simulation(20000, "fp64", eps=0.01) as small:
        assert small.get_symmetric() == (-1, False)   # 53 blocks: one-sided kernel
    with nb.Simulation(3000, "mixed", eps=0.01) as other:
        assert other.get_symmetric() == (-1, False)
        with pytest.raises(nb.NbodyError):
            other.set_symmetric(1)


def test_fp64_symmetric_massless_and_kdk(nb):
    """Massless tracers (binary64 fallback on their side of each pair) and a
    KDK trajectory through the each-pair-once path."""
    n = 2600
    w = nbody_ics.workload("plummer", n=n)
    mass = w["mass"].copy()
    mass[::5] = 0.0
    with nb.Simulation(n, "fp64", eps=0.01) as sim:
        sim.set_symmetric(1)
        acc, pot = sim.accel(w["pos"], mass)
        _check_fp64(acc, pot, w["pos"], mass, 0.01)
        sim.set_state(w["pos"], w["vel"], mass)
        sim.step(1e-3, 3)
        p, v, _, _ = sim.get_state()
    op, ov, _, _ = oracle.kdk(w["pos"], w["vel"], mass, 0.01, 1.0, 1e-3, 3)
    assert np.abs(p - op).max() <= 1e-12 * np.abs(op).max()
    assert np.abs(v - ov).max() <= 1e-12 * np.abs(ov).max()


# ------------------------------------------------------------------ KDK, Eq. 5-7 (Plummer N=4096)
def test_fp64_kdk_plummer4096_each_step(nb):
    """Plummer N=4096, eps=0.01, 10 KDK steps of dt=1e-3: a, pot, r, v and
    E, P, L compared with the oracle after every step."""
    w = nbody_ics.workload("plummer")
    pos, vel, mass, eps = w["pos"], w["vel"], w["mass"], w["eps"]
    n = len(mass)
    dt = 1e-3
    op, ov = pos.copy(), vel.copy()
    oa = None
    with nb.Simulation(n, "fp64", eps=eps) as sim:
        sim.set_state(pos, vel, mass)
        for k in range(10):
            sim.step(dt, 1)
            op, ov, oa, opot = oracle.kdk(op, ov, mass, eps, 1.0, dt, 1, acc0=oa)
            p, v, t, s = sim.get_state()
            acc, pot = sim.get_accel()
            assert s == k + 1 and abs(t - (k + 1) * dt) < 1e-15
            assert np.abs(p - op).max() <= 1e-12 * np.abs(op).max()
            assert np.abs(v - ov).max() <= 1e-12 * np.abs(ov).max()
            _, _, smag = oracle.accel(op, mass, eps)
            assert fp64_accel_gate(acc, oa, smag, n)[0].all()
            assert np.all(np.abs(pot - opot) <= 1e-12 * np.abs(opot))
            d = sim.diagnostics()
            od = oracle.diag(op, ov, mass, eps)
            assert abs(d["E"] - od["E"]) <= 1e-12 * abs(od["E"])
            assert np.abs(d["P"] - od["P"]).max() <= 1e-15
            assert np.abs(d["L"] - od["L"]).max() <= 1e-14


def test_fp64_kdk_multistep_equals_single_steps(nb):
    w = nbody_ics.workload("plummer", n=1500)
    with nb.Simulation(1500, "fp64", eps=0.01) as a, nb.Simulation(1500, "fp64", eps=0.01) as b:
        a.set_state(w["pos"], w["vel"], w["mass"])
        b.set_state(w["pos"], w["vel"], w["mass"])
        a.step(1e-3, 7)
        for _ in range(7):
            b.step(1e-3, 1)
        pa, va, _, _ = a.get_state()
        pb, vb, _, _ = b.get_state()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)


def test_fp64_rk4(nb):
    w = nbody_ics.workload("plummer", n=1000)
    with nb.Simulation(1000, "fp64", eps=0.01) as sim:
        sim.set_state(w["pos"], w["vel"], w["mass"])
        sim.step(2e-3, 4, "rk4")
        p, v, t, s = sim.get_state()
        acc, _ = sim.get_accel()
    op, ov, oa = oracle.rk4(w["pos"], w["vel"], w["mass"], 0.01, 1.0, 2e-3, 4)
    assert s == 4
    assert np.abs(p - op).max() <= 1e-12 * np.abs(op).max()
    assert np.abs(v - ov).max() <= 1e-12 * np.abs(ov).max()
    _, _, smag = oracle.accel(op, w["mass"], 0.01)
    assert fp64_accel_gate(acc, oa, smag, 1000)[0].all()


def test_fp64_fr4_each_step(nb):
    """Fourth-order composition of the KDK step, Plummer N = 2000: state,
    accelerations and potentials against the oracle after every step."""
    w = nbody_ics.workload("plummer", n=2000)
    mass, eps, dt = w["mass"], 0.01, 2e-3
    op, ov, oa = w["pos"].copy(), w["vel"].copy(), None
    with nb.Simulation(2000, "fp64", eps=eps) as sim:
        sim.set_state(w["pos"], w["vel"], mass)
        for k in range(4):
            sim.step(dt, 1, "fr4")
            op, ov, oa, opot = oracle.fr4(op, ov, mass, eps, 1.0, dt, 1, acc0=oa)
            p, v, t, s = sim.get_state()
            acc, pot = sim.get_accel()
            assert s == k + 1 and abs(t - (k + 1) * dt) < 1e-15
            assert np.abs(p - op).max() <= 1e-12 * np.abs(op).max()
            assert np.abs(v - ov).max() <= 1e-12 * np.abs(ov).max()
            _, _, smag = oracle.accel(op, mass, eps)
            assert fp64_accel_gate(acc, oa, smag, 2000)[0].all()
            assert np.all(np.abs(pot - opot) <= 1e-12 * np.abs(opot))


def test_fr4_multistep_equals_single_steps_and_launches(nb):
    w = nbody_ics.workload("plummer", n=1200)
    with nb.Simulation(1200, "fp64", eps=0.01) as a, nb.Simulation(1200, "fp64", eps=0.01) as b:
        a.set_state(w["pos"], w["vel"], w["mass"])
        b.set_state(w["pos"], w["vel"], w["mass"])
        a.step(1e-3, 1, "fr4")
        l0 = a.launch_count
        a.step(1e-3, 4, "fr4")
        per_step = (a.launch_count - l0) / 4
        for _ in range(5):
            b.step(1e-3, 1, "fr4")
        pa, va, _, _ = a.get_state()
        pb, vb, _, _ = b.get_state()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)
    # three force evaluations per step, each followed by one fused update
    assert per_step == 6, per_step


def test_kdk_fr4_rk4_switching(nb):
    w = nbody_ics.workload("plummer", n=600)
    args = (w["mass"], 0.02, 1.0)
    with nb.Simulation(600, "fp64", eps=0.02) as sim:
        sim.set_state(w["pos"], w["vel"], w["mass"])
        sim.step(1e-3, 2, "kdk")
        sim.step(1e-3, 2, "fr4")
        sim.step(1e-3, 1, "rk4")
        sim.step(2e-3, 1, "fr4")
        sim.step(2e-3, 1, "kdk")
        p, v, t, s = sim.get_state()
    op, ov, _, _ = oracle.kdk(w["pos"], w["vel"], *args, 1e-3, 2)
    op, ov, _, _ = oracle.fr4(op, ov, *args, 1e-3, 2)
    op, ov, _ = oracle.rk4(op, ov, *args, 1e-3, 1)
    op, ov, _, _ = oracle.fr4(op, ov, *args, 2e-3, 1)
    op, ov, _, _ = oracle.kdk(op, ov, *args, 2e-3, 1)
    assert s == 7 and abs(t - 9e-3) < 1e-15
    assert np.abs(p - op).max() <= 1e-12 * np.abs(op).max()
    assert np.abs(v - ov).max() <= 1e-12 * np.abs(ov).max()


@pytest.mark.parametrize("mode,tol", [("f64e", 1e-12), ("mixed", 1e-6), ("fp32", 1e-4)])
def test_fr4_reduced_precision_tracks_oracle(nb, mode, tol):
    w = nbody_ics.workload("plummer", n=3000)
    with nb.Simulation(3000, mode, eps=0.01) as sim:
        sim.set_state(w["pos"], w["vel"], w["mass"])
        sim.step(1e-3, 3, "fr4")
        p, v, t, s = sim.get_state()
    op, ov, _, _ = oracle.fr4(w["pos"], w["vel"], w["mass"], 0.01, 1.0, 1e-3, 3)
    assert s == 3
    assert np.abs(p - op).max() <= tol * np.abs(op).max()
    assert np.abs(v - ov).max() <= 100 * tol * np.abs(ov).max()


def test_kdk_then_rk4_then_kdk(nb):
    """Switching schemes keeps the state consistent (a(t) recomputed when stale)."""
    w = nbody_ics.workload("plummer", n=700)
    args = (w["mass"], 0.02, 1.0)
    with nb.Simulation(700, "fp64", eps=0.02) as sim:
        sim.set_state(w["pos"], w["vel"], w["mass"])
        sim.step(1e-3, 2, "kdk")
        sim.step(1e-3, 1, "rk4")
        sim.step(2e-3, 2, "kdk")
        p, v, t, s = sim.get_state()
    op, ov, _, _ = oracle.kdk(w["pos"], w["vel"], *args, 1e-3, 2)
    op, ov, _ = oracle.rk4(op, ov, *args, 1e-3, 1)
    op, ov, _, _ = oracle.kdk(op, ov, *args, 2e-3, 2)
    assert s == 5 and abs(t - 7e-3) < 1e-15
    assert np.abs(p - op).max() <= 1e-12 * np.abs(op).max()
    assert np.abs(v - ov).max() <= 1e-12 * np.abs(ov).max()


# ------------------------------------------------------------------ state handling
def test_set_state_rejects_non_finite(nb):
    w = nbody_ics.workload("plummer", n=300)
    with nb.Simulation(300, "fp64", eps=0.01) as sim:
        sim.set_state(w["pos"], w["vel"], w["mass"])
        bad = w["pos"].copy()
        bad[17, 1] = np.nan
        with pytest.raises(nb.NbodyError) as e:
            sim.set_state(bad, w["vel"], w["mass"])
        assert e.value.code == -1
        badm = w["mass"].copy()
        badm[3] = -1.0
        with pytest.raises(nb.NbodyError):
            sim.set_state(w["pos"], w["vel"], badm)
        p, v, _, _ = sim.get_state()  # previous state kept
        assert np.array_equal(p, w["pos"]) and np.array_equal(v, w["vel"])


def test_errors_before_state(nb):
    with nb.Simulation(10, "fp64", eps=0.01) as sim:
        with pytest.raises(nb.NbodyError) as e:
            sim.step(1e-3, 1)
        assert e.value.code == -5
        with pytest.raises(nb.NbodyError) as e:
            sim.step(-1e-3, 1)
        assert e.value.code == -1


# ------------------------------------------------------------------ reduced precision (measured)
def _measured(nb, mode, name, n, rows=512, seed=3):
    w = nbody_ics.workload(name, n=n)
    g = np.random.default_rng(seed)
    r = np.sort(g.choice(n, min(rows, n), replace=False))
    with nb.Simulation(n, mode, eps=w["eps"]) as sim:
        acc, pot = sim.accel(w["pos"], w["mass"])
    acc_o, pot_o, _ = oracle.accel(w["pos"], w["mass"], w["eps"], rows=r)
    e = rel_errors(acc[r], acc_o)
    ep = np.abs(pot[r] - pot_o) / np.abs(pot_o)
    return np.sqrt((e ** 2).mean()), e.max(), ep.max()


@pytest.mark.parametrize("n", [1000, 2 ** 14 + 7])
def test_mixed_force_error(nb, n):
    rms, mx, pmx = _measured(nb, "mixed", "disk_halo", n)
    print(f"mixed N={n}: rms {rms:.2e} max {mx:.2e} pot max {pmx:.2e}")
    assert rms <= 1e-6 and mx <= 2e-5 and pmx <= 1e-6


def _mixed_error(nb, pos, mass, eps, rows, order="spatial"):
    n = len(mass)
    with nb.Simulation(n, "mixed", eps=eps) as sim:
        sim.set_order(order)
        acc, pot = sim.accel(pos, mass)
    acc_o, pot_o, _ = oracle.accel(pos, mass, eps, rows=rows)
    e = rel_errors(acc[rows], acc_o)
    ep = np.abs(pot[rows] - pot_o) / np.abs(pot_o)
    return float(np.sqrt((e ** 2).mean())), float(e.max()), float(ep.max())


@pytest.mark.parametrize("n", [4099, 2 ** 16 + 3])
@pytest.mark.parametrize("dist", ["uniform", "plummer"])
@pytest.mark.parametrize("eps", [1e-3, 0.0])
def test_mixed_force_error_small_softening(nb, n, dist, eps):
    """Mixed mode with softening far below the mean separation (eps = 1e-3)
    and none at all (eps = 0), lognormal masses, ragged sizes: RMS relative
    acceleration error <= 1e-6 against the oracle (the bound the mixed mode
    states), with the default spatial order.  In input order the same cases
    reach ~1e-6 at N = 2^16 (the tiles span the whole cloud), printed for contrast."""
    s = nbody_ics.SEED_BASE + 3
    pos = (nbody_ics.uniform_sphere(n, s) if dist == "uniform" else nbody_ics.plummer(n, s))[0]
    mass = nbody_ics.lognormal_masses(n, s + 1)
    rows = np.sort(np.random.default_rng(n).choice(n, 384, replace=False))
    rms, mx, pmx = _mixed_error(nb, pos, mass, eps, rows)
    rms_in, _, _ = _mixed_error(nb, pos, mass, eps, rows, order="input")
    print(f"mixed {dist} N={n} eps={eps}: spatial rms {rms:.2e} max {mx:.2e} pot {pmx:.2e}; "
          f"input order rms {rms_in:.2e}")
    assert rms <= 1e-6 and pmx <= 1e-6
    if n > 2 ** 16:
        assert rms < rms_in   # where tiles in input order span the cloud, the order pays


def test_spatial_order_is_a_function_of_the_positions(nb):
    """The spatial order depends on the positions only: permuting the input
    permutes the mixed-mode result bit for bit (no two particles share a
    Morton cell here), and repeated calls agree bit for bit."""
    n = 20000
    w = nbody_ics.workload("sweep_uniform", n=n)
    perm = np.random.default_rng(5).permutation(n)
    with nb.Simulation(n, "mixed", eps=1e-3) as sim:
        assert sim.get_order() == "spatial"
        a1, p1 = sim.accel(w["pos"], w["mass"])
        a2, p2 = sim.accel(w["pos"][perm], w["mass"][perm])
        a3, _ = sim.accel(w["pos"], w["mass"])
    assert np.array_equal(a1[perm], a2) and np.array_equal(p1[perm], p2)
    assert np.array_equal(a1, a3)


@pytest.mark.parametrize("mode", ["fp64", "f64e"])
def test_spatial_order_in_binary64_modes(nb, mode):
    """FP64 and F64E accept the spatial order (one-sided and each-pair-once
    paths); results stay within the FP64 gate."""
    for n in (3001, 64 * 512 + 13):
        w = nbody_ics.workload("sweep_plummer", n=n)
        rows = np.sort(np.random.default_rng(n).choice(n, 256, replace=False))
        with nb.Simulation(n, mode, eps=w["eps"]) as sim:
            sim.set_order("spatial")
            acc, pot = sim.accel(w["pos"], w["mass"])
        _check_fp64(acc, pot, w["pos"], w["mass"], w["eps"], rows=rows)
    with nb.Simulation(10, "fp32", eps=0.01) as sim:
        with pytest.raises(nb.NbodyError):
            sim.set_order("spatial")


@pytest.mark.parametrize("n", [1000, 2 ** 14 + 7])
def test_fp32_force_error(nb, n):
    rms, mx, pmx = _measured(nb, "fp32", "disk_halo", n)
    print(f"fp32 N={n}: rms {rms:.2e} max {mx:.2e} pot max {pmx:.2e}")
    assert rms <= 1e-4 and mx <= 1e-3


def test_mixed_kdk_tracks_fp64(nb):
    """Mixed state stays binary64; after 20 KDK steps it is within the force
    error's effect of the oracle trajectory."""
    w = nbody_ics.workload("plummer", n=2048)
    with nb.Simulation(2048, "mixed", eps=0.01) as sim:
        sim.set_state(w["pos"], w["vel"], w["mass"])
        sim.step(1e-3, 20)
        p, v, _, _ = sim.get_state()
        d = sim.diagnostics()
    op, ov, _, _ = oracle.kdk(w["pos"], w["vel"], w["mass"], 0.01, 1.0, 1e-3, 20)
    od = oracle.diag(op, ov, w["mass"], 0.01)
    assert np.abs(p - op).max() <= 1e-9 * np.abs(op).max()
    assert np.abs(v - ov).max() <= 1e-6 * np.abs(ov).max()
    assert abs(d["E"] / od["E"] - 1) <= 1e-6


# ------------------------------------------------------------------ full-size workloads (sampled)
@pytest.mark.slow
def test_fp64_disk_halo_2_17_sampled(nb):
    w = nbody_ics.workload("disk_halo", n=2 ** 17)
    n = 2 ** 17
    rows = np.concatenate([np.arange(0, 64), np.arange(n - 64, n),
                           np.random.default_rng(0).choice(n, 128, replace=False)])
    with nb.Simulation(n, "fp64", eps=w["eps"]) as sim:
        acc, pot = sim.accel(w["pos"], w["mass"])
    _check_fp64(acc, pot, w["pos"], w["mass"], w["eps"], rows=rows)


@pytest.mark.slow
def test_fp64_and_mixed_disk_halo_2_20_sampled(nb):
    """The benchmark's workload (disk + halo, N = 2^20, eps = 0.02) in the
    default launch shape: FP64 on sampled particles within the FP64 gate,
    mixed RMS error <= 1e-6 on the same sample."""
    n = 2 ** 20
    w = nbody_ics.workload("disk_halo", n=n)
    rows = np.concatenate([np.arange(0, 32), np.arange(n - 32, n),
                           np.random.default_rng(1).choice(n, 64, replace=False)])
    acc_o, pot_o, smag = oracle.accel(w["pos"], w["mass"], w["eps"], rows=rows)
    with nb.Simulation(n, "mixed", eps=w["eps"]) as sim:
        accm, _ = sim.accel(w["pos"], w["mass"])
    e = rel_errors(accm[rows], acc_o)
    assert np.sqrt((e ** 2).mean()) <= 1e-6
    with nb.Simulation(n, "fp64", eps=w["eps"]) as sim:
        acc, pot = sim.accel(w["pos"], w["mass"])
    ok, err, amag = fp64_accel_gate(acc[rows], acc_o, smag, n)
    assert ok.all()
    assert np.all(np.abs(pot[rows] - pot_o) <= 1e-12 * np.abs(pot_o))


# ------------------------------------------------------------------ F64E (float-float, binary64-class)
def _f64e_errors(nb, pos, mass, eps, G=1.0, rows=None):
    n = len(mass)
    with nb.Simulation(n, "f64e", eps=eps, G=G) as sim:
        acc, pot = sim.accel(pos, mass)
    acc_o, pot_o, smag = oracle.accel(pos, mass, eps, G, rows=rows)
    a = acc if rows is None else acc[rows]
    p = pot if rows is None else pot[rows]
    ok, err, amag = fp64_accel_gate(a, acc_o, smag, n)
    rel = err / np.maximum(amag, 1e-300)
    prel = np.abs(p - pot_o) / np.abs(pot_o)
    return ok, rel, err / np.maximum(smag, 1e-300), prel


@pytest.mark.parametrize("n", [2, 3, 129, 1000, 5003])
@pytest.mark.parametrize("eps", [0.01, 0.0])
def test_f64e_accel_sizes(nb, n, eps):
    pos, _, _ = nbody_ics.plummer(n, 11 + n)
    mass = nbody_ics.lognormal_masses(n, 12 + n)
    ok, rel, rels, prel = _f64e_errors(nb, pos, mass, eps, 1.3)
    print(f"f64e n={n} eps={eps}: gate {ok.mean():.3f} rel max {rel.max():.2e} rms "
          f"{np.sqrt((rel ** 2).mean()):.2e} |da|/S max {rels.max():.2e} pot {prel.max():.2e}")
    assert ok.all() and prel.max() <= 1e-12          # the FP64 gate


def test_f64e_disk_halo_sampled(nb):
    n = 2 ** 17
    w = nbody_ics.workload("disk_halo", n=n)
    rows = np.random.default_rng(2).choice(n, 256, replace=False)
    ok, rel, rels, prel = _f64e_errors(nb, w["pos"], w["mass"], w["eps"], rows=rows)
    print(f"f64e disk_halo 2^17: gate {ok.mean():.3f} rel max {rel.max():.2e} rms "
          f"{np.sqrt((rel ** 2).mean()):.2e} |da|/S max {rels.max():.2e} pot {prel.max():.2e}")
    assert ok.all() and prel.max() <= 1e-12          # the FP64 gate


def test_f64e_kdk_tracks_oracle(nb):
    w = nbody_ics.workload("plummer", n=2048)
    with nb.Simulation(2048, "f64e", eps=0.01) as sim:
        sim.set_state(w["pos"], w["vel"], w["mass"])
        sim.step(1e-3, 10)
        p, v, _, _ = sim.get_state()
    op, ov, _, _ = oracle.kdk(w["pos"], w["vel"], w["mass"], 0.01, 1.0, 1e-3, 10)
    assert np.abs(p - op).max() <= 1e-12 * np.abs(op).max()
    assert np.abs(v - ov).max() <= 1e-11 * np.abs(ov).max()


def test_fp32_kdk_and_diagnostics(nb):
    """The paper's SP mode keeps its state in binary32: after 10 KDK steps the
    trajectory stays within float precision of the oracle's, and the Eq. 8-10
    diagnostics of that state are within float precision of the oracle's."""
    w = nbody_ics.workload("plummer", n=2048)
    with nb.Simulation(2048, "fp32", eps=0.01) as sim:
        sim.set_state(w["pos"], w["vel"], w["mass"])
        sim.step(1e-3, 10)
        p, v, t, s = sim.get_state()
        d = sim.diagnostics()
        sim.step(1e-3, 2, "rk4")
        p2, _, _, s2 = sim.get_state()
    op, ov, _, _ = oracle.kdk(w["pos"], w["vel"], w["mass"], 0.01, 1.0, 1e-3, 10)
    od = oracle.diag(op, ov, w["mass"], 0.01)
    assert s == 10 and s2 == 12
    assert np.abs(p - op).max() <= 1e-5 * np.abs(op).max()
    assert np.abs(v - ov).max() <= 1e-4 * np.abs(ov).max()
    assert abs(d["E"] / od["E"] - 1) <= 1e-5
    assert np.all(p.astype(np.float32).astype(np.float64) == p)      # state is binary32
    op2, _, _ = oracle.rk4(op, ov, w["mass"], 0.01, 1.0, 1e-3, 2)
    assert np.abs(p2 - op2).max() <= 1e-5 * np.abs(op2).max()


def test_golden_fixture_f64e(nb):
    from tests.test_oracle_pins import load_golden
    g = load_golden()
    n = len(g["mass"])
    with nb.Simulation(n, "f64e", eps=g["eps"], G=g["G"]) as sim:
        sim.set_state(g["pos"], g["vel"], g["mass"])
        acc, pot = sim.get_accel()
        sim.step(g["dt"], 10, "kdk")
        kp, kv, _, _ = sim.get_state()
    _, _, smag = oracle.accel(g["pos"], g["mass"], g["eps"])
    assert fp64_accel_gate(acc, g["acc"], smag, n)[0].all()
    assert np.abs(kp - g["kdk_pos"]).max() <= 1e-12 * np.abs(g["pos"]).max()
    assert np.abs(kv - g["kdk_vel"]).max() <= 1e-12 * np.abs(g["vel"]).max()
