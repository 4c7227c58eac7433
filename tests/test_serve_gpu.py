"""Batched serving path (nbody_batch_* C ABI and the continuous-batching
server) against the FP64 oracle and against the same simulations run alone."""
import numpy as np
import pytest

import nbody_ics
import oracle
from tests.gates import fp64_accel_gate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_1803_01190_gb300 as nb
    from paper_1803_01190_gb300 import serve
    return nb, serve


def _plummer(n, seed):
    return nbody_ics.plummer(n, seed)


def test_batch_fp64_matches_oracle(sv):
    """Three FP64 simulations of uneven size in one pool, 5 ticks = a(t0) + 4 KDK
    steps each, compared with the oracle's Eq. 5-7 per simulation."""
    nb, serve = sv
    b = serve.Batch(capacity=8192, max_sims=8)
    sims = [(300, 0.01, 1.0, 1e-3), (1000, 0.02, 0.7, 2e-3), (64, 0.05, 1.3, 5e-4)]
    slots, ics = [], []
    for k, (n, eps, G, dt) in enumerate(sims):
        p, v, m = _plummer(n, 40 + k)
        ics.append((p, v, m))
        slots.append(b.admit(p, v, m, "fp64", eps, G, dt))
    b.step(5)
    for (n, eps, G, dt), s, (p, v, m) in zip(sims, slots, ics):
        pos, vel, t, step = b.get_state(s)
        assert step == 4 and abs(t - 4 * dt) < 1e-15
        op, ov, oa, opot = oracle.kdk(p, v, m, eps, G, dt, 4)
        assert np.abs(pos - op).max() <= 1e-12 * np.abs(op).max()
        assert np.abs(vel - ov).max() <= 1e-12 * np.abs(ov).max()
        acc, pot = b.get_accel(s)
        _, _, smag = oracle.accel(op, m, eps, G)
        assert fp64_accel_gate(acc, oa, smag, n)[0].all()
        d = b.diagnostics(s)
        od = oracle.diag(op, ov, m, eps, G)
        assert abs(d["E"] - od["E"]) <= 1e-12 * abs(od["E"])
    b.close()


def test_batch_alone_equals_mix_bitwise(sv):
    """With a fixed launch shape, a simulation's trajectory does not depend on
    which other simulations share its ticks, nor on admissions and evictions
    around it: bit-for-bit equal to the same simulation alone in a pool."""
    nb, serve = sv
    p, v, m = nbody_ics.disk_halo(2000, 7)
    alone = serve.Batch(capacity=4096, max_sims=2)
    sa = alone.admit(p, v, m, "mixed", 0.02, 1.0, 5e-4)
    alone.step(13)
    ref = alone.get_state(sa)
    alone.close()
    mix = serve.Batch(capacity=65536, max_sims=16)
    o1 = mix.admit(*_plummer(5000, 1), "fp64", 0.01, 1.0, 1e-3)
    mix.step(2)
    sx = mix.admit(p, v, m, "mixed", 0.02, 1.0, 5e-4)
    o2 = mix.admit(*_plummer(700, 2), "mixed", 0.01, 1.0, 1e-3)
    mix.step(5)
    mix.evict(o1)
    o3 = mix.admit(*nbody_ics.disk_halo(3000, 3), "fp64", 0.02, 1.0, 5e-4)
    mix.step(8)
    got = mix.get_state(sx)
    assert got[3] == ref[3] == 12
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    for s in (o2, o3):
        mix.evict(s)
    mix.close()


def test_batch_matches_single_context(sv):
    """The same simulation through a batch and through a single context (other
    launch shapes, so other rounding order; both in input order): equal within
    1e-12 (FP64) and 1e-9 (MIXED) relative after 10 steps."""
    nb, serve = sv
    p, v, m = _plummer(1500, 9)
    for mode, tol in (("fp64", 1e-12), ("mixed", 1e-9)):
        b = serve.Batch(capacity=4096, max_sims=2)
        s = b.admit(p, v, m, mode, 0.01, 1.0, 1e-3)
        b.step(11)
        bp, bv, _, _ = b.get_state(s)
        b.close()
        with nb.Simulation(1500, mode, eps=0.01) as sim:
            sim.set_order("input")   # the pool sums in admission order
            sim.set_state(p, v, m)
            sim.step(1e-3, 10)
            sp, svv, _, _ = sim.get_state()
        assert np.abs(bp - sp).max() <= tol * np.abs(sp).max()
        assert np.abs(bv - svv).max() <= tol * np.abs(svv).max()


def test_batch_admission_limits(sv):
    nb, serve = sv
    b = serve.Batch(capacity=1024, max_sims=3)
    a = b.admit(*_plummer(600, 1), "fp64", 0.01, 1.0, 1e-3)
    assert a is not None
    assert b.admit(*_plummer(600, 2), "fp64", 0.01, 1.0, 1e-3) is None      # no range left
    c = b.admit(*_plummer(300, 3), "mixed", 0.01, 1.0, 1e-3)
    d = b.admit(*_plummer(60, 4), "fp64", 0.01, 1.0, 1e-3)
    assert c is not None and d is not None
    assert b.admit(*_plummer(10, 5), "fp64", 0.01, 1.0, 1e-3) is None       # no slot left
    b.step(2)
    b.evict(a)
    e = b.admit(*_plummer(600, 6), "fp64", 0.01, 1.0, 1e-3)                 # range reused
    assert e is not None
    b.step(2)
    assert b.get_state(e)[3] == 1 and b.get_state(c)[3] == 3
    bad = _plummer(50, 7)
    pbad = bad[0].copy()
    pbad[3, 0] = np.inf
    with pytest.raises(nb.NbodyError) as ex:
        b.admit(pbad, bad[1], bad[2], "fp64", 0.01, 1.0, 1e-3)
    assert ex.value.code == -1
    with pytest.raises(KeyError):
        b.admit(*bad, "fp32", 0.01, 1.0, 1e-3)
    b.close()


def test_server_continuous_batching_alone_vs_mix(sv):
    """A Poisson stream through the server (autotuner on): every request
    completes, and each result equals the same simulation run alone through
    a single context within 1e-12 (FP64) / 1e-9 (MIXED) relative."""
    nb, serve = sv
    reqs = serve.poisson_requests(14, rate=400.0, seed=5, n_range=(256, 3000), nsteps=12, dt=5e-4)
    srv = serve.Server(capacity=3 * 8192, max_sims=6, autotune=True)
    out = srv.run(reqs, duration=120)
    srv.close()
    assert out["completed"] == 14 and out["queued_at_end"] == 0
    assert out["tick_ms_p99"] >= out["tick_ms_p50"] > 0
    for rq in out["done"]:
        p, v, m = rq.make()
        with nb.Simulation(rq.n, rq.mode, eps=rq.eps, G=rq.G) as sim:
            sim.set_order("input")   # the pool sums in admission order
            sim.set_state(p, v, m)
            sim.step(rq.dt, rq.nsteps)
            sp, svv, _, _ = sim.get_state()
        bp, bv, t, step = rq.result
        assert step == rq.nsteps
        tol = 1e-12 if rq.mode == "fp64" else 1e-9
        assert np.abs(bp - sp).max() <= tol * np.abs(sp).max()
        assert np.abs(bv - svv).max() <= tol * np.abs(svv).max()


def test_batch_f64e_matches_oracle_and_single(sv):
    """F64E simulations in a pool (with FP64 and MIXED neighbours) against the
    oracle (FP64 gate on the final accelerations, positions to 1e-12) and
    against the same simulation in a single F64E context (same launch shape,
    other blocking of the work: 1e-12 relative)."""
    nb, serve = sv
    b = serve.Batch(capacity=16384, max_sims=6)
    p, v, m = _plummer(1200, 21)
    s = b.admit(p, v, m, "f64e", 0.01, 1.0, 1e-3)
    b.admit(*_plummer(900, 22), "fp64", 0.01, 1.0, 1e-3)
    b.admit(*_plummer(700, 23), "mixed", 0.01, 1.0, 1e-3)
    b.step(6)
    pos, vel, t, step = b.get_state(s)
    acc, _ = b.get_accel(s)
    b.close()
    op, ov, oa, _ = oracle.kdk(p, v, m, 0.01, 1.0, 1e-3, 5)
    assert step == 5
    assert np.abs(pos - op).max() <= 1e-12 * np.abs(op).max()
    assert np.abs(vel - ov).max() <= 1e-11 * np.abs(ov).max()
    _, _, smag = oracle.accel(op, m, 0.01)
    assert fp64_accel_gate(acc, oa, smag, 1200)[0].all()
    with nb.Simulation(1200, "f64e", eps=0.01) as sim:
        sim.set_state(p, v, m)
        sim.step(1e-3, 5)
        sp, svv, _, _ = sim.get_state()
    assert np.abs(pos - sp).max() <= 1e-12 * np.abs(sp).max()


def test_server_fp64_requests_on_f64e(sv):
    nb, serve = sv
    reqs = serve.poisson_requests(8, rate=400.0, seed=6, n_range=(256, 2000), nsteps=8, dt=5e-4)
    srv = serve.Server(capacity=2 * 8192, max_sims=4, autotune=True, fp64_kernel="f64e")
    out = srv.run(reqs, duration=120)
    srv.close()
    assert out["completed"] == 8
    for rq in out["done"]:
        p, v, m = rq.make()
        op, ov, _, _ = oracle.kdk(p, v, m, rq.eps, rq.G, rq.dt, rq.nsteps)
        bp = rq.result[0]
        tol = 1e-12 if rq.mode == "fp64" else 1e-7
        assert np.abs(bp - op).max() <= tol * np.abs(op).max(), (rq.mode, np.abs(bp - op).max())
