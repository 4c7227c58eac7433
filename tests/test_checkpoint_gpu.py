"""Checkpoint / resume: stopping after k steps, saving (pos, vel, mass, t,
step) on the host, and resuming in a fresh context continues the trajectory
bit for bit, in every precision mode (the kernels are deterministic and a(t)
is recomputed from the same positions)."""
import numpy as np
import pytest

import nbody_ics

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


@pytest.mark.parametrize("scheme", ["kdk", "fr4", "rk4"])
@pytest.mark.parametrize("mode", ["fp64", "f64e", "mixed", "fp32"])
def test_resume_is_bitwise(nb, mode, scheme):
    n, dt = 3000, 1e-3
    w = nbody_ics.workload("disk_halo", n=n)
    with nb.Simulation(n, mode, eps=w["eps"]) as a:
        a.set_state(w["pos"], w["vel"], w["mass"])
        a.step(dt, 8, scheme)
        ref = a.get_state()
    with nb.Simulation(n, mode, eps=w["eps"]) as b:
        b.set_state(w["pos"], w["vel"], w["mass"])
        b.step(dt, 5, scheme)
        pos, vel, t, s = b.get_state()                  # checkpoint to host memory
    with nb.Simulation(n, mode, eps=w["eps"]) as c:
        c.set_state(pos, vel, w["mass"])
        c.set_clock(t, s)
        c.step(dt, 3, scheme)
        got = c.get_state()
    assert got[3] == ref[3] == 8 and abs(got[2] - ref[2]) < 1e-15
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
