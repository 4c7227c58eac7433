"""Failure detection without a GPU fault: the bounded host wait.

A context's synchronising calls wait at most the time set with
nbody_set_timeout; here a wait of 1 microsecond on a force evaluation that
takes ~0.5 s must give up with NBODY_ETIMEOUT, leave the queued work running,
and leave the context usable once the limit is lifted."""
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


def test_wait_times_out_and_context_recovers(nb):
    n = 2 ** 17
    w = nbody_ics.workload("disk_halo", n=n)
    with nb.Simulation(n, "fp64", eps=w["eps"]) as sim:
        sim.set_state(w["pos"], w["vel"], w["mass"])
        sim.set_timeout(1e-6)
        sim.step(5e-4, 1)                      # queued: a(t0) plus one step, ~1 s of FP64 work
        with pytest.raises(nb.NbodyError) as e:
            sim.diagnostics()                  # its wait gives up
        assert e.value.code == -4
        sim.set_timeout(0)
        d = sim.diagnostics()                  # the same context, now waiting without limit
        p, v, t, s = sim.get_state()
    assert s == 1 and np.isfinite(d["E"]) and np.isfinite(p).all()
