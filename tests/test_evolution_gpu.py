"""Round-off-driven drift of the centre of mass and of the momentum (the
quantities behind the paper's Fig. 6 comparison of single and double
precision, section 3): the disk + halo model, started with the centre of mass
at rest at the origin, keeps it there to round-off in the binary64-class
modes, while the paper's single precision moves it by orders of magnitude
more.  Also checks the data that bench.py --evolution writes."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import nbody_ics

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_1803_01190_gb300 as m
    return m


def _com_drift(nb, mode, n=8192, steps=400):
    w = nbody_ics.workload("disk_halo", n=n)
    m = w["mass"]
    with nb.Simulation(n, mode, eps=w["eps"]) as sim:
        sim.set_state(w["pos"], w["vel"], w["mass"])
        p0, _, _, _ = sim.get_state()
        c0 = (m[:, None] * p0).sum(0) / m.sum()
        P0 = sim.diagnostics()["P"]
        sim.step(5e-4, steps)
        p1, _, _, _ = sim.get_state()
        P1 = sim.diagnostics()["P"]
    c1 = (m[:, None] * p1).sum(0) / m.sum()
    return float(np.linalg.norm(c1 - c0)), float(np.linalg.norm(P1 - P0))


@pytest.fixture(scope="module")
def fp32_drift(nb):
    return _com_drift(nb, "fp32")


@pytest.mark.parametrize("mode,bound_r,bound_p,factor", [("fp64", 1e-14, 1e-15, 100),
                                                         ("f64e", 1e-14, 1e-15, 100),
                                                         ("mixed", 1e-9, 1e-9, 10)])
def test_centre_of_mass_drift_by_mode(nb, fp32_drift, mode, bound_r, bound_p, factor):
    dr, dp = _com_drift(nb, mode)
    dr32, dp32 = fp32_drift
    print(f"{mode}: |dR_cm| {dr:.2e} |dP| {dp:.2e}; fp32: {dr32:.2e} {dp32:.2e}")
    assert dr <= bound_r and dp <= bound_p
    assert dr32 > factor * dr and dp32 > factor * dp


def test_evolution_data_file(nb, tmp_path):
    out = tmp_path / "evo.npz"
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--evolution", "fp64,fp32",
                        "--n", "4096", "--evolution-steps", "200", "--evolution-every", "100",
                        "--evolution-out", str(out)], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    assert line["summary"]["times"] == pytest.approx([0.0, 0.05, 0.1])
    d = np.load(out)
    assert d["fp64_sigma"].shape[0] == 3 and d["fp32_com"].shape == (3, 3)
    # the maps hold the disk's mass (M_d = 1: half the particles, all inside the grid at t = 0)
    area = (d["edges"][1] - d["edges"][0]) ** 2
    assert d["fp64_sigma"][0].sum() * area == pytest.approx(1.0, rel=1e-9)
