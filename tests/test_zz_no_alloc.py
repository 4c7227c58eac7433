"""The allocation-free force entry point (nbody_accel_f64_static).

It exists for callers that cannot let the library allocate GPU memory (an
application that owns all device memory through its own allocator, or a
timing-critical loop where cudaMalloc/cudaFree would stall the device).  Its
scratch is a fixed device array shared by all calls.  Here it is called
through the C ABI twice in a row, and each result is compared with the
context-based nbody_accel (FP64) within the FP64 gate used by the parity
tests; a second call with other inputs shows that the shared scratch carries
nothing over.  This file sorts last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import nbody_ics
import oracle
from tests.gates import fp64_accel_gate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_1803_01190_gb300 as nb
    f = nb.lib.nbody_accel_f64_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return torch, nb, f


def _static_call(torch, f, pos, mass, eps, G, with_pot=True):
    n = len(mass)
    dp = torch.tensor(pos, device="cuda")
    dm = torch.tensor(mass, device="cuda")
    acc = torch.full((n, 3), np.nan, dtype=torch.float64, device="cuda")
    pot = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    rc = f(n, dp.data_ptr(), dm.data_ptr(), eps, G, acc.data_ptr(),
           pot.data_ptr() if with_pot else None, st.cuda_stream)
    assert rc == 0
    st.synchronize()
    return acc.cpu().numpy(), pot.cpu().numpy()


def _check(nb, torch, f, pos, mass, eps, G):
    n = len(mass)
    a_s, p_s = _static_call(torch, f, pos, mass, eps, G)
    with nb.Simulation(n, "fp64", eps=eps, G=G) as sim:
        a_c, p_c = sim.accel(pos, mass)
    a_o, p_o, smag = oracle.accel(pos, mass, eps, G)
    ok, err, _ = fp64_accel_gate(a_s, a_c, smag, n)
    assert ok.all(), err.max()
    assert np.all(np.abs(p_s - p_c) <= 1e-12 * np.abs(p_c))
    # and directly against the oracle, within the same gate
    ok, err, _ = fp64_accel_gate(a_s, a_o, smag, n)
    assert ok.all(), err.max()
    assert np.all(np.abs(p_s - p_o) <= 1e-12 * np.abs(p_o))


def test_static_matches_context_entry_point_twice(env):
    torch, nb, f = env
    w = nbody_ics.workload("plummer", n=4096)
    _check(nb, torch, f, w["pos"], w["mass"], w["eps"], 1.0)
    # second call in a row: other size, masses, eps and G
    n2 = 3001
    pos2 = nbody_ics.uniform_sphere(n2, 9)[0]
    mass2 = nbody_ics.lognormal_masses(n2, 10)
    _check(nb, torch, f, pos2, mass2, 1e-3, 0.7)


def test_static_at_capacity_and_rejections(env):
    torch, nb, f = env
    nmax = 32768
    w = nbody_ics.workload("sweep_plummer", n=nmax)
    a1, p1 = _static_call(torch, f, w["pos"], w["mass"], w["eps"], 1.0)
    a2, p2 = _static_call(torch, f, w["pos"], w["mass"], w["eps"], 1.0)
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2)
    with nb.Simulation(nmax, "fp64", eps=w["eps"]) as sim:
        ac, pc = sim.accel(w["pos"], w["mass"])
    rows = np.arange(0, nmax, 97)
    _, _, smag = oracle.accel(w["pos"], w["mass"], w["eps"], rows=rows)
    assert fp64_accel_gate(a1[rows], ac[rows], smag, nmax)[0].all()
    d = torch.zeros(3 * (nmax + 1), dtype=torch.float64, device="cuda")
    assert f(nmax + 1, d.data_ptr(), d.data_ptr(), 0.01, 1.0, d.data_ptr(), None, None) == -1
    assert f(0, d.data_ptr(), d.data_ptr(), 0.01, 1.0, d.data_ptr(), None, None) == -1
    assert f(10, None, d.data_ptr(), 0.01, 1.0, d.data_ptr(), None, None) == -1


def test_static_without_potential_and_argument_errors(env):
    torch, nb, f = env
    w = nbody_ics.workload("plummer", n=2000)
    a_p, _ = _static_call(torch, f, w["pos"], w["mass"], w["eps"], 1.0)
    a_n, p_n = _static_call(torch, f, w["pos"], w["mass"], w["eps"], 1.0, with_pot=False)
    assert np.array_equal(a_p, a_n)          # pot = NULL: same accelerations, pot untouched
    assert np.isnan(p_n).all()
    d = torch.zeros(3 * 16, dtype=torch.float64, device="cuda")
    for eps, G in ((-1.0, 1.0), (float("nan"), 1.0), (float("inf"), 1.0), (0.01, float("inf")),
                   (0.01, float("nan"))):
        assert f(16, d.data_ptr(), d.data_ptr(), eps, G, d.data_ptr(), None, None) == -1
        assert b"eps" in nb.lib.nbody_last_error()


def test_static_allocates_nothing(env):
    """After a first call (which looks up the scratch address), further calls
    leave the device's free memory unchanged: nothing is allocated per call."""
    torch, nb, f = env
    n = 8192
    w = nbody_ics.workload("sweep_uniform", n=n)
    dp = torch.tensor(w["pos"], device="cuda")
    dm = torch.tensor(w["mass"], device="cuda")
    acc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty((n,), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    assert f(n, dp.data_ptr(), dm.data_ptr(), w["eps"], 1.0, acc.data_ptr(), pot.data_ptr(),
             st.cuda_stream) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert f(n, dp.data_ptr(), dm.data_ptr(), w["eps"], 1.0, acc.data_ptr(), pot.data_ptr(),
                 st.cuda_stream) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
