"""FP64 pair arithmetic at the ulp level, through the public API.

The FP64 force kernel evaluates 1/r and 1/r^2 (Eq. 1-2) on the integer and
binary32 pipes and forms m/r and (m/r)(1/r^2) with an integer binary64
multiply.  One massive particle at the origin and massless test particles on
the x axis isolate a single pair per test particle: with eps = 0 the kernel's
r^2 is the binary64 square of the distance, its potential is -G m/r with one
rounding of the mass times 1/r, and its acceleration is dx (m/r)(1/r^2) with
three roundings.  The references are computed in extended precision (numpy
longdouble: 64-bit or 113-bit significand) from the same binary64 r^2.
"""
import numpy as np
import pytest

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


def _ulps(got, exact):
    exact = np.asarray(exact, dtype=np.longdouble)
    _, e = np.frexp(exact)
    ulp = np.ldexp(np.ones_like(exact), e.astype(np.int64) - 53)
    return np.abs((np.asarray(got, dtype=np.longdouble) - exact) / ulp).astype(np.float64)


def _axis_positions(log2_lo, log2_hi, n, seed):
    rng = np.random.default_rng(seed)
    x = np.unique(np.exp2(rng.uniform(log2_lo, log2_hi, n)) * rng.choice([-1.0, 1.0], n))
    pos = np.zeros((len(x) + 1, 3))
    pos[1:, 0] = x
    return pos


def _axis_case(nb, m0, pos, sym=-1):
    """(pot ulps, acc ulps, pot) of the test particles against extended precision."""
    x = pos[1:, 0]
    mass = np.zeros(len(pos))
    mass[0] = m0
    with nb.Simulation(len(mass), "fp64", eps=0.0) as sim:
        sim.set_symmetric(sym)
        acc, pot = sim.accel(pos, mass)
    r2 = (x * x).astype(np.longdouble)  # the binary64 square, as the kernel forms it
    inv_r = 1 / np.sqrt(r2)
    pot_exact = -np.longdouble(m0) * inv_r
    ax_exact = -np.longdouble(m0) * x.astype(np.longdouble) * inv_r / r2
    assert np.all(acc[1:, 1:] == 0)
    return _ulps(pot[1:], pot_exact), _ulps(acc[1:, 0], ax_exact), pot[1:]


# Worst cases, in ulps of the result: 1/r and 1/r^2 are within 0.52 ulp, i.e.
# a relative error of at most 1.04 ulps of any product they enter; each
# binary64 rounding adds at most 0.5 ulp of its own result, 1 ulp of a
# later product.  pot = RN(m/r), acc = RN(dx RN(RN(m/r) / r^2)).


def test_longdouble_is_extended():
    assert np.finfo(np.longdouble).nmant >= 63


@pytest.mark.parametrize("sym", [0, 1])
@pytest.mark.parametrize("seed", [1, 2])
def test_unit_mass_potential_is_reciprocal_sqrt(nb, seed, sym):
    # |r^2| in [2^-59, 2^59]: the integer path; m = 1 makes pot exactly -(1/r);
    # sym = 1: each pair evaluated once for both particles
    pos = _axis_positions(-29.5, 29.5, 40000, 20180200 + seed)
    pot_ulp, acc_ulp, _ = _axis_case(nb, 1.0, pos, sym)
    assert pot_ulp.max() <= 0.55, pot_ulp.max()
    assert 0.2 <= pot_ulp.mean() <= 0.3  # near correctly rounded on average
    assert acc_ulp.max() <= 4.1, acc_ulp.max()


@pytest.mark.parametrize("sym", [0, 1])
def test_general_mass_product_is_binary64(nb, sym):
    pos = _axis_positions(-29.5, 29.5, 40000, 20180203)
    _, _, pot1 = _axis_case(nb, 1.0, pos, sym)
    m0 = 0.7371089013468521
    pot_ulp, acc_ulp, pot = _axis_case(nb, m0, pos, sym)
    # the integer multiply rounds m (1/r) exactly as binary64 does
    assert np.array_equal(pot, m0 * pot1)
    assert pot_ulp.max() <= 1.6, pot_ulp.max()
    assert acc_ulp.max() <= 5.1, acc_ulp.max()


@pytest.mark.parametrize("lo,hi", [(-40.0, -30.2), (30.2, 35.0)])
def test_outside_integer_range(nb, lo, hi):
    # r^2 outside [2^-60, 2^60): the binary64 fallback (sqrt, two divisions)
    pot_ulp, acc_ulp, _ = _axis_case(nb, 1.0, _axis_positions(lo, hi, 2000, 20180204))
    assert pot_ulp.max() <= 2.1, pot_ulp.max()
    assert acc_ulp.max() <= 5.1, acc_ulp.max()


def test_extreme_masses_use_fallback(nb):
    # masses outside [2^-895, 2^897) take the binary64 fallback as well
    pos = _axis_positions(-10.0, 10.0, 2000, 20180205)
    for m0 in (2.0 ** -960, 2.0 ** 950):
        pot_ulp, acc_ulp, _ = _axis_case(nb, m0, pos)
        assert pot_ulp.max() <= 3.1, (m0, pot_ulp.max())
        assert acc_ulp.max() <= 6.1, (m0, acc_ulp.max())
