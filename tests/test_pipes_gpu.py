"""The measured pipe rates that the rooflines divide by (nbody_measure_pipes):
plausible for a GB300 (the SM count of the device, 2 DFMA, 128 FP32 FMA
lane-ops and 16 SFU reciprocal square roots per clock per SM, within a few
percent), positive and consistent with each other, and argument errors."""
import ctypes

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


def test_measured_pipe_rates_are_plausible(nb):
    import torch
    p = nb.measure_pipes()
    assert p["sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert 500 < p["sm_mhz"] < 2500
    assert 1.8 < p["dfma_per_clk_sm"] < 2.2
    assert 115 < p["ffma2_lane_per_clk_sm"] < 135
    assert 14 < p["rsqrt_per_clk_sm"] < 18
    # absolute rates are the per-clock rates times SMs and clock
    clk = p["sm_mhz"] * 1e6 * p["sms"]
    per_clk = p["dfma_ginstr_s"] * 1e9 / clk
    assert abs(per_clk - p["dfma_per_clk_sm"]) <= 1e-9 * p["dfma_per_clk_sm"]
    assert p["ffma_glane_s"] > 0.8 * p["ffma2_glane_s"]


def test_measure_pipes_rejects_short_output(nb):
    out = (ctypes.c_double * 4)()
    assert nb.lib.nbody_measure_pipes(out, 4) == -1
    assert nb.lib.nbody_measure_pipes(None, 9) == -1
