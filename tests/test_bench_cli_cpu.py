"""The benchmark's command line, on the CPU: the options the measurement
contract and the experiment modes depend on are there, and the timing rules
it enforces reject a run before any GPU work."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                          capture_output=True, text=True, timeout=120, cwd=ROOT)


def test_help_lists_contract_and_experiment_options():
    r = _run("--help")
    assert r.returncode == 0, r.stderr
    for opt in ("--gpus", "--steps", "--warmup", "--impl", "--drift", "--drift-scheme",
                "--evolution", "--evolution-out", "--profile-force"):
        assert opt in r.stdout, opt


def test_fewer_than_three_warmup_steps_rejected():
    r = _run("--warmup", "2")
    assert r.returncode == 2 and "--warmup must be >= 3" in r.stderr


def test_unknown_scheme_and_impl_rejected():
    assert _run("--drift", "fp64", "--drift-scheme", "leapfrog4").returncode == 2
    assert _run("--impl", "other").returncode == 2


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PIPES = {"sms": 152.0, "sm_mhz": 2070.0, "dfma_ginstr_s": 629.28, "ffma_glane_s": 39000.0,
         "ffma2_glane_s": 40273.92, "rsqrt_g_s": 5034.0, "dfma_per_clk_sm": 2.0,
         "ffma2_lane_per_clk_sm": 128.0, "rsqrt_per_clk_sm": 16.0}


def test_fp64_roofline_arithmetic():
    """achieved = FP64-pipe instructions per interaction x N^2 / force time,
    against the measured DFMA rate; the 20-flop convention beside it."""
    b = _bench_module()
    n = 2 ** 20
    t_ms = 11570.0
    r = b.roofline_fp64(n, True, t_ms, t_ms + 1.0, PIPES)
    inter = float(n) * n
    assert r["bound"] == "alu" and r["instr_per_interaction"] == 6
    assert abs(r["achieved"] - 6 * inter / (t_ms * 1e-3) / 1e9) < 1e-9 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / 629.28) < 1e-12
    assert abs(r["convention_20flop"]["achieved"] - 20 * inter / (t_ms * 1e-3) / 1e12) < 1e-12
    one_sided = b.roofline_fp64(n, False, t_ms, t_ms, PIPES)
    assert one_sided["instr_per_interaction"] == 9 and one_sided["kernel"] == "k_force_f64"


def test_fp32_pipe_roofline_arithmetic():
    b = _bench_module()
    n = 2 ** 20
    r = b.roofline_fp32_pipe("k_force_mixed", 13, n, 440.0, PIPES)
    achieved = 13 * float(n) * n / 0.44 / 1e9
    assert abs(r["achieved"] - achieved) < 1e-9 * achieved
    assert abs(r["frac"] - achieved / 40273.92) < 1e-12 and r["unit"] == "G FMA-pipe lane-ops/s"


def test_fp64_traffic_reported_only_for_the_captured_kernel_source():
    """The stored DRAM traffic of the each-pair-once path applies to the kernel
    source it was captured from (a hash of the functions involved) and size."""
    b = _bench_module()
    assert b.traffic_f64(2 ** 20, True) == b.TRAFFIC["k_force_f64_sym"]["bytes"]
    assert b.traffic_f64(2 ** 18, True) is None
