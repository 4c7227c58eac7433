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
