"""C-ABI library checks that need no GPU: it builds, loads, exports every
function include/nbody.h declares, and rejects bad arguments before touching
the device."""
import ctypes
import os
import re
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "nbody.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(nbody_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def nbmod():
    import __graft_entry__ as g
    g.build()
    import paper_1803_01190_gb300 as nb
    return nb


def test_every_declared_function_is_exported(nbmod):
    names = header_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(nbmod.lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", nbmod.library_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (nbody_\w+)$", out, flags=re.M))
    assert set(names) <= exported, set(names) - exported


def test_version_and_strerror(nbmod):
    assert nbmod.version() >= 100
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert nbmod.lib.nbody_strerror(code)
    assert nbmod.lib.nbody_strerror(-99) == b"unknown error"


@pytest.mark.parametrize("n,mode,eps,G", [(0, 0, 0.1, 1.0), (-5, 0, 0.1, 1.0), (10, 7, 0.1, 1.0),
                                          (10, 0, -1.0, 1.0), (10, 0, float("nan"), 1.0),
                                          (10, 0, 0.1, float("inf")), (10, 2, 1e-30, 1.0)])
def test_create_rejects_bad_arguments(nbmod, n, mode, eps, G):
    h = ctypes.c_void_p()
    rc = nbmod.lib.nbody_create(ctypes.byref(h), n, mode, eps, G, None)
    assert rc == -1 and not h.value
    assert b"invalid argument" in nbmod.lib.nbody_last_error()


def test_null_context_rejected(nbmod):
    L = nbmod.lib
    assert L.nbody_step(None, 0, 1e-3, 1) == -1
    assert L.nbody_diagnostics(None, None, None, None) == -1
    assert L.nbody_get_state(None, None, None, None, None, 0) == -1
    assert L.nbody_destroy(None) == 0
    assert L.nbody_launch_count(None) == 0


def test_missing_library_fails_loudly(tmp_path):
    """Without libnbody.so the package refuses to import: no CPU fallback."""
    pkg = tmp_path / "paper_1803_01190_gb300"
    shutil.copytree(os.path.join(ROOT, "paper_1803_01190_gb300"), pkg,
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    r = subprocess.run([sys.executable, "-c", "import paper_1803_01190_gb300"], cwd=tmp_path,
                       capture_output=True, text=True)
    assert r.returncode != 0 and "libnbody.so is missing" in r.stderr


def test_product_never_imports_oracle():
    """The library package and its C sources never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_1803_01190_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "nbody_oracle" not in txt and "liboracle" not in txt, f
