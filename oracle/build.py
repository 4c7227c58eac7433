"""Compile the FP64 CPU oracle (test infrastructure) into oracle/liboracle.so,
and the plain CPU loop of the benchmark's CPU baseline into
oracle/libcpu_plain.so.

Oracle: plain gcc, -O2 with -ffp-contract=off so that no multiply-add is
fused (the oracle's roundings are the ones its source spells out), OpenMP
over particles.  Plain loop: -O3 with contraction and vectorisation allowed
and no -march flag, so it builds and runs alike on x86-64 and aarch64 hosts
(each uses its baseline vector unit).  Both build identically on either host.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "nbody_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
PLAIN_SRC = os.path.join(HERE, "cpu_plain.c")
PLAIN_LIB = os.path.join(HERE, "libcpu_plain.so")


def build(force: bool = False, src: str = SRC, lib: str = LIB) -> str:
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(src):
        return lib
    cc = os.environ.get("CC", "gcc")
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-Wall", "-Wextra", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def build_plain(force: bool = False) -> str:
    if not force and os.path.exists(PLAIN_LIB) and os.path.getmtime(PLAIN_LIB) >= os.path.getmtime(PLAIN_SRC):
        return PLAIN_LIB
    cc = os.environ.get("CC", "gcc")
    tmp = PLAIN_LIB + f".tmp{os.getpid()}"
    cmd = [cc, "-O3", "-std=c11", "-ffp-contract=fast", "-fno-math-errno", "-fopenmp",
           "-fPIC", "-shared", "-Wall", "-Wextra", "-o", tmp, PLAIN_SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, PLAIN_LIB)
    return PLAIN_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build_plain(force="--force" in sys.argv))
