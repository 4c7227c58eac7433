"""Write the oracle fixtures in this folder.  Calls only oracle/ and the seeded
input generators; run from the repository root:  python tests/golden/make_golden.py

plummer64.txt -- Plummer sphere, N = 64, seed 20180111, eps = 0.05, G = 1:
  the input state, the Eq. 1-2 accelerations and potentials at t = 0, the
  state after 10 KDK steps (Eq. 5-7) of dt = 1e-3, the state after 3 classical
  RK4 steps of dt = 1e-3, the Eq. 8-10 diagnostics at t = 0, and the state
  after 3 steps of dt = 1e-3 of the fourth-order composition of the KDK step.
Values are written with 17 significant digits (exact round trip of binary64).
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import nbody_ics  # noqa: E402
import oracle  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    n, eps, G, dt = 64, 0.05, 1.0, 1e-3
    pos, vel, mass = nbody_ics.plummer(n, nbody_ics.SEED_BASE)
    acc, pot, _ = oracle.accel(pos, mass, eps, G)
    kp, kv, ka, _ = oracle.kdk(pos, vel, mass, eps, G, dt, 10)
    rp, rv, _ = oracle.rk4(pos, vel, mass, eps, G, dt, 3)
    fp, fv, _, _ = oracle.fr4(pos, vel, mass, eps, G, dt, 3)
    d = oracle.diag(pos, vel, mass, eps, G)
    with open(os.path.join(HERE, "plummer64.txt"), "w") as f:
        f.write("# Plummer N=64 seed 20180111 eps=0.05 G=1 dt=1e-3; written by make_golden.py from oracle/\n")
        f.write("# columns: x y z vx vy vz m | ax ay az pot | kdk10: x y z vx vy vz | rk4x3: x y z vx vy vz | fr4x3: x y z vx vy vz\n")
        f.write("# diag E K W Px Py Pz Lx Ly Lz: " + " ".join("%.17g" % x for x in
                [d["E"], d["K"], d["W"], *d["P"], *d["L"]]) + "\n")
        for i in range(n):
            row = [*pos[i], *vel[i], mass[i], *acc[i], pot[i], *kp[i], *kv[i], *rp[i], *rv[i], *fp[i], *fv[i]]
            f.write(" ".join("%.17g" % x for x in row) + "\n")


if __name__ == "__main__":
    main()
