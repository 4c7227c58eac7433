"""FP64 CPU oracle for the direct PP N-body method (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package; the GPU library never does, and this package never
imports the GPU library.  It wraps the plain C oracle in nbody_oracle.c
(Eq. 1-2 force and potential, Eq. 5-7 KDK leapfrog, classical RK4 and the
fourth-order symplectic composition of the KDK step as the two readings of
the paper's fourth-order scheme, Eq. 8-10 diagnostics) with numpy arrays.  Arrays are float64, C-contiguous, positions/velocities shaped (n, 3).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int64)


def _d(a):
    return a.ctypes.data_as(_dp)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class Oracle:
    """The oracle's entry points bound to one compiled copy of nbody_oracle.c."""

    def __init__(self, path):
        lib = ctypes.CDLL(path)
        lib.oracle_accel.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int64, _ip, _dp, _dp, _dp, ctypes.c_int]
        lib.oracle_kdk.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int64, _dp, _dp, ctypes.c_int]
        lib.oracle_fr4.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int64, _dp, _dp, ctypes.c_int]
        lib.oracle_rk4.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int64, _dp, ctypes.c_int]
        lib.oracle_diag.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                    _dp, ctypes.c_int]
        for f in (lib.oracle_accel, lib.oracle_kdk, lib.oracle_fr4, lib.oracle_rk4, lib.oracle_diag):
            f.restype = ctypes.c_int
        lib.oracle_max_threads.restype = ctypes.c_int
        self.lib = lib
        self.path = path

    def max_threads(self) -> int:
        return self.lib.oracle_max_threads()

    def accel(self, pos, mass, eps, G=1.0, rows=None, threads=0):
        """Eq. 1-2: (acc (k,3), pot (k,), smag (k,)) for the particles in `rows`
        (all particles when rows is None).  smag_i = G sum_{j!=i} m_j |d_ij| / (d^2+eps^2)^{3/2}."""
        pos = _f64(pos, (-1, 3))
        mass = _f64(mass, (-1,))
        n = pos.shape[0]
        assert mass.shape[0] == n
        if rows is None:
            k, rp = n, None
        else:
            rows = np.ascontiguousarray(rows, dtype=np.int64)
            k, rp = rows.shape[0], rows.ctypes.data_as(_ip)
        acc = np.empty((k, 3))
        pot = np.empty(k)
        smag = np.empty(k)
        rc = self.lib.oracle_accel(n, _d(pos), _d(mass), float(eps), float(G), k, rp,
                                   _d(acc), _d(pot), _d(smag), int(threads))
        if rc != 0:
            raise ValueError("oracle_accel: bad argument")
        return acc, pot, smag

    def kdk(self, pos, vel, mass, eps, G, dt, nsteps, acc0=None, threads=0):
        """Eq. 5-7 for nsteps steps.  Returns (pos, vel, acc, pot) at the end;
        acc0 = a(t0) (evaluated here when None)."""
        pos = _f64(pos, (-1, 3)).copy()
        vel = _f64(vel, (-1, 3)).copy()
        mass = _f64(mass, (-1,))
        n = pos.shape[0]
        if acc0 is None:
            acc = self.accel(pos, mass, eps, G, threads=threads)[0]
        else:
            acc = _f64(acc0, (-1, 3)).copy()
        pot = np.empty(n)
        rc = self.lib.oracle_kdk(n, _d(pos), _d(vel), _d(mass), float(eps), float(G), float(dt),
                                 int(nsteps), _d(acc), _d(pot), int(threads))
        if rc != 0:
            raise ValueError("oracle_kdk: bad argument")
        return pos, vel, acc, pot

    def fr4(self, pos, vel, mass, eps, G, dt, nsteps, acc0=None, threads=0):
        """Fourth-order symplectic composition of Eq. 5-7 (three KDK steps of
        w1 dt, w0 dt, w1 dt).  Returns (pos, vel, acc, pot) at the end;
        acc0 = a(t0) (evaluated here when None)."""
        pos = _f64(pos, (-1, 3)).copy()
        vel = _f64(vel, (-1, 3)).copy()
        mass = _f64(mass, (-1,))
        n = pos.shape[0]
        if acc0 is None:
            acc = self.accel(pos, mass, eps, G, threads=threads)[0]
        else:
            acc = _f64(acc0, (-1, 3)).copy()
        pot = np.empty(n)
        rc = self.lib.oracle_fr4(n, _d(pos), _d(vel), _d(mass), float(eps), float(G), float(dt),
                                 int(nsteps), _d(acc), _d(pot), int(threads))
        if rc != 0:
            raise ValueError("oracle_fr4: bad argument")
        return pos, vel, acc, pot

    def rk4(self, pos, vel, mass, eps, G, dt, nsteps, threads=0):
        """Classical RK4 (the reading of the paper's fourth-order scheme).
        Returns (pos, vel, acc) at the end."""
        pos = _f64(pos, (-1, 3)).copy()
        vel = _f64(vel, (-1, 3)).copy()
        mass = _f64(mass, (-1,))
        n = pos.shape[0]
        acc = np.empty((n, 3))
        rc = self.lib.oracle_rk4(n, _d(pos), _d(vel), _d(mass), float(eps), float(G), float(dt),
                                 int(nsteps), _d(acc), int(threads))
        if rc != 0:
            raise ValueError("oracle_rk4: bad argument")
        return pos, vel, acc

    def diag(self, pos, vel, mass, eps, G=1.0, threads=0):
        """Eq. 8-10: dict with E, K, W, P (3,), L (3,) (L[2] is the paper's L)."""
        pos = _f64(pos, (-1, 3))
        vel = _f64(vel, (-1, 3))
        mass = _f64(mass, (-1,))
        out = np.empty(9)
        rc = self.lib.oracle_diag(pos.shape[0], _d(pos), _d(vel), _d(mass), float(eps), float(G),
                                  _d(out), int(threads))
        if rc != 0:
            raise ValueError("oracle_diag: bad argument")
        return {"E": out[0], "K": out[1], "W": out[2], "P": out[3:6].copy(), "L": out[6:9].copy()}


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(_build.build())
    return _default


def max_threads():
    return default().max_threads()


def accel(*a, **k):
    return default().accel(*a, **k)


def kdk(*a, **k):
    return default().kdk(*a, **k)


def fr4(*a, **k):
    return default().fr4(*a, **k)


def rk4(*a, **k):
    return default().rk4(*a, **k)


def diag(*a, **k):
    return default().diag(*a, **k)


_plain = None


def plain_accel(pos, mass, eps, G=1.0, rows=None, threads=0):
    """The plain (uncompensated, vectorised) binary64 CPU loop of cpu_plain.c:
    the benchmark's CPU throughput figure, never a parity reference.
    Returns (acc (k,3), pot (k,))."""
    global _plain
    if _plain is None:
        lib = ctypes.CDLL(_build.build_plain())
        lib.plain_accel.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int64, _ip, _dp, _dp, ctypes.c_int]
        lib.plain_accel.restype = ctypes.c_int
        lib.plain_max_threads.restype = ctypes.c_int
        _plain = lib
    pos = _f64(pos, (-1, 3))
    mass = _f64(mass, (-1,))
    n = pos.shape[0]
    if rows is None:
        k, rp = n, None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        k, rp = rows.shape[0], rows.ctypes.data_as(_ip)
    acc = np.empty((k, 3))
    pot = np.empty(k)
    if _plain.plain_accel(n, _d(pos), _d(mass), float(eps), float(G), k, rp, _d(acc), _d(pot),
                          int(threads)) != 0:
        raise ValueError("plain_accel: bad argument")
    return acc, pot
