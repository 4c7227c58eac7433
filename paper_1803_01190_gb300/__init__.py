"""GB300 direct-summation N-body library: Python binding of libnbody.so.

The computation (Eq. 1-2 force and potential, Eq. 5-7 KDK leapfrog, the
fourth-order scheme as classical RK4 or as the symplectic composition of the
KDK step, Eq. 8-10 diagnostics) runs in the CUDA kernels of
csrc/ behind the C ABI declared in include/nbody.h.  This module only
marshals arguments: it turns numpy arrays or torch tensors into pointers,
picks the current torch CUDA stream, and turns error codes into exceptions.
There is no CPU fallback: if the CUDA library is missing, importing the
binding's entry points raises.

Arrays: positions and velocities (n, 3) float64, masses (n,) float64,
C-contiguous.  A torch tensor on the GPU is passed as a device pointer
(on_device=1); a numpy array or CPU tensor as a host pointer.
"""
import ctypes
import os

import numpy as np

from . import _abi
from ._abi import (F64E, FP32, FP64, FR4, KDK, MIXED, RK4, NbodyError, check, lib,  # noqa: F401
                   library_path)

MODES = {"fp64": FP64, "mixed": MIXED, "fp32": FP32, "f64e": F64E}
SCHEMES = {"kdk": KDK, "rk4": RK4, "fr4": FR4}

__all__ = ["Simulation", "NbodyError", "MODES", "SCHEMES", "lib", "library_path", "build",
           "measure_pipes"]


def build(force=False):
    """Compile libnbody.so in-tree (nvcc, sm_103a)."""
    from . import build as _b
    return _b.build(force=force)


def _torch():
    try:
        import torch
        return torch
    except ImportError:  # pragma: no cover
        return None


def _is_cuda_tensor(a):
    t = _torch()
    return t is not None and isinstance(a, t.Tensor) and a.is_cuda


def _ptr_in(a, shape, keep):
    """Pointer and on_device flag for an input array; `keep` holds temporaries alive."""
    t = _torch()
    if t is not None and isinstance(a, t.Tensor):
        if a.dtype != t.float64:
            raise TypeError("expected a float64 tensor")
        a = a.contiguous()
        if tuple(a.shape) != shape:
            a = a.reshape(shape)
        keep.append(a)
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda)
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(shape)
    keep.append(a)
    return ctypes.c_void_p(a.ctypes.data), 0


def _current_stream():
    t = _torch()
    if t is not None and t.cuda.is_available():
        return ctypes.c_void_p(t.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


PIPE_FIELDS = ("sms", "sm_mhz", "dfma_ginstr_s", "ffma_glane_s", "ffma2_glane_s", "rsqrt_g_s",
               "dfma_per_clk_sm", "ffma2_lane_per_clk_sm", "rsqrt_per_clk_sm")


def measure_pipes():
    """Measured pipe issue rates of the current device (nbody_measure_pipes)."""
    out = (ctypes.c_double * len(PIPE_FIELDS))()
    check(lib.nbody_measure_pipes(out, len(PIPE_FIELDS)), "nbody_measure_pipes")
    return dict(zip(PIPE_FIELDS, (float(x) for x in out)))


class Simulation:
    """One N-body system resident on the GPU (a context of the C ABI).

    mode: "fp64" | "f64e" | "mixed" | "fp32"; eps: softening (the paper's delta);
    G: gravitational constant; stream: a torch.cuda.Stream (default: the
    current one at creation)."""

    def __init__(self, n, mode="fp64", eps=0.01, G=1.0, stream=None):
        self.n = int(n)
        self.mode = mode
        self.eps = float(eps)
        self.G = float(G)
        st = ctypes.c_void_p(stream.cuda_stream) if stream is not None else _current_stream()
        self._stream = stream
        h = ctypes.c_void_p()
        check(lib.nbody_create(ctypes.byref(h), self.n, MODES[mode], self.eps, self.G, st),
              "nbody_create")
        self._h = h

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.nbody_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- outputs
    def _out(self, shape, on_device):
        if on_device:
            t = _torch()
            o = t.empty(shape, dtype=t.float64, device="cuda")
            return o, ctypes.c_void_p(o.data_ptr())
        o = np.empty(shape)
        return o, ctypes.c_void_p(o.ctypes.data)

    # -- state
    def set_state(self, pos, vel, mass):
        keep = []
        pp, dev = _ptr_in(pos, (self.n, 3), keep)
        pv = None
        if vel is not None:
            pv, dv = _ptr_in(vel, (self.n, 3), keep)
            if dv != dev:
                raise ValueError("pos and vel must both be on the host or both on the device")
        pm, dm = _ptr_in(mass, (self.n,), keep)
        if dm != dev:
            raise ValueError("pos and mass must both be on the host or both on the device")
        check(lib.nbody_set_state(self._h, pp, pv, pm, dev), "nbody_set_state")

    def set_clock(self, t, step):
        """Model time and step counter (for resuming from a checkpoint)."""
        check(lib.nbody_set_clock(self._h, float(t), int(step)), "nbody_set_clock")

    def get_state(self, on_device=False):
        """(pos (n,3), vel (n,3), t, step) at the current step boundary."""
        pos, pp = self._out((self.n, 3), on_device)
        vel, pv = self._out((self.n, 3), on_device)
        t = ctypes.c_double()
        s = ctypes.c_int64()
        check(lib.nbody_get_state(self._h, pp, pv, ctypes.byref(t), ctypes.byref(s), int(on_device)),
              "nbody_get_state")
        return pos, vel, t.value, s.value

    def accel(self, pos, mass, on_device=None):
        """Eq. 1-2 for the given positions and masses: (acc (n,3), pot (n,))."""
        keep = []
        pp, dev = _ptr_in(pos, (self.n, 3), keep)
        pm, dm = _ptr_in(mass, (self.n,), keep)
        if dm != dev:
            raise ValueError("pos and mass must both be on the host or both on the device")
        od = dev if on_device is None else int(on_device)
        if od != dev:
            raise ValueError("outputs are returned where the inputs live")
        acc, pa = self._out((self.n, 3), dev)
        pot, po = self._out((self.n,), dev)
        check(lib.nbody_accel(self._h, pp, pm, pa, po, dev), "nbody_accel")
        return acc, pot

    def accel_rows(self, i0, ni, pos, mass):
        """Eq. 1-2 for the rows [i0, i0 + ni) against all n particles of pos and
        mass: (acc (ni,3), pot (ni,)), where the inputs live."""
        keep = []
        pp, dev = _ptr_in(pos, (self.n, 3), keep)
        pm, dm = _ptr_in(mass, (self.n,), keep)
        if dm != dev:
            raise ValueError("pos and mass must both be on the host or both on the device")
        acc, pa = self._out((int(ni), 3), dev)
        pot, po = self._out((int(ni),), dev)
        check(lib.nbody_accel_rows(self._h, int(i0), int(ni), pp, pm, pa, po, dev), "nbody_accel_rows")
        return acc, pot

    def get_accel(self, on_device=False):
        acc, pa = self._out((self.n, 3), on_device)
        pot, po = self._out((self.n,), on_device)
        check(lib.nbody_get_accel(self._h, pa, po, int(on_device)), "nbody_get_accel")
        return acc, pot

    def step(self, dt, nsteps=1, scheme="kdk"):
        check(lib.nbody_step(self._h, SCHEMES[scheme], float(dt), int(nsteps)), "nbody_step")

    def diagnostics(self):
        """Eq. 8-10: dict(E, K, W, P (3,), L (3,)); L[2] is the paper's L."""
        E, K, W = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        P = (ctypes.c_double * 3)()
        L = (ctypes.c_double * 3)()
        check(lib.nbody_diagnostics_ext(self._h, ctypes.byref(E), ctypes.byref(K), ctypes.byref(W),
                                        P, L), "nbody_diagnostics_ext")
        return {"E": E.value, "K": K.value, "W": W.value, "P": np.array(P[:]), "L": np.array(L[:])}

    def set_launch(self, ipt=0, jsplit=0):
        check(lib.nbody_set_launch(self._h, int(ipt), int(jsplit)), "nbody_set_launch")

    def set_symmetric(self, mode=-1):
        """FP64: evaluate each pair once for both particles (-1 auto, 0 off, 1 on)."""
        check(lib.nbody_set_symmetric(self._h, int(mode)), "nbody_set_symmetric")

    def get_symmetric(self):
        """(setting, whether the next force evaluation uses the each-pair-once path)."""
        m, a = ctypes.c_int(), ctypes.c_int()
        check(lib.nbody_get_symmetric(self._h, ctypes.byref(m), ctypes.byref(a)), "nbody_get_symmetric")
        return m.value, bool(a.value)

    def set_order(self, order):
        """Particle order of the force sum: "input" or "spatial" (Morton curve;
        the default in mixed mode)."""
        code = {"input": 0, "spatial": 1}[order]
        check(lib.nbody_set_order(self._h, code), "nbody_set_order")

    def get_order(self):
        o = ctypes.c_int()
        check(lib.nbody_get_order(self._h, ctypes.byref(o)), "nbody_get_order")
        return ("input", "spatial")[o.value]

    def get_launch(self):
        v = [ctypes.c_int() for _ in range(4)]
        check(lib.nbody_get_launch(self._h, *[ctypes.byref(x) for x in v]), "nbody_get_launch")
        return dict(zip(("ipt", "jsplit", "threads", "tile"), (x.value for x in v)))

    def set_timeout(self, seconds):
        check(lib.nbody_set_timeout(self._h, float(seconds)), "nbody_set_timeout")

    def profile(self, enable=True):
        """Time every force-kernel launch with CUDA events on this context's stream."""
        check(lib.nbody_profile(self._h, int(bool(enable))), "nbody_profile")

    def profile_read(self):
        """(summed force-kernel milliseconds, number of timed launches) since the last read."""
        ms = ctypes.c_double()
        k = ctypes.c_int64()
        check(lib.nbody_profile_read(self._h, ctypes.byref(ms), ctypes.byref(k)), "nbody_profile_read")
        return ms.value, k.value

    @property
    def launch_count(self):
        return int(lib.nbody_launch_count(self._h))


def accel(pos, mass, eps, G=1.0, mode="fp64", stream=None):
    """One-shot Eq. 1-2 evaluation through a temporary context."""
    n = int(np.shape(pos)[0]) if not _is_cuda_tensor(pos) else int(pos.shape[0])
    with Simulation(n, mode=mode, eps=eps, G=G, stream=stream) as sim:
        return sim.accel(pos, mass)


def version():
    return int(lib.nbody_version())


def loaded_library():
    """Absolute path of the CUDA library this process uses."""
    return os.path.realpath(library_path)
