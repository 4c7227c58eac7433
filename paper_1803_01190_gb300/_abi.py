"""ctypes declarations of the C ABI in include/nbody.h (libnbody.so).

Loading fails loudly when the compiled library is missing: there is no
fallback implementation.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libnbody.so")

if not os.path.exists(library_path):
    raise ImportError(
        f"{library_path} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()' or python -m paper_1803_01190_gb300.build)")

lib = ctypes.CDLL(library_path)

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESTATE, ENOSPC = 0, -1, -2, -3, -4, -5, -6
FP64, MIXED, FP32, F64E = 0, 1, 2, 3
KDK, RK4, FR4 = 0, 1, 2

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_d = ctypes.c_double
_i = ctypes.c_int
_dp = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "nbody_version": (_i, []),
    "nbody_strerror": (ctypes.c_char_p, [_i]),
    "nbody_last_error": (ctypes.c_char_p, []),
    "nbody_create": (_i, [ctypes.POINTER(_vp), _i64, _i, _d, _d, _vp]),
    "nbody_destroy": (_i, [_vp]),
    "nbody_set_timeout": (_i, [_vp, _d]),
    "nbody_set_state": (_i, [_vp, _vp, _vp, _vp, _i]),
    "nbody_get_state": (_i, [_vp, _vp, _vp, ctypes.POINTER(_d), ctypes.POINTER(_i64), _i]),
    "nbody_set_clock": (_i, [_vp, _d, _i64]),
    "nbody_accel": (_i, [_vp, _vp, _vp, _vp, _vp, _i]),
    "nbody_get_accel": (_i, [_vp, _vp, _vp, _i]),
    "nbody_accel_rows": (_i, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _i]),
    "nbody_step": (_i, [_vp, _i, _d, _i64]),
    "nbody_diagnostics": (_i, [_vp, _dp, _dp, _dp]),
    "nbody_diagnostics_ext": (_i, [_vp, _dp, _dp, _dp, _dp, _dp]),
    "nbody_set_launch": (_i, [_vp, _i, _i]),
    "nbody_get_launch": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                              ctypes.POINTER(_i)]),
    "nbody_set_symmetric": (_i, [_vp, _i]),
    "nbody_get_symmetric": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "nbody_set_order": (_i, [_vp, _i]),
    "nbody_get_order": (_i, [_vp, ctypes.POINTER(_i)]),
    "nbody_launch_count": (_i64, [_vp]),
    "nbody_profile": (_i, [_vp, _i]),
    "nbody_profile_read": (_i, [_vp, ctypes.POINTER(_d), ctypes.POINTER(_i64)]),
    "nbody_batch_bytes_per_particle": (_i64, []),
    "nbody_batch_last_error": (ctypes.c_char_p, []),
    "nbody_batch_create": (_i, [ctypes.POINTER(_vp), _i64, _i, _vp]),
    "nbody_batch_destroy": (_i, [_vp]),
    "nbody_batch_admit": (_i, [_vp, _i64, _i, _d, _d, _d, _vp, _vp, _vp, _i, ctypes.POINTER(_i)]),
    "nbody_batch_evict": (_i, [_vp, _i]),
    "nbody_batch_step": (_i, [_vp, _i64]),
    "nbody_batch_sync": (_i, [_vp]),
    "nbody_batch_query": (_i, [_vp]),
    "nbody_batch_get_state": (_i, [_vp, _i, _vp, _vp, ctypes.POINTER(_d), ctypes.POINTER(_i64), _i]),
    "nbody_batch_get_accel": (_i, [_vp, _i, _vp, _vp, _i]),
    "nbody_batch_diagnostics": (_i, [_vp, _i, _dp, _dp, _dp, _dp, _dp]),
    "nbody_batch_info": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "nbody_batch_slot_info": (_i, [_vp, _i, ctypes.POINTER(_i64), ctypes.POINTER(_i),
                                   ctypes.POINTER(_i64)]),
    "nbody_batch_set_launch": (_i, [_vp, _i, _i, _i64]),
    "nbody_batch_profile": (_i, [_vp, _i]),
    "nbody_batch_set_fp64_residency": (_i, [_vp, _i]),
    "nbody_batch_profile_read": (_i, [_vp, _i64, _vp, _vp, _vp, ctypes.POINTER(_i64)]),
    "nbody_batch_launch_count": (_i64, [_vp]),
    "nbody_accel_f64_static": (_i, [_i64, _vp, _vp, _d, _d, _vp, _vp, _vp]),
    "nbody_measure_pipes": (_i, [_dp, _i]),
}

for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class NbodyError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        getter = lib.nbody_batch_last_error if where.startswith("nbody_batch") else lib.nbody_last_error
        detail = getter().decode(errors="replace")
        super().__init__(f"{where} failed ({code}): {detail}")


def check(code, where="nbody"):
    if code != OK:
        raise NbodyError(code, where)
    return code
