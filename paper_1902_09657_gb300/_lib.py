"""ctypes declarations of the C ABI in include/kpdhg.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# KPDHG_CHECKED=1 loads the bounds-checked build (libkpdhg_checked.so, `_build --checked`)
LIB_PATH = os.path.join(HERE, "libkpdhg_checked.so" if os.environ.get("KPDHG_CHECKED") == "1" else "libkpdhg.so")

KP_OK, KP_EINVAL, KP_ENOMEM, KP_ECUDA, KP_ECUFFT, KP_EDIVERGED, KP_ENONFINITE, KP_ETIMEOUT, KP_EINTERNAL = range(9)
KP_C64, KP_C32_BF16, KP_C32_FP16 = 0, 1, 2
KP_REG_L2, KP_REG_L1_WAVELET, KP_REG_TV = 0, 1, 2


class KpParams(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("img", ctypes.c_int64 * 3),
        ("ncoils", ctypes.c_int),
        ("nsamples", ctypes.c_int64),
        ("oversamp", ctypes.c_float),
        ("kernel_width", ctypes.c_int),
        ("wavelet_levels", ctypes.c_int),
    ]


class KpStats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int),
        ("lmax", ctypes.c_double),
        ("pmin", ctypes.c_double),
        ("sigma_last", ctypes.c_double),
        ("tau_last", ctypes.c_double),
        ("final_obj", ctypes.c_double),
        ("phase_ms", ctypes.c_double * 12),
    ]


class KpState(ctypes.Structure):
    _fields_ = [
        ("x", ctypes.c_void_p),
        ("xbar", ctypes.c_void_p),
        ("u", ctypes.c_void_p),
        ("v", ctypes.c_void_p),
        ("k", ctypes.c_int),
    ]


PHASES = ["fwd_pre", "fft_fwd", "interp_dual", "spread", "spread_reduce", "fft_inv", "adj_primal",
          "dwt_fwd", "soft", "dwt_inv", "extrap", "counter"]


_vp = ctypes.c_void_p
_SIGS = {
    "kp_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "kp_last_error": (ctypes.c_char_p, []),
    "kp_plan_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(KpParams), _vp]),
    "kp_plan_destroy": (ctypes.c_int, [_vp]),
    "kp_plan_set_trajectory": (ctypes.c_int, [_vp, _vp, _vp]),
    "kp_plan_set_maps": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp]),
    "kp_sense_forward": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "kp_sense_adjoint": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp]),
    "kp_make_preconditioner": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "kp_max_eig": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _vp]),
    "kp_pdhg_solve": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                                     ctypes.c_double, _vp, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(KpStats), _vp]),
    "kp_pdhg_solve_host": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                                          ctypes.c_double, _vp, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(KpStats), _vp]),
    "kp_pdhg_solve_ex": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                                        ctypes.c_double, ctypes.POINTER(KpState), ctypes.POINTER(KpState),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(KpStats), _vp]),
    "kp_plan_set_wait_limit": (ctypes.c_int, [_vp, ctypes.c_longlong]),
    "kp_make_circulant_preconditioner": (ctypes.c_int, [_vp, _vp, _vp]),
    "kp_cg_l2_solve": (ctypes.c_int, [_vp, _vp, ctypes.c_float, ctypes.c_int, ctypes.c_int, _vp,
                                      ctypes.POINTER(ctypes.c_double), _vp]),
    "kp_fista_solve": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_float, ctypes.c_int, ctypes.c_double, _vp,
                                      ctypes.POINTER(ctypes.c_double), _vp]),
    "kp_plan_sync": (ctypes.c_int, [_vp, _vp]),
    "kp_wavelet": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "kp_plan_set_profiling": (ctypes.c_int, [_vp, ctypes.c_int]),
    "kp_plan_launch_count": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int64)]),
    "kp_bounds_report": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_uint32),
                                        ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_int64)]),
    "kp_sense_adjoint_noalloc": (ctypes.c_int, [ctypes.POINTER(KpParams), _vp, _vp, _vp, _vp, _vp]),
    "kp_sense_forward_traj_grad": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "kp_sense_adjoint_traj_grad": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "kp_unrolled_forward": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_float, ctypes.c_int, ctypes.c_double, _vp, _vp]),
    "kp_unrolled_backward": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(ctypes.c_double), _vp, _vp]),
    "kp_plan_tile_stats": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "kp_dual_l2_solve": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_float, ctypes.c_int, _vp,
                                        ctypes.POINTER(ctypes.c_double), _vp]),
    "kp_plan_spread_config": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "kp_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int]),
    "kp_batch_solve": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_vp),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float), ctypes.c_int,
                                      ctypes.POINTER(_vp), _vp]),
    "kp_batch_destroy": (ctypes.c_int, [_vp]),
    "kp_batch_set_form": (ctypes.c_int, [_vp, ctypes.c_int]),
}

_lib = None


class KpError(RuntimeError):
    def __init__(self, status, fn, msg):
        self.status = status
        super().__init__(f"{fn} failed: {status_name(status)}: {msg}")


def load():
    """Load libkpdhg.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{os.path.basename(LIB_PATH)} is not built ({LIB_PATH} missing); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'` first (the checked "
                           "variant: `python -m paper_1902_09657_gb300._build --checked`)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def status_name(s):
    try:
        return load().kp_status_string(s).decode()
    except Exception:  # pragma: no cover - only when the library is absent
        return str(s)


def check(status, fn):
    if status != KP_OK:
        msg = load().kp_last_error().decode()
        raise KpError(status, fn, msg)
