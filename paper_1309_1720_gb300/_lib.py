"""ctypes loader for libcardiac_gb300.so (the C ABI of include/cardiac_gb300.h).

Argument marshalling only.  If the shared library has not been built the
import of any entry point raises: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# CG_BOUNDS_CHECK=1 in the environment loads the checked build instead (every
# stage worker checks its indices before use; see cg_bounds_checked).
CHECKED = os.environ.get("CG_BOUNDS_CHECK", "") not in ("", "0")
LIB_PATH = os.path.join(HERE, "libcardiac_gb300_checked.so" if CHECKED else "libcardiac_gb300.so")

c_dp = ctypes.POINTER(ctypes.c_double)


class CProblem(ctypes.Structure):
    """Mirror of ``cg_problem``."""
    _fields_ = [
        ("abi_version", ctypes.c_int32), ("model", ctypes.c_int32),
        ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("Dxx", ctypes.c_double * 4), ("Dyy", ctypes.c_double * 4),
        ("stencil", ctypes.c_int32), ("bc", ctypes.c_int32),
        ("scheme", ctypes.c_int32), ("flags", ctypes.c_uint32),
        ("alpha_d", ctypes.c_double), ("dt", ctypes.c_double),
        ("params", c_dp), ("n_params", ctypes.c_int32), ("reserved0", ctypes.c_int32),
        ("barrier_timeout_s", ctypes.c_double),
    ]


class CTuning(ctypes.Structure):
    """Mirror of ``cg_tuning``."""
    _fields_ = [("cells_x", ctypes.c_int32), ("rows", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("schedule", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "cg_plan_create": (ctypes.c_int, [ctypes.POINTER(CProblem), ctypes.POINTER(ctypes.c_void_p)]),
    "cg_plan_create_tuned": (ctypes.c_int, [ctypes.POINTER(CProblem), ctypes.POINTER(CTuning),
                                            ctypes.POINTER(ctypes.c_void_p)]),
    "cg_batch_create": (ctypes.c_int, [ctypes.POINTER(CProblem), ctypes.c_int32, ctypes.POINTER(CTuning),
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "cg_batch_offsets": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "cg_plan_n_instances": (ctypes.c_int32, [ctypes.c_void_p]),
    "cg_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "cg_workspace_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "cg_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                              ctypes.c_void_p, ctypes.c_void_p]),
    "cg_get_device_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32)]),
    "cg_read_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_uint32)]),
    "cg_tlm_workspace_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    "cg_tlm_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.c_void_p]),
    "cg_tlm_linearized_workspace_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                                        ctypes.POINTER(ctypes.c_size_t)]),
    "cg_tlm_linearize": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "cg_tlm_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                    ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "cg_adjoint_workspace_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                                 ctypes.POINTER(ctypes.c_size_t)]),
    "cg_adjoint_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "cg_adjoint_checkpoint_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                                  ctypes.POINTER(ctypes.c_size_t)]),
    "cg_adjoint_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cg_adjoint_reverse": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "cg_newton_workspace_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    "cg_newton_gmres_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_double, ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                                            ctypes.c_void_p, ctypes.c_void_p]),
    "cg_newton_linearized_workspace_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                                           ctypes.POINTER(ctypes.c_size_t)]),
    "cg_newton_gmres_step_linearized": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                                       ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                                       ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p,
                                                       ctypes.c_void_p]),
    "cg_dot": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p]),
    "cg_axpby": (ctypes.c_int, [ctypes.c_double, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64,
                                ctypes.c_void_p]),
    "cg_run_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                      ctypes.c_void_p, ctypes.c_void_p]),
    "cg_host_workspace_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "cg_rhs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "cg_batch_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                    ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "cg_run_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                   ctypes.c_void_p, ctypes.c_void_p]),
    "cg_last_error": (ctypes.c_char_p, []),
    "cg_n_fields": (ctypes.c_int32, [ctypes.c_int32]),
    "cg_n_params": (ctypes.c_int32, [ctypes.c_int32]),
    "cg_default_params": (ctypes.c_int, [ctypes.c_int32, c_dp]),
    "cg_abi_version": (ctypes.c_int32, []),
    "cg_bounds_checked": (ctypes.c_int32, []),
    "cg_adjoint_schedule": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]),
    "cg_static_schedule": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int32), ctypes.c_int64,
                                          ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_int32)]),
    "cg_check_fastmath": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int64]),
    "cg_measure_fp64_rate": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double)]),
}


def lib() -> ctypes.CDLL:
    """Load the library (once) and attach the signatures."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    "%s is not built; run `python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class CGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("cg status %d: %s" % (status, msg))
        self.status = status


def check(status: int) -> None:
    if status != 0:
        raise CGError(status, lib().cg_last_error().decode(errors="replace"))
