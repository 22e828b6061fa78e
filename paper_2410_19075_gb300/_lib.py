"""ctypes loader for libsim.so (argument marshalling only).

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_2410_19075_gb300.build``).  There is no fallback: if the shared
library is missing or fails to load, every call raises.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsim.so")

SIM_OK, SIM_EINVAL, SIM_ENOMEM, SIM_EDEVICE, SIM_ETIMEOUT, SIM_ENONFINITE, SIM_EBUSY = 0, -1, -2, -3, -4, -5, -6
SIM_ESTEPS, SIM_ESMALL = -7, -8
STATUS_NAMES = {0: "SIM_OK", -1: "SIM_EINVAL", -2: "SIM_ENOMEM", -3: "SIM_EDEVICE", -4: "SIM_ETIMEOUT",
                -5: "SIM_ENONFINITE", -6: "SIM_EBUSY", -7: "SIM_ESTEPS", -8: "SIM_ESMALL"}


class DP5Opts(ctypes.Structure):
    _fields_ = [("t0", ctypes.c_double), ("t_end", ctypes.c_double), ("rtol", ctypes.c_double),
                ("atol", ctypes.c_double), ("h0", ctypes.c_double), ("h_max", ctypes.c_double),
                ("out_dt", ctypes.c_double), ("max_attempts", ctypes.c_int64)]


class DP5Stats(ctypes.Structure):
    _fields_ = [("accepted", ctypes.c_int64), ("rejected", ctypes.c_int64), ("t", ctypes.c_double),
                ("h_next", ctypes.c_double), ("status", ctypes.c_int)]


class SimError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None
_i64, _int, _uint, _dbl, _vp, _sz = ctypes.c_int64, ctypes.c_int, ctypes.c_uint, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
_dp = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes)
SIGNATURES = {
    "sim_workspace_bytes": (_sz, [_int, _int, _i64, _i64]),
    "sim_create": (_int, [ctypes.POINTER(_vp), _int, _int, _i64, _i64, _dp, _int, _uint, _vp]),
    "sim_create_in": (_int, [ctypes.POINTER(_vp), _int, _int, _i64, _i64, _dp, _int, _uint, _vp, _sz, _vp]),
    "sim_nodes": (_i64, [_vp]),
    "sim_dim": (_int, [_vp]),
    "sim_set_state": (_int, [_vp, _vp, _i64]),
    "sim_set_state_device": (_int, [_vp, _vp, _i64]),
    "sim_set_node_param": (_int, [_vp, _int, _vp, _i64]),
    "sim_step": (_int, [_vp, _i64, _dbl]),
    "sim_step_timed": (_int, [_vp, _i64, _dbl, _dp, ctypes.POINTER(_i64)]),
    "sim_get_state": (_int, [_vp, _vp, _i64]),
    "sim_get_state_device": (_int, [_vp, _vp, _i64]),
    "sim_rhs": (_int, [_vp, _vp, _i64]),
    "sim_observables": (_int, [_vp, _vp, _i64, ctypes.POINTER(_i64)]),
    "sim_sync": (_int, [_vp]),
    "sim_batch_create": (_int, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), _int, _vp]),
    "sim_batch_set_budgets": (_int, [_vp, ctypes.POINTER(_i64)]),
    "sim_batch_step": (_int, [_vp, _i64, _dbl]),
    "sim_batch_sync": (_int, [_vp]),
    "sim_batch_destroy": (None, [_vp]),
    "srv_create": (_int, [ctypes.POINTER(_vp), _sz, _int, _i64, _vp]),
    "srv_submit": (_int, [_vp, _int, _int, _i64, _i64, _dp, _int, _vp, _vp, _i64, _dbl, ctypes.POINTER(_i64)]),
    "srv_poll": (_int, [_vp, _i64, ctypes.POINTER(_int), _vp, _i64, _vp, _i64, ctypes.POINTER(_i64), _vp]),
    "srv_wait_idle": (_int, [_vp]),
    "srv_stats": (_int, [_vp, ctypes.POINTER(_i64)]),
    "srv_timings": (_int, [_vp, _dp]),
    "srv_memory": (_int, [_vp, ctypes.POINTER(_i64)]),
    "sim_autotune": (_int, [_vp, ctypes.c_double, _i64, ctypes.POINTER(_int), ctypes.POINTER(_int)]),
    "sim_tune_info": (_int, [_vp, ctypes.POINTER(_int), ctypes.POINTER(_int)]),
    "sim_batch_autotune": (_int, [_vp, ctypes.c_double, _i64, ctypes.POINTER(_int)]),
    "sim_tune_save": (_int, [ctypes.c_char_p]),
    "sim_tune_load": (_int, [ctypes.c_char_p]),
    "sim_tune_clear": (_int, []),
    "srv_destroy": (None, [_vp]),
    "sim_math_eval": (_int, [_int, _vp, _vp, _i64]),
    "sim_probe_peak": (_int, [_int, ctypes.POINTER(ctypes.c_double)]),
    "sim_ring_step_noalloc": (_int, [_int, _i64, _i64, _dp, _int, _uint, _vp, _vp, _i64, _dbl, _vp]),
    "sim_steps_done": (_i64, [_vp]),
    "sim_dp5": (_int, [_vp, ctypes.POINTER(DP5Opts), ctypes.POINTER(DP5Stats)]),
    "sim_create_graph": (_int, [ctypes.POINTER(_vp), _int, _i64, _vp, _vp, _dp, _int, _vp]),
    "sim_graph_info": (_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_sz)]),
    "sim_batch_dp5": (_int, [_vp, ctypes.POINTER(DP5Opts), ctypes.POINTER(DP5Stats)]),
    "sim_last_error": (ctypes.c_char_p, []),
    "sim_destroy": (None, [_vp]),
}


def lib():
    """Load libsim.so once and declare every signature."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it first with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status):
    if status != SIM_OK:
        raise SimError(status, lib().sim_last_error().decode())
    return status
