"""ctypes declarations of libquadsim.so (include/quadsim.h).  Marshalling only."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
#: QUADSIM_LIB points the binding at another build of the same sources (the
#: bounds-checked build, libquadsim_checked.so).
LIB_PATH = os.environ.get("QUADSIM_LIB") or os.path.join(HERE, "libquadsim.so")

SIM_OK = 0
SIM_ERR_ARG = -1
SIM_ERR_CUDA = -2
SIM_ERR_WORKSPACE = -3
SIM_ERR_TIMEOUT = -4
SIM_ERR_GROUP = -5
SIM_ERR_STALE = -6
SIM_OPEN_LOOP = 0
SIM_CLOSED_LOOP = 1
SIM_CLOSED_LOOP_PID = 2
SIM_TYPE_QUADROTOR, SIM_TYPE_CAR, SIM_TYPE_FIXED_WING = 0, 1, 2
SIM_MAX_GROUPS = 32
SIM_NTHETA = 16
SIM_NOALLOC_SCRATCH_BYTES = 32 << 20

#: Every entry point include/quadsim.h declares.
EXPORTS = ("sim_create", "sim_set_params", "sim_step", "sim_step_host", "sim_rollout_forward",
           "sim_workspace_bytes", "sim_rollout_backward", "sim_set_launch", "sim_get_launch", "sim_status",
           "sim_reset_status", "sim_graph_create", "sim_graph_launch", "sim_graph_destroy", "sim_step_launches",
           "sim_destroy", "sim_error_string", "sim_rollout_backward_noalloc",
           "sim_collide_workspace_bytes", "sim_collide", "sim_copy_status", "sim_run_rounds", "sim_load_status", "sim_compact", "sim_bounds_checks",
           "sim_group_stats")


class GroupParams(ctypes.Structure):
    """sim_group_params_t."""
    _fields_ = [("m", ctypes.c_float), ("Jxx", ctypes.c_float), ("Jyy", ctypes.c_float), ("Jzz", ctypes.c_float),
                ("L", ctypes.c_float), ("alpha", ctypes.c_float), ("kt", ctypes.c_float), ("kq", ctypes.c_float),
                ("tau_m", ctypes.c_float), ("c_d", ctypes.c_float), ("omega_max", ctypes.c_float),
                ("g", ctypes.c_float), ("kp", ctypes.c_float * 3), ("kd", ctypes.c_float * 3),
                ("katt", ctypes.c_float * 3), ("krate", ctypes.c_float * 3), ("a_max", ctypes.c_float),
                ("kI", ctypes.c_float * 3), ("kD", ctypes.c_float * 3), ("xi_max", ctypes.c_float * 3),
                ("type", ctypes.c_int32), ("veh", ctypes.c_float * 8)]


#: PID rate-loop fields and the values a group without them gets (P loop, no integrator limit).
PID_DEFAULTS = {"kI": [0.0] * 3, "kD": [0.0] * 3, "xi_max": [float("inf")] * 3}


def group_struct(g: dict) -> GroupParams:
    s = GroupParams()
    for k in ("m", "Jxx", "Jyy", "Jzz", "L", "alpha", "kt", "kq", "tau_m", "c_d", "omega_max", "g", "a_max"):
        setattr(s, k, float(g[k]))
    for k in ("kp", "kd", "katt", "krate"):
        getattr(s, k)[:] = [float(v) for v in g[k]]
    for k, d in PID_DEFAULTS.items():
        getattr(s, k)[:] = [float(v) for v in g.get(k, d)]
    s.type = int(g.get("type", SIM_TYPE_QUADROTOR))
    s.veh[:] = [float(v) for v in (list(g.get("veh", [])) + [0.0] * 8)[:8]]
    return s


class SimError(RuntimeError):
    pass


_lib = None


def lib():
    """The loaded library; raises if it was not built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise SimError(f"{LIB_PATH} is missing: build it with paper_2308_12698_b300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, I, I64, F, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t
    sig = {
        "sim_create": (I, [ctypes.POINTER(GroupParams), I, I64, P, I, ctypes.POINTER(P)]),
        "sim_set_params": (I, [P, ctypes.POINTER(GroupParams), I]),
        "sim_step": (I, [P, P, P, F, I64, I, P]),
        "sim_step_host": (I, [P, P, P, P, P, F, I64, I, P]),
        "sim_rollout_forward": (I, [P, P, P, F, I64, I, P, P, P]),
        "sim_workspace_bytes": (SZ, [P, I]),
        "sim_rollout_backward": (I, [P, P, P, F, I64, I, P, P, P, P, P, P, SZ, P]),
        "sim_rollout_backward_noalloc": (I, [P, P, P, F, I64, I, P, P, P, P, P, P]),
        "sim_collide_workspace_bytes": (SZ, [P]),
        "sim_collide": (I, [P, P, F, P, SZ, P]),
        "sim_copy_status": (I, [P, P, P]),
        "sim_load_status": (I, [P, P, P]),
        "sim_run_rounds": (I, [P, P, P, P, P, P, F, I64, I64, I, P]),
        "sim_set_launch": (I, [P, I, I, I, I]),
        "sim_get_launch": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
        "sim_status": (I, [P, ctypes.POINTER(I64), I, P]),
        "sim_reset_status": (I, [P, P]),
        "sim_compact": (I, [P, P]),
        "sim_group_stats": (I, [P, P, P, P]),
        "sim_bounds_checks": (I, [ctypes.POINTER(ctypes.c_uint64)]),
        "sim_graph_create": (I, [P, P, P, F, I64, I, P, ctypes.POINTER(P)]),
        "sim_graph_launch": (I, [P, P]),
        "sim_graph_destroy": (None, [P]),
        "sim_step_launches": (I64, [P, I64, I]),
        "sim_destroy": (None, [P]),
        "sim_error_string": (ctypes.c_char_p, [I]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(rc: int, what: str):
    if rc != SIM_OK:
        raise SimError(f"{what}: {lib().sim_error_string(rc).decode()} ({rc})")
