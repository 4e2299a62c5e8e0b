"""FP64 CPU checker for the batched quadrotor step -- TEST INFRASTRUCTURE ONLY.

This package is the slow, obviously-correct definition the CUDA library is
tested against.  Only ``tests/``, the smoke check and the bench's CPU-baseline
leg import it; the product path never does.  It shares no code with the CUDA
library: the model lives in ``quad_model.hpp`` (C++, FP64, agent by agent,
written from the equations of Sec. III-B of arXiv 2308.12698), compiled into
``liboracle.so`` and reached through ctypes.

Parity status: the rigid-body equations, rotor model, allocation and RK4
are pinned by closed forms and invariants in ``tests/test_oracle_pins.py``.
The cascaded controller is the build's own reading (the paper defers it to a
reference it does not include); it is pinned by hand-solved special cases and
by the closed-loop spectrum at hover, not by any printed value, so its parity
against the paper itself is unpinned.

``rollout_f32`` evaluates the same model on float (every operation rounded to
single precision).  It is not a reference for values: its distance from the
FP64 rollout sizes the tolerance of the FP32 CUDA path over long rollouts, and
``tests/test_oracle_fp32.py`` pins it to the FP64 model.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
#: ORACLE_LIB points the wrapper at another build of the same source (the
#: mutation test loads deliberately broken copies this way).
LIB_PATH = os.environ.get("ORACLE_LIB") or os.path.join(_HERE, "liboracle.so")
_SOURCES = ("oracle.cpp", "quad_model.hpp", "scalar_types.hpp", "vehicles.hpp")

NX = 17
NXP = 20  # PID mode: the 17 states and the rate-error integral xi
NPARAM = 43
NTHETA = 16
OPEN_LOOP = 0
CLOSED_LOOP = 1
CLOSED_LOOP_PID = 2
TYPE_QUAD, TYPE_CAR, TYPE_FIXED_WING = 0, 1, 2


def state_dim(mode: int) -> int:
    return NXP if mode == CLOSED_LOOP_PID else NX


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (-O2, FP64, no fast-math)."""
    src_m = max(os.path.getmtime(os.path.join(_HERE, s)) for s in _SOURCES)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= src_m:
        return LIB_PATH
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-pthread",
           os.path.join(_HERE, "oracle.cpp"), "-o", LIB_PATH + ".tmp"]
    subprocess.run(cmd, check=True)
    os.replace(LIB_PATH + ".tmp", LIB_PATH)
    return LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.environ.get("ORACLE_LIB"):
            build()
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        L.oracle_rollout.argtypes = [P, ctypes.c_int, P, ctypes.c_int64, P, P, ctypes.c_double,
                                     ctypes.c_int64, ctypes.c_int, ctypes.c_int, P]
        L.oracle_rollout_f32.argtypes = [P, ctypes.c_int, P, ctypes.c_int64, P, P, ctypes.c_double,
                                         ctypes.c_int64, ctypes.c_int, ctypes.c_int]
        L.oracle_grad.argtypes = [P, ctypes.c_int, P, ctypes.c_int64, P, P, ctypes.c_double,
                                  ctypes.c_int64, ctypes.c_int, P, ctypes.c_double, ctypes.c_int, P, P, P]
        L.oracle_derivative.argtypes = [P, P, P, P]
        L.oracle_controller.argtypes = [P, P, P, P]
        L.oracle_controller_pid.argtypes = [P, P, P, P, P, P]
        L.oracle_vehicle_controller.argtypes = [P, P, P, P]
        L.oracle_vehicle_derivative.argtypes = [P, P, P, P]
        L.oracle_vehicle_margins.argtypes = [P, ctypes.c_int, P, ctypes.c_int64, P, P, ctypes.c_double,
                                             ctypes.c_int64, ctypes.c_int, P]
        L.oracle_allocation.argtypes = [P, P, P, P]
        L.oracle_shepperd.argtypes = [P, P]
        L.oracle_count_ops.argtypes = [P, P, P, ctypes.c_double, ctypes.c_int, P]
        L.oracle_count_derivative_ops.argtypes = [P, P, P, P]
        L.oracle_count_adjoint_edges.argtypes = [P, P, P, ctypes.c_double, ctypes.c_int, P]
        L.oracle_collisions.argtypes = [P, P, P, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_int, P]
        L.oracle_clamp_margins.argtypes = [P, ctypes.c_int, P, ctypes.c_int64, P, P, ctypes.c_double, ctypes.c_int64,
                                           ctypes.c_int, ctypes.c_int, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def pack_group(g: dict) -> np.ndarray:
    """Packed FP64 parameter group: m Jxx Jyy Jzz L alpha kt kq tau_m c_d omega_max g kp kd katt krate a_max
    kI kD xi_max (the PID rate loop's gains and integrator limit; absent keys: 0, 0, 1e30), type and
    veh[8] (agent type 0 quadrotor, 1 car, 2 fixed-wing and its model's parameters; absent: 0)."""
    v = [g["m"], g["Jxx"], g["Jyy"], g["Jzz"], g["L"], g["alpha"], g["kt"], g["kq"], g["tau_m"], g["c_d"],
         g["omega_max"], g["g"], *g["kp"], *g["kd"], *g["katt"], *g["krate"], g["a_max"],
         *g.get("kI", [0.0] * 3), *g.get("kD", [0.0] * 3), *g.get("xi_max", [1e30] * 3),
         g.get("type", TYPE_QUAD), *(list(g.get("veh", [])) + [0.0] * 8)[:8]]
    a = np.asarray(v, dtype=np.float64)
    assert a.size == NPARAM
    return a


def pack_groups(groups) -> np.ndarray:
    return np.ascontiguousarray(np.concatenate([pack_group(g) for g in groups]))


def _threads(nthreads):
    return nthreads if nthreads else (os.cpu_count() or 1)


def _states(x0, mode):
    x = np.ascontiguousarray(np.asarray(x0, dtype=np.float64))
    if x.ndim != 2 or x.shape[1] != state_dim(mode):
        raise ValueError(f"states must be (n, {state_dim(mode)}) in mode {mode}")
    return x


def rollout(groups, gid, x0, cmd, h, nsteps, mode, nthreads=None, with_cost=False):
    """Advance every agent nsteps RK4 steps; returns the (n, 17) FP64 final state ((n, 20) in
    the PID mode) and, when asked, the per-agent running sum of Omega^2 over step ends."""
    x = _states(x0, mode).copy()
    n = x.shape[0]
    c = np.ascontiguousarray(np.asarray(cmd, dtype=np.float64))
    gi = np.ascontiguousarray(np.asarray(gid, dtype=np.int32))
    pg = pack_groups(groups)
    rc = np.zeros(n, dtype=np.float64)
    rcode = lib().oracle_rollout(_p(pg), len(groups), _p(gi), n, _p(x), _p(c), float(h), int(nsteps), int(mode),
                                 _threads(nthreads), _p(rc))
    if rcode != 0:
        raise ValueError("oracle_rollout rejected its arguments")
    return (x, rc) if with_cost else x


def rollout_f32(groups, gid, x0, cmd, h, nsteps, mode, nthreads=None):
    """The same rollout with the model evaluated in FP32 (every operation rounded to single
    precision, the state kept as float32 between steps); quadrotor groups only.  Returns the
    (n, state_dim) float32 final state.  Its distance from ``rollout`` measures what FP32 rounding
    does to the equations, independently of the CUDA path."""
    x = np.ascontiguousarray(np.asarray(x0, dtype=np.float32)).copy()
    if x.ndim != 2 or x.shape[1] != state_dim(mode):
        raise ValueError(f"states must be (n, {state_dim(mode)}) in mode {mode}")
    c = np.ascontiguousarray(np.asarray(cmd, dtype=np.float64))
    gi = np.ascontiguousarray(np.asarray(gid, dtype=np.int32))
    pg = pack_groups(groups)
    rcode = lib().oracle_rollout_f32(_p(pg), len(groups), _p(gi), x.shape[0], _p(x), _p(c), float(h),
                                     int(nsteps), int(mode), _threads(nthreads))
    if rcode != 0:
        raise ValueError("oracle_rollout_f32 rejected its arguments")
    return x


def grad(groups, gid, x0, cmd, h, nsteps, mode, goal, w_omega, nthreads=None):
    """Per-agent loss, dL/dx0 (n, 17; (n, 20) in the PID mode) and dL/dtheta (n, 16) by FP64
    reverse mode."""
    x = _states(x0, mode)
    n = x.shape[0]
    c = np.ascontiguousarray(np.asarray(cmd, dtype=np.float64))
    gi = np.ascontiguousarray(np.asarray(gid, dtype=np.int32))
    gl = np.ascontiguousarray(np.asarray(goal, dtype=np.float64))
    pg = pack_groups(groups)
    loss = np.zeros(n)
    dx0 = np.zeros((n, state_dim(mode)))
    dth = np.zeros((n, NTHETA))
    rcode = lib().oracle_grad(_p(pg), len(groups), _p(gi), n, _p(x), _p(c), float(h), int(nsteps), int(mode),
                              _p(gl), float(w_omega), _threads(nthreads), _p(loss), _p(dx0), _p(dth))
    if rcode != 0:
        raise ValueError("oracle_grad rejected its arguments")
    return loss, dx0, dth


def loss(groups, gid, x0, cmd, h, nsteps, mode, goal, w_omega, nthreads=None):
    """Per-agent loss |p_T - goal|^2 + w_omega * sum_{n=1..T} sum_i Omega_{n,i}^2 (FP64)."""
    xT, rc = rollout(groups, gid, x0, cmd, h, nsteps, mode, nthreads, with_cost=True)
    d = xT[:, 0:3] - np.asarray(goal, dtype=np.float64)
    return (d * d).sum(axis=1) + w_omega * rc


def clamp_margins(groups, gid, x0, cmd, h, nsteps, nthreads=None, mode=CLOSED_LOOP):
    """(n, 3) minima over a closed-loop trajectory of: |S|/omega_max^2 (rotor demand near the
    sqrt kink at 0), |S - omega_max^2|/omega_max^2 (rotor ceiling), ||ar| - a_max|/a_max
    (acceleration clamp; in the PID mode also the integrator clamp)."""
    x = _states(x0, mode)
    n = x.shape[0]
    c = np.ascontiguousarray(np.asarray(cmd, dtype=np.float64))
    gi = np.ascontiguousarray(np.asarray(gid, dtype=np.int32))
    pg = pack_groups(groups)
    out = np.zeros((n, 3))
    if lib().oracle_clamp_margins(_p(pg), len(groups), _p(gi), n, _p(x), _p(c), float(h), int(nsteps), int(mode),
                                  _threads(nthreads), _p(out)) != 0:
        raise ValueError("oracle_clamp_margins rejected its arguments")
    return out


def collisions(p, radius, alive, idx=None, nthreads=None):
    """uint8 flags: 1 where a live agent is closer than r_i + r_j to another live agent.

    Decided in FP32 without fused multiply-adds (the precision the kernel decides in):
    d2 = (dx*dx + dy*dy) + dz*dz < (r_i + r_j)^2.  With idx, only those agents are decided."""
    pp = np.ascontiguousarray(np.asarray(p, dtype=np.float32).reshape(-1, 3))
    n = pp.shape[0]
    rr = np.ascontiguousarray(np.asarray(radius, dtype=np.float32).reshape(n))
    al = np.ascontiguousarray(np.asarray(alive, dtype=np.uint8).reshape(n))
    if idx is None:
        out = np.zeros(n, dtype=np.uint8)
        rc = lib().oracle_collisions(_p(pp), _p(rr), _p(al), n, None, -1, _threads(nthreads), _p(out))
    else:
        ii = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
        out = np.zeros(ii.size, dtype=np.uint8)
        rc = lib().oracle_collisions(_p(pp), _p(rr), _p(al), n, _p(ii), ii.size, _threads(nthreads), _p(out))
    if rc != 0:
        raise ValueError("oracle_collisions rejected its arguments")
    return out


def derivative(group, x, w):
    pg = pack_group(group)
    xx = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    ww = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    dx = np.zeros(NX)
    lib().oracle_derivative(_p(pg), _p(xx), _p(ww), _p(dx))
    return dx


def controller(group, x, cmd):
    pg = pack_group(group)
    xx = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    cc = np.ascontiguousarray(np.asarray(cmd, dtype=np.float64))
    w = np.zeros(4)
    lib().oracle_controller(_p(pg), _p(xx), _p(cc), _p(w))
    return w


def controller_pid(group, x, cmd):
    """PID mode, one agent with its 20-state x: (rotor-speed commands (4), rate error (3),
    omega' at x (3))."""
    pg = pack_group(group)
    xx = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(NXP))
    cc = np.ascontiguousarray(np.asarray(cmd, dtype=np.float64))
    w, e, wd = np.zeros(4), np.zeros(3), np.zeros(3)
    lib().oracle_controller_pid(_p(pg), _p(xx), _p(cc), _p(w), _p(e), _p(wd))
    return w, e, wd


def allocation(group):
    pg = pack_group(group)
    G = np.zeros(16)
    Gi = np.zeros(16)
    tm = np.zeros(3)
    lib().oracle_allocation(_p(pg), _p(G), _p(Gi), _p(tm))
    return G.reshape(4, 4), Gi.reshape(4, 4), tm


def shepperd(R):
    RR = np.ascontiguousarray(np.asarray(R, dtype=np.float64).reshape(9))
    q = np.zeros(4)
    lib().oracle_shepperd(_p(RR), _p(q))
    return q


def count_adjoint_edges(group, x, cmd, h, mode):
    """Edges of the one-step reverse-mode tape (each costs a multiply and an add to sweep)."""
    pg = pack_group(group)
    xx = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    cc = np.ascontiguousarray(np.asarray(cmd, dtype=np.float64))
    out = np.zeros(1, dtype=np.int64)
    lib().oracle_count_adjoint_edges(_p(pg), _p(xx), _p(cc), float(h), int(mode), _p(out))
    return int(out[0])


def count_ops(group, x, cmd, h, mode):
    """Non-trivial FP64 operations of one step: dict(add, mul, div, sqrt, trig, cmp)."""
    pg = pack_group(group)
    xx = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    cc = np.ascontiguousarray(np.asarray(cmd, dtype=np.float64))
    out = np.zeros(6, dtype=np.int64)
    lib().oracle_count_ops(_p(pg), _p(xx), _p(cc), float(h), int(mode), _p(out))
    return dict(zip(("add", "mul", "div", "sqrt", "trig", "cmp"), out.tolist()))


def count_derivative_ops(group, x, w):
    """Non-trivial FP64 operations of one time-derivative evaluation: dict(add, mul, div, sqrt, trig, cmp)."""
    pg = pack_group(group)
    xx = np.ascontiguousarray(np.asarray(x, dtype=np.float64)[:NX])
    ww = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    out = np.zeros(6, dtype=np.int64)
    lib().oracle_count_derivative_ops(_p(pg), _p(xx), _p(ww), _p(out))
    return dict(zip(("add", "mul", "div", "sqrt", "trig", "cmp"), out.tolist()))


def vehicle_controller(group, x, cmd):
    """Car or fixed-wing agent: its controller's inputs (3) at the 17-state x."""
    pg = pack_group(group)
    xx = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(NX))
    cc = np.ascontiguousarray(np.asarray(cmd, dtype=np.float64))
    u = np.zeros(3)
    if lib().oracle_vehicle_controller(_p(pg), _p(xx), _p(cc), _p(u)) != 0:
        raise ValueError("not a car or fixed-wing group")
    return u


def vehicle_derivative(group, x, u):
    """Car or fixed-wing agent: time derivative (17) at state x for held inputs u (3)."""
    pg = pack_group(group)
    xx = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(NX))
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(3))
    dx = np.zeros(NX)
    if lib().oracle_vehicle_derivative(_p(pg), _p(xx), _p(uu), _p(dx)) != 0:
        raise ValueError("not a car or fixed-wing group")
    return dx


def vehicle_margins(groups, gid, x0, cmd, h, nsteps, nthreads=None):
    """(n,) minimum over the trajectory of pi - |course error| for fixed-wing agents (the atan2
    jump when the waypoint passes straight behind); inf for cars and quadrotors."""
    x = _states(x0, CLOSED_LOOP)
    n = x.shape[0]
    c = np.ascontiguousarray(np.asarray(cmd, dtype=np.float64))
    gi = np.ascontiguousarray(np.asarray(gid, dtype=np.int32))
    pg = pack_groups(groups)
    out = np.zeros(n)
    if lib().oracle_vehicle_margins(_p(pg), len(groups), _p(gi), n, _p(x), _p(c), float(h), int(nsteps),
                                    _threads(nthreads), _p(out)) != 0:
        raise ValueError("oracle_vehicle_margins rejected its arguments")
    return out
