"""Pins of the checker's car and fixed-wing models (CPU only).

The paper lists cars and fixed-wing drones among the simulator's robot types and cites their
models without equations (Sec. III-B).  The readings are the kinematic bicycle under pure pursuit
and the coordinated-turn guidance model with first-order autopilot loops.  Each pin ties a piece
of them to a fact outside the checker: an exact solution of the motion (straight line, circle of
radius 1/kappa or V^2/(g tan phi), exponential and second-order responses), a controller output
solved by hand, or a norm the motion preserves.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from paper_2308_12698_b300 import workload as W

CL = W.CLOSED_LOOP


def _car_state(p=(0.0, 0.0), v=0.0, psi=0.0):
    x = np.zeros(17)
    x[0:2] = p
    x[3] = v
    x[6], x[7] = math.cos(psi), math.sin(psi)
    return x


def _fw_state(p=(0.0, 0.0), h=100.0, V=20.0, psi=0.0, phi=0.0, hdot=0.0):
    x = np.zeros(17)
    x[0:3] = (p[0], p[1], h)
    x[3] = V
    x[5] = hdot
    x[6], x[7] = math.cos(psi), math.sin(psi)
    x[10] = phi
    return x


def _run(orc, g, x, cmd, h, n):
    return orc.rollout([g], [0], np.asarray(x, float)[None], np.asarray(cmd, float)[None], h, n, CL)[0]


# ------------------------------------------------------------------ car --

def test_car_straight_line(orc):
    """Waypoint dead ahead, at the target speed: a straight line at constant speed."""
    g = W.car_group()
    x0 = _car_state(p=(1.0, 2.0), v=10.0, psi=0.3)
    far = (1.0 + 1e4 * math.cos(0.3), 2.0 + 1e4 * math.sin(0.3), 0.0, 10.0)
    x = _run(orc, g, x0, far, 1e-3, 2000)
    np.testing.assert_allclose(x[0:2], [1.0 + 20 * math.cos(0.3), 2.0 + 20 * math.sin(0.3)], rtol=0, atol=1e-9)
    np.testing.assert_allclose(x[[3, 6, 7]], x0[[3, 6, 7]], rtol=0, atol=1e-12)


def test_car_speed_response(orc):
    """a = k_v (v_c - v) unclamped, evaluated once per step and held: v_n = v_c + (v0 - v_c)
    (1 - k_v h)^n exactly (RK4 integrates a held constant exactly), which tends to the
    continuous exp(-k_v t) as h -> 0."""
    g = W.car_group()
    kv = g["veh"][3]
    x0 = _car_state(v=8.0)
    x = _run(orc, g, x0, (1e5, 0.0, 0.0, 9.5), 1e-3, 3000)
    np.testing.assert_allclose(x[3], 9.5 + (8.0 - 9.5) * (1 - kv * 1e-3) ** 3000, rtol=0, atol=1e-12)
    assert abs(x[3] - (9.5 - 1.5 * math.exp(-kv * 3.0))) < 2e-4


def test_car_full_lock_circle(orc):
    """Waypoint 3 m to the left: the pursuit curvature 2 sin(alpha) / l_min exceeds the steering
    limit all the way round, so kappa = tan(delta_max)/L_w and at constant speed the car runs on
    a circle of radius 1/kappa, turning by v kappa t."""
    g = W.car_group()
    Lw, tmax = g["veh"][0], g["veh"][1]
    kappa = tmax / Lw
    v = 6.0
    x0 = _car_state(v=v)
    cmd = (0.0, 3.0, 0.0, v)
    n = 3000
    x = _run(orc, g, x0, cmd, 1e-3, n)
    ang = v * kappa * n * 1e-3  # about 4.7 rad: most of a lap
    np.testing.assert_allclose(x[0:2], [math.sin(ang) / kappa, (1 - math.cos(ang)) / kappa], rtol=0, atol=1e-10)
    np.testing.assert_allclose(x[6:8], [math.cos(ang), math.sin(ang)], rtol=0, atol=1e-12)
    assert orc.vehicle_controller(g, x, cmd)[0] == pytest.approx(kappa, rel=1e-15)  # still saturated


@pytest.mark.parametrize("bearing,dist", [(0.3, 40.0), (-0.7, 12.0), (1.2, 3.0), (0.2, 3.0), (2.8, 60.0),
                                          (-3.0, 25.0)])
def test_car_pure_pursuit_by_hand(orc, bearing, dist):
    """Target at bearing alpha (ahead or behind) and distance d: kappa = 2 sin(alpha) /
    max(d, l_min), clamped to tan(delta_max)/L_w; a = clamp(k_v (v_c - v), +-a_max)."""
    g = W.car_group()
    Lw, tmax, amax, kv, lmin = g["veh"][:5]
    psi = 0.4
    x0 = _car_state(p=(3.0, -1.0), v=7.0, psi=psi)
    cmd = (3.0 + dist * math.cos(psi + bearing), -1.0 + dist * math.sin(psi + bearing), 0.0, 12.0)
    u = orc.vehicle_controller(g, x0, cmd)
    k = float(np.clip(2 * math.sin(bearing) / max(dist, lmin), -tmax / Lw, tmax / Lw))
    np.testing.assert_allclose(u[:2], [k, float(np.clip(kv * 5.0, -amax, amax))], rtol=1e-12, atol=1e-15)


def test_car_derivative_by_hand(orc):
    g = W.car_group()
    x = _car_state(p=(1, 2), v=4.0, psi=0.9)
    dx = orc.vehicle_derivative(g, x, [0.1, 0.5, 0.0])
    ref = np.zeros(17)
    ref[0:2] = 4.0 * math.cos(0.9), 4.0 * math.sin(0.9)
    ref[3] = 0.5
    ref[6:8] = -math.sin(0.9) * 0.4, math.cos(0.9) * 0.4
    np.testing.assert_allclose(dx, ref, rtol=1e-14, atol=1e-15)


# ------------------------------------------------------------ fixed-wing --

def test_fixed_wing_straight_level(orc):
    """Waypoint dead ahead at the commanded altitude and airspeed, wings level: a straight line."""
    g = W.fixed_wing_group()
    x0 = _fw_state(p=(10.0, -5.0), h=80.0, V=20.0, psi=-1.1)
    cmd = (10.0 + 1e5 * math.cos(-1.1), -5.0 + 1e5 * math.sin(-1.1), 80.0, 20.0)
    x = _run(orc, g, x0, cmd, 1e-3, 3000)
    np.testing.assert_allclose(x[0:2], [10.0 + 60 * math.cos(-1.1), -5.0 + 60 * math.sin(-1.1)], rtol=0,
                               atol=1e-9)
    np.testing.assert_allclose(x[[2, 3, 5, 10]], [80.0, 20.0, 0.0, 0.0], rtol=0, atol=1e-10)


def test_fixed_wing_airspeed_and_altitude_responses(orc):
    """V' = b_V (V_c - V): exponential; (h, h') follow the linear second-order loop
    h'' = -b_hd h' + b_h (h_c - h): the matrix exponential."""
    g = W.fixed_wing_group()
    bhd, bh, bV = g["veh"][3], g["veh"][4], g["veh"][5]
    x0 = _fw_state(h=100.0, V=18.0, hdot=1.5)
    x = _run(orc, g, x0, (1e6, 0.0, 130.0, 24.0), 1e-3, 4000)
    np.testing.assert_allclose(x[3], 24.0 + (18.0 - 24.0) * math.exp(-bV * 4.0), rtol=0, atol=1e-11)
    A = np.array([[0.0, 1.0], [-bh, -bhd]])
    e = expm(A * 4.0) @ np.array([100.0 - 130.0, 1.5])
    np.testing.assert_allclose([x[2] - 130.0, x[5]], e, rtol=0, atol=1e-10)


def test_fixed_wing_steady_turn(orc):
    """Banked at the limit with the waypoint behind (the command stays saturated): a
    coordinated turn at rate g tan(phi)/V on a circle of radius V^2 / (g tan(phi))."""
    g = W.fixed_wing_group()
    phi = g["veh"][1]
    V = 20.0
    x0 = _fw_state(V=V, phi=phi)
    rate = g["g"] * math.tan(phi) / V
    n = int(round(0.7 / rate / 1e-3))  # 0.7 rad of turn: the waypoint stays far behind
    x = _run(orc, g, x0, (-1e6, 1e3, 100.0, V), 1e-3, n)
    ang = rate * n * 1e-3
    R = V * V / (g["g"] * math.tan(phi))
    np.testing.assert_allclose(x[0:2], [R * math.sin(ang), R * (1 - math.cos(ang))], rtol=0, atol=1e-9)
    np.testing.assert_allclose(x[10], phi, rtol=0, atol=1e-15)


@pytest.mark.parametrize("bearing", [0.2, -0.35, 2.5, -3.0])
def test_fixed_wing_bank_command_by_hand(orc, bearing):
    """Course error = the waypoint's bearing off the nose (atan2, any quadrant): phi_c =
    clamp(k_chi bearing, +-phi_max); the altitude and airspeed commands pass through."""
    g = W.fixed_wing_group()
    bphi, phimax, kchi = g["veh"][:3]
    psi = 2.0
    x0 = _fw_state(p=(5.0, 7.0), psi=psi, phi=0.1)
    cmd = (5.0 + 300 * math.cos(psi + bearing), 7.0 + 300 * math.sin(psi + bearing), 90.0, 22.0)
    u = orc.vehicle_controller(g, x0, cmd)
    np.testing.assert_allclose(u, [float(np.clip(kchi * bearing, -phimax, phimax)), 90.0, 22.0], rtol=1e-12)
    dx = orc.vehicle_derivative(g, x0, u)
    np.testing.assert_allclose(dx[10], bphi * (u[0] - 0.1), rtol=1e-14)
    turn = g["g"] * math.tan(0.1) / 20.0
    np.testing.assert_allclose(dx[6:8], [-math.sin(psi) * turn, math.cos(psi) * turn], rtol=1e-13)


# ---------------------------------------------------------------- mixed --

def test_mixed_swarm_each_type_runs_its_own_model(orc):
    """One rollout over quadrotor, car and fixed-wing groups equals each group run alone, and
    the heading vectors of cars and drones keep unit length: no renormalisation, and RK4's
    local error on a rotation whose rate varies within the step (speed, bank) leaves a drift
    under 1e-7 over 20 s."""
    wl = W.multi_type(sizes=(20, 20, 20), shuffle=True)
    both = orc.rollout(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, 5000, wl.mode)
    for gi in range(3):
        sel = wl.gid == gi
        alone = orc.rollout([wl.groups[gi]], np.zeros(sel.sum(), np.int32), wl.x0[sel], wl.cmd[sel], wl.dt, 5000,
                            wl.mode)
        np.testing.assert_array_equal(both[sel], alone)
    xT = orc.rollout(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, 20000, wl.mode)
    veh = wl.gid > 0
    assert np.abs(np.hypot(xT[veh, 6], xT[veh, 7]) - 1).max() < 1e-7


def test_vehicle_types_only_in_the_closed_loop(orc):
    g = W.car_group()
    with pytest.raises(ValueError):
        orc.rollout([g], [0], np.zeros((1, 17)), np.zeros((1, 4)), 1e-3, 1, W.OPEN_LOOP)
    with pytest.raises(ValueError):
        orc.grad([g], [0], np.zeros((1, 17)), np.zeros((1, 4)), 1e-3, 1, CL, np.zeros((1, 3)), 0.0)


def test_vehicle_margins(orc):
    """The course-error jump margin over one step start: 0 for a drone whose waypoint is
    straight behind, pi - |bearing| otherwise, and inf for cars and quadrotors; over more steps
    the minimum along the trajectory."""
    gq, gc, gf = W.base_group(), W.car_group(), W.fixed_wing_group()
    x = np.stack([_fw_state(), _fw_state(), _car_state(v=5.0), np.zeros(17)])
    x[3, 6] = 1.0
    cmd = np.array([[-500.0, 0.0, 100.0, 20.0], [100.0, 300.0, 100.0, 20.0], [-50.0, 1e-9, 0.0, 5.0],
                    [1.0, 1.0, 1.0, 0.0]])
    m = orc.vehicle_margins([gq, gc, gf], [2, 2, 1, 0], x, cmd, 1e-3, 1)
    assert m[0] == 0.0
    np.testing.assert_allclose(m[1], math.pi - math.atan2(300.0, 100.0), rtol=1e-12)
    assert m[2] > 1e299 and m[3] > 1e299
    m50 = orc.vehicle_margins([gq, gc, gf], [2, 2, 1, 0], x, cmd, 1e-3, 50)
    assert m50[0] == 0.0 and m50[1] <= m[1]
