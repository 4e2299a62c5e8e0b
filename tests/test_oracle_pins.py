"""Pins of the FP64 checker against facts fixed outside it (CPU only).

Each test ties one part of the checker's model to something it does not
compute itself: a closed-form solution, an invariant of the equations, a
library routine, the sign pattern printed in Eq. 3, or an independently
derived linearisation.  Plausible slips (a dropped term, a flipped sign, a
swapped operand or index) each fail at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2308_12698_b300 import workload as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _group(**kw):
    g = W.base_group()
    g.update(kw)
    return g


def _state(p=(0, 0, 0), v=(0, 0, 0), q=(1, 0, 0, 0), w=(0, 0, 0), Om=(0, 0, 0, 0)):
    return np.array([*p, *v, *q, *w, *Om], dtype=np.float64)


def _run(orc, group, x, cmd, h, n, mode=0):
    return orc.rollout([group], [0], np.asarray(x, float)[None], np.asarray(cmd, float)[None], h, n, mode)[0]


def _quat_mul(a, b):
    # Hamilton product written from the definition (i^2 = j^2 = k^2 = ijk = -1)
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _rot(q):
    """scipy rotation of a scalar-first quaternion."""
    q = np.asarray(q, float)
    return Rotation.from_quat([q[1], q[2], q[3], q[0]])


def _tilted_q(seed=0):
    r = Rotation.from_rotvec(np.random.default_rng(seed).normal(0, 0.6, 3))
    x, y, z, w = r.as_quat()
    return np.array([w, x, y, z])


# ----------------------------------------------------------- Eq. 3 / Eq. 2 --

def _printed_G(g):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "allocation_signs_eq3.txt")) if l.strip() and l[0] != "#"]
    mag = {"one": 1.0, "L_sin_alpha": g["L"] * math.sin(g["alpha"]), "L_cos_alpha": g["L"] * math.cos(g["alpha"]),
           "kq_over_kt": g["kq"] / g["kt"]}
    return np.array([[mag[r[1]] * float(s) for s in r[2:6]] for r in rows])


def test_allocation_matrix_is_the_printed_one(orc):
    g = W.base_group()
    G, Ginv, taumax = orc.allocation(g)
    np.testing.assert_allclose(G, _printed_G(g), rtol=0, atol=1e-15)
    np.testing.assert_allclose(G @ Ginv, np.eye(4), rtol=0, atol=1e-13)
    om2 = g["omega_max"] ** 2
    np.testing.assert_allclose(taumax, [2 * g["L"] * math.sin(g["alpha"]) * g["kt"] * om2,
                                        2 * g["L"] * math.cos(g["alpha"]) * g["kt"] * om2,
                                        2 * g["kq"] * om2], rtol=1e-14)


def test_torques_match_rotor_geometry(orc):
    """Roll/pitch rows of G equal r_i x (0, 0, f_i) for an X frame (FLU body):
    rotor 1 front-left, 2 front-right, 3 rear-right, 4 rear-left."""
    g = _group(alpha=0.61)  # not pi/4, so sin and cos rows differ
    Lc, Ls = g["L"] * math.cos(g["alpha"]), g["L"] * math.sin(g["alpha"])
    r = np.array([[Lc, Ls, 0], [Lc, -Ls, 0], [-Lc, -Ls, 0], [-Lc, Ls, 0]])
    Om = np.array([610.0, 580.0, 655.0, 540.0])
    f = g["kt"] * Om ** 2
    tau = sum(np.cross(r[i], [0, 0, f[i]]) for i in range(4))
    tau[2] = g["kq"] * (Om[0] ** 2 - Om[1] ** 2 + Om[2] ** 2 - Om[3] ** 2)
    dx = orc.derivative(g, _state(Om=Om), Om)  # omega = 0: omega' = tau / J
    J = np.array([g["Jxx"], g["Jyy"], g["Jzz"]])
    np.testing.assert_allclose(dx[10:13] * J, tau, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(dx[5], f.sum() / g["m"] - g["g"], rtol=1e-13)


def test_yaw_sign():
    """Rotors 1 and 3 faster than 2 and 4 give positive yaw acceleration (Eq. 3, row 4)."""
    import oracle
    g = W.base_group()
    Om = np.array([650.0, 560.0, 650.0, 560.0])
    dx = oracle.derivative(g, _state(Om=Om), Om)
    assert dx[12] > 0 and abs(dx[10]) < 1e-12 and abs(dx[11]) < 1e-12


# ---------------------------------------------------------- closed forms --

def test_free_fall(orc):
    """Rotors off, no drag: p = p0 + v0 t - g t^2/2 e3 (RK4 is exact on polynomials)."""
    g = _group(c_d=0.0)
    q = _tilted_q(1)
    x0 = _state(p=(1.0, -2.0, 30.0), v=(0.3, -0.7, 2.0), q=q)
    h, n = 1e-3, 1000
    x = _run(orc, g, x0, [0, 0, 0, 0], h, n)
    t = h * n
    p = x0[0:3] + x0[3:6] * t - 0.5 * g["g"] * t * t * np.array([0, 0, 1])
    v = x0[3:6] - g["g"] * t * np.array([0, 0, 1])
    np.testing.assert_allclose(x[0:3], p, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(x[3:6], v, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(x[6:10], q, rtol=0, atol=1e-15)


def test_linear_drag_closed_form(orc):
    """Rotors off: v(t) = v_inf + (v0 - v_inf) exp(-c t / m), v_inf = -(m g / c) e3."""
    g = _group(c_d=0.3)
    x0 = _state(p=(0.0, 0.0, 10.0), v=(4.0, -3.0, 1.0))
    h, n = 1e-3, 2000
    x = _run(orc, g, x0, [0, 0, 0, 0], h, n)
    t, k = h * n, g["c_d"] / g["m"]
    vinf = np.array([0, 0, -g["g"] / k])
    v = vinf + (x0[3:6] - vinf) * math.exp(-k * t)
    p = x0[0:3] + vinf * t + (x0[3:6] - vinf) * (1 - math.exp(-k * t)) / k
    np.testing.assert_allclose(x[3:6], v, rtol=0, atol=1e-11)
    np.testing.assert_allclose(x[0:3], p, rtol=0, atol=1e-11)


def test_thrust_along_body_z(orc):
    """Equal rotors at their command, no rates: constant acceleration R(q) e3 f_c / m - g e3."""
    g = _group(c_d=0.0)
    q = _tilted_q(2)
    Om = np.full(4, 700.0)
    x0 = _state(v=(0.5, 0.1, -0.2), q=q, Om=Om)
    h, n = 1e-3, 500
    x = _run(orc, g, x0, Om, h, n)
    t = h * n
    a = _rot(q).apply([0, 0, 1]) * 4 * g["kt"] * 700.0 ** 2 / g["m"] - np.array([0, 0, g["g"]])
    np.testing.assert_allclose(x[3:6], x0[3:6] + a * t, rtol=0, atol=1e-11)
    np.testing.assert_allclose(x[0:3], x0[0:3] + x0[3:6] * t + 0.5 * a * t * t, rtol=0, atol=1e-11)


def test_rotor_lag_is_rk4_of_a_linear_ode(orc):
    """Omega' = (u - Omega)/tau: RK4 multiplies the offset by R(z) = 1+z+z^2/2+z^3/6+z^4/24, z=-h/tau."""
    g = W.base_group()
    u = np.array([640.0, 580.0, 700.0, 500.0])
    x0 = _state(Om=(606.5, 606.5, 606.5, 606.5))
    h, tau = 1e-3, g["tau_m"]
    z = -h / tau
    Rz = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    for n in (1, 7, 30, 200):
        x = _run(orc, g, x0, u, h, n)
        off = x0[13:17] - u
        np.testing.assert_allclose(x[13:17], u + off * Rz ** n, rtol=1e-13)
        # and the exact exponential within the RK4 local error bound
        assert np.all(np.abs(x[13:17] - (u + off * math.exp(z * n))) <= n * abs(z) ** 5 / 120 * np.abs(off) + 1e-12)


def test_torque_free_principal_spin(orc):
    """omega = (0, 0, w0), rotors off: omega constant, q(t) = q0 (x) (cos(w0 t/2), 0, 0, sin(w0 t/2))."""
    g = W.base_group()
    q0 = _tilted_q(3)
    w0 = 2.5
    x0 = _state(q=q0, w=(0, 0, w0))
    h, n = 1e-3, 1500
    x = _run(orc, g, x0, [0, 0, 0, 0], h, n)
    t = h * n
    q = _quat_mul(q0, [math.cos(w0 * t / 2), 0, 0, math.sin(w0 * t / 2)])
    np.testing.assert_array_equal(x[10:13], [0, 0, w0])
    np.testing.assert_allclose(x[6:10], q, rtol=0, atol=1e-12)


def test_torque_free_invariants(orc):
    """Rotors off, asymmetric body: kinetic energy and inertial angular momentum R(q) J omega are conserved."""
    g = _group(Jxx=0.03, Jyy=0.05, Jzz=0.09)
    J = np.array([0.03, 0.05, 0.09])
    x0 = _state(q=_tilted_q(4), w=(0.9, -1.3, 0.6))
    x = _run(orc, g, x0, [0, 0, 0, 0], 1e-3, 3000)
    w0, w1 = x0[10:13], x[10:13]
    E0, E1 = 0.5 * w0 @ (J * w0), 0.5 * w1 @ (J * w1)
    H0 = _rot(x0[6:10]).apply(J * w0)
    H1 = _rot(x[6:10] / np.linalg.norm(x[6:10])).apply(J * w1)
    assert abs(E1 - E0) <= 1e-11 * E0
    np.testing.assert_allclose(H1, H0, rtol=0, atol=1e-11 * np.linalg.norm(H0))
    # the motion is not trivial: omega changed in the body frame
    assert np.linalg.norm(w1 - w0) > 0.1


def test_rk4_fourth_order(orc):
    """Open loop, error against a fine solution shrinks 16x per halving of h."""
    g = _group(tau_m=0.1)
    x0 = _state(p=(1, 2, 3), v=(0.5, -0.3, 0.2), q=_tilted_q(5), w=(0.8, -0.5, 0.3),
                Om=(560, 640, 610, 590))
    u = np.array([630.0, 575.0, 640.0, 600.0])
    T = 1.0
    ref = _run(orc, g, x0, u, T / 3200, 3200)
    errs = []
    for h in (0.02, 0.01, 0.005):
        x = _run(orc, g, x0, u, h, int(round(T / h)))
        errs.append(np.max(np.abs(x - ref) / np.maximum(np.abs(ref), 1.0)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 14 <= r1 <= 18 and 14 <= r2 <= 18, (errs, r1, r2)


def test_unit_quaternion_preserved_without_renormalisation(orc):
    g = W.base_group()
    wh = W.hover_speed(g)
    x0 = _state(q=_tilted_q(6), w=(0.4, -0.2, 0.9), Om=(wh, wh, wh, wh))
    x = _run(orc, g, x0, [wh * 1.01, wh * 0.99, wh * 1.01, wh * 0.99], 1e-3, 10000)
    assert abs(np.linalg.norm(x[6:10]) - 1.0) <= 1e-9


def test_hover_equilibrium_open_loop(orc):
    g = W.base_group()
    wh = W.hover_speed(g)
    x0 = _state(p=(3, -4, 5), q=(math.cos(0.3), 0, 0, math.sin(0.3)), Om=(wh,) * 4)
    x = _run(orc, g, x0, [wh] * 4, 1e-3, 1000)
    np.testing.assert_allclose(x, x0, rtol=0, atol=1e-12)


# ------------------------------------------------------------- controller --

def _level(psi):
    return (math.cos(psi / 2), 0, 0, math.sin(psi / 2))


@pytest.mark.parametrize("psi", [0.0, 0.7, -2.9, 3.1])
def test_controller_fixed_point_at_waypoint(orc, psi):
    """Level at the waypoint with the commanded heading, rotors at hover: nothing moves."""
    g = W.base_group()
    wh = W.hover_speed(g)
    x0 = _state(p=(3, -4, 5), q=_level(psi), Om=(wh,) * 4)
    cmd = [3, -4, 5, psi]
    np.testing.assert_allclose(orc.controller(g, x0, cmd), [wh] * 4, rtol=1e-12)
    x = _run(orc, g, x0, cmd, 1e-3, 1000, mode=1)
    np.testing.assert_allclose(x, x0, rtol=0, atol=1e-9)


@pytest.mark.parametrize("dz,az", [(1.0, 4.0), (0.5, 3.0), (-2.0, -4.0)])
def test_controller_vertical(orc, dz, az):
    """Waypoint straight above/below: a_z = clamp(kp dz, +-a_max), all rotors sqrt(m (g + a_z) / (4 kt))."""
    g = W.base_group()
    x0 = _state(q=_level(0.0))
    w = orc.controller(g, x0, [0, 0, dz, 0])
    np.testing.assert_allclose(w, [math.sqrt(g["m"] * (g["g"] + az) / (4 * g["kt"]))] * 4, rtol=1e-12)


def test_controller_roll_error(orc):
    """Rolled by th at the waypoint, heading 0: R_des = I, q_e = (cos th/2, -sin th/2, 0, 0),
    tau_x = krate taumax_x (-2 katt sin(th/2)), f_c = m g cos th; solved by the orthogonal rows of G."""
    g = W.base_group()
    th = 0.2
    x0 = _state(q=(math.cos(th / 2), math.sin(th / 2), 0, 0))
    w = orc.controller(g, x0, [0, 0, 0, 0])
    Ls = g["L"] * math.sin(g["alpha"])
    taumax = 2 * Ls * g["kt"] * g["omega_max"] ** 2
    tx = g["krate"][0] * taumax * (-2 * g["katt"][0] * math.sin(th / 2))
    fc = g["m"] * g["g"] * math.cos(th)
    f = fc / 4 + np.array([1, -1, -1, 1]) * tx / (4 * Ls)
    np.testing.assert_allclose(w, np.sqrt(f / g["kt"]), rtol=1e-12)


@pytest.mark.parametrize("psi", [0.0, 0.9, -2.5])
def test_controller_roll_error_under_heading(orc, psi):
    """Yawed to the commanded heading psi, then rolled by th about the body x axis: the error is a
    pure body-x roll whatever psi is (q_e = q^* o q_d is the body-frame error), so the rotor
    commands equal the unyawed roll case."""
    g = W.base_group()
    th = 0.2
    qy = np.array([math.cos(psi / 2), 0, 0, math.sin(psi / 2)])
    qr = np.array([math.cos(th / 2), math.sin(th / 2), 0, 0])
    x0 = _state(q=_quat_mul(qy, qr))
    w = orc.controller(g, x0, [0, 0, 0, psi])
    Ls = g["L"] * math.sin(g["alpha"])
    taumax = 2 * Ls * g["kt"] * g["omega_max"] ** 2
    tx = g["krate"][0] * taumax * (-2 * g["katt"][0] * math.sin(th / 2))
    fc = g["m"] * g["g"] * math.cos(th)
    f = fc / 4 + np.array([1, -1, -1, 1]) * tx / (4 * Ls)
    np.testing.assert_allclose(w, np.sqrt(f / g["kt"]), rtol=1e-10)


def test_controller_yaw_error(orc):
    """Level, yawed by phi, heading 0: q_e = (cos phi/2, 0, 0, -sin phi/2)."""
    g = W.base_group()
    phi = 0.3
    x0 = _state(q=_level(phi))
    w = orc.controller(g, x0, [0, 0, 0, 0])
    c = g["kq"] / g["kt"]
    tz = g["krate"][2] * 2 * g["kq"] * g["omega_max"] ** 2 * (-2 * g["katt"][2] * math.sin(phi / 2))
    f = g["m"] * g["g"] / 4 + np.array([1, -1, 1, -1]) * tz / (4 * c)
    np.testing.assert_allclose(w, np.sqrt(f / g["kt"]), rtol=1e-12)


def test_controller_rotor_clamp(orc):
    """Huge yaw error drives two rotors to the floor (0) and two to the ceiling (omega_max)."""
    g = _group(katt=[8.0, 8.0, 400.0])
    x0 = _state(q=_level(1.5))
    w = orc.controller(g, x0, [0, 0, 0, 0])
    np.testing.assert_allclose(w, [0.0, g["omega_max"], 0.0, g["omega_max"]], rtol=1e-15)


def test_shepperd_matches_library():
    import oracle
    rng = np.random.default_rng(7)
    rots = [Rotation.from_rotvec(v) for v in rng.normal(0, 1.5, (200, 3))]
    for ax in np.eye(3):
        for ang in (math.pi, 0.999 * math.pi, 2.5, -3.0):
            rots.append(Rotation.from_rotvec(ax * ang))
    branches = set()
    for r in rots:
        R = r.as_matrix()
        q = oracle.shepperd(R)
        x, y, z, w = r.as_quat()
        ref = np.array([w, x, y, z])
        s = 1.0 if q @ ref >= 0 else -1.0
        np.testing.assert_allclose(q, s * ref, rtol=0, atol=1e-12)
        tr = np.trace(R)
        branches.add("w" if tr > 0 else "xyz"[int(np.argmax(np.diag(R)))])
    assert branches == {"w", "x", "y", "z"}


def _spectrum(orc, g, h=1e-4):
    wh = W.hover_speed(g)
    x0 = _state(Om=(wh,) * 4)
    J = np.zeros((17, 17))
    e = 1e-6
    for j in range(17):
        d = np.zeros(17)
        d[j] = e
        J[:, j] = (_run(orc, g, x0 + d, [0, 0, 0, 0], h, 1, 1) - _run(orc, g, x0 - d, [0, 0, 0, 0], h, 1, 1)) / (2 * e)
    return np.log(np.linalg.eigvals(J).astype(complex)) / h


def _linear_spectrum(g, K):
    """Small-angle hover linearisation built by hand, chain by chain.

    roll/pitch: (pos, vel, angle, rate, lagged torque) with
      vel' = +-g angle - (c_d/m) vel, angle_des = -+(kp pos + kd vel)/g,
      tau_cmd = K (katt (angle_des - angle) - rate), tau' = (tau_cmd - tau)/tau_m;
    height: (z, vz, thrust deviation) with thrust' = (m(-kp z - kd vz) - thrust)/tau_m;
    yaw: (psi, rate, lagged torque); plus the neutral quaternion-norm mode.
    """
    m, cd, gr, tm = g["m"], g["c_d"], g["g"], g["tau_m"]
    kp, kd, ka = g["kp"][0], g["kd"][0], g["katt"][0]

    def chain(K, J, sgn):
        A = np.zeros((5, 5))
        A[0, 1] = 1
        A[1, 1] = -cd / m
        A[1, 2] = sgn * gr
        A[2, 3] = 1
        A[3, 4] = 1 / J
        A[4, 0] = -K * ka * sgn * kp / gr / tm
        A[4, 1] = -K * ka * sgn * kd / gr / tm
        A[4, 2] = -K * ka / tm
        A[4, 3] = -K / tm
        A[4, 4] = -1 / tm
        return np.linalg.eigvals(A)

    z = np.linalg.eigvals(np.array([[0, 1, 0], [0, -cd / m, 1 / m], [-m * kp / tm, -m * kd / tm, -1 / tm]]))
    yaw = np.linalg.eigvals(np.array([[0, 1, 0], [0, 0, 1 / g["Jzz"]],
                                      [-K[2] * g["katt"][2] / tm, -K[2] / tm, -1 / tm]]))
    return np.concatenate([chain(K[0], g["Jxx"], -1), chain(K[1], g["Jyy"], 1), z, yaw, [0.0]])


def _match(a, b, tol):
    a = list(a)
    for lam in b:
        i = int(np.argmin([abs(lam - x) for x in a]))
        assert abs(lam - a[i]) <= tol + 2e-3 * abs(lam), (lam, a[i])
        a.pop(i)


@pytest.mark.parametrize("reading", ["normalised", "literal"])
def test_closed_loop_spectrum_at_hover(orc, reading):
    """Eigenvalues of the checker's closed-loop step map at hover equal those of the hand linearisation.

    'literal' uses a rate gain of 0.2 N m s/rad on every axis; that reading is
    unstable (roll and pitch modes with positive real part), which is why the
    rate gain is scaled by the axis torque limit."""
    g = W.base_group()
    _, _, taumax = orc.allocation(g)
    if reading == "literal":
        g["krate"] = [0.2 / t for t in taumax]
    K = np.array(g["krate"]) * taumax
    lam = _spectrum(orc, g)
    _match(lam, _linear_spectrum(g, K), 0.03)
    if reading == "normalised":
        assert lam.real.max() < 1e-6 and sorted(lam.real)[-2] < -0.3
    else:
        assert lam.real.max() > 0.2


# ------------------------------------------------------------ reverse mode --

@pytest.mark.parametrize("w_omega", [1e-6, 1e-3])
def test_reverse_mode_matches_central_differences(orc, w_omega):
    """FP64 reverse mode vs FP64 central differences, step 1e-6 relative to each parameter
    (and 1e-6 max(1, |x|) for states), within 1e-5 relative per component."""
    wl = W.differentiable(n_per_group=2, n_groups=2, nsteps=300, w_omega=w_omega)
    n = wl.n
    x0 = wl.x0.astype(np.float64)
    loss, dx0, dth = orc.grad(wl.groups, wl.gid, x0, wl.cmd, wl.dt, wl.nsteps, wl.mode, wl.goal, w_omega)
    keys = [("kp", 0), ("kp", 1), ("kp", 2), ("kd", 0), ("kd", 1), ("kd", 2), ("katt", 0), ("katt", 1), ("katt", 2),
            ("krate", 0), ("krate", 1), ("krate", 2), ("m", None), ("Jxx", None), ("Jyy", None), ("Jzz", None)]
    h = 1e-6

    def L(a, groups, x):
        return orc.loss(groups, [0], x[None], wl.cmd[a:a + 1], wl.dt, wl.nsteps, wl.mode, wl.goal[a:a + 1],
                        w_omega, nthreads=1)[0]

    checked = 0
    for a in range(n):
        g0 = dict(wl.groups[wl.gid[a]])
        g0 = {k: (list(v) if isinstance(v, list) else v) for k, v in g0.items()}
        assert abs(L(a, [g0], x0[a]) - loss[a]) <= 1e-12 * abs(loss[a])
        fd = []
        for k, i in keys:
            vals = []
            for s in (+1, -1):
                gg = {kk: (list(v) if isinstance(v, list) else v) for kk, v in g0.items()}
                base = gg[k][i] if i is not None else gg[k]
                step = h * abs(base)  # relative: J of the light airframes is ~1e-4
                if i is None:
                    gg[k] = base + s * step
                else:
                    gg[k][i] = base + s * step
                vals.append(L(a, [gg], x0[a]))
            fd.append((vals[0] - vals[1]) / (2 * step))
        for j in range(17):
            step = h * max(1.0, abs(x0[a, j]))
            xp, xm = x0[a].copy(), x0[a].copy()
            xp[j] += step
            xm[j] -= step
            fd.append((L(a, [g0], xp) - L(a, [g0], xm)) / (2 * step))
        fd = np.array(fd)
        ad = np.concatenate([dth[a], dx0[a]])
        scale = np.abs(ad).max()
        err = np.abs(fd - ad)
        assert np.all(err <= 1e-5 * np.maximum(np.abs(ad), 1e-3 * scale)), (a, err / np.maximum(np.abs(ad), 1e-3 * scale))
        checked += 1
    assert checked == n
