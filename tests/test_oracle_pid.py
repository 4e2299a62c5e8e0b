"""Pins of the checker's PID body-rate loop (mode CLOSED_LOOP_PID), CPU only.

The paper names a "PID body rate controller" (Sec. III-B) and gives no gains.  The reading:
per axis tau_i = taumax_i (krate_i e_i + kI_i xi_i - kD_i omega'_i), e = omega_des - omega,
xi the integral of e (three extra states) advanced once per step by xi <- clamp(xi + h e,
+-xi_max), omega' taken on the measurement from Eq. (qd4) at the step start.  Each pin ties a
part of that to a fact outside the checker: the P loop it must reduce to, hand-solved controller
outputs, and the hover spectrum of a hand linearisation with the integrator and derivative terms.
"""
import math

import numpy as np
import pytest

from paper_2308_12698_b300 import workload as W

PID = W.CLOSED_LOOP_PID


def _state20(p=(0, 0, 0), v=(0, 0, 0), q=(1, 0, 0, 0), w=(0, 0, 0), Om=(0, 0, 0, 0), xi=(0, 0, 0)):
    return np.array([*p, *v, *q, *w, *Om, *xi], dtype=np.float64)


def _level(psi):
    return (math.cos(psi / 2), 0, 0, math.sin(psi / 2))


def test_zero_gains_give_the_p_loop(orc):
    """kI = kD = 0: the 17 states follow the P-loop trajectory whatever xi holds."""
    wl = W.closed_loop(n=16, nsteps=800)
    g = dict(W.base_group())
    g.update(kI=[0.0] * 3, kD=[0.0] * 3, xi_max=[2.0] * 3)
    x20 = np.concatenate([wl.x0.astype(np.float64), np.random.default_rng(1).uniform(-1, 1, (16, 3))], axis=1)
    a = orc.rollout([g], wl.gid, x20, wl.cmd, wl.dt, 800, PID)
    b = orc.rollout([g], wl.gid, wl.x0, wl.cmd, wl.dt, 800, W.CLOSED_LOOP)
    np.testing.assert_allclose(a[:, :17], b, rtol=0, atol=1e-9 * np.abs(b).max())


def test_integrator_accumulates_h_times_the_rate_error(orc):
    """xi after n steps equals xi0 plus the sum of h e_k, with e_k the controller's rate error at
    each step start (re-evaluated here through the checker's controller)."""
    wl = W.closed_loop_pid(n=4, nsteps=300)
    g = wl.groups[0]
    for a in range(4):
        x = wl.x0[a].astype(np.float64)
        acc = x[17:20].copy()
        for _ in range(300):
            _, e, _ = orc.controller_pid(g, x, wl.cmd[a])
            acc = np.clip(acc + wl.dt * e, -2.0, 2.0)
            x = orc.rollout([g], [0], x[None], wl.cmd[a:a + 1], wl.dt, 1, PID)[0]
        np.testing.assert_allclose(x[17:20], acc, rtol=1e-13, atol=1e-15)


def test_integrator_one_step_by_hand(orc):
    """Level at the waypoint and heading, hover rotors, spinning at omega: q_e = identity, so
    e = -omega and xi1 = xi0 - h omega; the clamp holds xi at +-xi_max."""
    g = W.pid_group()
    wh = W.hover_speed(g)
    om = np.array([0.3, -0.2, 0.1])
    x0 = _state20(p=(1, 2, 3), q=_level(0.4), w=om, Om=(wh,) * 4, xi=(0.1, -0.05, -1.99995))
    _, e, _ = orc.controller_pid(g, x0, [1, 2, 3, 0.4])
    np.testing.assert_allclose(e, -om, rtol=0, atol=1e-15)
    x1 = orc.rollout([g], [0], x0[None], np.array([[1, 2, 3, 0.4]]), 1e-3, 1, PID)[0]
    np.testing.assert_allclose(x1[17:19], [0.1 - 1e-3 * 0.3, -0.05 + 1e-3 * 0.2], rtol=1e-15)
    assert x1[19] == -2.0  # -1.99995 - 1e-4 clamped to -xi_max


def test_integral_term_rotor_commands_by_hand(orc):
    """Hovering level at the waypoint and heading with omega = 0 and balanced rotors (omega' = 0):
    the only torque demand is taumax kI xi, solved through the orthogonal rows of G."""
    g = W.pid_group()
    wh = W.hover_speed(g)
    xi = np.array([0.4, -0.3, 0.5])
    x0 = _state20(q=_level(0.0), Om=(wh,) * 4, xi=xi)
    w, e, wd = orc.controller_pid(g, x0, [0, 0, 0, 0])
    np.testing.assert_allclose(np.concatenate([e, wd]), 0.0, atol=1e-15)
    Ls, Lc, c = g["L"] * math.sin(g["alpha"]), g["L"] * math.cos(g["alpha"]), g["kq"] / g["kt"]
    om2 = g["omega_max"] ** 2
    taumax = np.array([2 * Ls * g["kt"] * om2, 2 * Lc * g["kt"] * om2, 2 * g["kq"] * om2])
    tau = taumax * np.array(g["kI"]) * xi
    f = (g["m"] * g["g"] / 4 + np.array([1, -1, -1, 1]) * tau[0] / (4 * Ls)
         + np.array([-1, -1, 1, 1]) * tau[1] / (4 * Lc) + np.array([1, -1, 1, -1]) * tau[2] / (4 * c))
    np.testing.assert_allclose(w, np.sqrt(f / g["kt"]), rtol=1e-12)


def test_derivative_term_on_measured_angular_acceleration(orc):
    """Level, at rest, rotors unbalanced by +-d: Eq. 2 and Eq. 3 give the body torques, Eq. (qd4)
    omega' = tau / J (omega = 0, no gyroscopic term); the demand adds -taumax kD omega'."""
    g = W.pid_group()
    wh = W.hover_speed(g)
    Om = np.array([wh + 30, wh - 10, wh - 25, wh + 5])
    x0 = _state20(q=_level(0.0), Om=Om)
    w, e, wd = orc.controller_pid(g, x0, [0, 0, 0, 0])
    f = g["kt"] * Om ** 2
    Ls, Lc, c = g["L"] * math.sin(g["alpha"]), g["L"] * math.cos(g["alpha"]), g["kq"] / g["kt"]
    tau_b = np.array([Ls * (f[0] - f[1] - f[2] + f[3]), Lc * (-f[0] - f[1] + f[2] + f[3]),
                      c * (f[0] - f[1] + f[2] - f[3])])
    np.testing.assert_allclose(wd, tau_b / np.array([g["Jxx"], g["Jyy"], g["Jzz"]]), rtol=1e-12)
    om2 = g["omega_max"] ** 2
    taumax = np.array([2 * Ls * g["kt"] * om2, 2 * Lc * g["kt"] * om2, 2 * g["kq"] * om2])
    tau = -taumax * np.array(g["kD"]) * wd
    fc = g["m"] * g["g"]
    ff = (fc / 4 + np.array([1, -1, -1, 1]) * tau[0] / (4 * Ls) + np.array([-1, -1, 1, 1]) * tau[1] / (4 * Lc)
          + np.array([1, -1, 1, -1]) * tau[2] / (4 * c))
    np.testing.assert_allclose(w, np.sqrt(ff / g["kt"]), rtol=1e-12)


def _spectrum_pid(orc, g, h=1e-4):
    wh = W.hover_speed(g)
    x0 = _state20(Om=(wh,) * 4)
    J = np.zeros((20, 20))
    e = 1e-6
    for j in range(20):
        d = np.zeros(20)
        d[j] = e
        xp = orc.rollout([g], [0], (x0 + d)[None], np.zeros((1, 4)), h, 1, PID)[0]
        xm = orc.rollout([g], [0], (x0 - d)[None], np.zeros((1, 4)), h, 1, PID)[0]
        J[:, j] = (xp - xm) / (2 * e)
    return np.log(np.linalg.eigvals(J).astype(complex)) / h


def _linear_spectrum_pid(g, taumax):
    """Small-angle hover linearisation by hand, chain by chain, with the PID rate loop.

    roll/pitch: (pos, vel, angle, rate, lagged torque, xi) with
      vel' = +-g angle - (c_d/m) vel, angle_des = -+(kp pos + kd vel)/g,
      e = katt (angle_des - angle) - rate, rate' = tau / J,
      tau_cmd = taumax (krate e + kI xi - kD tau / J), tau' = (tau_cmd - tau)/tau_m, xi' = e;
    height: (z, vz, thrust deviation); yaw: (psi, rate, lagged torque, xi); the neutral
    quaternion-norm mode."""
    m, cd, gr, tm = g["m"], g["c_d"], g["g"], g["tau_m"]
    kp, kd, ka = g["kp"][0], g["kd"][0], g["katt"][0]

    def chain(i, J, sgn):
        P, I, D = (taumax[i] * g[k][i] for k in ("krate", "kI", "kD"))
        e = np.array([-ka * sgn * kp / gr, -ka * sgn * kd / gr, -ka, -1.0, 0.0, 0.0])
        A = np.zeros((6, 6))
        A[0, 1] = 1
        A[1, 1] = -cd / m
        A[1, 2] = sgn * gr
        A[2, 3] = 1
        A[3, 4] = 1 / J
        A[4] = P * e / tm
        A[4, 4] += -1 / tm - D / (J * tm)
        A[4, 5] += I / tm
        A[5] = e
        return np.linalg.eigvals(A)

    P, I, D = (taumax[2] * g[k][2] for k in ("krate", "kI", "kD"))
    ka_z = g["katt"][2]
    ey = np.array([-ka_z, -1.0, 0.0, 0.0])
    Ay = np.zeros((4, 4))
    Ay[0, 1] = 1
    Ay[1, 2] = 1 / g["Jzz"]
    Ay[2] = P * ey / tm
    Ay[2, 2] += -1 / tm - D / (g["Jzz"] * tm)
    Ay[2, 3] += I / tm
    Ay[3] = ey
    z = np.linalg.eigvals(np.array([[0, 1, 0], [0, -cd / m, 1 / m], [-m * kp / tm, -m * kd / tm, -1 / tm]]))
    return np.concatenate([chain(0, g["Jxx"], -1), chain(1, g["Jyy"], 1), z, np.linalg.eigvals(Ay), [0.0]])


def _match(a, b, tol):
    a = list(a)
    for lam in b:
        i = int(np.argmin([abs(lam - x) for x in a]))
        assert abs(lam - a[i]) <= tol + 2e-3 * abs(lam), (lam, a[i])
        a.pop(i)


@pytest.mark.parametrize("kI,kD,stable", [(0.05, 0.005, True), (0.1, 0.0, True), (0.3, 0.005, False)])
def test_pid_spectrum_at_hover(orc, kI, kD, stable):
    """Eigenvalues of the checker's 20-state PID step map at hover equal those of the hand
    linearisation, for a stable and an unstable integral gain."""
    g = dict(W.pid_group())
    g.update(kI=[kI] * 3, kD=[kD] * 3)
    g = W.round_group(g)
    _, _, taumax = orc.allocation(g)
    lam = _spectrum_pid(orc, g)
    _match(lam, _linear_spectrum_pid(g, taumax), 0.03)
    assert (lam.real.max() < 1e-6) == stable


def test_pid_reverse_mode_matches_central_differences(orc):
    """The checker's reverse mode on the 20-state PID step vs FP64 central differences (step 1e-5
    relative per parameter, 1e-5 max(1, |x|) per state), within 1e-5 relative per component.
    The step is 10x the P loop's: through omega' the inertias enter the loss more steeply, and
    at 1e-6 the difference quotient of J (about 3e-8 kg m^2 per step) loses 1e-5 to rounding;
    at 1e-4 and 1e-5 it converges on the reverse-mode value to 1e-7."""
    wl = W.differentiable_pid(n_per_group=2, n_groups=2, nsteps=300)
    x0 = wl.x0.astype(np.float64)
    x0[:, 17:20] = np.random.default_rng(9).uniform(-0.3, 0.3, (wl.n, 3))  # a nonzero integral to start
    loss, dx0, dth = orc.grad(wl.groups, wl.gid, x0, wl.cmd, wl.dt, wl.nsteps, PID, wl.goal, wl.w_omega)
    keys = [("kp", 0), ("kp", 1), ("kp", 2), ("kd", 0), ("kd", 1), ("kd", 2), ("katt", 0), ("katt", 1), ("katt", 2),
            ("krate", 0), ("krate", 1), ("krate", 2), ("m", None), ("Jxx", None), ("Jyy", None), ("Jzz", None)]
    h = 1e-5

    def L(a, g, x):
        return orc.loss([g], [0], x[None], wl.cmd[a:a + 1], wl.dt, wl.nsteps, PID, wl.goal[a:a + 1], wl.w_omega,
                        nthreads=1)[0]

    for a in range(wl.n):
        g0 = {k: (list(v) if isinstance(v, list) else v) for k, v in wl.groups[wl.gid[a]].items()}
        fd = []
        for k, i in keys:
            vals = []
            for s in (+1, -1):
                gg = {kk: (list(v) if isinstance(v, list) else v) for kk, v in g0.items()}
                base = gg[k][i] if i is not None else gg[k]
                step = h * abs(base)
                if i is None:
                    gg[k] = base + s * step
                else:
                    gg[k][i] = base + s * step
                vals.append(L(a, gg, x0[a]))
            fd.append((vals[0] - vals[1]) / (2 * step))
        for j in range(20):
            step = h * max(1.0, abs(x0[a, j]))
            xp, xm = x0[a].copy(), x0[a].copy()
            xp[j] += step
            xm[j] -= step
            fd.append((L(a, g0, xp) - L(a, g0, xm)) / (2 * step))
        fd = np.array(fd)
        ad = np.concatenate([dth[a], dx0[a]])
        scale = np.abs(ad).max()
        err = np.abs(fd - ad)
        assert np.all(err <= 1e-5 * np.maximum(np.abs(ad), 1e-3 * scale)), (a, err / np.maximum(np.abs(ad), 1e-3 * scale))
        assert np.abs(dx0[a, 17:20]).max() > 0  # the integral does reach the loss
