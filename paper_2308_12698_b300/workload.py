"""Seeded synthetic workloads for the batched quadrotor step.

This module only draws inputs: parameter groups, initial states, commands and
goals.  It holds none of the simulation arithmetic (no controller, no
dynamics, no integrator), so the CUDA path and the CPU checker can both take
their inputs from here without sharing any of the method.

Conventions
-----------
* Per-agent state, 17 values in this order: p(3), v(3), q(4: w, x, y, z;
  Hamilton, scalar first, body->inertial), omega(3, body rates), Omega(4,
  rotor speeds in rad/s).  Frames: ENU inertial, FLU body (Sec. III-B).
* Every floating value is rounded to float32 here, so the FP32 device path
  and the FP64 checker see the same problem (the checker upcasts exactly).
* ``cmd`` is one float4 per agent.  Open loop: four rotor-speed commands.
  Closed loop: waypoint x, y, z and heading psi.

Parameter groups are plain dicts with keys ``m, Jxx, Jyy, Jzz, L, alpha, kt,
kq, tau_m, c_d, omega_max, g, kp, kd, katt, krate, a_max`` (the last gains
are 3-vectors).  ``kt``/``kq`` are the thrust/torque coefficients of Eq. 2,
``L``/``alpha`` the arm geometry of the allocation matrix in Eq. 3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

#: Seeds follow one rule: base seed plus the workload index.
BASE_SEED = 20230823

STATE_DIM = 17
THETA_NAMES = ("kp_x", "kp_y", "kp_z", "kd_x", "kd_y", "kd_z",
               "katt_x", "katt_y", "katt_z", "krate_x", "krate_y", "krate_z",
               "m", "Jxx", "Jyy", "Jzz")

OPEN_LOOP = 0
CLOSED_LOOP = 1
CLOSED_LOOP_PID = 2
#: state components in the PID mode: the 17 and the rate-error integral xi (3)
STATE_DIM_PID = 20
#: agent types of a parameter group
TYPE_QUAD, TYPE_CAR, TYPE_FIXED_WING = 0, 1, 2

#: Fixed group sizes of the uneven heterogeneous swarm (sum 600,000).
HETERO_SIZES = (100, 900, 5000, 19000, 55000, 130000, 190000, 200000)


def _f32(x):
    return float(np.float32(x))


def base_group() -> dict:
    """The reference quadrotor: 1.5 kg X-frame, 0.225 m arms, lag 0.03 s.

    Gains: position PD (6, 4.5), attitude P 8, normalised rate P 0.2 per
    axis, per-axis acceleration clamp 4 m/s^2, rotor clamp [0, 1200] rad/s.
    """
    g = dict(m=1.5, Jxx=0.0347, Jyy=0.0458, Jzz=0.0977, L=0.225,
             alpha=math.pi / 4, kt=1e-5, kq=1.6e-7, tau_m=0.03, c_d=0.1,
             omega_max=1200.0, g=9.81, kp=[6.0] * 3, kd=[4.5] * 3,
             katt=[8.0] * 3, krate=[0.2] * 3, a_max=4.0)
    return round_group(g)


def pid_group() -> dict:
    """The reference quadrotor with a PID body-rate loop: the P gain 0.2 of the base group plus
    integral gain kI = 0.05 and derivative gain kD = 0.005 per axis (normalised by the axis
    torque limit like the P gain) and integrator limit |xi| <= 2 rad.  At hover the slowest
    closed-loop pole sits at -0.23 1/s and the fastest rate mode is damped to |Im| = 7.6 rad/s
    (0.05 < kI < 0.2 is the stable band at kD = 0.005)."""
    g = dict(base_group())
    g.update(kI=[0.05] * 3, kD=[0.005] * 3, xi_max=[2.0] * 3)
    return round_group(g)


def car_group() -> dict:
    """A road car under pure pursuit (kinematic bicycle): wheelbase 2.7 m, steering lock 35 deg
    (tan = 0.7), acceleration clamp 3 m/s^2, speed gain 1 /s, minimum look-ahead 5 m.  The
    quadrotor fields are those of base_group and unused."""
    g = dict(base_group())
    g.update(type=TYPE_CAR, veh=[2.7, 0.7, 3.0, 1.0, 5.0, 0.0, 0.0, 0.0])
    return round_group(g)


def fixed_wing_group() -> dict:
    """A small fixed-wing drone (coordinated-turn guidance model): bank response 3 /s, bank
    limit 35 deg (0.61 rad), course gain 1.5 rad of bank per rad of course error, altitude loop
    b_hd = 2 /s, b_h = 1 /s^2 (critically damped), airspeed response 0.5 /s."""
    g = dict(base_group())
    g.update(type=TYPE_FIXED_WING, veh=[3.0, 0.61, 1.5, 2.0, 1.0, 0.5, 0.0, 0.0])
    return round_group(g)


def round_group(g: dict) -> dict:
    out = {}
    for k, v in g.items():
        out[k] = [_f32(e) for e in v] if isinstance(v, (list, tuple)) else _f32(v)
    return out


def hover_speed(g: dict) -> float:
    """Rotor speed at which four rotors carry the weight: sqrt(m g / (4 kt))."""
    return math.sqrt(g["m"] * g["g"] / (4.0 * g["kt"]))


def scaled_group(m: float, omega_h: float) -> dict:
    """One member of a heterogeneous family, scaled from the base airframe.

    Arm r = 0.225 (m/1.5)^(1/3); inertia J_base (m/1.5)(r/0.225)^2;
    kt = m g / (4 omega_h^2) keeps hover at omega_h; kq = 0.016 kt;
    omega_max = 1.979 omega_h keeps thrust/weight; drag c_d = (0.1/1.5) m.
    Gains are the normalised ones of the base group.
    """
    b = base_group()
    s = m / 1.5
    r = 0.225 * s ** (1.0 / 3.0)
    jscale = s * (r / 0.225) ** 2
    kt = m * 9.81 / (4.0 * omega_h ** 2)
    g = dict(b)
    g.update(m=m, Jxx=0.0347 * jscale, Jyy=0.0458 * jscale, Jzz=0.0977 * jscale,
             L=r, kt=kt, kq=0.016 * kt, omega_max=1.979 * omega_h,
             c_d=0.1 / 1.5 * m)
    return round_group(g)


def draw_groups(rng: np.random.Generator, n_groups: int) -> list[dict]:
    """Mass log-uniform in [0.03, 5] kg, hover speed log-uniform in [400, 1000] rad/s."""
    ms = np.exp(rng.uniform(math.log(0.03), math.log(5.0), n_groups))
    ws = np.exp(rng.uniform(math.log(400.0), math.log(1000.0), n_groups))
    return [scaled_group(float(m), float(w)) for m, w in zip(ms, ws)]


@dataclass
class Workload:
    """Inputs of one batched rollout, host side, float32."""
    name: str
    mode: int
    groups: list[dict]
    gid: np.ndarray          # (N,) uint8 group index per agent
    x0: np.ndarray           # (N, 17) float32 initial state
    cmd: np.ndarray          # (N, 4) float32 command
    dt: float
    nsteps: int
    goal: np.ndarray | None = None   # (N, 3) float32 terminal goal (differentiable rollout)
    w_omega: float = 0.0             # weight of the rotor-speed running cost
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x0.shape[0])


def _initial_states(rng: np.random.Generator, n: int, omega_h: np.ndarray):
    """p ~ U[-10,10]^3, v ~ N(0, 0.5), omega ~ N(0, 0.1), tilt <= 10 deg, Omega = hover.

    q = q_axis((cos phi, sin phi, 0), theta) (x) q_z(psi) with phi ~ U[0, 2 pi),
    theta ~ U[0, 10 deg], psi ~ U[-pi, pi).  Returns (x0, psi): psi is the
    drawn heading, which closed-loop agents are commanded to hold.
    """
    x = np.zeros((n, STATE_DIM), dtype=np.float64)
    x[:, 0:3] = rng.uniform(-10.0, 10.0, (n, 3))
    x[:, 3:6] = rng.normal(0.0, 0.5, (n, 3))
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    th = rng.uniform(0.0, math.radians(10.0), n)
    psi = rng.uniform(-math.pi, math.pi, n)
    # tilt quaternion about the horizontal axis (cos phi, sin phi, 0)
    a_w = np.cos(th / 2)
    a_x = np.sin(th / 2) * np.cos(phi)
    a_y = np.sin(th / 2) * np.sin(phi)
    # yaw quaternion (cos psi/2, 0, 0, sin psi/2); product a (x) b written out
    b_w = np.cos(psi / 2)
    b_z = np.sin(psi / 2)
    x[:, 6] = a_w * b_w
    x[:, 7] = a_x * b_w + a_y * b_z
    x[:, 8] = a_y * b_w - a_x * b_z
    x[:, 9] = a_w * b_z
    x[:, 10:13] = rng.normal(0.0, 0.1, (n, 3))
    x[:, 13:17] = omega_h[:, None]
    return x.astype(np.float32), psi


def _hover_per_agent(groups, gid):
    wh = np.array([hover_speed(g) for g in groups], dtype=np.float64)
    return wh[gid]


def open_loop(n: int = 64, nsteps: int = 1000, dt: float = 1e-3, seed: int = BASE_SEED + 0) -> Workload:
    """Reference quadrotors flying open loop on rotor commands hover x (1 +- 5 %)."""
    rng = np.random.default_rng(seed)
    groups = [base_group()]
    gid = np.zeros(n, dtype=np.uint8)
    wh = _hover_per_agent(groups, gid)
    x0, _ = _initial_states(rng, n, wh)
    cmd = (wh[:, None] * (1.0 + rng.uniform(-0.05, 0.05, (n, 4)))).astype(np.float32)
    return Workload("open-loop", OPEN_LOOP, groups, gid, x0, cmd, dt, nsteps)


def closed_loop(n: int = 5000, nsteps: int = 10000, dt: float = 1e-3, seed: int = BASE_SEED + 1,
                name: str = "closed-loop") -> Workload:
    """Reference quadrotors under the cascaded controller, waypoints ~ U[-50, 50]^3.

    Each agent is commanded to hold its initial heading (cmd[3] = drawn yaw).
    A common heading of 0 against yaws spread over [-pi, pi) saturates the
    mixer on yaw for seconds, and the swarm does not reach its waypoints.
    """
    rng = np.random.default_rng(seed)
    groups = [base_group()]
    gid = np.zeros(n, dtype=np.uint8)
    wh = _hover_per_agent(groups, gid)
    x0, psi = _initial_states(rng, n, wh)
    cmd = np.zeros((n, 4), dtype=np.float64)
    cmd[:, 0:3] = rng.uniform(-50.0, 50.0, (n, 3))
    cmd[:, 3] = psi
    return Workload(name, CLOSED_LOOP, groups, gid, x0, cmd.astype(np.float32), dt, nsteps)


def closed_loop_pid(n: int = 5000, nsteps: int = 1000, dt: float = 1e-3, seed: int = BASE_SEED + 7,
                    name: str = "closed-loop-pid") -> Workload:
    """Reference quadrotors under the cascade with the PID rate loop (pid_group), waypoints
    ~ U[-50, 50]^3, heading hold; 20-component states with the integral xi starting at 0."""
    rng = np.random.default_rng(seed)
    groups = [pid_group()]
    gid = np.zeros(n, dtype=np.uint8)
    wh = _hover_per_agent(groups, gid)
    x17, psi = _initial_states(rng, n, wh)
    x0 = np.zeros((n, STATE_DIM_PID), dtype=np.float32)
    x0[:, :STATE_DIM] = x17
    cmd = np.zeros((n, 4), dtype=np.float64)
    cmd[:, 0:3] = rng.uniform(-50.0, 50.0, (n, 3))
    cmd[:, 3] = psi
    return Workload(name, CLOSED_LOOP_PID, groups, gid, x0, cmd.astype(np.float32), dt, nsteps)


def scale_sweep(n: int, nsteps: int = 1000, dt: float = 1e-3) -> Workload:
    """Closed-loop swarm of the reference quadrotor at size n (1e3 .. 1e7)."""
    return closed_loop(n=n, nsteps=nsteps, dt=dt, seed=BASE_SEED + 2, name=f"closed-loop-{n}")


def heterogeneous(sizes=HETERO_SIZES, nsteps: int = 1000, dt: float = 1e-3, seed: int = BASE_SEED + 3,
                  shuffle: bool = False) -> Workload:
    """Eight scaled airframes in uneven groups, one launch; ids sorted or shuffled."""
    rng = np.random.default_rng(seed)
    groups = draw_groups(rng, len(sizes))
    gid = np.concatenate([np.full(s, i, dtype=np.uint8) for i, s in enumerate(sizes)])
    if shuffle:
        gid = gid[rng.permutation(gid.size)]
    n = gid.size
    wh = _hover_per_agent(groups, gid)
    x0, psi = _initial_states(rng, n, wh)
    cmd = np.zeros((n, 4), dtype=np.float64)
    cmd[:, 0:3] = rng.uniform(-50.0, 50.0, (n, 3))
    cmd[:, 3] = psi
    return Workload("heterogeneous", CLOSED_LOOP, groups, gid, x0, cmd.astype(np.float32), dt, nsteps,
                    extra=dict(sizes=list(sizes), shuffled=shuffle))


def differentiable(n_per_group: int = 1024, n_groups: int = 4, nsteps: int = 2000, dt: float = 1e-3,
                   seed: int = BASE_SEED + 4, w_omega: float = 1e-6) -> Workload:
    """Goal-reaching rollout for gradients: goal = p0 + U[-5, 5]^3, also the waypoint.

    Loss = sum_a |p_T - goal|^2 + w_omega sum_a sum_{n=1..T} sum_i Omega_{n,i}^2.
    """
    rng = np.random.default_rng(seed)
    groups = draw_groups(rng, n_groups)
    gid = np.repeat(np.arange(n_groups, dtype=np.uint8), n_per_group)
    n = gid.size
    wh = _hover_per_agent(groups, gid)
    x0, psi = _initial_states(rng, n, wh)
    goal = (x0[:, 0:3].astype(np.float64) + rng.uniform(-5.0, 5.0, (n, 3))).astype(np.float32)
    cmd = np.zeros((n, 4), dtype=np.float32)
    cmd[:, 0:3] = goal
    cmd[:, 3] = psi
    return Workload("differentiable", CLOSED_LOOP, groups, gid, x0, cmd, dt, nsteps,
                    goal=goal, w_omega=w_omega)


def differentiable_pid(n_per_group: int = 1024, n_groups: int = 4, nsteps: int = 2000, dt: float = 1e-3,
                       seed: int = BASE_SEED + 8, w_omega: float = 1e-6) -> Workload:
    """The goal-reaching rollout of :func:`differentiable` with the PID body-rate loop: each
    drawn airframe gets pid_group's kI, kD and xi_max; 20-component states, xi starting at 0."""
    base = differentiable(n_per_group, n_groups, nsteps, dt, seed, w_omega)
    pid = pid_group()
    groups = []
    for g in base.groups:
        g = dict(g)
        g.update(kI=pid["kI"], kD=pid["kD"], xi_max=pid["xi_max"])
        groups.append(round_group(g))
    x0 = np.zeros((base.n, STATE_DIM_PID), dtype=np.float32)
    x0[:, :STATE_DIM] = base.x0
    return Workload("differentiable-pid", CLOSED_LOOP_PID, groups, base.gid, x0, base.cmd, dt, nsteps,
                    goal=base.goal, w_omega=w_omega)


def _vehicle_states(rng: np.random.Generator, kind: int, n: int):
    """Initial 17-states and commands of n cars or fixed-wing drones (the unused components 0)."""
    x = np.zeros((n, STATE_DIM))
    cmd = np.zeros((n, 4))
    psi = rng.uniform(-math.pi, math.pi, n)
    x[:, 6], x[:, 7] = np.cos(psi), np.sin(psi)
    if kind == TYPE_CAR:
        x[:, 0:2] = rng.uniform(-50.0, 50.0, (n, 2))
        x[:, 3] = rng.uniform(0.0, 15.0, n)
        cmd[:, 0:2] = rng.uniform(-100.0, 100.0, (n, 2))
        cmd[:, 3] = rng.uniform(5.0, 20.0, n)
    else:
        x[:, 0:2] = rng.uniform(-500.0, 500.0, (n, 2))
        x[:, 2] = rng.uniform(50.0, 150.0, n)
        x[:, 3] = rng.uniform(15.0, 25.0, n)
        x[:, 10] = rng.uniform(-0.2, 0.2, n)
        cmd[:, 0:2] = rng.uniform(-1000.0, 1000.0, (n, 2))
        cmd[:, 2] = rng.uniform(50.0, 150.0, n)
        cmd[:, 3] = rng.uniform(15.0, 25.0, n)
    return x, cmd


#: Agents per type of the mixed swarm: quadrotors, cars, fixed-wing drones (sum 600,000).
MULTI_TYPE_SIZES = (200000, 200000, 200000)


def multi_type(sizes=MULTI_TYPE_SIZES, nsteps: int = 1000, dt: float = 1e-3, seed: int = BASE_SEED + 9,
               shuffle: bool = False) -> Workload:
    """Quadrotors, cars and fixed-wing drones in one closed-loop swarm (three groups, one type
    each): the quadrotors as in closed_loop, cars with waypoints ~ U[-100, 100]^2 and target
    speeds U[5, 20] m/s, drones with waypoints ~ U[-1000, 1000]^2, altitudes U[50, 150] m and
    airspeeds U[15, 25] m/s.  Group ids sorted by type, or shuffled."""
    rng = np.random.default_rng(seed)
    groups = [base_group(), car_group(), fixed_wing_group()]
    xs, cs = [], []
    wh = hover_speed(groups[0])
    xq, psi = _initial_states(rng, sizes[0], np.full(sizes[0], wh))
    cq = np.zeros((sizes[0], 4))
    cq[:, 0:3] = rng.uniform(-50.0, 50.0, (sizes[0], 3))
    cq[:, 3] = psi
    xs.append(xq.astype(np.float64))
    cs.append(cq)
    for kind, m in ((TYPE_CAR, sizes[1]), (TYPE_FIXED_WING, sizes[2])):
        x, c = _vehicle_states(rng, kind, m)
        xs.append(x)
        cs.append(c)
    gid = np.concatenate([np.full(m, i, dtype=np.uint8) for i, m in enumerate(sizes)])
    x0 = np.concatenate(xs).astype(np.float32)
    cmd = np.concatenate(cs).astype(np.float32)
    if shuffle:
        perm = rng.permutation(gid.size)
        gid, x0, cmd = gid[perm], x0[perm], cmd[perm]
    return Workload("multi-type", CLOSED_LOOP, groups, gid, np.ascontiguousarray(x0), np.ascontiguousarray(cmd),
                    dt, nsteps, extra=dict(sizes=list(sizes), shuffled=shuffle))


def thrust_down(n: int = 4096, nsteps: int = 1, dt: float = 1e-3, seed: int = BASE_SEED + 6) -> Workload:
    """Demanded force pointing downwards: the reference airframe with its acceleration clamp
    raised to 25 m/s^2 (above g), climbing at 2-10 m/s towards waypoints 5-20 m below,
    attitudes uniform over all rotations (half of them inverted), headings uniform in
    [-pi, pi).  Goal = waypoint, for gradients."""
    rng = np.random.default_rng(seed)
    g = dict(base_group())
    g["a_max"] = 25.0
    groups = [round_group(g)]
    wh = hover_speed(groups[0])
    x = np.zeros((n, STATE_DIM))
    x[:, 0:3] = rng.uniform(-10.0, 10.0, (n, 3))
    x[:, 3:5] = rng.normal(0.0, 1.0, (n, 2))
    x[:, 5] = rng.uniform(2.0, 10.0, n)
    q = rng.normal(size=(n, 4))
    x[:, 6:10] = q / np.linalg.norm(q, axis=1, keepdims=True)
    x[:, 10:13] = rng.normal(0.0, 0.5, (n, 3))
    x[:, 13:17] = wh * rng.uniform(0.5, 1.5, (n, 4))
    cmd = np.zeros((n, 4))
    cmd[:, 0:2] = x[:, 0:2] + rng.uniform(-5.0, 5.0, (n, 2))
    cmd[:, 2] = x[:, 2] - rng.uniform(5.0, 20.0, n)
    cmd[:, 3] = rng.uniform(-math.pi, math.pi, n)
    x, cmd = x.astype(np.float32), cmd.astype(np.float32)
    return Workload("thrust-down", CLOSED_LOOP, groups, np.zeros(n, np.uint8), x, cmd, dt, nsteps,
                    goal=cmd[:, 0:3].copy(), w_omega=1e-6)


# --- layout helpers (data movement only) -----------------------------------

def to_planes(x: np.ndarray) -> np.ndarray:
    """(N, 17) or (N, 20) agent-major -> flat planar layout used on the device.

    Planes 0..3 hold float4 groups of state components (0-3, 4-7, 8-11,
    12-15) for all agents; plane 4 holds the rest (component 16, or 16-19 in
    the PID mode) interleaved per agent.  Returns a flat float32 array.
    """
    n, nx = x.shape
    out = np.empty(nx * n, dtype=np.float32)
    for k in range(4):
        out[4 * k * n: 4 * k * n + 4 * n] = x[:, 4 * k:4 * k + 4].reshape(-1)
    out[16 * n:] = x[:, 16:].reshape(-1)
    return out


def from_planes(flat: np.ndarray, n: int) -> np.ndarray:
    """Inverse of :func:`to_planes` (17 or 20 components, from the size)."""
    flat = np.asarray(flat)
    nx = flat.size // n
    x = np.empty((n, nx), dtype=flat.dtype)
    for k in range(4):
        x[:, 4 * k:4 * k + 4] = flat[4 * k * n: 4 * k * n + 4 * n].reshape(n, 4)
    x[:, 16:] = flat[16 * n: nx * n].reshape(n, nx - 16)
    return x


def collision_field(n: int, spacing: float = 2.0, planted: float = 0.01, seed: int = BASE_SEED + 5,
                    nsteps: int = 1, dt: float = 1e-3) -> Workload:
    """Reference quadrotors spread uniformly over a cube of side spacing * n^(1/3) (mean spacing
    `spacing` m), with a fraction `planted` of agents moved next to another one at a distance
    U[0.2, 0.6] m along a random direction (two reference airframes collide below 0.45 m).
    Waypoints are the agents' own positions (hover); heading held."""
    rng = np.random.default_rng(seed)
    groups = [base_group()]
    gid = np.zeros(n, dtype=np.uint8)
    wh = _hover_per_agent(groups, gid)
    x0, psi = _initial_states(rng, n, wh)
    side = spacing * max(n, 1) ** (1.0 / 3.0)
    pos = rng.uniform(-side / 2, side / 2, (n, 3))
    k = int(planted * n)
    if k and n > 1:
        a = rng.choice(n, k, replace=False)
        b = rng.integers(0, n, k)
        b = np.where(b == a, (b + 1) % n, b)
        u = rng.normal(size=(k, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        pos[a] = pos[b] + u * rng.uniform(0.2, 0.6, (k, 1))
    x0[:, 0:3] = pos.astype(np.float32)
    cmd = np.zeros((n, 4), dtype=np.float32)
    cmd[:, 0:3] = x0[:, 0:3]
    cmd[:, 3] = psi
    return Workload("collision-field", CLOSED_LOOP, groups, gid, x0, cmd, dt, nsteps,
                    extra=dict(side=side, planted=k))
