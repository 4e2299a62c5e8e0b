"""Cars and fixed-wing drones beside quadrotors in one launch, on the GPU through the C ABI,
against the FP64 checker.

Tolerances: one step, 1e-5 relative with floor 1 per component.  n steps: position 1e-3 m plus
n half-ulps of FP32 at its magnitude, n 2^-24 |p| (a drone 300 m out adds its 2 cm per step to
a position whose ulp is 3e-5 m, and the roundings can pile up over the steps), heading angle
1e-4 rad, speed 1e-4 relative, climb rate 1e-3 m/s, bank 1e-4 rad.  Quadrotors in the same
launch keep their own bars.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2308_12698_b300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def gpu_run(wl, dev, nsteps, K=0, x0=None, groups=None, block=0):
    from paper_2308_12698_b300.sim import Sim, planar, unplanar
    groups = wl.groups if groups is None else groups
    g = torch.from_numpy(wl.gid).to(dev) if len(groups) > 1 else None
    sim = Sim(groups, wl.n, wl.mode, gid=g)
    if block:
        sim.set_launch(block=block)
    x = planar(torch.from_numpy(wl.x0 if x0 is None else x0)).to(dev)
    cmd = torch.from_numpy(wl.cmd).to(dev).reshape(-1)
    sim.step(x, cmd, wl.dt, nsteps, K=K)
    torch.cuda.synchronize()
    out = unplanar(x, wl.n).cpu().numpy()
    sim.close()
    return out


def ref_run(orc, wl, nsteps, x0=None):
    return orc.rollout(wl.groups, wl.gid, wl.x0 if x0 is None else x0, wl.cmd, wl.dt, nsteps, wl.mode)


def check_vehicles(got, ref, nsteps):
    got = got.astype(np.float64)
    dp = np.abs(got[:, 0:3] - ref[:, 0:3]).max(axis=1)
    tol = 1e-3 + nsteps * 2.0 ** -24 * np.abs(ref[:, 0:3]).max(axis=1)
    assert (dp <= tol).all(), (dp.max(), (dp / tol).max())
    ang = np.abs(np.arctan2(got[:, 7] * ref[:, 6] - got[:, 6] * ref[:, 7], got[:, 6] * ref[:, 6] + got[:, 7] * ref[:, 7]))
    assert ang.max() <= 1e-4, ang.max()
    assert (np.abs(got[:, 3] - ref[:, 3]) <= 1e-4 * np.maximum(np.abs(ref[:, 3]), 1.0)).all()
    assert np.abs(got[:, 10] - ref[:, 10]).max() <= 1e-4
    assert np.abs(got[:, 5] - ref[:, 5]).max() <= 1e-3


def check_quads(got, ref):
    perr = np.abs(got[:, 0:3].astype(np.float64) - ref[:, 0:3]).max()
    qa = got[:, 6:10] / np.linalg.norm(got[:, 6:10], axis=1, keepdims=True)
    qb = ref[:, 6:10] / np.linalg.norm(ref[:, 6:10], axis=1, keepdims=True)
    aerr = (2 * np.arccos(np.clip(np.abs((qa * qb).sum(axis=1)), 0, 1))).max()
    assert perr <= 1e-3 and aerr <= 1e-3, (perr, aerr)


@pytest.mark.parametrize("kind", [W.TYPE_CAR, W.TYPE_FIXED_WING])
def test_vehicle_one_step(dev, orc, kind):
    sizes = (0, 4097, 0) if kind == W.TYPE_CAR else (0, 0, 4097)
    wl = W.multi_type(sizes=sizes)
    g = wl.groups[kind]
    one = W.Workload("one", W.CLOSED_LOOP, [g], np.zeros(wl.n, np.uint8), wl.x0, wl.cmd, wl.dt, 1)
    got, ref = gpu_run(one, dev, 1, K=1), ref_run(orc, one, 1)
    tol = 1e-5 * np.maximum(np.abs(ref), 1.0)
    assert (np.abs(got.astype(np.float64) - ref) <= tol).all(), (np.abs(got - ref) / tol).max()


@pytest.mark.parametrize("shuffle", [False, True])
def test_mixed_swarm_1000_steps(dev, orc, shuffle):
    """Every car, every quadrotor and every drone whose course error stays 1e-3 rad away from
    the atan2 jump at +-pi (waypoint straight behind) meets the bars."""
    wl = W.multi_type(sizes=(3000, 3000, 3000), shuffle=shuffle)
    got, ref = gpu_run(wl, dev, 1000, K=100), ref_run(orc, wl, 1000)
    q = wl.gid == W.TYPE_QUAD
    check_quads(got[q], ref[q])
    m = orc.vehicle_margins(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, 1000)
    ok = ~q & (m > 1e-3)
    assert ok.sum() >= 5900, ok.sum()
    check_vehicles(got[ok], ref[ok], 1000)


def test_mixed_launch_is_bitwise_each_group_alone(dev):
    wl = W.multi_type(sizes=(700, 900, 1100), shuffle=True)
    both = gpu_run(wl, dev, 200, K=200)
    for gi in range(3):
        idx = np.flatnonzero(wl.gid == gi)
        one = W.Workload("one", W.CLOSED_LOOP, [wl.groups[gi]], np.zeros(idx.size, np.uint8),
                         np.ascontiguousarray(wl.x0[idx]), np.ascontiguousarray(wl.cmd[idx]), wl.dt, 200)
        np.testing.assert_array_equal(both[idx], gpu_run(one, dev, 200, K=200))


def test_mixed_fused_is_bitwise_plain(dev):
    wl = W.multi_type(sizes=(500, 500, 501), shuffle=True)
    a = gpu_run(wl, dev, 60, K=1)
    np.testing.assert_array_equal(a, gpu_run(wl, dev, 60, K=60))
    np.testing.assert_array_equal(a, gpu_run(wl, dev, 60, K=7, block=64))


def test_vehicle_handles_refuse_rollouts_and_open_loop(dev):
    from paper_2308_12698_b300 import _lib
    from paper_2308_12698_b300.sim import Sim
    wl = W.multi_type(sizes=(10, 10, 10))
    gid = torch.from_numpy(wl.gid).to(dev)
    with pytest.raises(_lib.SimError):
        Sim(wl.groups, wl.n, W.OPEN_LOOP, gid=gid)
    with pytest.raises(_lib.SimError):
        Sim(wl.groups, wl.n, W.CLOSED_LOOP_PID, gid=gid)
    sim = Sim(wl.groups, wl.n, wl.mode, gid=gid)
    x = torch.zeros(17 * wl.n, device=dev)
    c = torch.zeros(4 * wl.n, device=dev)
    ck = torch.zeros(2 * 17 * wl.n, device=dev)
    rc = _lib.lib().sim_rollout_forward(sim.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(c.data_ptr()),
                                        1e-3, 10, 10, ctypes.c_void_p(ck.data_ptr()), None, None)
    assert rc == _lib.SIM_ERR_ARG
    sim.close()


def test_vehicle_parameter_checks(dev):
    from paper_2308_12698_b300 import _lib
    from paper_2308_12698_b300.sim import Sim
    for bad in (dict(W.car_group(), veh=[0.0, 0.7, 3.0, 1.0, 5.0, 0, 0, 0]),        # wheelbase 0
                dict(W.fixed_wing_group(), veh=[3.0, 1.6, 1.5, 2.0, 1.0, 0.5, 0, 0]),  # bank limit >= pi/2
                dict(W.car_group(), type=7)):                                        # unknown type
        with pytest.raises(_lib.SimError):
            Sim([bad], 4, W.CLOSED_LOOP)


def test_stalled_drone_is_frozen_and_counted(dev):
    """A drone at zero airspeed divides by zero in g tan(phi) / V: it is marked dead and kept at
    its last finite state; the cars and quadrotors of the launch step on."""
    from paper_2308_12698_b300.sim import Sim, planar, unplanar
    wl = W.multi_type(sizes=(64, 64, 64))
    x0 = wl.x0.copy()
    bad = int(np.flatnonzero(wl.gid == W.TYPE_FIXED_WING)[5])
    x0[bad, 3] = 0.0
    x0[bad, 10] = 0.3
    sim = Sim(wl.groups, wl.n, wl.mode, gid=torch.from_numpy(wl.gid).to(dev))
    x = planar(torch.from_numpy(x0)).to(dev)
    sim.step(x, torch.from_numpy(wl.cmd).to(dev).reshape(-1), wl.dt, 50, K=10)
    assert sim.n_dead() == 1
    st = sim.status().cpu().numpy()
    assert st[bad] == 1 and (np.delete(st, bad) == 0).all()
    got = unplanar(x, wl.n).cpu().numpy()
    np.testing.assert_array_equal(got[bad], x0[bad])
    assert np.isfinite(got).all()
    sim.close()


def test_mixed_swarm_collisions(dev, orc):
    """Collision detection over quadrotors, cars and drones: each group's L is its radius."""
    from paper_2308_12698_b300.sim import Sim, planar
    wl = W.multi_type(sizes=(300, 300, 300), shuffle=True)
    x0 = wl.x0.copy()
    x0[:, 0:3] = np.random.default_rng(11).uniform(-6.0, 6.0, (wl.n, 3)).astype(np.float32)
    groups = [dict(g, L=r) for g, r in zip(wl.groups, (0.225, 1.5, 0.9))]
    sim = Sim(groups, wl.n, wl.mode, gid=torch.from_numpy(wl.gid).to(dev))
    x = planar(torch.from_numpy(x0)).to(dev)
    sim.collide(x, radius_scale=1.0)
    got = (sim.status().cpu().numpy() == 2).astype(np.uint8)
    radius = np.array([0.225, 1.5, 0.9], np.float32)[wl.gid]
    ref = orc.collisions(x0[:, 0:3], radius, np.ones(wl.n, np.uint8))
    np.testing.assert_array_equal(got, ref)
    assert 0 < ref.sum() < wl.n
    sim.close()


def test_mixed_swarm_host_entry_and_rounds_are_bitwise_sim_step(dev):
    """The host-buffer pipeline and the decision rounds run the mixed launch like sim_step."""
    from paper_2308_12698_b300.sim import Sim, planar, unplanar
    wl = W.multi_type(sizes=(70_000, 40_000, 50_001), shuffle=True)
    direct = gpu_run(wl, dev, 40, K=20)
    sim = Sim(wl.groups, wl.n, wl.mode, gid=torch.from_numpy(wl.gid).to(dev))
    h_state = planar(torch.from_numpy(wl.x0)).pin_memory()
    h_cmd = torch.from_numpy(wl.cmd).reshape(-1).contiguous().pin_memory()
    d_state = torch.empty(17 * wl.n, device=dev)
    d_cmd = torch.empty(4 * wl.n, device=dev)
    sim.step_host(h_state, h_cmd, d_state, d_cmd, wl.dt, 40, K=20)
    np.testing.assert_array_equal(unplanar(h_state, wl.n).numpy(), direct)
    x = planar(torch.from_numpy(wl.x0)).to(dev)
    h_cmds = torch.from_numpy(wl.cmd).reshape(1, -1).repeat(4, 1).contiguous().pin_memory()
    sim.run_rounds(x, h_cmds, 10, wl.dt, K=10)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(unplanar(x, wl.n).cpu().numpy(), direct)
    sim.close()


@pytest.mark.parametrize("shuffle", [False, True], ids=["contiguous", "interleaved"])
def test_mixed_swarm_full_size_sampled(dev, orc, shuffle):
    """The bench's mixed-type legs (600,000 agents, one launch of K = 1000; the types' ids
    contiguous, or in random order through the group-sorted order): 1000 sampled agents of each
    type against the checker."""
    from paper_2308_12698_b300.sim import Sim, planar, unplanar
    wl = W.multi_type(nsteps=1000, shuffle=shuffle)
    sim = Sim(wl.groups, wl.n, wl.mode, gid=torch.from_numpy(wl.gid).to(dev))
    x = planar(torch.from_numpy(wl.x0)).to(dev)
    sim.step(x, torch.from_numpy(wl.cmd).to(dev).reshape(-1), wl.dt, 1000, K=1000)
    rng = np.random.default_rng(22)
    idx = np.concatenate([rng.choice(np.flatnonzero(wl.gid == t), 1000, replace=False) for t in range(3)])
    got = unplanar(x, wl.n)[torch.from_numpy(idx).to(dev)].cpu().numpy()
    sub = dict(gid=wl.gid[idx], x0=wl.x0[idx], cmd=wl.cmd[idx])
    ref = orc.rollout(wl.groups, sub["gid"], sub["x0"], sub["cmd"], wl.dt, 1000, wl.mode)
    q = sub["gid"] == W.TYPE_QUAD
    check_quads(got[q], ref[q])
    m = orc.vehicle_margins(wl.groups, sub["gid"], sub["x0"], sub["cmd"], wl.dt, 1000)
    ok = ~q & (m > 1e-3)
    assert ok.sum() >= 1990
    check_vehicles(got[ok], ref[ok], 1000)
    assert sim.n_dead() == 0
    sim.close()


def test_vehicles_at_and_near_their_waypoints(dev, orc):
    """Degenerate guidance geometry: a car or a drone exactly on its waypoint (zero distance: no
    curvature, no course error), a car inside the look-ahead floor l_min (the floor sets the
    pursuit radius), and both types straight ahead of the waypoint's direction.  One step and 50
    steps against the checker."""
    cars = W.multi_type(sizes=(0, 6, 0))
    drones = W.multi_type(sizes=(0, 0, 6))
    for base, kind in ((cars, W.TYPE_CAR), (drones, W.TYPE_FIXED_WING)):
        x0, cmd = base.x0.copy(), base.cmd.copy()
        c, s = x0[:, 6], x0[:, 7]
        cmd[0, 0:2] = x0[0, 0:2]                                   # on the waypoint
        cmd[1, 0:2] = x0[1, 0:2] + 0.5 * np.array([-s[1], c[1]])   # 0.5 m to the side: inside l_min
        cmd[2, 0:2] = x0[2, 0:2] + 50.0 * np.array([c[2], s[2]])   # straight ahead
        cmd[3, 0:2] = x0[3, 0:2] + 0.3 * np.array([c[3], s[3]])    # just ahead, inside l_min
        if kind == W.TYPE_FIXED_WING:
            cmd[:, 2] = x0[:, 2]                                   # hold altitude as well
        wl = W.Workload("wp", W.CLOSED_LOOP, [base.groups[kind]], np.zeros(6, np.uint8), x0, cmd, base.dt, 50)
        got, ref = gpu_run(wl, dev, 1, K=1), ref_run(orc, wl, 1)
        tol = 1e-5 * np.maximum(np.abs(ref), 1.0)
        assert (np.abs(got.astype(np.float64) - ref) <= tol).all(), (kind, (np.abs(got - ref) / tol).max())
        got, ref = gpu_run(wl, dev, 50, K=10), ref_run(orc, wl, 50)
        dp = np.abs(got[:, 0:3].astype(np.float64) - ref[:, 0:3]).max(axis=1)
        assert (dp <= 1e-3 + 50 * 2.0 ** -24 * np.abs(ref[:, 0:3]).max(axis=1)).all(), (kind, dp)
