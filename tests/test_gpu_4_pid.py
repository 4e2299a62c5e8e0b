"""PID body-rate loop (SIM_CLOSED_LOOP_PID, 20-component states) on the GPU, through the C ABI,
against the FP64 checker.

Tolerances as for the P loop: one step 1e-5 relative with floors (xi: floor 1 rad); 1000 steps
1e-3 m in position, 1e-3 rad in attitude, and 1e-3 rad in xi.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2308_12698_b300 import workload as W

pytestmark = pytest.mark.gpu

FLOOR = np.array([1.0] * 3 + [1.0] * 3 + [1.0] * 4 + [1.0] * 3 + [100.0] * 4 + [1.0] * 3)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def gpu_run(wl, dev, nsteps, K=0, x0=None, groups=None, block=0, mode=None):
    from paper_2308_12698_b300.sim import Sim, planar, unplanar
    groups = wl.groups if groups is None else groups
    g = torch.from_numpy(wl.gid).to(dev) if len(groups) > 1 else None
    sim = Sim(groups, wl.n, wl.mode if mode is None else mode, gid=g)
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


def check_one_step(got, ref):
    tol = 1e-5 * np.maximum(np.abs(ref), FLOOR)
    bad = np.abs(got.astype(np.float64) - ref) > tol
    assert not bad.any(), (np.argwhere(bad)[:5], (np.abs(got - ref) / tol).max())


def attitude_err(qa, qb):
    qa = qa / np.linalg.norm(qa, axis=1, keepdims=True)
    qb = qb / np.linalg.norm(qb, axis=1, keepdims=True)
    return 2.0 * np.arccos(np.clip(np.abs(np.sum(qa * qb, axis=1)), 0.0, 1.0))


def check_traj(got, ref, tol=1e-3):
    perr = np.abs(got[:, 0:3].astype(np.float64) - ref[:, 0:3]).max()
    aerr = attitude_err(got[:, 6:10].astype(np.float64), ref[:, 6:10]).max()
    xerr = np.abs(got[:, 17:20].astype(np.float64) - ref[:, 17:20]).max()
    assert perr <= tol and aerr <= tol and xerr <= tol, (perr, aerr, xerr)


@pytest.mark.parametrize("n", [1, 33, 4097])
def test_pid_one_step(dev, orc, n):
    wl = W.closed_loop_pid(n=n)
    check_one_step(gpu_run(wl, dev, 1, K=1), ref_run(orc, wl, 1))


def test_pid_one_step_from_advanced_states(dev, orc):
    """One step from states 1.5 s into the transient: tilted, spinning, xi built up (some clamped)."""
    wl = W.closed_loop_pid(n=2000)
    xs = ref_run(orc, wl, 1500).astype(np.float32)
    assert np.abs(xs[:, 17:20]).max() > 0.05
    check_one_step(gpu_run(wl, dev, 1, K=1, x0=xs), ref_run(orc, wl, 1, x0=xs))


@pytest.mark.parametrize("K", [1, 10, 1000])
def test_pid_1000_steps(dev, orc, K):
    wl = W.closed_loop_pid(n=5000)
    check_traj(gpu_run(wl, dev, 1000, K=K), ref_run(orc, wl, 1000))


def test_pid_fused_is_bitwise_plain(dev):
    wl = W.closed_loop_pid(n=3001)
    a = gpu_run(wl, dev, 120, K=1)
    np.testing.assert_array_equal(a, gpu_run(wl, dev, 120, K=120))
    np.testing.assert_array_equal(a, gpu_run(wl, dev, 120, K=7, block=128))


def test_pid_zero_gains_is_bitwise_the_p_loop(dev):
    """kI = kD = 0: the PID kernel's 17 states are bit for bit the P-loop kernel's, whatever xi is."""
    wl = W.closed_loop_pid(n=4097)
    g = dict(wl.groups[0])
    g.update(kI=[0.0] * 3, kD=[0.0] * 3)
    x0 = wl.x0.copy()
    x0[:, 17:20] = np.random.default_rng(3).uniform(-1, 1, (wl.n, 3)).astype(np.float32)
    a = gpu_run(wl, dev, 200, K=50, x0=x0, groups=[g])
    wl17 = W.Workload("p", W.CLOSED_LOOP, [g], wl.gid, np.ascontiguousarray(x0[:, :17]), wl.cmd, wl.dt, 200)
    b = gpu_run(wl17, dev, 200, K=50)
    np.testing.assert_array_equal(a[:, :17], b)


def _hetero_pid(n_per=700):
    base = W.closed_loop_pid(n=3 * n_per)
    gs = []
    for i, (kI, kD, xm) in enumerate([(0.05, 0.005, 2.0), (0.08, 0.0, 0.5), (0.02, 0.01, 2.0)]):
        g = dict(W.scaled_group(0.5 + i, 500.0 + 150 * i))
        g.update(kI=[kI] * 3, kD=[kD] * 3, xi_max=[xm] * 3)
        gs.append(W.round_group(g))
    gid = np.random.default_rng(4).permutation(np.repeat(np.arange(3, dtype=np.uint8), n_per))
    x0 = base.x0.copy()
    x0[:, 13:17] = np.array([W.hover_speed(g) for g in gs], dtype=np.float32)[gid][:, None]
    return W.Workload("pid-hetero", W.CLOSED_LOOP_PID, gs, gid, x0, base.cmd, base.dt, 1000)


def test_pid_heterogeneous_parity(dev, orc):
    wl = _hetero_pid()
    check_traj(gpu_run(wl, dev, 1000, K=100), ref_run(orc, wl, 1000))


def test_pid_heterogeneous_is_bitwise_each_group_alone(dev):
    wl = _hetero_pid(300)
    both = gpu_run(wl, dev, 100, K=100)
    for gi in range(3):
        idx = np.flatnonzero(wl.gid == gi)
        one = W.Workload("one", W.CLOSED_LOOP_PID, [wl.groups[gi]], np.zeros(idx.size, np.uint8),
                         np.ascontiguousarray(wl.x0[idx]), np.ascontiguousarray(wl.cmd[idx]), wl.dt, 100)
        np.testing.assert_array_equal(both[idx], gpu_run(one, dev, 100, K=100))


def test_pid_graph_host_entry_and_rounds_are_bitwise_sim_step(dev):
    from paper_2308_12698_b300.sim import Sim, planar, unplanar
    wl = W.closed_loop_pid(n=150_001)
    direct = gpu_run(wl, dev, 30, K=10)
    sim = Sim(wl.groups, wl.n, wl.mode)
    x = planar(torch.from_numpy(wl.x0)).to(dev)
    cmd = torch.from_numpy(wl.cmd).to(dev).reshape(-1)
    gr = sim.graph(x, cmd, wl.dt, 30, K=10)
    gr.launch()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(unplanar(x, wl.n).cpu().numpy(), direct)
    gr.close()
    h_state = planar(torch.from_numpy(wl.x0)).pin_memory()
    h_cmd = torch.from_numpy(wl.cmd).reshape(-1).contiguous().pin_memory()
    d_state = torch.empty(20 * wl.n, device=dev)
    d_cmd = torch.empty(4 * wl.n, device=dev)
    sim.step_host(h_state, h_cmd, d_state, d_cmd, wl.dt, 30, K=10)
    np.testing.assert_array_equal(unplanar(h_state, wl.n).numpy(), direct)
    # decision rounds: 3 rounds of 10 steps with the same commands, positions observed after each
    x = planar(torch.from_numpy(wl.x0)).to(dev)
    h_cmds = torch.from_numpy(np.tile(wl.cmd.reshape(1, -1), (3, 1))).contiguous().pin_memory()
    h_obs = torch.empty((3, 4 * wl.n), dtype=torch.float32).pin_memory()
    sim.run_rounds(x, h_cmds, 10, wl.dt, K=10, h_obs=h_obs)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(unplanar(x, wl.n).cpu().numpy(), direct)
    np.testing.assert_array_equal(h_obs[2].numpy().reshape(wl.n, 4), direct[:, 0:4])
    sim.close()


SQRT_MARGIN, CLAMP_MARGIN = 1e-3, 1e-5


def check_grad(got, ref, what, loose=False):
    """The gradient bars of the P loop: strict 1e-3 |r| + 1e-4 max|r|, cosine >= 0.9999; near a
    kink 2e-2 |r| + 2e-3 max|r|, cosine >= 0.999."""
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    cos = got @ ref / (np.linalg.norm(got) * np.linalg.norm(ref) + 1e-300)
    a, b, c = (2e-2, 2e-3, 0.999) if loose else (1e-3, 1e-4, 0.9999)
    tol = a * np.abs(ref) + b * np.abs(ref).max()
    err = np.abs(got - ref)
    assert cos >= c and np.all(err <= tol), (what, cos, (err / tol).max())


def pid_grads(wl, dev, C, block_adj=0):
    from paper_2308_12698_b300.sim import Sim, planar, unplanar
    gid = torch.from_numpy(wl.gid).to(dev)
    sim = Sim(wl.groups, wl.n, wl.mode, gid=gid)
    if block_adj:
        sim.set_launch(block_adj=block_adj)
    x0 = planar(torch.from_numpy(wl.x0)).to(dev)
    cmd = torch.from_numpy(wl.cmd).to(dev).reshape(-1)
    ckpt, rc = sim.rollout_forward(x0, cmd, wl.dt, wl.nsteps, C=C)
    xT = unplanar(ckpt[-1], wl.n)
    g = torch.zeros_like(xT)
    g[:, 0:3] = 2 * (xT[:, 0:3] - torch.from_numpy(wl.goal).to(dev))
    w = torch.full((wl.n,), wl.w_omega, device=dev)
    dx0, dth, dtha = sim.rollout_backward(ckpt, cmd, wl.dt, wl.nsteps, planar(g), w, C=C, per_agent=True)
    torch.cuda.synchronize()
    out = (unplanar(dx0, wl.n).cpu().numpy(), dth.cpu().numpy(), dtha.cpu().numpy(), xT.cpu().numpy(),
           rc.cpu().numpy())
    sim.close()
    return out


def test_pid_rollout_forward_is_bitwise_sim_step(dev, orc):
    """The checkpointed forward runs the same PID step: its last checkpoint equals sim_step's
    state bit for bit, and its running cost matches the checker's."""
    wl = W.differentiable_pid(n_per_group=300, n_groups=3, nsteps=400)
    _, _, _, xT, rc = pid_grads(wl, dev, C=50)
    from paper_2308_12698_b300.sim import Sim, planar, unplanar
    sim = Sim(wl.groups, wl.n, wl.mode, gid=torch.from_numpy(wl.gid).to(dev))
    x = planar(torch.from_numpy(wl.x0)).to(dev)
    sim.step(x, torch.from_numpy(wl.cmd).to(dev).reshape(-1), wl.dt, wl.nsteps, K=37)
    np.testing.assert_array_equal(unplanar(x, wl.n).cpu().numpy(), xT)
    sim.close()
    _, rref = orc.rollout(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, wl.nsteps, wl.mode, with_cost=True)
    np.testing.assert_allclose(rc, rref, rtol=2e-4)


def test_pid_adjoint_matches_fp64_reverse_mode(dev, orc):
    """Per-agent dL/dtheta and dL/dx0 (20 components, the integral included) against the
    checker's reverse mode on the PID step; agents whose FP64 trajectory comes near a kink (rotor
    demand near 0 or the ceiling, acceleration or integrator clamp) take the looser bar."""
    wl = W.differentiable_pid(n_per_group=16, n_groups=4, nsteps=2000)
    dx0, dth, dtha, _, _ = pid_grads(wl, dev, C=100)
    _, rdx0, rdth = orc.grad(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, wl.nsteps, wl.mode, wl.goal, wl.w_omega)
    m = orc.clamp_margins(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, wl.nsteps, mode=wl.mode)
    fl = (m[:, 0] < SQRT_MARGIN) | (m[:, 1] < CLAMP_MARGIN) | (m[:, 2] < CLAMP_MARGIN)
    assert (~fl).sum() >= 16, fl.sum()
    assert np.abs(rdx0[:, 17:20]).max() > 0
    for a in range(wl.n):
        check_grad(dtha[a], rdth[a], f"theta agent {a}", loose=fl[a])
        check_grad(dx0[a], rdx0[a], f"x0 agent {a}", loose=fl[a])
    for gi in range(len(wl.groups)):
        check_grad(dth[gi], rdth[wl.gid == gi].sum(axis=0), f"theta group {gi}", loose=True)


def test_pid_adjoint_shared_and_global_scratch_agree(dev):
    """C = 2 keeps the segment in shared memory, C = 40 in the global workspace: same
    checkpointed states and per-step arithmetic, so per-agent gradients agree bit for bit."""
    wl = W.differentiable_pid(n_per_group=500, n_groups=2, nsteps=200)
    a = pid_grads(wl, dev, C=2)
    b = pid_grads(wl, dev, C=40)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[2], b[2])


def test_pid_empty_swarm(dev):
    from paper_2308_12698_b300.sim import Sim
    sim = Sim([W.pid_group()], 0, W.CLOSED_LOOP_PID)
    x = torch.zeros(0, device=dev)
    sim.step(x, torch.zeros(0, device=dev), 1e-3, 10)
    assert sim.n_dead() == 0
    sim.close()


def test_pid_full_size_sampled(dev, orc):
    """The bench's PID leg (1e6 agents, one launch of K = 1000): 2048 sampled agents."""
    from paper_2308_12698_b300.sim import Sim, planar, unplanar
    wl = W.closed_loop_pid(n=1_000_000, nsteps=1000)
    sim = Sim(wl.groups, wl.n, wl.mode)
    x = planar(torch.from_numpy(wl.x0)).to(dev)
    sim.step(x, torch.from_numpy(wl.cmd).to(dev).reshape(-1), wl.dt, 1000, K=1000)
    idx = np.random.default_rng(21).choice(wl.n, 2048, replace=False)
    got = unplanar(x, wl.n)[torch.from_numpy(idx).to(dev)].cpu().numpy()
    ref = orc.rollout(wl.groups, wl.gid[idx], wl.x0[idx], wl.cmd[idx], wl.dt, 1000, wl.mode)
    check_traj(got, ref)
    assert sim.n_dead() == 0
    sim.close()


def test_pid_autograd_function(dev):
    """torch.autograd through QuadRollout in the PID mode equals the direct adjoint call."""
    from paper_2308_12698_b300.sim import QuadRollout, Sim, planar, unplanar
    wl = W.differentiable_pid(n_per_group=64, n_groups=2, nsteps=300)
    sim = Sim(wl.groups, wl.n, wl.mode, gid=torch.from_numpy(wl.gid).to(dev))
    theta = torch.tensor(sim.theta(), requires_grad=True)
    x0 = planar(torch.from_numpy(wl.x0)).to(dev).requires_grad_(True)
    cmd = torch.from_numpy(wl.cmd).to(dev).reshape(-1)
    goal = torch.from_numpy(wl.goal).to(dev)
    xT, rc = QuadRollout.apply(theta, x0, sim, cmd, wl.dt, wl.nsteps, 30)
    loss = ((unplanar(xT, wl.n)[:, 0:3] - goal) ** 2).sum() + wl.w_omega * rc.sum()
    loss.backward()
    sim.close()
    dx0, dth, _, _, _ = pid_grads(wl, dev, C=30)
    np.testing.assert_allclose(theta.grad.cpu().numpy(), dth, rtol=1e-5, atol=1e-6 * np.abs(dth).max())
    np.testing.assert_allclose(unplanar(x0.grad, wl.n).cpu().numpy(), dx0, rtol=1e-5, atol=1e-7)
    assert x0.grad.shape[0] == 20 * wl.n
