"""Differentiable rollout on the GPU: the hand-written FP32 adjoint against the
checker's FP64 reverse mode and FP64 central differences.

Loss = sum_a |p_T - goal_a|^2 + w sum_a sum_{n=1..T} sum_i Omega_{n,i}^2.
Acceptance per gradient block (theta of one agent or group: 16 values;
dL/dx0 of one agent: 17 values): cosine >= 0.9999, and every component within
1e-3 of itself plus 1e-4 of the block's largest component.  The floor is the
FP32 accumulation bound: a 2000-step adjoint of ~1e3 operations per step
carries a random-walk rounding error of order sqrt(2e6) * 6e-8 ~ 1e-4 of the
block's scale, which a purely component-relative bar would charge to its
smallest components.

Agents whose trajectory passes next to a kink of the controller are flagged
(from the FP64 trajectory): a rotor demand S = Omega_cmd^2 within 1e-3
Omega_max^2 of 0 (sqrt has an unbounded derivative there and S is a difference
of terms ~Omega_max^2, so rounding-level state noise moves that step's
contribution by ~eps Omega_max^2 / S), or within 1e-5 of the rotor ceiling or
of the acceleration clamp.  Flagged agents are reported separately and held
to a conditioning bar (cosine >= 0.999, components within 2e-2 of themselves
plus 2e-3 of the block's largest); unflagged agents to the bar above.
"""
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


SQRT_MARGIN, CLAMP_MARGIN = 1e-3, 1e-5


def flagged(orc, wl, idx=None):
    sel = slice(None) if idx is None else idx
    m = orc.clamp_margins(wl.groups, wl.gid[sel], wl.x0[sel], wl.cmd[sel], wl.dt, wl.nsteps)
    return (m[:, 0] < SQRT_MARGIN) | (m[:, 1] < CLAMP_MARGIN) | (m[:, 2] < CLAMP_MARGIN)


def check_loose(got, ref, what):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    cos = got @ ref / (np.linalg.norm(got) * np.linalg.norm(ref) + 1e-300)
    err = np.abs(got - ref)
    tol = 2e-2 * np.abs(ref) + 2e-3 * np.abs(ref).max()
    assert cos >= 0.999 and np.all(err <= tol), (what, cos, err / tol)


def check_block(got, ref, what):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    cos = got @ ref / (np.linalg.norm(got) * np.linalg.norm(ref) + 1e-300)
    err = np.abs(got - ref)
    tol = 1e-3 * np.abs(ref) + 1e-4 * np.abs(ref).max()
    worst = int(np.argmax(err / tol))
    assert cos >= 0.9999 and np.all(err <= tol), (what, cos, worst, err[worst] / tol[worst], got[worst], ref[worst])


def gpu_grad(wl, dev, C, per_agent=True, run=1):
    from paper_2308_12698_b300.sim import Sim, planar, unplanar
    gid = torch.from_numpy(wl.gid).to(dev)
    sim = Sim(wl.groups, wl.n, wl.mode, gid=gid)
    x0 = planar(torch.from_numpy(wl.x0)).to(dev)
    cmd = torch.from_numpy(wl.cmd).to(dev).reshape(-1)
    ckpt, rc = sim.rollout_forward(x0, cmd, wl.dt, wl.nsteps, C=C)
    xT = unplanar(ckpt[-1], wl.n)
    goal = torch.from_numpy(wl.goal).to(dev)
    d = xT[:, 0:3] - goal
    loss = (d * d).sum(dim=1) + wl.w_omega * rc
    g = torch.zeros_like(xT)
    g[:, 0:3] = 2 * d
    w = torch.full((wl.n,), wl.w_omega, device=dev)
    outs = []
    for _ in range(run):
        dx0, dth, dth_a = sim.rollout_backward(ckpt, cmd, wl.dt, wl.nsteps, planar(g), w, C=C, per_agent=per_agent)
        torch.cuda.synchronize()
        outs.append((unplanar(dx0, wl.n).cpu().numpy(), dth.cpu().numpy(),
                     None if dth_a is None else dth_a.cpu().numpy()))
    res = dict(loss=loss.cpu().numpy(), rc=rc.cpu().numpy(), xT=xT.cpu().numpy(), outs=outs)
    sim.close()
    return res


def test_adjoint_matches_fp64_reverse_mode(dev, orc):
    wl = W.differentiable(n_per_group=8, n_groups=4, nsteps=2000)
    r = gpu_grad(wl, dev, C=100)
    dx0, dth, dth_a = r["outs"][0]
    loss, rdx0, rdth = orc.grad(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, wl.nsteps, wl.mode, wl.goal, wl.w_omega)
    np.testing.assert_allclose(r["loss"], loss, rtol=2e-4, atol=1e-6)
    fl = flagged(orc, wl)
    assert (~fl).sum() >= 8, fl.sum()
    for a in range(wl.n):
        chk = check_loose if fl[a] else check_block
        chk(dth_a[a], rdth[a], f"theta agent {a}")
        chk(dx0[a], rdx0[a], f"x0 agent {a}")
    for gi in range(len(wl.groups)):
        check_loose(dth[gi], rdth[wl.gid == gi].sum(axis=0), f"theta group {gi}")


def gentle(n_per_group, n_groups, nsteps):
    """Start at rest, level, at the commanded heading, 0.1 m from the goal, headings over all of
    [-pi, pi) (every Shepperd branch of the desired attitude): no agent comes near a kink."""
    base = W.differentiable(n_per_group=n_per_group, n_groups=n_groups, nsteps=nsteps)
    rng = np.random.default_rng(11)
    goal = (base.x0[:, 0:3] + rng.uniform(-0.1, 0.1, (base.n, 3))).astype(np.float32)
    cmd = base.cmd.copy()
    cmd[:, 0:3] = goal
    cmd[:, 3] = np.linspace(-np.pi, np.pi, base.n, endpoint=False).astype(np.float32)
    x0 = base.x0.copy()
    half = cmd[:, 3].astype(np.float64) / 2  # start level at the commanded heading
    x0[:, 6:10] = np.stack([np.cos(half), 0 * half, 0 * half, np.sin(half)], 1).astype(np.float32)
    x0[:, 3:6] = 0.0
    x0[:, 10:13] = 0.0
    return W.Workload("gentle", base.mode, base.groups, base.gid, x0, cmd, base.dt, base.nsteps, goal=goal,
                      w_omega=1e-6)


def test_adjoint_gentle_rollout_every_agent_strict(dev, orc):
    """No agent of the gentle rollout comes near a kink, so every agent meets the strict bar."""
    wl = gentle(64, 2, 400)
    assert not flagged(orc, wl).any()
    r = gpu_grad(wl, dev, C=50)
    dx0, dth, dth_a = r["outs"][0]
    _, rdx0, rdth = orc.grad(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, wl.nsteps, wl.mode, wl.goal, wl.w_omega)
    for a in range(wl.n):
        check_block(dth_a[a], rdth[a], f"theta agent {a}")
        check_block(dx0[a], rdx0[a], f"x0 agent {a}")
    for gi in range(len(wl.groups)):
        check_block(dth[gi], rdth[wl.gid == gi].sum(axis=0), f"theta group {gi}")


#: theta's parameter families (gains per loop, mass, inertia): their units and scales differ
THETA_FAMILIES = {"kp": slice(0, 3), "kd": slice(3, 6), "katt": slice(6, 9), "krate": slice(9, 12),
                  "m": slice(12, 13), "J": slice(13, 16)}


def test_group_sums_strict_against_fp64(dev, orc):
    """The per-group reduction (warp butterflies, per-warp accumulators, per-block partials, the
    fixed-order second pass) on 4,096 kink-free agents in 4 airframe groups: each group's
    dL/dtheta_g against the sum of the FP64 reverse mode's per-agent gradients over that group,
    at the strict bar, on the whole 16-vector and on each parameter family alone (so that the
    mass gradient, orders of magnitude above the gains', sets no floor for them)."""
    wl = gentle(1024, 4, 400)
    assert not flagged(orc, wl).any()
    r = gpu_grad(wl, dev, C=50, per_agent=False)
    _, dth, _ = r["outs"][0]
    _, _, rdth = orc.grad(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, wl.nsteps, wl.mode, wl.goal, wl.w_omega)
    worst = 0.0
    for gi in range(len(wl.groups)):
        ref = rdth[wl.gid == gi].sum(axis=0)
        check_block(dth[gi], ref, f"theta group {gi}")
        for fam, sl in THETA_FAMILIES.items():
            check_block(dth[gi][sl], ref[sl], f"theta group {gi} {fam}")
        worst = max(worst, float(np.max(np.abs(dth[gi] - ref) / np.abs(ref))))
    print(f"group sums: worst component relative error {worst:.2e}")


def test_running_cost_matches(dev, orc):
    wl = W.differentiable(n_per_group=16, n_groups=2, nsteps=500)
    r = gpu_grad(wl, dev, C=50, per_agent=False)
    xT, rc = orc.rollout(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, wl.nsteps, wl.mode, with_cost=True)
    np.testing.assert_allclose(r["rc"], rc, rtol=1e-5)
    np.testing.assert_allclose(r["xT"][:, 0:3], xT[:, 0:3], rtol=0, atol=1e-3)


@pytest.mark.parametrize("nsteps,C", [(250, 100), (37, 5), (100, 1), (64, 200)])
def test_segment_tails(dev, orc, nsteps, C):
    wl = W.differentiable(n_per_group=4, n_groups=2, nsteps=nsteps)
    r = gpu_grad(wl, dev, C=C)
    dx0, dth, dth_a = r["outs"][0]
    _, rdx0, rdth = orc.grad(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, wl.nsteps, wl.mode, wl.goal, wl.w_omega)
    fl = flagged(orc, wl)
    for a in range(wl.n):
        chk = check_loose if fl[a] else check_block
        chk(dth_a[a], rdth[a], f"theta agent {a}")
        chk(dx0[a], rdx0[a], f"x0 agent {a}")


def test_open_loop_adjoint(dev, orc):
    base = W.open_loop(n=16, nsteps=300)
    goal = base.x0[:, 0:3] + 1.0
    wl = W.Workload("ol", base.mode, base.groups, base.gid, base.x0, base.cmd, base.dt, 300, goal=goal,
                    w_omega=1e-6)
    r = gpu_grad(wl, dev, C=30)
    dx0, dth, dth_a = r["outs"][0]
    _, rdx0, rdth = orc.grad(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, wl.nsteps, wl.mode, wl.goal, wl.w_omega)
    assert np.all(dth_a[:, :12] == 0)  # gains do not act open loop
    for a in range(wl.n):
        check_block(dth_a[a, 12:], rdth[a, 12:], f"m,J agent {a}")
        check_block(dx0[a], rdx0[a], f"x0 agent {a}")


def test_adjoint_is_deterministic(dev):
    wl = W.differentiable(n_per_group=300, n_groups=3, nsteps=200)
    r = gpu_grad(wl, dev, C=50, run=2)
    (a0, b0, c0), (a1, b1, c1) = r["outs"]
    np.testing.assert_array_equal(a0, a1)
    np.testing.assert_array_equal(b0, b1)
    np.testing.assert_array_equal(c0, c1)
    # group sums are the per-agent contributions summed
    for gi in range(3):
        np.testing.assert_allclose(b0[gi], c0[wl.gid == gi].astype(np.float64).sum(axis=0), rtol=1e-4,
                                   atol=1e-6 * np.abs(b0[gi]).max())


def _fd_theta(orc, wl, agents, h=1e-6):
    """FP64 central differences of each sampled agent's loss w.r.t. its 16 group parameters."""
    from paper_2308_12698_b300.sim import theta_of, with_theta
    groups, gid, x0, cmd, goal, meta = [], [], [], [], [], []
    for a in agents:
        g0 = wl.groups[wl.gid[a]]
        th = np.array(theta_of(g0))
        for k in range(16):
            for s in (+1, -1):
                t = th.copy()
                t[k] += s * h * abs(th[k])
                groups.append(with_theta(g0, t))
                gid.append(len(groups) - 1)
                x0.append(wl.x0[a])
                cmd.append(wl.cmd[a])
                goal.append(wl.goal[a])
                meta.append((a, k, s, h * abs(th[k])))
    L = orc.loss(groups, np.array(gid), np.array(x0), np.array(cmd), wl.dt, wl.nsteps, wl.mode, np.array(goal),
                 wl.w_omega)
    out = np.zeros((len(agents), 16))
    for j in range(0, len(meta), 2):
        a, k, _, step = meta[j]
        out[list(agents).index(a), k] = (L[j] - L[j + 1]) / (2 * step)
    return out


def test_full_size_adjoint_sampled_against_fd(dev, orc):
    """4096 agents in 4 groups, 2000 steps, C = 100; 16 sampled agents checked against FP64
    reverse mode (theta and x0) and FP64 central differences (theta)."""
    wl = W.differentiable()
    r = gpu_grad(wl, dev, C=100)
    dx0, dth, dth_a = r["outs"][0]
    # 16 agents: the first 8 unflagged and the first 8 flagged of a seeded permutation
    perm = np.random.default_rng(5).permutation(wl.n)[:256]
    fl = flagged(orc, wl, perm)
    agents = np.concatenate([perm[~fl][:8], perm[fl][:8]])
    fla = np.concatenate([np.zeros(8, bool), np.ones(len(agents) - 8, bool)])
    sub = lambda v: v[agents]  # noqa: E731
    groups_sub = wl.groups
    _, rdx0, rdth = orc.grad(groups_sub, sub(wl.gid), sub(wl.x0), sub(wl.cmd), wl.dt, wl.nsteps, wl.mode,
                             sub(wl.goal), wl.w_omega)
    fd = _fd_theta(orc, wl, agents)
    # worst component error as a fraction of the strict bar 1e-3 |r| + 1e-4 max|r| (1 = at the bar)
    rel = lambda g, r: float(np.max(np.abs(g - r) / (1e-3 * np.abs(r) + 1e-4 * np.abs(r).max())))  # noqa: E731
    cosine = lambda g, r: float(g @ r / (np.linalg.norm(g) * np.linalg.norm(r)))  # noqa: E731
    strict = [j for j in range(len(agents)) if not fla[j]]
    print(f"differentiable workload: {fl.mean():.3f} of 256 sampled agents flagged at a kink; unflagged agents, "
          f"worst error as a fraction of the strict bar: theta vs FP64 reverse "
          f"{max(rel(dth_a[agents[j]], rdth[j]) for j in strict):.3f} "
          f"(cosine >= {min(cosine(dth_a[agents[j]], rdth[j]) for j in strict):.7f}), theta vs FD "
          f"{max(rel(dth_a[agents[j]], fd[j]) for j in strict):.3f}, x0 vs reverse "
          f"{max(rel(dx0[agents[j]], rdx0[j]) for j in strict):.3f}; flagged agents theta vs reverse "
          f"{max(rel(dth_a[agents[j]], rdth[j]) for j in range(len(agents)) if fla[j]):.3f} of the strict bar")
    for j, a in enumerate(agents):
        if fla[j]:
            # FD itself straddles the kink for these; reverse mode is the reference
            check_loose(dth_a[a], rdth[j], f"theta agent {a} vs reverse (flagged)")
            check_loose(dx0[a], rdx0[j], f"x0 agent {a} vs reverse (flagged)")
        else:
            check_block(dth_a[a], rdth[j], f"theta agent {a} vs reverse")
            check_block(dx0[a], rdx0[j], f"x0 agent {a} vs reverse")
            check_block(dth_a[a], fd[j], f"theta agent {a} vs FD")


def test_autograd_function(dev):
    from paper_2308_12698_b300.sim import QuadRollout, Sim, planar, unplanar
    wl = W.differentiable(n_per_group=64, n_groups=2, nsteps=300)
    gid = torch.from_numpy(wl.gid).to(dev)
    sim = Sim(wl.groups, wl.n, wl.mode, gid=gid)
    theta = torch.tensor(sim.theta(), requires_grad=True)
    x0 = planar(torch.from_numpy(wl.x0)).to(dev).requires_grad_(True)
    cmd = torch.from_numpy(wl.cmd).to(dev).reshape(-1)
    goal = torch.from_numpy(wl.goal).to(dev)
    xT, rc = QuadRollout.apply(theta, x0, sim, cmd, wl.dt, wl.nsteps, 30)
    p = unplanar(xT, wl.n)[:, 0:3]
    loss = ((p - goal) ** 2).sum() + wl.w_omega * rc.sum()
    loss.backward()
    ref = gpu_grad(wl, dev, C=30, per_agent=False)
    dx0, dth, _ = ref["outs"][0]
    np.testing.assert_allclose(theta.grad.cpu().numpy(), dth, rtol=1e-5, atol=1e-6 * np.abs(dth).max())
    np.testing.assert_allclose(unplanar(x0.grad, wl.n).cpu().numpy(), dx0, rtol=1e-5, atol=1e-7)
    sim.close()


def test_autograd_two_forwards_at_different_theta(dev):
    """Two rollouts of one handle at different theta, summed into one loss: each backward runs
    under the theta its own forward used, so the gradients equal separate forward/backward pairs
    on handles of their own, bit for bit; the handle keeps the later forward's theta."""
    from paper_2308_12698_b300.sim import QuadRollout, Sim, planar, unplanar, with_theta
    wl = W.differentiable(n_per_group=64, n_groups=2, nsteps=200)
    gid = torch.from_numpy(wl.gid).to(dev)
    sim = Sim(wl.groups, wl.n, wl.mode, gid=gid)
    th0 = sim.theta()
    th1 = th0.copy()
    th1[:, 0:3] *= 1.25  # kp
    th1[:, 12] *= 1.1  # mass
    x0 = planar(torch.from_numpy(wl.x0)).to(dev)
    cmd = torch.from_numpy(wl.cmd).to(dev).reshape(-1)
    goal = torch.from_numpy(wl.goal).to(dev)

    def loss_of(xT, rc):
        p = unplanar(xT, wl.n)[:, 0:3]
        return ((p - goal) ** 2).sum() + wl.w_omega * rc.sum()

    ta, tb = torch.tensor(th0, requires_grad=True), torch.tensor(th1, requires_grad=True)
    xa, xb = x0.clone().requires_grad_(True), x0.clone().requires_grad_(True)
    loss = loss_of(*QuadRollout.apply(ta, xa, sim, cmd, wl.dt, wl.nsteps, 20)) + \
        loss_of(*QuadRollout.apply(tb, xb, sim, cmd, wl.dt, wl.nsteps, 20))
    loss.backward()
    assert np.array_equal(sim.theta(), th1)
    assert not torch.equal(ta.grad, tb.grad)
    for th, tgrad, xgrad in ((th0, ta.grad, xa.grad), (th1, tb.grad, xb.grad)):
        alone = Sim([with_theta(g, t) for g, t in zip(wl.groups, th)], wl.n, wl.mode, gid=gid)
        t = torch.tensor(th, requires_grad=True)
        x = x0.clone().requires_grad_(True)
        loss_of(*QuadRollout.apply(t, x, alone, cmd, wl.dt, wl.nsteps, 20)).backward()
        assert torch.equal(t.grad, tgrad)
        assert torch.equal(x.grad, xgrad)
        alone.close()
    sim.close()


def test_shared_and_global_scratch_agree(dev):
    """C = 8 keeps the segment in shared memory, C = 40 in the global workspace, C = 1 needs no
    scratch at all: the same checkpointed or recomputed states and per-step arithmetic, so
    per-agent gradients are bitwise equal."""
    from paper_2308_12698_b300.sim import Sim, planar
    wl = W.differentiable(n_per_group=500, n_groups=3, nsteps=240)
    gid = torch.from_numpy(wl.gid).to(dev)
    sim = Sim(wl.groups, wl.n, wl.mode, gid=gid)
    sim.set_launch(block_adj=128)  # 40 steps x 68 B x 128 threads exceed the shared-memory scratch
    x0 = planar(torch.from_numpy(wl.x0)).to(dev)
    cmd = torch.from_numpy(wl.cmd).reshape(-1).to(dev)
    gT = torch.zeros(17 * wl.n, device=dev)
    gT[: 3 * wl.n] = 1.0
    w = torch.full((wl.n,), wl.w_omega, device=dev)
    out = {}
    for C in (1, 8, 40):
        ckpt, _ = sim.rollout_forward(x0, cmd, wl.dt, wl.nsteps, C=C)
        assert sim.workspace_bytes(C) > 0
        out[C] = sim.rollout_backward(ckpt, cmd, wl.dt, wl.nsteps, gT, w, C=C, per_agent=True)
    torch.cuda.synchronize()
    assert sim.workspace_bytes(8) < sim.workspace_bytes(40)  # no global scratch for C = 8
    assert torch.equal(out[8][0], out[40][0]) and torch.equal(out[1][0], out[40][0])
    assert torch.equal(out[8][2], out[40][2]) and torch.equal(out[1][2], out[40][2])
    np.testing.assert_allclose(out[8][1].cpu().numpy(), out[40][1].cpu().numpy(), rtol=1e-5,
                               atol=1e-6 * out[40][1].abs().max().item())
    sim.close()


@pytest.mark.parametrize("C,block_adj", [(1, 128), (2, 64)])
def test_adjoint_full_size_bench_configuration(dev, orc, C, block_adj):
    """1e6 agents x 1000 steps in the launch shapes the bench's autotuner picks (C = 1 or 2,
    shared scratch, 128- or 64-thread blocks): 24 sampled agents' gradients against FP64
    reverse mode."""
    from paper_2308_12698_b300.sim import Sim, planar, unplanar
    base = W.scale_sweep(1_000_000, nsteps=1000)
    goal = base.cmd[:, 0:3].copy()
    wl = W.Workload("full", base.mode, base.groups, base.gid, base.x0, base.cmd, base.dt, 1000, goal=goal,
                    w_omega=1e-6)
    sim = Sim(wl.groups, wl.n, wl.mode)
    sim.set_launch(block_adj=block_adj)
    x0 = planar(torch.from_numpy(wl.x0)).to(dev)
    cmd = torch.from_numpy(wl.cmd).reshape(-1).to(dev)
    ckpt, rc = sim.rollout_forward(x0, cmd, wl.dt, wl.nsteps, C=C)
    xT = unplanar(ckpt[-1], wl.n)
    g = torch.zeros_like(xT)
    g[:, 0:3] = 2 * (xT[:, 0:3] - torch.from_numpy(goal).to(dev))
    w = torch.full((wl.n,), wl.w_omega, device=dev)
    dx0, dth, dtha = sim.rollout_backward(ckpt, cmd, wl.dt, wl.nsteps, planar(g), w, C=C, per_agent=True)
    torch.cuda.synchronize()
    idx = np.random.default_rng(12).choice(wl.n, 24, replace=False)
    sel = torch.from_numpy(idx).to(dev)
    got_dx = unplanar(dx0, wl.n)[sel].cpu().numpy()
    got_th = dtha[sel].cpu().numpy()
    _, rdx0, rdth = orc.grad(wl.groups, wl.gid[idx], wl.x0[idx], wl.cmd[idx], wl.dt, wl.nsteps, wl.mode, goal[idx],
                             wl.w_omega)
    m = orc.clamp_margins(wl.groups, wl.gid[idx], wl.x0[idx], wl.cmd[idx], wl.dt, wl.nsteps)
    fl = (m[:, 0] < SQRT_MARGIN) | (m[:, 1] < CLAMP_MARGIN) | (m[:, 2] < CLAMP_MARGIN)
    for j in range(len(idx)):
        chk = check_loose if fl[j] else check_block
        chk(got_th[j], rdth[j], f"theta agent {idx[j]}")
        chk(got_dx[j], rdx0[j], f"x0 agent {idx[j]}")
    # the group sum is the sum of the per-agent contributions
    np.testing.assert_allclose(dth.cpu().numpy()[0], dtha.double().sum(0).cpu().numpy(), rtol=1e-4,
                               atol=1e-6 * dth.abs().max().item())
    sim.close()


def test_adjoint_thrust_pointing_down(dev, orc):
    """Gradients through the roll half-angle's second formula (demanded force pointing down,
    inverted and upright bodies, all headings): 5-step rollouts against FP64 reverse mode."""
    wl = W.thrust_down(2048, nsteps=5)
    g = wl.groups[0]
    az = np.clip(g["kp"][2] * (wl.cmd[:, 2].astype(np.float64) - wl.x0[:, 2]) - g["kd"][2] * wl.x0[:, 5],
                 -g["a_max"], g["a_max"])
    down = az + g["g"] < 0  # first demanded force points down
    r = gpu_grad(wl, dev, C=5)
    dx0, _, dth_a = r["outs"][0]
    _, rdx0, rdth = orc.grad(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, wl.nsteps, wl.mode, wl.goal, wl.w_omega)
    fl = flagged(orc, wl)
    strict = ~fl & down
    assert strict.sum() > 500, strict.sum()
    for a in np.flatnonzero(~fl):
        check_block(dth_a[a], rdth[a], f"theta agent {a}")
        check_block(dx0[a], rdx0[a], f"x0 agent {a}")
    for a in np.flatnonzero(fl):
        check_loose(dx0[a], rdx0[a], f"x0 agent {a} (near a kink)")


@pytest.mark.parametrize("pid", [False, True])
def test_dead_agents_get_the_frozen_gradient(dev, pid):
    """Agents marked dead before the rollout are frozen through it (checkpoints x_0, running cost 0),
    so the adjoint gives them dL/dx_0 = dL/dx_T, zero per-agent theta rows and no share of the group
    sums (the output buffers start as NaN: every element is written).  The live agents' gradients
    are bit for bit those of the same swarm with nobody dead."""
    import ctypes

    from paper_2308_12698_b300 import _lib
    from paper_2308_12698_b300.sim import Sim, planar
    wl = (W.differentiable_pid if pid else W.differentiable)(n_per_group=300, n_groups=2, nsteps=120)
    gid = torch.from_numpy(wl.gid).to(dev)
    x0 = planar(torch.from_numpy(wl.x0)).to(dev)
    cmd = torch.from_numpy(wl.cmd).to(dev).reshape(-1)
    gT = torch.randn(x0.numel(), generator=torch.Generator().manual_seed(3)).to(dev)
    w = torch.full((wl.n,), wl.w_omega, device=dev)
    dead = np.zeros(wl.n, np.uint8)
    dead[::5] = 2
    out = {}
    for name, status in (("all_alive", np.zeros(wl.n, np.uint8)), ("some_dead", dead)):
        sim = Sim(wl.groups, wl.n, wl.mode, gid=gid)
        sim.load_status(torch.from_numpy(status).to(dev))
        ckpt, rc = sim.rollout_forward(x0, cmd, wl.dt, wl.nsteps, C=40)
        ws = sim.workspace_bytes(40)
        buf = torch.empty(ws, dtype=torch.uint8, device=dev)
        dx0 = torch.full_like(x0, float("nan"))
        dth = torch.full((2, 16), float("nan"), device=dev)
        dtha = torch.full((wl.n, 16), float("nan"), device=dev)
        p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
        assert _lib.lib().sim_rollout_backward(sim.handle, p(ckpt), p(cmd), wl.dt, wl.nsteps, 40, p(gT), p(w),
                                               p(dx0), p(dth), p(dtha), p(buf), ws, None) == _lib.SIM_OK
        torch.cuda.synchronize()
        out[name] = (ckpt, rc, dx0, dth, dtha)
        sim.close()
    from paper_2308_12698_b300.sim import unplanar
    ckpt, rc, dx0, dth, dtha = out["some_dead"]
    d = torch.from_numpy(dead != 0).to(dev)
    assert torch.equal(unplanar(ckpt[-1], wl.n)[d], unplanar(x0, wl.n)[d])
    assert torch.all(rc[d] == 0)
    assert torch.equal(unplanar(dx0, wl.n)[d], unplanar(gT, wl.n)[d])
    assert torch.all(dtha[d] == 0)
    a = out["all_alive"]
    assert torch.equal(unplanar(dx0, wl.n)[~d], unplanar(a[2], wl.n)[~d])
    assert torch.equal(dtha[~d], a[4][~d])
    assert bool(torch.isfinite(dth).all())
    live = ~d.cpu().numpy()
    ref = np.stack([dtha.cpu().numpy()[live & (wl.gid == g)].astype(np.float64).sum(axis=0) for g in range(2)])
    np.testing.assert_allclose(dth.cpu().numpy(), ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())


@pytest.mark.parametrize("n,pid", [(1, False), (3, False), (5, False), (33, False), (1001, False), (3, True),
                                   (1001, True)])
def test_rollout_and_adjoint_any_agent_count(dev, orc, n, pid):
    """Checkpoint states start 16-byte aligned whatever the agent count: the stride from one to the
    next is the state's 17 N (20 N) floats rounded up to a multiple of 4.  A swarm of N agents, N not
    a multiple of 4, gives bit for bit the checkpoints and per-agent gradients of the same agents in
    a swarm whose count is (whose checkpoints need no gap), and the unflagged agents meet the strict
    bar against the checker's reverse mode."""
    from paper_2308_12698_b300.sim import Sim, planar, unplanar
    nx = 20 if pid else 17
    big = (W.differentiable_pid if pid else W.differentiable)(n_per_group=(n + 3) // 4 * 4 + 4, n_groups=1,
                                                              nsteps=90)
    cut = lambda v: np.ascontiguousarray(v[:n])  # noqa: E731
    wl = W.Workload("odd", big.mode, big.groups, cut(big.gid), cut(big.x0), cut(big.cmd), big.dt, big.nsteps,
                    goal=cut(big.goal), w_omega=big.w_omega)
    res = {}
    for name, w in (("odd", wl), ("aligned", big)):
        sim = Sim(w.groups, w.n, w.mode)
        x0 = planar(torch.from_numpy(w.x0)).to(dev)
        ckpt, _ = sim.rollout_forward(x0, torch.from_numpy(w.cmd).to(dev).reshape(-1), w.dt, w.nsteps, C=20)
        torch.cuda.synchronize()
        assert ckpt.shape == (6, nx * w.n) and ckpt.stride(0) == (nx * w.n + 3) // 4 * 4
        cks = np.stack([unplanar(ckpt[s], w.n).cpu().numpy()[:n] for s in range(6)])
        sim.close()
        r = gpu_grad(w, dev, C=20)
        dx0, _, dth_a = r["outs"][0]
        res[name] = (cks, dx0[:n], dth_a[:n])
    for a, b in zip(res["odd"], res["aligned"]):
        np.testing.assert_array_equal(a, b)
    _, rdx0, rdth = orc.grad(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, wl.nsteps, wl.mode, wl.goal, wl.w_omega)
    m = orc.clamp_margins(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, wl.nsteps, mode=wl.mode)
    fl = (m[:, 0] < SQRT_MARGIN) | (m[:, 1] < CLAMP_MARGIN) | (m[:, 2] < CLAMP_MARGIN)
    _, dx0, dth_a = res["odd"]
    for a in np.flatnonzero(~fl):
        chk = check_loose if pid else check_block
        chk(dth_a[a], rdth[a], f"theta agent {a}")
        chk(dx0[a], rdx0[a], f"x0 agent {a}")
