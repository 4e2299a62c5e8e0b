"""sim_compact: only the live agents are stepped (Sec. III-A: agents marked dead are
excluded from the computation).

The live agents' order changes which warp holds which agent, never an agent's
arithmetic: every case compares a compacted handle with an uncompacted one bit
for bit, state and status bytes, over launches that take the order (2 steps or
more, any K for mixed agent types) and launches that do not (K = 1).
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


def _workload(kind):
    if kind == "one_group":
        return W.closed_loop(n=5000, nsteps=100)
    if kind == "contiguous":
        return W.heterogeneous(sizes=(700, 1000, 300, 5), nsteps=100, shuffle=False)
    if kind == "interleaved":
        return W.heterogeneous(sizes=(700, 1000, 300, 5), nsteps=100, shuffle=True)
    if kind == "mixed_types":
        return W.multi_type(sizes=(600, 500, 400), nsteps=100, shuffle=True)
    return W.closed_loop_pid(n=3000, nsteps=100)


def _dead(n, frac, seed):
    st = np.zeros(n, np.uint8)
    st[np.random.default_rng(seed).random(n) < frac] = 2
    return st


def _sim(wl, dev):
    from paper_2308_12698_b300.sim import Sim
    gid = torch.from_numpy(wl.gid).to(dev) if len(wl.groups) > 1 else None
    return Sim(wl.groups, wl.n, wl.mode, gid=gid)


def _run(wl, dev, status, nsteps, K, compact, x0=None):
    from paper_2308_12698_b300.sim import planar, unplanar
    sim = _sim(wl, dev)
    sim.load_status(torch.from_numpy(status).to(dev))
    if compact:
        sim.compact()
    x = planar(torch.from_numpy(wl.x0 if x0 is None else x0)).to(dev)
    cmd = torch.from_numpy(wl.cmd).reshape(-1).to(dev)
    sim.step(x, cmd, wl.dt, nsteps, K=K)
    torch.cuda.synchronize()
    out = unplanar(x, wl.n).cpu().numpy()
    st = sim.status().cpu().numpy()
    sim.close()
    return out, st


@pytest.mark.parametrize("kind", ["one_group", "contiguous", "interleaved", "mixed_types", "pid"])
@pytest.mark.parametrize("K", [1, 40, 100])
def test_compacted_steps_are_bitwise_the_same(dev, kind, K):
    """Half the agents dead at random; 100 steps (K = 40: launches of 40, 40 and 20)."""
    wl = _workload(kind)
    status = _dead(wl.n, 0.5, 1)
    a, sa = _run(wl, dev, status, 100, K, compact=False)
    b, sb = _run(wl, dev, status, 100, K, compact=True)
    np.testing.assert_array_equal(b, a)
    np.testing.assert_array_equal(sb, sa)
    dead = status != 0
    np.testing.assert_array_equal(b[dead], wl.x0[dead])  # dead agents are not stepped


def test_agents_dying_after_compaction(dev):
    """Agents that go non-finite after the compaction (eight spinning past RK4's stability bound)
    are frozen at their last finite state, as without it."""
    wl = W.closed_loop(n=4000, nsteps=300)
    x0 = wl.x0.copy()
    spin = [3, 9, 17, 22, 35, 41, 50, 63]
    x0[spin, 10:13] = 0.0
    x0[spin, 12] = [5900.0, 6000.0, 6100.0, 6200.0, 6500.0, 7000.0, 8000.0, 9000.0]
    status = _dead(wl.n, 0.3, 2)
    status[spin] = 0
    a, sa = _run(wl, dev, status, 300, 100, compact=False, x0=x0)
    b, sb = _run(wl, dev, status, 300, 100, compact=True, x0=x0)
    np.testing.assert_array_equal(b, a)
    np.testing.assert_array_equal(sb, sa)
    assert (sb[spin] == 1).all()


def test_status_reset_drops_the_order(dev):
    """After sim_reset_status or sim_load_status the revived agents are stepped again: the same
    bits as a handle that was never compacted."""
    from paper_2308_12698_b300.sim import planar, unplanar
    wl = W.heterogeneous(sizes=(700, 1000, 300, 5), nsteps=100, shuffle=True)
    cmd = torch.from_numpy(wl.cmd).reshape(-1).to(dev)
    ref, _ = _run(wl, dev, np.zeros(wl.n, np.uint8), 100, 50, compact=False)
    for how in ("reset", "load"):
        sim = _sim(wl, dev)
        sim.load_status(torch.from_numpy(_dead(wl.n, 0.5, 3)).to(dev))
        sim.compact()
        if how == "reset":
            sim.reset_status()
        else:
            sim.load_status(torch.zeros(wl.n, dtype=torch.uint8, device=dev))
        x = planar(torch.from_numpy(wl.x0)).to(dev)
        sim.step(x, cmd, wl.dt, 100, K=50)
        np.testing.assert_array_equal(unplanar(x, wl.n).cpu().numpy(), ref)
        assert sim.n_dead() == 0
        sim.close()


def test_graphs_captured_before_an_order_change_are_refused(dev):
    from paper_2308_12698_b300 import _lib
    from paper_2308_12698_b300.sim import planar, unplanar
    wl = W.closed_loop(n=3000, nsteps=100)
    status = _dead(wl.n, 0.5, 4)
    ref, _ = _run(wl, dev, status, 200, 50, compact=False)
    sim = _sim(wl, dev)
    sim.load_status(torch.from_numpy(status).to(dev))
    x = planar(torch.from_numpy(wl.x0)).to(dev)
    cmd = torch.from_numpy(wl.cmd).reshape(-1).to(dev)
    before = sim.graph(x, cmd, wl.dt, 100, K=50)
    sim.compact()
    stream = torch.cuda.current_stream().cuda_stream
    import ctypes
    assert _lib.lib().sim_graph_launch(before._g, ctypes.c_void_p(stream)) == _lib.SIM_ERR_STALE
    after = sim.graph(x, cmd, wl.dt, 100, K=50)  # captured on the live agents' order
    after.launch()
    after.launch()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(unplanar(x, wl.n).cpu().numpy(), ref)
    sim.compact()  # every new order makes the graphs before it stale
    assert _lib.lib().sim_graph_launch(after._g, ctypes.c_void_p(stream)) == _lib.SIM_ERR_STALE
    again = sim.graph(x, cmd, wl.dt, 100, K=50)
    sim.reset_status()  # dropping the order too
    assert _lib.lib().sim_graph_launch(again._g, ctypes.c_void_p(stream)) == _lib.SIM_ERR_STALE
    for g in (before, after, again):
        g.close()
    sim.close()


@pytest.mark.parametrize("kind", ["interleaved", "mixed_types"])
def test_compacted_host_pipeline(dev, kind):
    """300k agents in 9 host-pipeline chunks, half of them dead: the chunks' launches take the
    live agents' order chunk by chunk; bitwise the device entry without compaction."""
    from paper_2308_12698_b300.sim import planar, unplanar
    if kind == "mixed_types":
        wl = W.multi_type(sizes=(100_000, 150_000, 50_001), nsteps=80, shuffle=True)
    else:
        wl = W.heterogeneous(sizes=(100_000, 150_000, 50_001), nsteps=80, shuffle=True)
    status = _dead(wl.n, 0.5, 5)
    ref, sref = _run(wl, dev, status, 80, 40, compact=False)
    sim = _sim(wl, dev)
    sim.load_status(torch.from_numpy(status).to(dev))
    sim.compact()
    h_state = planar(torch.from_numpy(wl.x0)).pin_memory()
    h_cmd = torch.from_numpy(wl.cmd).reshape(-1).pin_memory()
    d_state = torch.full((17 * wl.n,), float("nan"), device=dev)
    d_cmd = torch.empty(4 * wl.n, device=dev)
    sim.step_host(h_state, h_cmd, d_state, d_cmd, wl.dt, 80, K=40)
    np.testing.assert_array_equal(unplanar(h_state, wl.n).numpy(), ref)
    np.testing.assert_array_equal(sim.status().cpu().numpy(), sref)
    sim.close()


def test_all_dead_and_empty(dev):
    wl = W.heterogeneous(sizes=(300, 200), nsteps=64, shuffle=True)
    status = np.full(wl.n, 2, np.uint8)
    out, st = _run(wl, dev, status, 64, 64, compact=True)
    np.testing.assert_array_equal(out, wl.x0)
    assert (st == 2).all()
    from paper_2308_12698_b300.sim import Sim
    empty = Sim([W.base_group()], 0, W.CLOSED_LOOP)
    empty.compact()
    empty.close()


def test_full_size_half_dead_bitwise(dev):
    """The bench's half-dead leg in its launch shape: 1e6 agents, half dead at random, one launch
    of K = 1000; compacted and in place give the same bits."""
    wl = W.scale_sweep(1_000_000, nsteps=1000)
    status = _dead(wl.n, 0.5, 7)
    a, sa = _run(wl, dev, status, 1000, 1000, compact=False)
    b, sb = _run(wl, dev, status, 1000, 1000, compact=True)
    np.testing.assert_array_equal(b, a)
    np.testing.assert_array_equal(sb, sa)


def _rollout(wl, dev, status, C, compact, x0, gT):
    from paper_2308_12698_b300.sim import planar
    sim = _sim(wl, dev)
    sim.load_status(torch.from_numpy(status).to(dev))
    if compact:
        sim.compact()
    x = planar(torch.from_numpy(x0)).to(dev)
    cmd = torch.from_numpy(wl.cmd).reshape(-1).to(dev)
    w = torch.full((wl.n,), wl.w_omega, device=dev)
    ckpt, rc = sim.rollout_forward(x, cmd, wl.dt, wl.nsteps, C=C)
    st_fwd = sim.status().cpu().numpy()
    dx0, dth, dtha = sim.rollout_backward(ckpt, cmd, wl.dt, wl.nsteps, gT, w, C=C, per_agent=True)
    torch.cuda.synchronize()
    out = [t.cpu().numpy() for t in (ckpt, rc, dx0, dth, dtha)] + [st_fwd]
    sim.close()
    return out


@pytest.mark.parametrize("pid", [False, True], ids=["p-loop", "pid-loop"])
@pytest.mark.parametrize("C", [1, 8, 40])
def test_compacted_rollout_and_adjoint(dev, pid, C):
    """Checkpointed rollout and adjoint over the live agents' order: checkpoints, running costs,
    status, dL/dx0 and per-agent theta rows bit for bit as without the order, group sums within
    summation-order rounding.  Half the agents dead before the rollout; eight more spin past
    RK4's stability bound and die during it (their checkpoints are the kernel's, not the
    frozen pass's, which runs first)."""
    make = W.differentiable_pid if pid else W.differentiable
    wl = make(n_per_group=500, n_groups=4, nsteps=240)
    x0 = wl.x0.copy()
    status = _dead(wl.n, 0.5, 8)
    spin = np.flatnonzero(status == 0)[:8]
    x0[spin, 10:13] = 0.0
    x0[spin, 12] = np.linspace(8000.0, 12000.0, 8)
    nx = x0.shape[1]
    gT = torch.zeros(nx * wl.n, device=dev)
    gT[: 3 * wl.n] = 1.0
    a = _rollout(wl, dev, status, C, False, x0, gT)
    b = _rollout(wl, dev, status, C, True, x0, gT)
    for k, name in ((0, "checkpoints"), (1, "running cost"), (2, "dL/dx0"), (4, "theta rows"), (5, "status")):
        np.testing.assert_array_equal(b[k], a[k], err_msg=name)
    assert (a[5][spin] == 1).sum() >= 6, a[5][spin]
    scale = np.abs(a[3]).max()
    np.testing.assert_allclose(b[3], a[3], rtol=1e-5, atol=1e-6 * scale)
