"""Collision detection on the GPU (spatial hash) against the checker's brute force.

The decision is integer (a flag per agent), taken in FP32 on both sides with
the same rounding, so the flags must agree bit for bit.
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


def _radii(wl, scale=1.0):
    arm = np.array([np.float32(g["L"]) for g in wl.groups], np.float32)
    return (arm[wl.gid] * np.float32(scale)).astype(np.float32)


def gpu_collide(wl, dev, scale=1.0, x0=None, runs=1):
    from paper_2308_12698_b300.sim import Sim, planar
    g = torch.from_numpy(wl.gid).to(dev) if len(wl.groups) > 1 else None
    sim = Sim(wl.groups, wl.n, wl.mode, gid=g)
    x = planar(torch.from_numpy(wl.x0 if x0 is None else x0)).to(dev)
    outs = []
    for _ in range(runs):
        sim.reset_status()
        sim.collide(x, scale)
        outs.append(sim.status().cpu().numpy())
    torch.cuda.synchronize()
    sim.close()
    return outs if runs > 1 else outs[0]


@pytest.mark.parametrize("n", [1, 2, 33, 1000, 50_000])
def test_flags_bit_exact(dev, orc, n):
    wl = W.collision_field(n, planted=0.05)
    st = gpu_collide(wl, dev)
    ref = orc.collisions(wl.x0[:, 0:3], _radii(wl), np.ones(wl.n))
    np.testing.assert_array_equal((st == 2).astype(np.uint8), ref)
    if n >= 1000:
        assert ref.sum() > 0


def test_two_agents_at_and_inside_threshold(dev, orc):
    wl = W.collision_field(4, planted=0.0)
    x0 = wl.x0.copy()
    x0[:, 0:3] = [[0, 0, 0], [0.45, 0, 0], [5, 5, 5], [5.449, 5, 5]]
    st = gpu_collide(wl, dev, x0=x0)
    ref = orc.collisions(x0[:, 0:3], _radii(wl), np.ones(4))
    np.testing.assert_array_equal((st == 2).astype(np.uint8), ref)


def test_heterogeneous_radii_and_scale(dev, orc):
    wl = W.heterogeneous(sizes=(300, 700, 2000), nsteps=1, shuffle=True)
    x0 = wl.x0.copy()
    rng = np.random.default_rng(2)
    x0[:, 0:3] = rng.uniform(-6, 6, (wl.n, 3))
    for scale in (0.5, 1.0, 2.0):
        st = gpu_collide(wl, dev, scale=scale, x0=x0)
        ref = orc.collisions(x0[:, 0:3], _radii(wl, scale), np.ones(wl.n))
        np.testing.assert_array_equal((st == 2).astype(np.uint8), ref)


def test_dead_agents_are_excluded(dev, orc):
    from paper_2308_12698_b300.sim import Sim, planar
    wl = W.collision_field(5000, planted=0.05)
    x0 = wl.x0.copy()
    dead = np.arange(0, wl.n, 7)
    x0[dead, 3] = np.nan  # non-finite velocity: the first step marks these dead
    sim = Sim(wl.groups, wl.n, wl.mode)
    x = planar(torch.from_numpy(x0)).to(dev)
    cmd = torch.from_numpy(wl.cmd).reshape(-1).to(dev)
    sim.step(x, cmd, wl.dt, 1, K=1)
    st0 = sim.status().cpu().numpy()
    assert set(np.nonzero(st0)[0]) == set(dead)
    sim.collide(x, 1.0)
    st = sim.status().cpu().numpy()
    from paper_2308_12698_b300.sim import unplanar
    pos = unplanar(x, wl.n).cpu().numpy()[:, 0:3]
    alive = (st0 == 0).astype(np.uint8)
    ref = orc.collisions(pos, _radii(wl), alive)
    np.testing.assert_array_equal((st == 2).astype(np.uint8), ref)
    assert np.all(st[dead] == 1)
    sim.close()


def test_collided_agents_are_frozen(dev):
    from paper_2308_12698_b300.sim import Sim, planar, unplanar
    wl = W.collision_field(2000, planted=0.05)
    sim = Sim(wl.groups, wl.n, wl.mode)
    x = planar(torch.from_numpy(wl.x0)).to(dev)
    cmd = torch.from_numpy(wl.cmd).reshape(-1).to(dev)
    sim.collide(x, 1.0)
    before = unplanar(x, wl.n).cpu().numpy()
    st = sim.status().cpu().numpy()
    sim.step(x, cmd, wl.dt, 20, K=5)
    after = unplanar(x, wl.n).cpu().numpy()
    hit = st == 2
    assert hit.any() and (~hit).any()
    np.testing.assert_array_equal(after[hit], before[hit])
    assert np.any(after[~hit] != before[~hit])
    assert sim.n_dead() == int(hit.sum())
    sim.close()


def test_deterministic_and_full_size_sampled(dev, orc):
    """1e6 agents in the bench's launch shape: two runs agree, 4096 sampled agents match brute force."""
    wl = W.collision_field(1_000_000)
    a, b = gpu_collide(wl, dev, runs=2)
    np.testing.assert_array_equal(a, b)
    idx = np.random.default_rng(4).choice(wl.n, 4096, replace=False)
    planted_hits = np.nonzero(a == 2)[0][:512]
    idx = np.unique(np.concatenate([idx, planted_hits]))
    ref = orc.collisions(wl.x0[:, 0:3], _radii(wl), np.ones(wl.n), idx=idx)
    np.testing.assert_array_equal((a[idx] == 2).astype(np.uint8), ref)
    assert ref.sum() >= 256


def test_detection_between_rounds_of_flight(dev, orc):
    """Detection outside the main loop, every 500 steps, while the swarm flies: each agent's waypoint
    is another agent's start, so paths cross.  At every check the new flags equal brute force over
    the live agents at the GPU's positions, agents already dead keep their status and their state
    through later steps, and agents keep dying round after round."""
    from paper_2308_12698_b300.sim import Sim, planar, unplanar
    wl = W.collision_field(20_000, spacing=2.0, planted=0.0)
    cmd = wl.cmd.copy()
    cmd[:, 0:3] = wl.x0[np.random.default_rng(11).permutation(wl.n), 0:3]
    sim = Sim(wl.groups, wl.n, wl.mode)
    x = planar(torch.from_numpy(wl.x0)).to(dev)
    c = torch.from_numpy(cmd).reshape(-1).to(dev)
    radii = _radii(wl)
    prev_x, prev_st, deaths = None, None, []
    for _ in range(5):
        sim.step(x, c, wl.dt, 500, K=100)
        xs = unplanar(x, wl.n).cpu().numpy()
        st0 = sim.status().cpu().numpy()
        if prev_x is not None:
            dead = prev_st != 0
            np.testing.assert_array_equal(st0, prev_st)
            np.testing.assert_array_equal(xs[dead], prev_x[dead])
        sim.collide(x, 1.0)
        st = sim.status().cpu().numpy()
        ref = orc.collisions(xs[:, 0:3], radii, (st0 == 0).astype(np.uint8)).astype(bool)
        np.testing.assert_array_equal((st == 2) & (st0 == 0), ref)
        np.testing.assert_array_equal(st[st0 != 0], st0[st0 != 0])
        deaths.append(int(ref.sum()))
        prev_x, prev_st = xs, st
    assert all(d > 0 for d in deaths), deaths
    sim.close()


@pytest.mark.parametrize("n_per", [0, 5000, 70_000])
def test_group_stats(dev, n_per):
    """sim_group_stats against numpy on the same state and status bytes: counts exact, means
    within FP64 summation-order rounding, and bitwise the same on a second call.  Groups
    interleaved, one of them empty when n_per = 0, agents non-finite and collided."""
    from paper_2308_12698_b300.sim import Sim, planar
    sizes = (n_per, 3000, 2 * n_per + 17) if n_per else (0, 3000, 17)
    wl = W.heterogeneous(sizes=sizes, nsteps=1, shuffle=True)
    x0 = wl.x0.copy()
    status = np.zeros(wl.n, np.uint8)
    rng = np.random.default_rng(11)
    status[rng.random(wl.n) < 0.1] = 1
    status[rng.random(wl.n) < 0.1] = 2
    gid = torch.from_numpy(wl.gid).to(dev)
    sim = Sim(wl.groups, wl.n, wl.mode, gid=gid)
    sim.load_status(torch.from_numpy(status).to(dev))
    x = planar(torch.from_numpy(x0)).to(dev)
    got = sim.group_stats(x)
    again = sim.group_stats(x)
    np.testing.assert_array_equal(got, again)
    for g in range(len(wl.groups)):
        m = wl.gid == g
        live = m & (status == 0)
        assert got[g, 0] == live.sum()
        assert got[g, 1] == (m & (status == 1)).sum()
        assert got[g, 2] == (m & (status == 2)).sum()
        mean = x0[live, 0:3].astype(np.float64).mean(axis=0) if live.any() else np.zeros(3)
        np.testing.assert_allclose(got[g, 3:6], mean, rtol=1e-12, atol=1e-12)
    sim.close()
