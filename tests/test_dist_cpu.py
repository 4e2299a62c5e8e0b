"""Two gloo ranks on CPU: sharded per-agent gradients summed over ranks equal the
single-process sum (the adjoint's only exchange), and sharding covers every agent."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2308_12698_b300 import dist as D
from paper_2308_12698_b300 import workload as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import oracle
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = W.differentiable(n_per_group=6, n_groups=2, nsteps=150)
    lo, hi = D.shard_range(wl.n, rank, world)
    sel = slice(lo, hi)
    loss, _, dth = oracle.grad(wl.groups, wl.gid[sel], wl.x0[sel], wl.cmd[sel], wl.dt, wl.nsteps, wl.mode,
                               wl.goal[sel], wl.w_omega, nthreads=1)
    g = np.zeros((len(wl.groups), 16))
    for gi in range(len(wl.groups)):
        g[gi] = dth[wl.gid[sel] == gi].sum(axis=0)
    t = torch.from_numpy(g)
    L = torch.tensor([loss.sum()], dtype=torch.float64)
    D.allreduce_grads(t, L)
    out[rank] = (t.numpy().copy(), float(L.item()))
    dist.destroy_process_group()


def test_two_rank_gradient_sum_equals_single_process(orc):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    wl = W.differentiable(n_per_group=6, n_groups=2, nsteps=150)
    loss, _, dth = orc.grad(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, wl.nsteps, wl.mode, wl.goal, wl.w_omega)
    ref = np.stack([dth[wl.gid == gi].sum(axis=0) for gi in range(2)])
    for r in range(2):
        g, L = out[r]
        np.testing.assert_allclose(g, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        assert abs(L - loss.sum()) <= 1e-12 * abs(loss.sum())


@pytest.mark.parametrize("n,world", [(10, 3), (1_000_000, 8), (5, 8), (0, 2)])
def test_shard_ranges_cover_everything(n, world):
    r = [D.shard_range(n, k, world) for k in range(world)]
    assert r[0][0] == 0 and r[-1][1] == n
    assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
    sizes = [hi - lo for lo, hi in r]
    assert max(sizes) - min(sizes) <= 1


def test_shard_by_groups_prefers_group_boundaries():
    gid = np.repeat(np.arange(4, dtype=np.uint8), [100, 900, 1000, 2000])
    cuts = D.shard_by_groups(gid, 2)
    assert cuts[0][0] == 0 and cuts[-1][1] == gid.size and cuts[0][1] == cuts[1][0]
    assert cuts[0][1] in (2000,)

