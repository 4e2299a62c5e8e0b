"""bench.py's multi-rank timing on two gloo ranks (CPU): the barrier holds, the time is the
slowest rank's, and the whole-job rate counts every rank's agents."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    mx = bench.max_over_ranks(10.0 * (rank + 1), world)
    rate = bench.job_rate(world, 1_000_000, 1000, 10, mx)
    out[rank] = (mx, rate)
    dist.destroy_process_group()


def test_two_rank_max_and_rate():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        mx, rate = out[r]
        assert mx == 20.0
        assert rate == 2 * 1_000_000 * 1000 * 10 / 0.020
