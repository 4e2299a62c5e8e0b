"""sim_rollout_backward_noalloc: the adjoint for callers that cannot allocate.

Some callers may not allocate device memory once they are running -- a
real-time control loop that reserves all of its memory at start-up, or a
plug-in whose host application owns every device allocation -- so they cannot
hand sim_rollout_backward a workspace.  The workspace-free entry point runs
the same adjoint out of a fixed 32 MiB array inside the library.  This test
calls it through the C ABI three times in a row (the array keeps the previous
call's contents; the first call differentiates another terminal cotangent) and
compares each call with the workspace entry point on the same input, for the
P and the PID rate loop: per-agent gradients bit for bit, per-group sums
within 1e-5 (the capped grid partitions the agents over fewer blocks, so the
group sums are added in another order).  The file name makes pytest collect
it last.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("block_adj", [128, 0], ids=["block128", "default-block"])
@pytest.mark.parametrize("pid", [False, True], ids=["p-loop", "pid-loop"])
def test_noalloc_adjoint_matches_workspace_adjoint_on_two_calls(pid, block_adj):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2308_12698_b300 import _lib
    from paper_2308_12698_b300 import workload as W
    from paper_2308_12698_b300.sim import Sim, planar

    L = _lib.lib()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    # one checkpoint segment of 400 steps: 400 x 68 B (80 B with the PID loop's
    # integral) per thread, so the fixed array holds fewer resident blocks than
    # the 16 blocks of 128 threads (or the 64 blocks of 32 threads that the
    # default block size gives 2,048 agents) the agents need, and each block of
    # the capped grid takes several agents in turn
    T, C = 400, 400
    make = W.differentiable_pid if pid else W.differentiable
    wl = make(n_per_group=512, n_groups=4, nsteps=T)
    gid = torch.from_numpy(wl.gid).to(dev)
    sim = Sim(wl.groups, wl.n, wl.mode, gid=gid)
    sim.set_launch(block_adj=block_adj)
    nx = sim.nx
    x0 = planar(torch.from_numpy(wl.x0)).to(dev)
    cmd = torch.from_numpy(wl.cmd).reshape(-1).to(dev)
    ckpt, _ = sim.rollout_forward(x0, cmd, wl.dt, T, C=C)
    gT = torch.zeros(nx * wl.n, device=dev)
    gT[: 3 * wl.n] = 1.0
    # another terminal cotangent, for a call whose leftovers the next call must not see
    g_other = torch.from_numpy(np.random.default_rng(5).normal(size=nx * wl.n).astype(np.float32)).to(dev)
    w = torch.full((wl.n,), wl.w_omega, device=dev)
    refs = {}
    for name, g in (("other", g_other), ("loss", gT)):
        refs[name] = sim.rollout_backward(ckpt, cmd, wl.dt, T, g, w, C=C, per_agent=True)
    torch.cuda.synchronize()
    for r in refs.values():
        assert all(torch.isfinite(t).all() for t in r)

    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # three calls in a row: the first with the other cotangent, then two with the loss's
    for name, g in (("other", g_other), ("loss", gT), ("loss", gT)):
        ref_dx0, ref_dth, ref_dtha = refs[name]
        dx0 = torch.full_like(ref_dx0, float("nan"))
        dth = torch.full_like(ref_dth, float("nan"))
        dtha = torch.full_like(ref_dtha, float("nan"))
        rc = L.sim_rollout_backward_noalloc(sim.handle, _p(ckpt), _p(cmd), wl.dt, T, C, _p(g), _p(w), _p(dx0),
                                            _p(dth), _p(dtha), stream)
        assert rc == _lib.SIM_OK, L.sim_error_string(rc)
        torch.cuda.synchronize()
        assert torch.equal(dx0, ref_dx0)
        assert torch.equal(dtha, ref_dtha)
        scale = ref_dth.abs().max().item()
        np.testing.assert_allclose(dth.cpu().numpy(), ref_dth.cpu().numpy(), rtol=1e-5, atol=1e-6 * scale)

    # a checkpoint interval whose scratch cannot fit even one block is refused
    dx0 = torch.empty_like(refs["loss"][0])
    dth = torch.empty_like(refs["loss"][1])
    rc = L.sim_rollout_backward_noalloc(sim.handle, _p(ckpt), _p(cmd), wl.dt, 100_000, 100_000, _p(gT), _p(w),
                                        _p(dx0), _p(dth), None, stream)
    assert rc == _lib.SIM_ERR_WORKSPACE
    sim.close()
