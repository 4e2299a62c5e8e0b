"""The device bounds checks fire (runs only against the bounds-checked build).

The checked-build test runs the GPU suite with QUADSIM_LIB pointing at
libquadsim_checked.so; this file then checks that a check does fire.  A group
id is overwritten on the device after sim_create has validated the ids (the
host cannot see it): the step kernel's check records site 5 with the bad id and
skips that agent, the others step as usual.  Before any launch the test makes
sure the checks are compiled in, so the product library never meets that input.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2308_12698_b300 import workload as W

pytestmark = pytest.mark.gpu


def test_a_bad_group_id_is_caught_and_skipped():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2308_12698_b300 import _lib
    from paper_2308_12698_b300.sim import Sim, planar, unplanar
    word = ctypes.c_uint64()
    if _lib.lib().sim_bounds_checks(ctypes.byref(word)) != 1:
        pytest.skip("device bounds checks are not compiled into this library")
    assert word.value == 0
    dev = torch.device("cuda:0")
    wl = W.heterogeneous(sizes=(300, 300), nsteps=10, shuffle=True)
    gid = torch.from_numpy(wl.gid).to(dev)
    sim = Sim(wl.groups, wl.n, wl.mode, gid=gid)
    ref = Sim(wl.groups, wl.n, wl.mode, gid=gid.clone())
    x = planar(torch.from_numpy(wl.x0)).to(dev)
    xr = x.clone()
    cmd = torch.from_numpy(wl.cmd).reshape(-1).to(dev)
    ref.step(xr, cmd, wl.dt, 10, K=1)
    gid[5] = 7  # two groups: id 7 indexes past the group table
    sim.step(x, cmd, wl.dt, 10, K=1)  # K = 1: the persistent kernel reads the id of every agent
    torch.cuda.synchronize()
    assert _lib.lib().sim_bounds_checks(ctypes.byref(word)) == 1
    assert word.value >> 48 == 5 and word.value & ((1 << 48) - 1) == 7, hex(word.value)
    got, want = unplanar(x, wl.n).cpu().numpy(), unplanar(xr, wl.n).cpu().numpy()
    np.testing.assert_array_equal(got[5], wl.x0[5])  # the agent with the bad id was skipped
    keep = np.arange(wl.n) != 5
    np.testing.assert_array_equal(got[keep], want[keep])
    assert _lib.lib().sim_bounds_checks(ctypes.byref(word)) == 1 and word.value == 0  # read clears it
    sim.close()
    ref.close()
