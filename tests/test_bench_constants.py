"""The work figures bench.py divides by are the checker's own counts."""
import numpy as np

import bench
from paper_2308_12698_b300 import workload as W


def test_flops_per_agent_step_is_the_checkers_count(orc):
    """The constant is the smallest count over the bench workload's states (a conservative figure)."""
    wl = W.scale_sweep(bench.N_AGENTS)
    counts = []
    for a in range(0, wl.n, wl.n // 256):
        c = orc.count_ops(wl.groups[0], wl.x0[a].astype(np.float64), wl.cmd[a], wl.dt, W.CLOSED_LOOP)
        counts.append(c["add"] + c["mul"] + c["div"] + c["sqrt"])
    assert min(counts) == bench.FLOPS_PER_AGENT_STEP, (min(counts), max(counts))
    assert max(counts) <= 1.03 * bench.FLOPS_PER_AGENT_STEP


def test_plain_bytes_per_agent_step():
    # state 17 floats in + out, one float4 command, one uint8 group id, one uint8 status
    assert bench.BYTES_PER_AGENT_STEP_PLAIN == 17 * 4 * 2 + 16 + 1 + 1
