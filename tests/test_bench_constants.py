"""The work figures bench.py divides by: the method's hand count (the roofline's numerator)
and, beside it for context, the checker's own operation counts along its plain route."""
import numpy as np

import bench
from paper_2308_12698_b300 import workload as W


def test_hand_counts():
    """The roofline's work per agent-step: 75 per derivative at four stages, 120 for the RK4
    updates, 150 for the controller; the PID loop adds 4 FMAs per axis; forward + adjoint counts
    the forward, its recomputation and a reverse sweep of 2.5 forwards."""
    assert bench.FLOPS_PER_AGENT_STEP == 4 * 75 + 120 + 150 == 570
    assert bench.FLOPS_PER_AGENT_STEP_PID == 570 + 24
    assert bench.FWD_ADJ_FLOPS_PER_AGENT_STEP == 2565
    # the method's count stays below the checker's deliberately plain route
    assert bench.FLOPS_PER_AGENT_STEP < bench.CHECKER_FLOPS_PER_AGENT_STEP


def test_issue_fraction():
    # 418 thread instructions per agent-step at 8.09e10 agent-steps/s on 148 SMs at 2032 MHz
    f = bench.issue_frac(418, 8.09e10, 148, 2032.0)
    assert abs(f - 418 * 8.09e10 / (148 * 4 * 32 * 2032e6)) < 1e-12 and 0.87 < f < 0.89
    assert bench.issue_frac(None, 1.0, 148, 2032.0) is None


def test_checker_flops_per_agent_step_is_the_checkers_count(orc):
    """The constant is the smallest count seen over the bench workload's states (a conservative figure)."""
    wl = W.scale_sweep(bench.N_AGENTS)
    counts = []
    for a in range(0, wl.n, wl.n // 256):
        c = orc.count_ops(wl.groups[0], wl.x0[a].astype(np.float64), wl.cmd[a], wl.dt, W.CLOSED_LOOP)
        counts.append(c["add"] + c["mul"] + c["div"] + c["sqrt"])
    # conservative: never above any sampled state's count, and within 1 % of the smallest
    assert bench.CHECKER_FLOPS_PER_AGENT_STEP <= min(counts) <= 1.01 * bench.CHECKER_FLOPS_PER_AGENT_STEP, \
        (min(counts), max(counts))
    assert max(counts) <= 1.03 * bench.CHECKER_FLOPS_PER_AGENT_STEP


def test_plain_bytes_per_agent_step():
    # state 17 floats in + out, one float4 command, one uint8 status (the bench's swarm is one
    # group: the kernel takes its parameters from the launch and reads no group id)
    assert bench.BYTES_PER_AGENT_STEP_PLAIN == 17 * 4 * 2 + 16 + 1


def test_adjoint_tape_edges_are_the_checkers_count(orc):
    wl = W.scale_sweep(bench.N_AGENTS)
    edges = [orc.count_adjoint_edges(wl.groups[0], wl.x0[a].astype(np.float64), wl.cmd[a], wl.dt, W.CLOSED_LOOP)
             for a in range(0, wl.n, wl.n // 256)]
    assert bench.CHECKER_ADJ_TAPE_EDGES_PER_AGENT_STEP <= min(edges) <= \
        1.01 * bench.CHECKER_ADJ_TAPE_EDGES_PER_AGENT_STEP, (min(edges), max(edges))


def test_checker_pid_flops_per_agent_step_is_the_checkers_count(orc):
    """PID step: the checker's count less its second evaluation of the time derivative (for
    omega', which the kernel takes from the first RK4 stage); minimum over the PID workload."""
    wl = W.closed_loop_pid(n=bench.N_AGENTS)
    counts = []
    for a in range(0, wl.n, wl.n // 256):
        x = wl.x0[a].astype(np.float64)
        c = orc.count_ops(wl.groups[0], x, wl.cmd[a], wl.dt, W.CLOSED_LOOP_PID)
        d = orc.count_derivative_ops(wl.groups[0], x, x[13:17])
        counts.append(sum(c[k] - d[k] for k in ("add", "mul", "div", "sqrt")))
    assert bench.CHECKER_FLOPS_PER_AGENT_STEP_PID <= min(counts) <= 1.01 * bench.CHECKER_FLOPS_PER_AGENT_STEP_PID, \
        (min(counts),)
    assert max(counts) <= 1.03 * bench.CHECKER_FLOPS_PER_AGENT_STEP_PID


def test_vehicle_flops_per_agent_step_are_the_checkers_count(orc):
    wl = W.multi_type(sizes=(0, 2000, 2000))
    for kind, const in ((W.TYPE_CAR, bench.FLOPS_PER_AGENT_STEP_CAR),
                        (W.TYPE_FIXED_WING, bench.FLOPS_PER_AGENT_STEP_FIXED_WING)):
        counts = []
        for a in np.flatnonzero(wl.gid == kind)[::16]:
            c = orc.count_ops(wl.groups[kind], wl.x0[a].astype(np.float64), wl.cmd[a], wl.dt, W.CLOSED_LOOP)
            counts.append(c["add"] + c["mul"] + c["div"] + c["sqrt"])
        assert const <= min(counts) <= 1.01 * const, (kind, min(counts))
        assert max(counts) <= 1.05 * const
