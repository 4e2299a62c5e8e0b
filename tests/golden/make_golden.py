"""Writes tests/golden/oracle_regression.json and tests/golden/kinks_differentiable.json
from the FP64 checker alone.

The first fixture freezes a few short rollouts of the checker (closed loop, open
loop, heterogeneous groups, the PID rate loop, a swarm of quadrotors, cars and
fixed-wing drones) so that an accidental change of its arithmetic
shows up as a failing test.  A deliberate change must regenerate it and name,
in the commit message, the equation or reading that justifies the change.

The second records, for the differentiable-rollout workload (4,096 agents in 4
airframe groups, 2000 steps), how many agents pass next to a kink of the
controller on the checker's FP64 trajectory: a rotor demand within 1e-3
Omega_max^2 of zero, or within 1e-5 (relative) of the rotor ceiling or of the
acceleration clamp.  Their FP32 gradients are ill-conditioned and are held to
the looser gradient bar; the bench reports the share beside the leg's rate.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2308_12698_b300 import workload as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression.json")
KINKS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "kinks_differentiable.json")
#: margins below which an agent counts as passing a kink: rotor demand near 0 (relative to
#: Omega_max^2), near the rotor ceiling, near the acceleration clamp
SQRT_MARGIN, CLAMP_MARGIN = 1e-3, 1e-5


def cases():
    yield "closed_loop", W.closed_loop(n=6, nsteps=250)
    yield "open_loop", W.open_loop(n=4, nsteps=250)
    yield "heterogeneous", W.heterogeneous(sizes=(2, 1, 3), nsteps=250, shuffle=True)
    yield "pid", W.closed_loop_pid(n=4, nsteps=250)
    yield "multi_type", W.multi_type(sizes=(2, 2, 2), nsteps=250, shuffle=True)


def main():
    out = {}
    for name, wl in cases():
        xT, rc = oracle.rollout(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, wl.nsteps, wl.mode, nthreads=1,
                                with_cost=True)
        out[name] = dict(nsteps=wl.nsteps, xT=xT.tolist(), run_cost=rc.tolist())
    with open(OUT, "w") as f:
        json.dump(out, f, indent=0)
    print("wrote", OUT)
    wl = W.differentiable()
    m = oracle.clamp_margins(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, wl.nsteps)
    kinds = {"rotor_demand_near_zero": m[:, 0] < SQRT_MARGIN, "rotor_ceiling": m[:, 1] < CLAMP_MARGIN,
             "acceleration_clamp": m[:, 2] < CLAMP_MARGIN}
    fl = kinds["rotor_demand_near_zero"] | kinds["rotor_ceiling"] | kinds["acceleration_clamp"]
    k = dict(workload="differentiable rollout: 4096 agents in 4 groups, 2000 steps of 1 ms",
             margins=dict(rotor_demand_near_zero=SQRT_MARGIN, rotor_ceiling=CLAMP_MARGIN,
                          acceleration_clamp=CLAMP_MARGIN),
             n_agents=int(wl.n), flagged=int(fl.sum()), share=float(fl.mean()),
             by_kind={n: int(v.sum()) for n, v in kinds.items()},
             share_by_group=[float(fl[wl.gid == g].mean()) for g in range(len(wl.groups))])
    with open(KINKS, "w") as f:
        json.dump(k, f, indent=1)
    print("wrote", KINKS)


if __name__ == "__main__":
    main()
