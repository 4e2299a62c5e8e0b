"""Writes tests/golden/oracle_regression.json from the FP64 checker alone.

The fixture freezes a few short rollouts of the checker (closed loop, open
loop, heterogeneous groups, the PID rate loop, a swarm of quadrotors, cars and
fixed-wing drones) so that an accidental change of its arithmetic
shows up as a failing test.  A deliberate change must regenerate it and name,
in the commit message, the equation or reading that justifies the change.

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


if __name__ == "__main__":
    main()
