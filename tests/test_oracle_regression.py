"""The checker still reproduces its committed fixture (written by tests/golden/make_golden.py)."""
import json
import os

import numpy as np

from paper_2308_12698_b300 import workload as W
from tests.golden.make_golden import CLAMP_MARGIN, KINKS, OUT, SQRT_MARGIN, cases


def test_oracle_matches_committed_fixture(orc):
    ref = json.load(open(OUT))
    for name, wl in cases():
        xT, rc = orc.rollout(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, wl.nsteps, wl.mode, nthreads=1, with_cost=True)
        np.testing.assert_allclose(xT, np.array(ref[name]["xT"]), rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(rc, np.array(ref[name]["run_cost"]), rtol=1e-13)


def test_kink_fixture_matches_the_checker(orc):
    """The share of the differentiable workload's agents that pass next to a controller kink
    (the bench prints it beside the leg) is still the checker's."""
    ref = json.load(open(KINKS))
    wl = W.differentiable()
    m = orc.clamp_margins(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, wl.nsteps)
    fl = (m[:, 0] < SQRT_MARGIN) | (m[:, 1] < CLAMP_MARGIN) | (m[:, 2] < CLAMP_MARGIN)
    assert int(fl.sum()) == ref["flagged"] and ref["n_agents"] == wl.n
    assert abs(fl.mean() - ref["share"]) < 1e-12
