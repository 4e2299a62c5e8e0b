"""The checker still reproduces its committed fixture (written by tests/golden/make_golden.py)."""
import json
import os

import numpy as np

from tests.golden.make_golden import OUT, cases


def test_oracle_matches_committed_fixture(orc):
    ref = json.load(open(OUT))
    for name, wl in cases():
        xT, rc = orc.rollout(wl.groups, wl.gid, wl.x0, wl.cmd, wl.dt, wl.nsteps, wl.mode, nthreads=1, with_cost=True)
        np.testing.assert_allclose(xT, np.array(ref[name]["xT"]), rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(rc, np.array(ref[name]["run_cost"]), rtol=1e-13)
