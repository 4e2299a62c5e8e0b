"""The GPU suite again on the bounds-checked build of the library.

libquadsim_checked.so is the same source compiled with QS_CHECKED: each
instrumented device access first tests its index against its buffer's extent,
and a failed test records the site and index in a device word and skips the
access (no trap, no assert).  This test runs every other GPU test against that
build in a child process (QUADSIM_LIB points the binding at it), among them the
control in test_gpu_9_checks_fire.py, which makes a check fire on purpose; the
child's session ends by reading the word, and any other recorded failure fails
it.  A stand-in for a device memory checker, which this pool does not offer.
"""
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_gpu_suite_on_the_checked_build():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_12698_b300 import build
    build.build()
    env = dict(os.environ, QUADSIM_LIB=build.LIB_CHECKED)
    r = subprocess.run([sys.executable, "-m", "pytest", "tests", "-m", "gpu", "-x", "-q", "-rs", "-p",
                        "no:cacheprovider", "--ignore", os.path.join("tests", os.path.basename(__file__))],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=3000)
    tail = (r.stdout + r.stderr)[-4000:]
    assert r.returncode == 0, tail
    assert "bounds checks: no failure" in r.stdout, tail
    # the control in test_gpu_9_checks_fire.py ran (a check fired and was read back), not skipped
    assert "not compiled into this library" not in r.stdout, tail
