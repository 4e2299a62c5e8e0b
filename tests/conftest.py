import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


def pytest_sessionfinish(session, exitstatus):
    """On a run against the bounds-checked library (QUADSIM_LIB set, as the checked-build test
    does), read the device check word once the tests are done: a failed index check fails the
    run with its site and index."""
    if not os.environ.get("QUADSIM_LIB"):
        return
    import ctypes

    import torch
    if not torch.cuda.is_available():
        return
    from paper_2308_12698_b300 import _lib
    word = ctypes.c_uint64()
    rc = _lib.lib().sim_bounds_checks(ctypes.byref(word))
    if rc != 1:
        print(f"\nbounds checks: not compiled into {_lib.LIB_PATH} (rc {rc})")
        session.exitstatus = 1
    elif word.value:
        print(f"\nbounds checks: FAILED at site {word.value >> 48}, index {word.value & ((1 << 48) - 1)}")
        session.exitstatus = 1
    else:
        print("\nbounds checks: no failure")
