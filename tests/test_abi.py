"""The C ABI library loads, exports every declared entry point and rejects bad
arguments on the host (no GPU needed for any of these)."""
import ctypes
import os
import re

import pytest

from paper_2308_12698_b300 import _lib
from paper_2308_12698_b300 import workload as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2308_12698_b300 import build
    build.build()
    return _lib.lib()


def declared():
    src = open(os.path.join(ROOT, "include", "quadsim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sim_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(_lib.EXPORTS)


def test_error_strings(L):
    for code in (0, -1, -2, -3, -4, -5, -6, -99):
        assert isinstance(L.sim_error_string(code), bytes)
    assert L.sim_error_string(-1) == b"invalid argument"


def _groups(n=1, **kw):
    g = W.base_group()
    g.update(kw)
    return (_lib.GroupParams * n)(*[_lib.group_struct(g) for _ in range(n)])


def test_create_rejects_bad_arguments_before_any_cuda_call(L):
    h = ctypes.c_void_p()
    ok = _groups()
    assert L.sim_create(None, 1, 10, None, 1, ctypes.byref(h)) == _lib.SIM_ERR_ARG
    assert L.sim_create(ok, 0, 10, None, 1, ctypes.byref(h)) == _lib.SIM_ERR_ARG
    assert L.sim_create(ok, 33, 10, None, 1, ctypes.byref(h)) == _lib.SIM_ERR_ARG
    assert L.sim_create(ok, 1, -1, None, 1, ctypes.byref(h)) == _lib.SIM_ERR_ARG
    assert L.sim_create(ok, 1, 10, None, 7, ctypes.byref(h)) == _lib.SIM_ERR_ARG
    assert L.sim_create(ok, 1, 10, None, 1, None) == _lib.SIM_ERR_ARG
    assert L.sim_create(_groups(2), 2, 10, None, 1, ctypes.byref(h)) == _lib.SIM_ERR_ARG  # ids missing
    for bad in (dict(m=0.0), dict(Jxx=-1.0), dict(kt=float("nan")), dict(tau_m=0.0), dict(alpha=2.0),
                dict(omega_max=float("inf")), dict(a_max=-1.0), dict(c_d=-0.1)):
        assert L.sim_create(_groups(**bad), 1, 10, None, 1, ctypes.byref(h)) == _lib.SIM_ERR_ARG, bad
    assert not h.value


def test_null_handle_calls_fail_cleanly(L):
    assert L.sim_step(None, None, None, 1e-3, 1, 1, None) == _lib.SIM_ERR_ARG
    assert L.sim_set_launch(None, 128, 128, 1, 1) == _lib.SIM_ERR_ARG
    assert L.sim_workspace_bytes(None, 100) == 0
    assert L.sim_step_launches(None, 10, 1) == 0
    assert L.sim_graph_launch(None, None) == _lib.SIM_ERR_ARG
    L.sim_destroy(None)
    L.sim_graph_destroy(None)


def test_checked_build_exports_the_same_entry_points(L):
    from paper_2308_12698_b300 import build
    checked = ctypes.CDLL(build.LIB_CHECKED)
    for n in declared():
        assert hasattr(checked, n), n


def test_product_build_has_no_device_checks(L):
    # the product library answers without touching the device: checks not compiled in
    word = ctypes.c_uint64(123)
    assert L.sim_bounds_checks(ctypes.byref(word)) == 0
    assert word.value == 0
    assert L.sim_bounds_checks(None) == _lib.SIM_ERR_ARG
