"""Pins of the checker's FP32 evaluation (CPU only).

``oracle.rollout_f32`` runs the checker's model instantiated on float: every
operation rounded to single precision, the state stored as float between
steps.  The GPU tests use its distance from the FP64 rollout as the measure of
what FP32 rounding alone does to the equations over thousands of steps.  For
that it must (a) be the same model as the pinned FP64 checker, up to FP32
rounding, and (b) really round in single precision, not compute in double and
round once at the end.
"""
import numpy as np
import pytest

from paper_2308_12698_b300 import workload as W

FLOOR = np.array([1.0] * 13 + [100.0] * 4 + [1.0] * 3)


def _both(orc, wl, nsteps):
    x0 = np.asarray(wl.x0, np.float32)
    a = orc.rollout(wl.groups, wl.gid, x0.astype(np.float64), wl.cmd, wl.dt, nsteps, wl.mode)
    b = orc.rollout_f32(wl.groups, wl.gid, x0, wl.cmd, wl.dt, nsteps, wl.mode)
    return a, b


@pytest.mark.parametrize("kind", ["open", "closed", "pid"])
def test_one_step_is_the_fp64_model(orc, kind):
    wl = {"open": W.open_loop, "closed": W.closed_loop, "pid": W.closed_loop_pid}[kind](n=2000)
    a, b = _both(orc, wl, 1)
    assert b.dtype == np.float32 and b.shape == a.shape
    tol = 1e-5 * np.maximum(np.abs(a), FLOOR[: a.shape[1]])
    assert (np.abs(b.astype(np.float64) - a) <= tol).all()


def test_thousand_closed_loop_steps_within_the_fp32_bar(orc):
    # the FP32 trajectory bar after 1000 closed-loop steps: 1e-3 m and 1e-3 rad for every agent
    a, b = _both(orc, W.closed_loop(n=2000, nsteps=1000), 1000)
    b = b.astype(np.float64)
    assert np.abs(b[:, 0:3] - a[:, 0:3]).max() <= 1e-3
    qa = a[:, 6:10] / np.linalg.norm(a[:, 6:10], axis=1, keepdims=True)
    qb = b[:, 6:10] / np.linalg.norm(b[:, 6:10], axis=1, keepdims=True)
    assert (2 * np.arccos(np.clip(np.abs((qa * qb).sum(1)), 0, 1))).max() <= 1e-3


def test_rounds_every_step_in_single_precision(orc):
    # one step: about half the agents land on the FP64 result rounded to float, the rest one
    # rounding away; after 100 steps every agent has collected roundings of its own
    wl = W.closed_loop(n=2000)
    a1, b1 = _both(orc, wl, 1)
    share1 = (b1 == a1.astype(np.float32)).all(axis=1).mean()
    assert 0.05 < share1 < 0.95, share1
    a100, b100 = _both(orc, wl, 100)
    assert not (b100 == a100.astype(np.float32)).all(axis=1).any()


def test_quaternion_norm_drifts_at_fp32_rounding(orc):
    # torque-free spin (no rotor speed, open loop) for 10,000 steps: the FP64 checker keeps |q| = 1
    # to ~1e-12, single-precision rounding of q every step moves it by some 1e-7 and more
    g = W.base_group()
    x0 = np.array([[0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 3.0, -2.0, 5.0, 0, 0, 0, 0]], np.float32)
    cmd = np.zeros((1, 4))
    a = orc.rollout([g], [0], x0.astype(np.float64), cmd, 1e-3, 10_000, 0)
    b = orc.rollout_f32([g], [0], x0, cmd, 1e-3, 10_000, 0)
    da = abs(np.linalg.norm(a[0, 6:10]) - 1)
    db = abs(np.linalg.norm(b[0, 6:10].astype(np.float64)) - 1)
    assert da < 1e-11 and 1e-8 < db < 1e-3, (da, db)


def test_refuses_other_agent_types(orc):
    wl = W.multi_type(nsteps=10)
    with pytest.raises(ValueError):
        orc.rollout_f32(wl.groups, wl.gid, np.asarray(wl.x0, np.float32), wl.cmd, wl.dt, 1, wl.mode)
