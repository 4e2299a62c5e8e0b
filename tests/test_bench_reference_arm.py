"""The bench's reference arm: the FP64 checker timed on the host cores, one JSON line from rank 0."""
import argparse
import contextlib
import io
import json

import bench


def run_arm(monkeypatch, world, rank, steps=2, warmup=3):
    # a 64-agent sample instead of one sized for seconds of CPU work per step
    monkeypatch.setattr(bench, "cpu_sample_size", lambda target_s, threads, nsteps: 64)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(argparse.Namespace(steps=steps, warmup=warmup, gpus=world), world, rank)
    return buf.getvalue().strip().splitlines()


def test_reference_arm_line(monkeypatch):
    lines = run_arm(monkeypatch, 1, 0)
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert (d["metric"], d["unit"], d["higher_is_better"]) == (bench.METRIC, bench.UNIT, True)
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 3)
    assert d["value"] > 0 and d["ms_per_step"] > 0
    # the same workload description as the native arm's line
    assert d["config"]["workload"] == bench.workload_config(None)["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"] and cb["cores"] >= 1
    assert "64 agents" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # value is agents x physics steps x timed steps over the timed seconds
    assert abs(d["value"] - 64 * bench.T_STEPS * 2 / (2 * d["ms_per_step"] / 1e3)) <= 1e-6 * d["value"]


def test_reference_arm_other_ranks_print_nothing(monkeypatch):
    assert run_arm(monkeypatch, 2, 1) == []
