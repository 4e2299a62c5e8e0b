"""Launch-configuration autotuner: threads per block, fused steps per launch
(K) and checkpoint interval (C), timed with CUDA events on the real swarm and
cached per (agents, groups, mode, device).

The tuner only times library calls; it changes no result: every candidate is
bitwise identical on the forward path
(tests/test_gpu_1_forward.py::test_autotuner_pick_is_bitwise_any_other).
"""
from __future__ import annotations

import json
import os

import torch

from .sim import Sim

BLOCKS = (32, 64, 128, 256)
KS = (10, 50, 100, 250, 1000)
CS = (1, 2, 4, 8, 16, 25, 50, 100)


def _cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "quadsim_b300", "autotune.json")


def _key(sim: Sim, kind: str, nsteps: int, candidates) -> str:
    name = torch.cuda.get_device_name()
    return f"{kind}|n={sim.n}|g={sim.n_groups}|mode={sim.mode}|T={nsteps}|{name}|{candidates}"


def _load() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache: dict):
    p = _cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        with open(p + ".tmp", "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(p + ".tmp", p)
    except OSError:
        pass


def _time(fn, reps: int = 3) -> float:
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def pick_step(results, tie: float = 0.005):
    """The (ms, block, K) to use from timed candidates: among those within `tie` of the fastest
    (the timing's spread), the largest block, then the largest K -- fewer blocks per launch for
    calls over part of the swarm."""
    best = min(r[0] for r in results)
    return max((r for r in results if r[0] <= best * (1.0 + tie)), key=lambda r: (r[1], r[2]))


def tune_step(sim: Sim, state: torch.Tensor, cmd: torch.Tensor, dt: float, nsteps: int, use_cache: bool = True,
              blocks=BLOCKS, ks=KS) -> dict:
    """Pick (block, K) for sim_step over nsteps; applies and returns it."""
    cache = _load() if use_cache else {}
    key = _key(sim, "step", nsteps, (tuple(blocks), tuple(ks)))
    if key in cache:
        cfg = cache[key]
    else:
        work = state.clone()
        results = []
        for b in blocks:
            sim.set_launch(block=b)
            for k in ks:
                if k > nsteps:
                    continue
                work.copy_(state)
                ms = _time(lambda: sim.step(work, cmd, dt, nsteps, K=k))
                results.append((ms, b, k))
        ms, b, k = pick_step(results)
        cfg = dict(block=b, K=k, ms=ms, candidates=[list(r) for r in results])
        cache[key] = cfg
        _store(cache)
    sim.set_launch(block=cfg["block"], K=cfg["K"])
    return cfg


def tune_adjoint(sim: Sim, x0: torch.Tensor, cmd: torch.Tensor, dt: float, nsteps: int, use_cache: bool = True,
                 cs=CS, blocks=(32, 64, 128)) -> dict:
    """Pick (block, C) for the checkpointed forward + adjoint; applies and returns it."""
    cache = _load() if use_cache else {}
    key = _key(sim, "adjoint", nsteps, (tuple(blocks), tuple(cs)))
    if key in cache:
        cfg = cache[key]
    else:
        g = torch.zeros(sim.nx * sim.n, dtype=torch.float32, device=x0.device)
        g[: 3 * sim.n] = 1.0
        results = []
        for b in blocks:
            sim.set_launch(block_adj=b)
            for c in cs:
                if c > nsteps:
                    continue
                ws = torch.empty(max(sim.workspace_bytes(c), 1), dtype=torch.uint8, device=x0.device)

                def run():
                    ckpt, _ = sim.rollout_forward(x0, cmd, dt, nsteps, C=c)
                    sim.rollout_backward(ckpt, cmd, dt, nsteps, g, None, C=c, workspace=ws)

                # checkpoints cost (T/C + 1) states: skip intervals whose checkpoints would
                # take more than half of the free device memory
                free, _ = torch.cuda.mem_get_info()
                if (nsteps // c + 2) * sim.nx * 4 * sim.n > free // 2:
                    del ws
                    continue
                results.append((_time(run, reps=2), b, c))
                del ws
                torch.cuda.empty_cache()
        ms, b, c = min(results)
        cfg = dict(block=b, C=c, ms=ms, candidates=[list(r) for r in results])
        cache[key] = cfg
        _store(cache)
    sim.set_launch(block_adj=cfg["block"], C=cfg["C"])
    return cfg
