#!/usr/bin/env python
"""Throughput of the batched quadrotor step on B300.

Workload (one bench step): a closed-loop swarm of 1,000,000 quadrotors of the
reference airframe (1.5 kg X-frame, cascaded controller, rotor lag, RK4 with
dt = 1 ms) advanced 1000 physics steps, replayed as a CUDA graph of fused
K-substep launches.  Inputs are seeded synthetic (positions U[-10,10]^3,
waypoints U[-50,50]^3, tilts <= 10 deg) and resident in HBM before timing;
L2 is flushed (256 MB write) and the initial state restored, both untimed,
before every timed step.

Metric: agent-steps/s (agents x physics steps / device time), whole job over
all ranks.  Beside it: the plain one-step-per-launch kernel, the checkpointed
forward + adjoint rollout and the heterogeneous 8-group batch, each in
agent-steps/s on the same GPU, the roofline of the dominant kernel, clocks
sampled during the timed region, an end-to-end figure through the host-buffer
C-ABI call, and the FP64 checker timed on host cores on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "agent-steps/s at 1M quadrotors (fwd; fwd+adjoint) vs plain kernel, % roofline"
UNIT = "agent-steps/s"
N_AGENTS = 1_000_000
T_STEPS = 1000
DT = 1e-3
# The paper's own timing of this workload size (Table I), quoted for context only: another GPU,
# PyTorch/TorchScript, and a "round" that may include more than the step
PAPER_1000 = {"ms_per_round": 0.8452, "agent_steps_per_s": 1000 / 0.8452e-3, "n_agents": 1000,
              "hardware": "NVIDIA GTX 1660 SUPER + Intel i7-10700", "software": "Python 3.8, PyTorch 1.10.0+cu102",
              "source": "arXiv 2308.12698, Table I"}

#: Algorithmic work of one closed-loop agent-step, the roofline's numerator: the method's
#: FP32 operations counted by hand (a fused multiply-add counts 2): the time derivative
#: (Eq. qd1-qd4 with Eq. 2-3 and drag) about 75, at each of the four RK4 stages (300); the RK4
#: stage states and weighted combination about 120; the cascaded controller (position PD,
#: desired attitude, attitude P, rate P, mixer, rotor clamp and square root) about 150.
FLOPS_DERIVATIVE, FLOPS_RK4_UPDATES, FLOPS_CONTROLLER = 75, 120, 150
FLOPS_PER_AGENT_STEP = 4 * FLOPS_DERIVATIVE + FLOPS_RK4_UPDATES + FLOPS_CONTROLLER  # 570
#: The PID body-rate loop adds, per axis, the rate error, the integral and derivative terms and
#: the integrator update: four fused multiply-adds (24 flops per agent-step).
FLOPS_PER_AGENT_STEP_PID = FLOPS_PER_AGENT_STEP + 3 * 4 * 2  # 594
#: Forward + adjoint per agent-step, one rule for every checkpoint interval: the forward step
#: (1x), its recomputation inside the backward sweep (1x) and the reverse sweep (2.5x the
#: forward).  The extra forward pass over a segment that a checkpoint interval C > 1 adds is
#: not counted: it is the price of the smaller checkpoint memory, not work of the method.
FWD_ADJ_FLOPS_PER_AGENT_STEP = int(4.5 * FLOPS_PER_AGENT_STEP)  # 2565
#: The checker's count of non-trivial floating operations (add/sub, mul, div, sqrt) of one
#: closed-loop agent-step along its deliberately plain route (desired attitude as a matrix
#: converted by Shepperd's method, G^-1 by Gauss-Jordan, divisions), the minimum over the bench
#: workload's states (748..762); reported beside the method's count, for context only.
CHECKER_FLOPS_PER_AGENT_STEP = 748
#: The same count for one step with the PID body-rate loop (minimum over the PID workload's
#: states, 760..774), less the checker's second evaluation of the time derivative for omega'.
CHECKER_FLOPS_PER_AGENT_STEP_PID = 760
#: Tape edges of one closed-loop step in the checker's reverse mode (minimum over the
#: workload's states, 1348..1367).
CHECKER_ADJ_TAPE_EDGES_PER_AGENT_STEP = 1348
#: The checker's count for one step of a car (98..101) and of a fixed-wing drone (156, plus
#: five transcendental functions: four tan and one atan2, not counted), minimum over the mixed
#: swarm's states.  No hand count of these models exists; the mixed swarm's work weights them
#: with these figures and the quadrotors with the hand count.
FLOPS_PER_AGENT_STEP_CAR = 98
FLOPS_PER_AGENT_STEP_FIXED_WING = 156
#: Bytes one plain step of a one-group swarm moves per agent: state 68 read +
#: 68 written, command 16, status 1 (with one group the group id is not read).
BYTES_PER_AGENT_STEP_PLAIN = 153
#: FP32 lanes per SM (Blackwell), warp schedulers per SM (each issues one warp instruction per
#: clock) and the largest SM clock of the part.
FP32_LANES_PER_SM = 128
SCHEDULERS_PER_SM = 4
SM_MAX_MHZ = 2032.0
L2_FLUSH_BYTES = 256 << 20
#: The sources of each profiled kernel: a committed ncu figure is used only while the
#: fingerprint of its sources is the one it was taken on.
CSRC = "paper_2308_12698_b300/csrc/"
STEP_SOURCES = (CSRC + "model_fwd.cuh", CSRC + "step_kernel.cuh")
KERNEL_SOURCES = {"step": STEP_SOURCES,
                  "adjoint": STEP_SOURCES + (CSRC + "model_adj.cuh", CSRC + "adjoint_kernel.cuh"),
                  "collide": (CSRC + "collide.cuh",),
                  "multi": STEP_SOURCES + (CSRC + "vehicles.cuh",)}


def kernel_sha(family: str = "step") -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[family]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled(kernel: str, workload: str, family: str = "step") -> dict:
    """ncu figures of one kernel on one workload from a committed profiles/ summary (its
    `bench_counters:` line), if they were taken on the current kernel sources: DRAM bytes
    per launch and thread instructions per unit of work.  Empty if there is none."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return {}
    sha = kernel_sha(family)
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith(".md"):
            continue
        for line in open(os.path.join(pdir, fn)):
            if not line.startswith("bench_counters:"):
                continue
            kv = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
            if kv.get("kernel") == kernel and kv.get("workload") == workload and kv.get("source_sha") == sha:
                out = {"profile": "profiles/" + fn}
                for k in ("bytes_per_launch", "inst_per_unit"):
                    if k in kv:
                        out[k] = float(kv[k])
                return out
    return {}


def issue_frac(inst_per_unit, rate: float, sms: int, mhz: float):
    """Fraction of the issue slots (SMs x schedulers x 32 threads x clock) that rate units per
    second take at the profiled thread instructions per unit."""
    if not inst_per_unit:
        return None
    return inst_per_unit * rate / (sms * SCHEDULERS_PER_SM * 32 * mhz * 1e6)


def alu_roofline(flops: float, rate: float, sms: int, clocks: dict | None, prof: dict, kernel: str, **extra) -> dict:
    """The FP32 roofline object of an ALU-bound leg: achieved = flops per unit x rate against
    SMs x 128 lanes x 2 x the maximum clock, plus the issue-slot fraction from ncu."""
    peak = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    achieved = flops * rate / 1e12
    r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
         "flops_per_agent_step": flops, "kernel": kernel,
         "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 (FMA) x {SM_MAX_MHZ:.0f} MHz max clock",
         "traffic": None, "issue_frac": issue_frac(prof.get("inst_per_unit"), rate, sms, SM_MAX_MHZ),
         "inst_per_agent_step": prof.get("inst_per_unit"), "counters": prof.get("profile")}
    mhz = (clocks or {}).get("sm_mhz")
    if mhz:
        r["frac_at_measured_clock"] = r["frac"] * SM_MAX_MHZ / mhz
        if r["issue_frac"] is not None:
            r["issue_frac_at_measured_clock"] = r["issue_frac"] * SM_MAX_MHZ / mhz
    r.update(extra)
    return r


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------ clocks --

class _Nvml:
    """Read-only NVML queries through the driver's libnvidia-ml (ctypes): SM clock (MHz),
    power (W) and the current clock-event reason bits (0x4 sw power cap, 0x8 hw slowdown,
    0x20 sw thermal, 0x40 hw thermal)."""

    def __init__(self, index: int):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.dev = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.dev)) != 0:
            raise RuntimeError("no NVML device")
        self.reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def max_sm_mhz(self) -> int:
        v = self.ct.c_uint()
        if self.lib.nvmlDeviceGetMaxClockInfo(self.dev, 1, self.ct.byref(v)) != 0:
            raise RuntimeError("nvmlDeviceGetMaxClockInfo failed")
        return v.value

    def sample(self):
        sm, mw, rs = self.ct.c_uint(), self.ct.c_uint(), self.ct.c_ulonglong()
        if (self.lib.nvmlDeviceGetClockInfo(self.dev, 1, self.ct.byref(sm)) != 0 or
                self.lib.nvmlDeviceGetPowerUsage(self.dev, self.ct.byref(mw)) != 0 or
                self.reasons(self.dev, self.ct.byref(rs)) != 0):
            raise RuntimeError("NVML read failed")
        return sm.value, mw.value / 1000.0, rs.value

    def close(self):
        try:
            self.lib.nvmlShutdown()
        except Exception:
            pass


class ClockSampler:
    """SM clock, power and throttle reasons sampled while the timed region runs.

    In-process NVML reads every 5 ms on a background thread (enough samples even
    for a timed region of a tenth of a second); nvidia-smi at 200 ms if the NVML
    library cannot be loaded.  Reads only: no setting is changed."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, period_s: float = 0.005):
        self.index = index
        self.period = period_s
        self.proc = None
        self.rows = []
        self.nvml = None
        self.path = os.path.join("/tmp", f"quadsim_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            import threading
            self.nvml = _Nvml(self.index)
            self.smax = self.nvml.max_sm_mhz()
            self.stop = threading.Event()
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            return self
        except Exception:
            self.nvml = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def _poll(self):
        nv = self.nvml
        while not self.stop.is_set():
            try:
                sm, pw, rs = nv.sample()
                self.rows.append(dict(sm=float(sm), smax=float(self.smax), power=pw, hw=bool(rs & 0x8),
                                      hwt=bool(rs & 0x40), swt=bool(rs & 0x20), pcap=bool(rs & 0x4)))
            except Exception:
                pass
            self.stop.wait(self.period)

    def __exit__(self, *exc):
        if self.nvml is not None:
            self.stop.set()
            self.thread.join(timeout=5)
            self.nvml.close()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    self.rows.append(dict(sm=float(p[1]), smax=float(p[2]), power=float(p[3]),
                                          hw=p[5].lower() == "active", hwt=p[6].lower() == "active",
                                          swt=p[7].lower() == "active", pcap=p[8].lower() == "active"))
                except ValueError:
                    continue
            os.unlink(self.path)

    def summary(self) -> dict:
        rows = self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        loaded = [r for r in rows if r["power"] > 200.0] or rows
        sm = sorted(r["sm"] for r in loaded)
        reasons = [name for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                                          ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap"))
                   if any(r[key] for r in loaded)]
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r["smax"] for r in rows), "reasons": reasons,
                "samples": len(rows), "samples_under_load": len(loaded),
                "power_w_max": max(r["power"] for r in rows),
                "source": "nvml" if self.nvml is not None else "nvidia-smi"}


# ------------------------------------------------------------- distributed --

def dist_setup(gpus: int):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world: int):
    import torch
    if torch.cuda.is_available():
        torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """The largest of the ranks' values (NCCL on GPUs, gloo on CPU)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    on_gpu = dist.get_backend() == "nccl"
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if on_gpu else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, agents_per_rank: int, physics_steps: int, bench_steps: int, max_ms: float) -> float:
    """Whole-job agent-steps/s: every rank's agents and steps over the slowest rank's time."""
    return world * agents_per_rank * physics_steps * bench_steps / (max_ms / 1e3)


# -------------------------------------------------------------- CPU legs --

_WL_CACHE = {}


def oracle_rate(n_agents: int, nsteps: int, threads: int):
    """The FP64 checker, as it stands, on n_agents x nsteps of the bench workload."""
    import oracle
    from paper_2308_12698_b300 import workload as W
    if "wl" not in _WL_CACHE:
        _WL_CACHE["wl"] = W.scale_sweep(N_AGENTS)
    wl = _WL_CACHE["wl"]
    sel = slice(0, n_agents)
    t0 = time.perf_counter()
    oracle.rollout(wl.groups, wl.gid[sel], wl.x0[sel], wl.cmd[sel], wl.dt, nsteps, wl.mode, nthreads=threads)
    dt = time.perf_counter() - t0
    return n_agents * nsteps / dt, dt


def cpu_sample_size(target_s: float, threads: int, nsteps: int) -> int:
    """Agents of a sample that keeps the checker busy about target_s seconds
    (calibrated on samples grown until one takes at least 0.3 s)."""
    n = 16 * threads
    while True:
        rate, secs = oracle_rate(n, nsteps, threads)
        if secs >= 0.3 or n >= N_AGENTS:
            break
        n = min(N_AGENTS, n * 4)
    return max(256, min(N_AGENTS, int(rate * target_s / nsteps)))


def cpu_baseline(target_s: float = 10.0) -> dict:
    threads = os.cpu_count() or 1
    n = cpu_sample_size(target_s, threads, T_STEPS)
    rate, secs = oracle_rate(n, T_STEPS, threads)
    return {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {n} agents of the 1e6-agent workload x {T_STEPS} steps, FP64 C++ checker, "
                      f"std::thread over {threads} host cores, {secs:.1f} s"}


#: First agents of each sweep point's workload, kept by the GPU sweep for the checker's rate
_SWEEP_SLICES = {}
#: Agents and steps of the checker's sample at each sweep point: all agents up to 1e5 (1000
#: steps up to 1e4 agents, else 100), a 1e5-agent slice beyond (the rate is linear in N)
CPU_SWEEP_MAX_AGENTS = 100_000


def cpu_sweep_rates() -> dict:
    import oracle
    threads = os.cpu_count() or 1
    out = {}
    for n, (groups, gid, x0, cmd, mode) in sorted(_SWEEP_SLICES.items()):
        steps = T_STEPS if n <= 10_000 else 100
        t0 = time.perf_counter()
        oracle.rollout(groups, gid, x0, cmd, DT, steps, mode, nthreads=threads)
        secs = time.perf_counter() - t0
        out[str(n)] = {"value": len(gid) * steps / secs, "unit": UNIT, "cores": threads, "kind": "oracle",
                       "sample": f"first {len(gid)} agents x {steps} steps", "seconds": secs}
    return out


def run_reference(args, world: int, rank: int):
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    # each step: a bounded sample sized so the whole run stays within ~2-3 minutes
    per_step_s = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    n = cpu_sample_size(per_step_s, threads, T_STEPS)
    for _ in range(args.warmup):
        oracle_rate(n, T_STEPS, threads)
    times = []
    for _ in range(args.steps):
        _, s = oracle_rate(n, T_STEPS, threads)
        times.append(s)
    total = sum(times)
    value = n * T_STEPS * len(times) / total
    sample = (f"first {n} agents of the 1e6-agent workload x {T_STEPS} steps per bench step, FP64 C++ checker "
              f"on {threads} host cores")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(None),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(tuned) -> dict:
    c = {"workload": "closed-loop quadrotor swarm: 1,000,000 reference quadrotors (1.5 kg X-frame, cascaded "
                     "PD/attitude/rate controller, rotor lag, linear drag), 1000 RK4 steps of 1 ms per bench step",
         "n_agents_per_gpu": N_AGENTS, "physics_steps_per_bench_step": T_STEPS, "dt_s": DT,
         "inputs": "seeded synthetic, resident in HBM",
         "l2": "flushed (256 MB write) and initial state restored before every timed step, untimed",
         "parallelism": "agent data parallel, one rank per GPU, no collective on the forward path"}
    if tuned:
        c.update(tuned)
    return c


# ------------------------------------------------------------ GPU legs --

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-extra", action="store_true", help="headline only (no side measurements)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--agents", type=int, default=N_AGENTS, help="agents per GPU (profiling cases)")
    ap.add_argument("--physics-steps", type=int, default=T_STEPS, help="physics steps per bench step")
    ap.add_argument("--K", type=int, default=0, help="fix the fused steps per launch (skips the tuner)")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="time only the checkpointed forward + adjoint (profiling case)")
    ap.add_argument("--C", type=int, default=0, help="fix the checkpoint interval (with --adjoint-only)")
    ap.add_argument("--block-adj", type=int, default=0, help="fix the adjoint block size (with --adjoint-only)")
    ap.add_argument("--pid-only", action="store_true",
                    help="time only the PID-rate-loop swarm at --agents x --physics-steps (profiling case)")
    ap.add_argument("--multi-only", action="store_true",
                    help="time only the quadrotor / car / fixed-wing swarm (equal thirds) at --agents x "
                         "--physics-steps (profiling case)")
    ap.add_argument("--hetero-only", action="store_true",
                    help="time only the 8-group heterogeneous swarm (600,000 agents) over --physics-steps "
                         "(profiling case)")
    ap.add_argument("--collide-only", action="store_true",
                    help="time only collision detection on --agents agents (profiling case)")
    ap.add_argument("--block", type=int, default=0, help="fix the forward block size (with --pid-only, --multi-only)")
    ap.add_argument("--interleaved", action="store_true",
                    help="with --multi-only or --hetero-only: the groups' ids in random order")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2308_12698_b300 import autotune
    from paper_2308_12698_b300 import workload as W
    from paper_2308_12698_b300.sim import Sim, planar

    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    if args.adjoint_only:
        run_adjoint_only(args, world, rank, dev)
        return
    if args.pid_only or args.multi_only or args.hetero_only:
        run_swarm_only(args, world, rank, dev, "pid" if args.pid_only else "multi" if args.multi_only else "hetero")
        return
    if args.collide_only:
        run_collide_only(args, rank, dev)
        return
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count

    NA, TS = args.agents, args.physics_steps
    wl = W.scale_sweep(NA, nsteps=TS)
    x0 = planar(torch.from_numpy(wl.x0)).to(dev)
    cmd = torch.from_numpy(wl.cmd).reshape(-1).to(dev)
    x = x0.clone()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sim = Sim(wl.groups, wl.n, wl.mode)
    if args.K:
        sim.set_launch(K=args.K)
        tune = {"block": sim.launch()["block"], "K": args.K, "tuned": False}
    else:
        tune = autotune.tune_step(sim, x0, cmd, DT, TS)
    K = tune["K"]
    graph = sim.graph(x, cmd, DT, TS, K=K)
    launches = graph.launches_per_replay

    def timed_steps(run, n, reset=None):
        """Per-step device times (ms) with untimed reset + L2 flush before each."""
        out = []
        for _ in range(n):
            if reset:
                reset()
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run()
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
        return out

    reset = lambda: x.copy_(x0)  # noqa: E731
    timed_steps(graph.launch, args.warmup, reset)
    barrier(world)
    with ClockSampler(local) as clk:
        times = timed_steps(graph.launch, args.steps, reset)
        barrier(world)
    total_ms = max_over_ranks(sum(times), world)
    ms_step = total_ms / args.steps
    value = job_rate(world, NA, TS, args.steps, total_ms)
    clocks = clk.summary()
    # the paper's method (Sec. IV): three repeats, mean and standard deviation
    reps3 = [times[i::3] for i in range(3)] if args.steps >= 3 else [times]
    rates = [world * NA * TS * len(r) / (sum(r) / 1e3) for r in reps3 if r]
    spread = {"repeats": len(rates), "mean": float(np.mean(rates)), "sd": float(np.std(rates, ddof=1)) if
              len(rates) > 1 else 0.0, "unit": UNIT}

    # roofline of the dominant kernel: the fused step kernel, FP32-ALU bound.  Its average launch
    # time is the timed region over the step launches (the one short pass per replay that
    # reads the status bytes for agents gone non-finite is charged to them)
    step_launches = -(-TS // K)
    launch_s = (sum(times) / args.steps / step_launches) / 1e3
    kernel_rate = NA * min(K, TS) / launch_s
    prof = profiled("group_kernel<1,one_group>", f"closed-loop-{NA}-K{K}")
    roof = alu_roofline(FLOPS_PER_AGENT_STEP, kernel_rate, sms, clocks, prof,
                        f"group_kernel<closed loop, one group>, K={K} fused steps, block {tune['block']}",
                        avg_launch_us=launch_s * 1e6)
    roof["traffic"] = prof.get("bytes_per_launch")
    roof["frac_checker_count"] = CHECKER_FLOPS_PER_AGENT_STEP * kernel_rate / 1e12 / roof["peak"]

    # end to end through the host-buffer C-ABI call
    h_state0 = planar(torch.from_numpy(wl.x0)).pin_memory()
    h_state = h_state0.clone().pin_memory()
    h_cmd = torch.from_numpy(wl.cmd).reshape(-1).contiguous().pin_memory()
    d_state = torch.empty_like(x0)
    d_cmd = torch.empty_like(cmd)
    for _ in range(args.warmup):
        h_state.copy_(h_state0)
        sim.step_host(h_state, h_cmd, d_state, d_cmd, DT, TS, K=K)
    barrier(world)
    e2e_s = 0.0
    for _ in range(args.steps):
        h_state.copy_(h_state0)
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step_host(h_state, h_cmd, d_state, d_cmd, DT, TS, K=K)
        e2e_s += time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world)
    e2e = {"value": world * NA * TS * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(h_state.numel() * 4 + h_cmd.numel() * 4),
           "d2h_bytes_per_step": int(h_state.numel() * 4),
           "call": "sim_step_host (pinned host state+cmd in, state out, stream wait)"}

    extra = {}
    if not args.no_extra and NA == N_AGENTS and TS == T_STEPS:
        extra = side_measurements(args, world, sim, wl, x0, cmd, x, flush, stream, timed_steps, sms, clocks)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config({"K": K, "block": tune["block"], "graph_launches_per_step": launches,
                                       "n_agents_per_gpu": NA, "physics_steps_per_bench_step": TS}),
            "roofline": roof, "clocks": clocks, "e2e": e2e, "gpu_launches": launches * args.steps,
            "repeat_spread": spread}
    line.update(extra)
    if world == 1 and rank == 0:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        if "sweep" in line:
            # the checker beside each sweep point, on a bounded slice of that point's workload
            rates = cpu_sweep_rates()
            line["cpu_baseline"]["sweep"] = rates
            for row in line["sweep"]:
                row["oracle"] = rates.get(str(row["n_agents"]))
    if rank == 0:
        print(json.dumps(line), flush=True)
    graph.close()
    sim.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_adjoint_only(args, world, rank, dev):
    """Checkpointed forward + adjoint on --agents x --physics-steps, --C (or tuned)."""
    import torch

    from paper_2308_12698_b300 import autotune
    from paper_2308_12698_b300 import workload as W
    from paper_2308_12698_b300.sim import Sim, planar
    NA, TS = args.agents, args.physics_steps
    wl = W.scale_sweep(NA, nsteps=TS)
    sim = Sim(wl.groups, wl.n, wl.mode)
    x0 = planar(torch.from_numpy(wl.x0)).to(dev)
    cmd = torch.from_numpy(wl.cmd).reshape(-1).to(dev)
    if args.block_adj:
        sim.set_launch(block_adj=args.block_adj)
    if args.C:
        C = args.C
    else:
        C = autotune.tune_adjoint(sim, x0, cmd, DT, TS)["C"]
    ckpt = sim.ckpt_buffer(TS, C, device=dev)
    rc = torch.empty(sim.n, dtype=torch.float32, device=dev)
    gT = torch.zeros(17 * sim.n, dtype=torch.float32, device=dev)
    gT[: 3 * sim.n] = 1.0
    w = torch.full((sim.n,), 1e-6, dtype=torch.float32, device=dev)
    ws = torch.empty(max(sim.workspace_bytes(C), 1), dtype=torch.uint8, device=dev)

    def run():
        sim.rollout_forward(x0, cmd, DT, TS, C=C, ckpt=ckpt, run_cost=rc)
        sim.rollout_backward(ckpt, cmd, DT, TS, gT, w, C=C, workspace=ws)

    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        run()
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / args.steps
    if rank == 0:
        print(json.dumps({"leg": "fwd_adjoint", "agents": NA, "physics_steps": TS, "C": C, "ms_per_step": ms,
                          "value": NA * TS / (ms / 1e3), "unit": UNIT, "launch": sim.launch()}), flush=True)
    sim.close()


def run_swarm_only(args, world, rank, dev, kind: str):
    """One swarm on --agents x --physics-steps, --K and --block (or tuned): kind "pid" is the
    PID-rate-loop swarm, "multi" the quadrotor / car / fixed-wing swarm in equal thirds,
    "hetero" the 8-group swarm of 600,000 agents (--agents ignored)."""
    import torch

    from paper_2308_12698_b300 import autotune
    from paper_2308_12698_b300 import workload as W
    from paper_2308_12698_b300.sim import Sim, planar
    NA, TS = args.agents, args.physics_steps
    if kind == "pid":
        wl = W.closed_loop_pid(n=NA, nsteps=TS)
        flops = FLOPS_PER_AGENT_STEP_PID
    elif kind == "hetero":
        wl = W.heterogeneous(nsteps=TS, shuffle=args.interleaved)
        NA = wl.n
        flops = FLOPS_PER_AGENT_STEP
    else:
        sizes = (NA // 3, NA // 3, NA - 2 * (NA // 3))
        wl = W.multi_type(sizes=sizes, nsteps=TS, shuffle=args.interleaved)
        flops = (sizes[0] * FLOPS_PER_AGENT_STEP + sizes[1] * FLOPS_PER_AGENT_STEP_CAR +
                 sizes[2] * FLOPS_PER_AGENT_STEP_FIXED_WING) / NA
    gid = torch.from_numpy(wl.gid).to(dev) if len(wl.groups) > 1 else None
    sim = Sim(wl.groups, wl.n, wl.mode, gid=gid)
    x0 = planar(torch.from_numpy(wl.x0)).to(dev)
    cmd = torch.from_numpy(wl.cmd).reshape(-1).to(dev)
    x = x0.clone()
    if args.K:
        sim.set_launch(block=args.block, K=args.K)
    else:
        autotune.tune_step(sim, x0, cmd, DT, TS)
        if args.block:
            sim.set_launch(block=args.block)
    g = sim.graph(x, cmd, DT, TS)
    for _ in range(args.warmup):
        x.copy_(x0)
        g.launch()
    torch.cuda.synchronize()
    ms = 0.0
    for _ in range(args.steps):
        x.copy_(x0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.launch()
        b.record()
        b.synchronize()
        ms += a.elapsed_time(b) / args.steps
    if rank == 0:
        rate = NA * TS / (ms / 1e3)
        print(json.dumps({"leg": kind, "agents": NA, "physics_steps": TS, "ms_per_step": ms, "value": rate,
                          "unit": UNIT, "flops_per_agent_step": flops, "tflops": flops * rate / 1e12,
                          "launch": sim.launch()}), flush=True)
    g.close()
    sim.close()


def timed_fwd_adj(sim, x0, cmd, nsteps: int, C: int, timed_steps, reps: int):
    """Checkpointed forward + adjoint of the loss |p_T - goal|^2 + w sum Omega^2 at interval C:
    (ms per rollout pair, checkpoint MB, workspace MB)."""
    import torch
    dev = x0.device
    ckpt = sim.ckpt_buffer(nsteps, C, device=dev)
    rc = torch.empty(sim.n, dtype=torch.float32, device=dev)
    gT = torch.zeros(sim.nx * sim.n, dtype=torch.float32, device=dev)
    gT[: 3 * sim.n] = 1.0
    w = torch.full((sim.n,), 1e-6, dtype=torch.float32, device=dev)
    ws = torch.empty(max(sim.workspace_bytes(C), 1), dtype=torch.uint8, device=dev)

    def run():
        sim.rollout_forward(x0, cmd, DT, nsteps, C=C, ckpt=ckpt, run_cost=rc)
        sim.rollout_backward(ckpt, cmd, DT, nsteps, gT, w, C=C, workspace=ws)

    timed_steps(run, 2)
    t = timed_steps(run, reps)
    out = (sum(t) / reps, (ckpt.shape[0] * sim.ckpt_stride()) * 4 / 1e6, ws.numel() / 1e6)
    del ckpt, ws
    torch.cuda.empty_cache()
    return out


def fwd_adj_entry(world, sim, x0, cmd, nsteps, C, timed_steps, reps, sms, clocks) -> dict:
    ms, ck_mb, ws_mb = timed_fwd_adj(sim, x0, cmd, nsteps, C, timed_steps, reps)
    ms = max_over_ranks(ms, world)
    rate = sim.n * nsteps / (ms / 1e3)
    pa = profiled("adjoint_kernel<1>", f"closed-loop-C{C}", "adjoint")
    pf = profiled("ckpt_kernel<1>", "closed-loop", "adjoint")
    inst = pa["inst_per_unit"] + pf["inst_per_unit"] if ("inst_per_unit" in pa and "inst_per_unit" in pf) else None
    roof = alu_roofline(FWD_ADJ_FLOPS_PER_AGENT_STEP, rate, sms, clocks, {"inst_per_unit": inst},
                        "ckpt_kernel + adjoint_kernel + reduce_partials",
                        basis="forward 1x + recomputation 1x + reverse sweep 2.5x the forward step's 570 flops")
    roof["counters"] = [q.get("profile") for q in (pf, pa) if q]
    return {"value": world * rate, "unit": UNIT, "ms_per_step": ms, "n_agents": sim.n, "physics_steps": nsteps,
            "C": C, "block_adj": sim.launch()["block_adj"], "checkpoint_MB": ck_mb, "workspace_MB": ws_mb,
            "roofline": roof}


def sm_fill(n: int, block: int, sms: int) -> str:
    """How a swarm of n agents lands on the GPU at this block size."""
    blocks = -(-n // block)
    return f"{n:,} agents in {blocks} blocks of {block} fill {min(blocks, sms)} of the {sms} SMs"


def swarm_leg(world, wl, dev, timed_steps, reps, **sim_kw):
    """A tuned swarm in one graph per bench step: (sim, tuned config, ms per bench step)."""
    import torch

    from paper_2308_12698_b300 import autotune
    from paper_2308_12698_b300.sim import Sim, planar
    gid = torch.from_numpy(wl.gid).to(dev) if len(wl.groups) > 1 else None
    s = Sim(wl.groups, wl.n, wl.mode, gid=gid)
    x0 = planar(torch.from_numpy(wl.x0)).to(dev)
    cmd = torch.from_numpy(wl.cmd).reshape(-1).to(dev)
    xx = x0.clone()
    tune = autotune.tune_step(s, x0, cmd, DT, wl.nsteps)
    g = s.graph(xx, cmd, DT, wl.nsteps, K=tune["K"])
    reset = lambda: xx.copy_(x0)  # noqa: E731
    timed_steps(g.launch, 2, reset)
    t = timed_steps(g.launch, reps, reset)
    ms = max_over_ranks(sum(t), world) / reps
    g.close()
    s.close()
    return tune, ms


def copy_rate(dst, src, nbytes: int, reps: int = 20) -> float:
    """GB/s of copying src into dst (torch tensors, pinned host or device): reps copies
    enqueued back to back between two events, best of three such runs."""
    import torch
    for _ in range(3):
        dst.copy_(src, non_blocking=True)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            dst.copy_(src, non_blocking=True)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / reps)
    return nbytes / (best / 1e3) / 1e9


def duplex_rate(d_in, h_in, h_out, d_out, nbytes: int, reps: int = 20) -> float:
    """GB/s per direction with host-to-device copies (h_in -> d_in) and device-to-host copies
    (d_out -> h_out) on two streams at once: reps of each, timed from the first start to the
    last end; best of three."""
    import torch
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    best = float("inf")
    for _ in range(4):
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        s1.wait_event(e0)
        s2.wait_event(e0)
        with torch.cuda.stream(s1):
            for _ in range(reps):
                d_in.copy_(h_in, non_blocking=True)
            e1.record(s1)
        with torch.cuda.stream(s2):
            for _ in range(reps):
                h_out.copy_(d_out, non_blocking=True)
            e2.record(s2)
        e1.synchronize()
        e2.synchronize()
        best = min(best, max(e0.elapsed_time(e1), e0.elapsed_time(e2)) / reps)
    return nbytes / (best / 1e3) / 1e9


def l2_copy_bandwidth(nbytes: int = 32 << 20) -> float:
    """GB/s (read + write bytes) of a device-to-device copy small enough to stay in L2."""
    import torch
    a = torch.ones(nbytes // 4, device="cuda")
    b = torch.empty_like(a)
    return copy_rate(b, a, 2 * nbytes)


#: Algorithmic bytes per agent of one collision call (1e6 agents at 2 m mean spacing, 2^22
#: buckets, cells of 0.909 m for the reference arm), as the kernels touch them.  Insert:
#: status 1, position 16, arm length 4, its 32-byte record written, bucket head exchange 4.
#: Query: status 1, own record 16, 8 bucket heads x 4, and per candidate on those lists
#: (8 x 1e6 / 2^22 = 1.9 unrelated agents plus 0.8 within the 8 cells: 2.7 expected) 20 bytes
#: of its record (position, radius, link); hit byte 1.  Apply: hit and status 2.
COLLIDE_BYTES_PER_AGENT = (1 + 16 + 4 + 32 + 4) + (1 + 16 + 8 * 4 + 2.7 * 20 + 1) + 2


def run_collide_only(args, rank, dev):
    """Collision detection on the collision field of --agents agents: --warmup then --steps calls."""
    import torch

    from paper_2308_12698_b300 import workload as W
    from paper_2308_12698_b300.sim import Sim, planar
    cw = W.collision_field(args.agents)
    cs = Sim(cw.groups, cw.n, cw.mode)
    cx = planar(torch.from_numpy(cw.x0)).to(dev)
    cws = torch.empty(max(cs.collide_workspace_bytes(), 1), dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        cs.reset_status()
        cs.collide(cx, 1.0, cws)
    torch.cuda.synchronize()
    ms = 0.0
    for _ in range(args.steps):
        cs.reset_status()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        cs.collide(cx, 1.0, cws)
        b.record()
        b.synchronize()
        ms += a.elapsed_time(b) / args.steps
    if rank == 0:
        print(json.dumps({"leg": "collide", "agents": cw.n, "ms_per_call": ms, "value": cw.n / (ms / 1e3),
                          "unit": "agents/s", "bytes_per_agent": COLLIDE_BYTES_PER_AGENT}), flush=True)
    cs.close()


def side_measurements(args, world, sim, wl, x0, cmd, x, flush, stream, timed_steps, sms, clocks) -> dict:
    """The other legs on the same GPU (3 timed repeats each unless stated)."""
    import torch

    from paper_2308_12698_b300 import autotune
    from paper_2308_12698_b300 import workload as W
    from paper_2308_12698_b300.sim import Sim, planar
    reps = 3
    out = {}
    dev = x0.device
    reset = lambda: x.copy_(x0)  # noqa: E731
    hbm = measured_peaks().get("hbm_gbs")

    # plain one-step kernel: 1000 launches per bench step (graph); the 1e6-agent state and
    # commands (84 MB) stay in the 126 MB L2 between launches, so this is not an HBM figure
    # (the sweep's 1e7 point is)
    g1 = sim.graph(x, cmd, DT, T_STEPS, K=1)
    timed_steps(g1.launch, 2, reset)
    t = timed_steps(g1.launch, reps, reset)
    ms = max_over_ranks(sum(t), world) / reps
    launch_s = ms / 1e3 / T_STEPS
    gbs = BYTES_PER_AGENT_STEP_PLAIN * N_AGENTS / launch_s / 1e9
    out["plain"] = {"value": world * N_AGENTS * T_STEPS / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                    "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": None,
                                 "l2_equiv_frac": gbs / hbm if hbm else None,
                                 "bytes_per_agent_step": BYTES_PER_AGENT_STEP_PLAIN,
                                 "note": "L2-resident: the 1e6-agent state (68 MB) and commands fit in the 126 MB "
                                         "L2 between launches; the HBM-bound case is sweep n_agents=1e7"}}
    g1.close()

    # checkpointed forward + adjoint at 1e6 x 1000: the tuned interval and C = 100
    cfg = autotune.tune_adjoint(sim, x0, cmd, DT, T_STEPS)
    fa = {}
    for C in sorted({cfg["C"], 100}):
        sim.set_launch(block_adj=cfg["block"])
        fa[f"C{C}"] = fwd_adj_entry(world, sim, x0, cmd, T_STEPS, C, timed_steps, reps, sms, clocks)
    out["fwd_adjoint"] = dict(fa[f"C{cfg['C']}"], tuned_C=cfg["C"], by_C=fa)

    # the differentiable-rollout workload: 4,096 agents in 4 groups, 2000 steps, C = 100
    dw = W.differentiable()
    ds = Sim(dw.groups, dw.n, dw.mode, gid=torch.from_numpy(dw.gid).to(dev))
    dx0 = planar(torch.from_numpy(dw.x0)).to(dev)
    dcmd = torch.from_numpy(dw.cmd).reshape(-1).to(dev)
    c4 = fwd_adj_entry(world, ds, dx0, dcmd, dw.nsteps, 100, timed_steps, reps, sms, clocks)
    # beside the workload's own interval, the tuner's pick of C and block for this swarm
    c4t = autotune.tune_adjoint(ds, dx0, dcmd, DT, dw.nsteps)
    tuned = fwd_adj_entry(world, ds, dx0, dcmd, dw.nsteps, c4t["C"], timed_steps, reps, sms, clocks)
    c4["tuned"] = {k: tuned[k] for k in ("value", "ms_per_step", "C", "block_adj", "checkpoint_MB")}
    c4["tuned"]["frac"] = tuned["roofline"]["frac"]
    kinks = {}
    try:
        with open(os.path.join(ROOT, "tests", "golden", "kinks_differentiable.json")) as f:
            kinks = json.load(f)
    except (OSError, ValueError):
        pass
    c4.update(groups=len(dw.groups), kink_share=kinks.get("share"), kinks_by_kind=kinks.get("by_kind"),
              kink_note="agents whose FP64 trajectory passes next to a controller kink (held to the looser "
                        "gradient bar); counted by the checker, tests/golden/kinks_differentiable.json",
              note=sm_fill(dw.n, c4["block_adj"], sms) + " in the reverse sweep, one warp each: "
                   "latency-bound, not a throughput figure")
    out["fwd_adjoint_config4"] = c4
    ds.close()
    del dx0, dcmd

    # heterogeneous: 8 groups, uneven sizes (600k), a launch per group range per K steps, side by side
    # on the handle's streams, in a graph;
    # beside it the one-group swarm at the same agent count
    hw = W.heterogeneous(nsteps=T_STEPS, shuffle=False)
    ht, ms = swarm_leg(world, hw, dev, timed_steps, reps)
    hrate = hw.n * T_STEPS / (ms / 1e3)
    st_, ms1 = swarm_leg(world, W.scale_sweep(hw.n, nsteps=T_STEPS), dev, timed_steps, reps)
    rate1 = hw.n * T_STEPS / (ms1 / 1e3)
    hp = profiled("group_kernel<1>", f"heterogeneous-{hw.n}-K{ht['K']}")
    out["hetero"] = {"value": world * hrate, "unit": UNIT, "ms_per_step": ms,
                     "n_agents": hw.n, "groups": len(hw.groups), "sizes": list(W.HETERO_SIZES), "K": ht["K"],
                     "block": ht["block"],
                     "one_group_same_n": {"value": world * rate1, "K": st_["K"], "block": st_["block"]},
                     "ratio_to_one_group": hrate / rate1,
                     "roofline": alu_roofline(FLOPS_PER_AGENT_STEP, hrate, sms, clocks, hp,
                                              "group_kernel<closed loop>: a launch per group range, side by "
                                              "side; the group's constants in the kernel's parameters",
                                              note="every group runs the same operations")}
    # the same agents with the groups' ids interleaved at random: the handle's group-sorted order
    hi, msi = swarm_leg(world, W.heterogeneous(nsteps=T_STEPS, shuffle=True), dev, timed_steps, reps)
    hirate = hw.n * T_STEPS / (msi / 1e3)
    hip = profiled("group_kernel<1,false,true>", f"heterogeneous-interleaved-{hw.n}-K{hi['K']}")
    out["hetero"]["interleaved"] = {"value": world * hirate, "ms_per_step": msi,
                                    "K": hi["K"], "block": hi["block"], "ratio_to_contiguous": ms / msi,
                                    "how": "ids in random order; group_kernel through the group-sorted order",
                                    "roofline": alu_roofline(FLOPS_PER_AGENT_STEP, hirate, sms, clocks, hip,
                                                             "group_kernel<closed loop, ORDER>")}

    # PID body-rate loop: 1e6 agents with 20-component states
    pw = W.closed_loop_pid(n=N_AGENTS, nsteps=T_STEPS)
    pt, ms = swarm_leg(world, pw, dev, timed_steps, reps)
    rate = pw.n * T_STEPS / (ms / 1e3)
    pp = profiled("group_kernel<2,one_group>", f"closed-loop-pid-{pw.n}-K{pt['K']}")
    out["pid"] = {"value": world * rate, "unit": UNIT, "ms_per_step": ms, "n_agents": pw.n, "K": pt["K"],
                  "block": pt["block"],
                  "roofline": alu_roofline(FLOPS_PER_AGENT_STEP_PID, rate, sms, clocks, pp,
                                           "group_kernel<PID rate loop, one group>")}

    # quadrotors, cars and fixed-wing drones (200,000 each): a launch per type's group, side by side
    mw = W.multi_type(nsteps=T_STEPS)
    mt, ms = swarm_leg(world, mw, dev, timed_steps, reps)
    sizes = W.MULTI_TYPE_SIZES
    rate = mw.n * T_STEPS / (ms / 1e3)
    flops = (sizes[0] * FLOPS_PER_AGENT_STEP + sizes[1] * FLOPS_PER_AGENT_STEP_CAR +
             sizes[2] * FLOPS_PER_AGENT_STEP_FIXED_WING) / mw.n
    mp = profiled("group_kernel<1,multi>", f"multi-type-{mw.n}-K{mt['K']}", "multi")
    out["multi_type"] = {"value": world * rate, "unit": UNIT, "ms_per_step": ms,
                         "n_agents": mw.n, "sizes": {"quadrotor": sizes[0], "car": sizes[1], "fixed_wing": sizes[2]},
                         "K": mt["K"], "block": mt["block"],
                         "roofline": alu_roofline(flops, rate, sms, clocks, mp, "group_kernel<mixed agent types>: a launch per type's group",
                                                  note="quadrotors at the hand count, cars and fixed-wing drones "
                                                       "at the checker's count; tan/atan2 not counted")}
    # the same swarm with the agent types interleaved at random: the group-sorted order keeps each
    # warp on one type
    mi, msi = swarm_leg(world, W.multi_type(nsteps=T_STEPS, shuffle=True), dev, timed_steps, reps)
    mirate = mw.n * T_STEPS / (msi / 1e3)
    mip = profiled("group_kernel<1,multi,true>", f"multi-type-interleaved-{mw.n}-K{mi['K']}", "multi")
    out["multi_type"]["interleaved"] = {"value": world * mirate, "ms_per_step": msi,
                                        "K": mi["K"], "block": mi["block"], "ratio_to_contiguous": ms / msi,
                                        "how": "ids in random order; group_kernel through the group-sorted order",
                                        "roofline": alu_roofline(flops, mirate, sms, clocks, mip,
                                                                 "group_kernel<mixed agent types, ORDER>")}

    # the closed-loop configuration at its own shape: 5,000 agents x 10,000 steps, tuned
    cw1 = W.closed_loop()
    c1t, ms = swarm_leg(world, cw1, dev, timed_steps, reps)
    out["closed_loop_5000"] = {"value": world * cw1.n * cw1.nsteps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                               "n_agents": cw1.n, "physics_steps": cw1.nsteps, "K": c1t["K"],
                               "block": c1t["block"],
                               "note": sm_fill(cw1.n, c1t["block"], sms) + " at the tuned block: latency-bound"}

    # half of the agents dead at random (as collisions leave them): live agent-steps/s with the
    # dead agents skipped by the threads that hold them, then after sim_compact
    import numpy as np
    dwl = W.scale_sweep(N_AGENTS, nsteps=T_STEPS)
    dead = np.zeros(dwl.n, np.uint8)
    dead[np.random.default_rng(7).random(dwl.n) < 0.5] = 2
    live = int((dead == 0).sum())
    dx0 = planar(torch.from_numpy(dwl.x0)).to(dev)
    dcmd = torch.from_numpy(dwl.cmd).reshape(-1).to(dev)
    dh = {}
    for compact in (False, True):
        ds = Sim(dwl.groups, dwl.n, dwl.mode)
        ds.load_status(torch.from_numpy(dead).to(dev))
        if compact:
            ds.compact()  # the first call also allocates the order's buffers
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ds.compact()
            dh["compact_ms"] = (time.perf_counter() - t0) * 1e3
        dxx = dx0.clone()
        dg = ds.graph(dxx, dcmd, DT, T_STEPS, K=T_STEPS)
        dreset = lambda: dxx.copy_(dx0)  # noqa: E731
        timed_steps(dg.launch, 2, dreset)
        dms = max_over_ranks(sum(timed_steps(dg.launch, reps, dreset)), world) / reps
        dh["compacted" if compact else "in_place"] = {"value": world * live * T_STEPS / (dms / 1e3),
                                                      "ms_per_step": dms}
        dg.close()
        # forward with checkpoints + adjoint over the same swarm (C = 100)
        fms, _, _ = timed_fwd_adj(ds, dx0, dcmd, T_STEPS, 100, timed_steps, reps)
        fms = max_over_ranks(fms, world)
        dh.setdefault("fwd_adjoint_C100", {})["compacted" if compact else "in_place"] = {
            "value": world * live * T_STEPS / (fms / 1e3), "ms_per_step": fms}
        ds.close()
    out["half_dead"] = dict(dh, unit=UNIT, n_agents=dwl.n, live_agents=live, K=T_STEPS,
                            note="live agent-steps/s; 50 % of the agents dead at random positions in the ids")
    del dx0, dcmd

    # decision rounds: commands from pinned host memory every M steps, positions back after
    # each round, both overlapped with the physics (1000 steps per bench step); beside them the
    # pinned copy bandwidth of this machine's host link, per direction, for one round's 16 MB
    rounds = {}
    link = {}
    for M in (10, 100):
        R = T_STEPS // M
        h_cmds = torch.from_numpy(wl.cmd).reshape(1, -1).repeat(R, 1).contiguous().pin_memory()
        h_obs = torch.empty((R, 4 * N_AGENTS), dtype=torch.float32).pin_memory()
        cmd2 = torch.empty(8 * N_AGENTS, dtype=torch.float32, device=dev)
        obs2 = torch.empty(8 * N_AGENTS, dtype=torch.float32, device=dev)
        if not link:
            # the host link as the rounds see it: one round's 16 MB between the same buffers,
            # each direction alone and both at once (the rounds move both at once)
            link = {"h2d_GBs": copy_rate(cmd2[: 4 * N_AGENTS], h_cmds[0], 16 * N_AGENTS),
                    "d2h_GBs": copy_rate(h_obs[0], obs2[: 4 * N_AGENTS], 16 * N_AGENTS),
                    "both_directions_GBs_each": duplex_rate(cmd2[: 4 * N_AGENTS], h_cmds[0], h_obs[0],
                                                            obs2[: 4 * N_AGENTS], 16 * N_AGENTS),
                    "bytes": 16 * N_AGENTS,
                    "how": "one round's 16 MB command plane in and observation plane out, between the rounds' "
                           "own pinned and device buffers, 20 copies back to back per direction (alone, then "
                           "both directions on two streams at once), CUDA events"}
        Kr = min(sim.launch()["K"], M)
        rrun = lambda: sim.run_rounds(x, h_cmds, M, DT, K=Kr, h_obs=h_obs, cmd2=cmd2, obs2=obs2)  # noqa: E731
        timed_steps(rrun, 2, reset)
        t = timed_steps(rrun, reps, reset)
        ms = max_over_ranks(sum(t), world) / reps
        per_dir = 16 * N_AGENTS * R / (ms / 1e3) / 1e9
        rounds[f"M{M}"] = {"value": world * N_AGENTS * T_STEPS / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                           "rounds": R, "K": Kr, "h2d_bytes_per_round": 16 * N_AGENTS,
                           "d2h_bytes_per_round": 16 * N_AGENTS, "link_GBs_per_direction": per_dir,
                           "h2d_frac_of_link": per_dir / link["h2d_GBs"], "d2h_frac_of_link": per_dir / link["d2h_GBs"],
                           "frac_of_link_both_directions": per_dir / link["both_directions_GBs_each"]}
    out["decision_rounds"] = dict(rounds, link=link)

    # collision detection: 1e6 agents at 2 m mean spacing, 1 % planted near pairs
    cw = W.collision_field(N_AGENTS)
    cs = Sim(cw.groups, cw.n, cw.mode)
    cx = planar(torch.from_numpy(cw.x0)).to(dev)
    cws = torch.empty(max(cs.collide_workspace_bytes(), 1), dtype=torch.uint8, device=dev)
    crun = lambda: cs.collide(cx, 1.0, cws)  # noqa: E731
    timed_steps(crun, 2, cs.reset_status)
    t = timed_steps(crun, reps, cs.reset_status)
    ms = max_over_ranks(sum(t), world) / reps
    hits = int((cs.status() == 2).sum().item())
    l2 = l2_copy_bandwidth()
    achieved = COLLIDE_BYTES_PER_AGENT * cw.n / (ms / 1e3) / 1e9
    cp = profiled("collide_query", f"collision-field-{cw.n}", "collide")
    out["collide"] = {"value": world * cw.n / (ms / 1e3), "unit": "agents/s", "ms_per_call": ms,
                      "n_agents": cw.n, "collided": hits, "table_and_lists_MB": cws.numel() / 1e6,
                      "method": "spatial hash of cells twice the contact distance, 32-byte records in "
                                "linked lists, 2 x 2 x 2-cell search",
                      "roofline": {"bound": "l2", "achieved": achieved, "peak": l2, "unit": "GB/s",
                                   "frac": achieved / l2, "bytes_per_agent": COLLIDE_BYTES_PER_AGENT,
                                   "peak_basis": "measured in this run: 32 MB device-to-device copies that stay "
                                                 "in L2, 20 back to back (read + write bytes)",
                                   "traffic": cp.get("bytes_per_launch"), "counters": cp.get("profile"),
                                   "note": "the table, lists and positions (8 + 4 + 16 MB) stay in L2; random "
                                           "4- and 16-byte reads"}}
    cs.close()
    del cx, cws

    # scale sweep 1e3 .. 1e7 agents, 1000 closed-loop steps: plain K = 1, fused K = 10 and 100,
    # and fused at the tuned K
    sweep = []
    l2_bytes = 126e6
    for n in (1_000, 10_000, 100_000, 1_000_000, 10_000_000):
        sw = W.scale_sweep(n, nsteps=T_STEPS)
        m = min(n, CPU_SWEEP_MAX_AGENTS)
        _SWEEP_SLICES[n] = (sw.groups, sw.gid[:m].copy(), sw.x0[:m].copy(), sw.cmd[:m].copy(), sw.mode)
        ss = Sim(sw.groups, sw.n, sw.mode)
        sx0 = planar(torch.from_numpy(sw.x0)).to(dev)
        scmd = torch.from_numpy(sw.cmd).reshape(-1).to(dev)
        sx = sx0.clone()
        st = autotune.tune_step(ss, sx0, scmd, DT, T_STEPS)
        sreset = lambda: sx.copy_(sx0)  # noqa: E731
        row = {"n_agents": n}
        for label, k in (("plain", 1), ("K10", 10), ("K100", 100), ("fused", st["K"])):
            gr = ss.graph(sx, scmd, DT, T_STEPS, K=k)
            timed_steps(gr.launch, 1, sreset)
            t = timed_steps(gr.launch, 2, sreset)
            ms = sum(t) / len(t)
            rate = n * T_STEPS / (ms / 1e3)
            row[label] = {"value": rate, "unit": UNIT, "ms_per_1000_steps": ms, "K": k,
                          "tflops": FLOPS_PER_AGENT_STEP * rate / 1e12,
                          "alu_frac": alu_roofline(FLOPS_PER_AGENT_STEP, rate, sms, None, {}, "")["frac"]}
            if k == 1:
                gbs = BYTES_PER_AGENT_STEP_PLAIN * rate / 1e9
                row[label]["hbm_gbs_equiv"] = gbs
                if n * 84 > l2_bytes:  # state + commands exceed L2: an HBM figure
                    row[label]["hbm_frac"] = gbs / hbm if hbm else None
                else:
                    row[label]["hbm_frac"] = None
                    row[label]["l2_equiv_frac"] = gbs / hbm if hbm else None
                    row[label]["note"] = "state and commands stay in L2 between launches"
            gr.close()
        ss.close()
        sweep.append(row)
        del sx0, sx, scmd
    out["sweep"] = sweep
    big = sweep[-1]["plain"]
    out["plain"]["hbm_case"] = {"n_agents": sweep[-1]["n_agents"], "value": big["value"],
                                "achieved_GBs": big["hbm_gbs_equiv"], "frac": big.get("hbm_frac")}
    pl = profiled("step_kernel<1,false,plain>", f"closed-loop-{sweep[-1]['n_agents']}-K1")
    if pl:  # DRAM bytes of one launch from the committed ncu summary, against the algorithmic bytes
        out["plain"]["hbm_case"].update(traffic=pl["bytes_per_launch"], profile=pl["profile"],
                                        algorithmic_bytes=BYTES_PER_AGENT_STEP_PLAIN * sweep[-1]["n_agents"])

    # the paper's own measurement point: 1000 quadrotors, per-round time (context only)
    pw = W.scale_sweep(1000, nsteps=T_STEPS)
    pt, ms = swarm_leg(world, pw, dev, timed_steps, reps)
    out["n1000"] = {"value": 1000 * T_STEPS / (ms / 1e3), "unit": UNIT, "us_per_physics_step": ms,
                    "K": pt["K"], "block": pt["block"],
                    "note": "latency bound: " + sm_fill(1000, pt["block"], sms),
                    "paper_context": PAPER_1000}
    return out


if __name__ == "__main__":
    main()
