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
import re
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

#: Non-trivial floating operations (add/sub, mul, div, sqrt) of one
#: closed-loop agent-step in the checker's definition, the minimum over the
#: bench workload's states (748..762; operands that are exactly 0 or 1 are not
#: counted); tests pin it to the checker's operation counter.
FLOPS_PER_AGENT_STEP = 748
#: Tape edges of one closed-loop step in the checker's reverse mode (minimum
#: over the workload's states, 1348..1367); sweeping one costs a multiply and
#: an add.  Algorithmic work of forward + adjoint per agent-step: the forward
#: step, the step again to linearise it, and the reverse sweep.  The extra
#: forward recomputation that checkpointing adds is not counted.
ADJ_TAPE_EDGES_PER_AGENT_STEP = 1348
FWD_ADJ_FLOPS_PER_AGENT_STEP = 2 * FLOPS_PER_AGENT_STEP + 2 * ADJ_TAPE_EDGES_PER_AGENT_STEP
#: The same count for one step with the PID body-rate loop (minimum over the PID workload's
#: states, 760..774), less the checker's second evaluation of the time derivative for omega'
#: (a step takes omega' from its first RK4 stage).
FLOPS_PER_AGENT_STEP_PID = 760
#: The checker's count for one step of a car (98..101) and of a fixed-wing drone (156, plus
#: five transcendental functions: four tan and one atan2, not counted), minimum over the mixed
#: swarm's states.
FLOPS_PER_AGENT_STEP_CAR = 98
FLOPS_PER_AGENT_STEP_FIXED_WING = 156
#: Bytes one plain step of a one-group swarm moves per agent: state 68 read +
#: 68 written, command 16, status 1 (with one group the group id is not read).
BYTES_PER_AGENT_STEP_PLAIN = 153
#: FP32 lanes per SM (Blackwell) and the largest SM clock of the part.
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2032.0
L2_FLUSH_BYTES = 256 << 20
#: The sources that define the headline step kernel: a committed ncu figure is
#: used only while their fingerprint is the one it was taken on.  (vehicles.cuh
#: enters only the mixed-type instantiations.)
KERNEL_SOURCES = ("paper_2308_12698_b300/csrc/model_fwd.cuh", "paper_2308_12698_b300/csrc/step_kernel.cuh")


def kernel_sha() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str):
    """dram bytes per launch from a committed ncu summary, if taken on the current kernel source."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    sha = kernel_sha()
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith(".md"):
            continue
        txt = open(os.path.join(pdir, fn)).read()
        m = re.search(r"^bench_traffic:\s*kernel=(\S+)\s+workload=(\S+)\s+source_sha=(\w+)\s+bytes_per_launch=([\d.eE+]+)",
                      txt, re.M)
        if m and m.group(1) == kernel and m.group(2) == workload and m.group(3) == sha:
            return float(m.group(4))
    return None


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
    ap.add_argument("--block", type=int, default=0, help="fix the forward block size (with --pid-only, --multi-only)")
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
    if args.pid_only or args.multi_only:
        run_swarm_only(args, world, rank, dev, "pid" if args.pid_only else "multi")
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

    # roofline of the dominant kernel: the fused step kernel, FP32-ALU bound
    launch_s = (sum(times) / args.steps / launches) / 1e3
    flops_launch = FLOPS_PER_AGENT_STEP * NA * min(K, TS)
    peak_tflops = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    achieved = flops_launch / launch_s / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
            "traffic": profiled_traffic("step_kernel<1,false>", f"closed-loop-{NA}-K{K}"),
            "kernel": f"step_kernel<closed loop, one group>, K={K} fused steps, block {tune['block']}",
            "flops_per_agent_step": FLOPS_PER_AGENT_STEP,
            "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 (FMA) x {SM_MAX_MHZ:.0f} MHz max clock",
            "avg_launch_us": launch_s * 1e6}
    if clocks.get("sm_mhz"):
        roof["frac_at_measured_clock"] = achieved / (peak_tflops * clocks["sm_mhz"] / SM_MAX_MHZ)

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
        extra = side_measurements(args, world, sim, wl, x0, cmd, x, flush, stream, timed_steps, sms)

    peaks = measured_peaks()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config({"K": K, "block": tune["block"], "graph_launches_per_step": launches,
                                       "n_agents_per_gpu": NA, "physics_steps_per_bench_step": TS}),
            "roofline": roof, "clocks": clocks, "e2e": e2e, "gpu_launches": launches * args.steps,
            "repeat_spread": spread}
    line.update(extra)
    if "hbm_gbs" in peaks and "plain" in line:
        line["plain"]["roofline"]["peak"] = peaks["hbm_gbs"]
        line["plain"]["roofline"]["frac"] = line["plain"]["roofline"]["achieved"] / peaks["hbm_gbs"]
    if world == 1 and rank == 0:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
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
    PID-rate-loop swarm, "multi" the quadrotor / car / fixed-wing swarm in equal thirds."""
    import torch

    from paper_2308_12698_b300 import autotune
    from paper_2308_12698_b300 import workload as W
    from paper_2308_12698_b300.sim import Sim, planar
    NA, TS = args.agents, args.physics_steps
    if kind == "pid":
        wl = W.closed_loop_pid(n=NA, nsteps=TS)
        flops = FLOPS_PER_AGENT_STEP_PID
    else:
        sizes = (NA // 3, NA // 3, NA - 2 * (NA // 3))
        wl = W.multi_type(sizes=sizes, nsteps=TS)
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


def side_measurements(args, world, sim, wl, x0, cmd, x, flush, stream, timed_steps, sms) -> dict:
    """Plain kernel, fwd+adjoint and heterogeneous batch on the same GPU (3 timed reps each)."""
    import torch

    from paper_2308_12698_b300 import autotune
    from paper_2308_12698_b300 import workload as W
    from paper_2308_12698_b300.sim import Sim, planar
    reps = 3
    out = {}
    reset = lambda: x.copy_(x0)  # noqa: E731

    # plain one-step kernel: 1000 launches per bench step (graph), HBM bound
    g1 = sim.graph(x, cmd, DT, T_STEPS, K=1)
    timed_steps(g1.launch, 2, reset)
    t = timed_steps(g1.launch, reps, reset)
    ms = max_over_ranks(sum(t), world) / reps
    launch_s = ms / 1e3 / T_STEPS
    gbs = BYTES_PER_AGENT_STEP_PLAIN * N_AGENTS / launch_s / 1e9
    out["plain"] = {"value": world * N_AGENTS * T_STEPS / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                    "roofline": {"bound": "hbm", "achieved": gbs, "peak": None, "unit": "GB/s", "frac": None,
                                 "bytes_per_agent_step": BYTES_PER_AGENT_STEP_PLAIN,
                                 "note": "1e6-agent state (68 MB) + commands fit in the 126 MB L2 between launches"}}
    g1.close()

    # checkpointed forward + adjoint, 1e6 agents x 1000 steps, loss |p_T - goal|^2 + w sum Omega^2
    cfg = autotune.tune_adjoint(sim, x0, cmd, DT, T_STEPS)
    C = cfg["C"]
    ckpt = sim.ckpt_buffer(T_STEPS, C, device=x0.device)
    rc = torch.empty(sim.n, dtype=torch.float32, device=x0.device)
    gT = torch.zeros(17 * sim.n, dtype=torch.float32, device=x0.device)
    gT[: 3 * sim.n] = 1.0
    w = torch.full((sim.n,), 1e-6, dtype=torch.float32, device=x0.device)
    ws = torch.empty(max(sim.workspace_bytes(C), 1), dtype=torch.uint8, device=x0.device)

    def fwd_adj():
        sim.rollout_forward(x0, cmd, DT, T_STEPS, C=C, ckpt=ckpt, run_cost=rc)
        sim.rollout_backward(ckpt, cmd, DT, T_STEPS, gT, w, C=C, workspace=ws)

    timed_steps(fwd_adj, 2)
    t = timed_steps(fwd_adj, reps)
    ms = max_over_ranks(sum(t), world) / reps
    rate = N_AGENTS * T_STEPS / (ms / 1e3)
    peak_tf = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    out["fwd_adjoint"] = {"value": world * rate, "unit": UNIT, "ms_per_step": ms,
                          "C": C, "block_adj": cfg["block"], "workspace_MB": ws.numel() / 1e6,
                          "checkpoint_MB": ckpt.numel() * 4 / 1e6,
                          "roofline": {"bound": "alu", "achieved": FWD_ADJ_FLOPS_PER_AGENT_STEP * rate / 1e12,
                                       "peak": peak_tf, "unit": "TFLOP/s",
                                       "frac": FWD_ADJ_FLOPS_PER_AGENT_STEP * rate / 1e12 / peak_tf,
                                       "flops_per_agent_step": FWD_ADJ_FLOPS_PER_AGENT_STEP,
                                       "basis": "forward + linearised forward + reverse sweep (2 flops per tape edge)"}}
    del ckpt, ws

    # heterogeneous: 8 groups, uneven sizes (600k), one persistent launch per K steps, graph
    hw = W.heterogeneous(nsteps=T_STEPS, shuffle=False)
    gid = torch.from_numpy(hw.gid).to(x0.device)
    hs = Sim(hw.groups, hw.n, hw.mode, gid=gid)
    hx0 = planar(torch.from_numpy(hw.x0)).to(x0.device)
    hcmd = torch.from_numpy(hw.cmd).reshape(-1).to(x0.device)
    hx = hx0.clone()
    ht = autotune.tune_step(hs, hx0, hcmd, DT, T_STEPS)
    hg = hs.graph(hx, hcmd, DT, T_STEPS, K=ht["K"])
    hreset = lambda: hx.copy_(hx0)  # noqa: E731
    timed_steps(hg.launch, 2, hreset)
    t = timed_steps(hg.launch, reps, hreset)
    ms = max_over_ranks(sum(t), world) / reps
    hrate = hw.n * T_STEPS / (ms / 1e3)
    out["hetero"] = {"value": world * hrate, "unit": UNIT, "ms_per_step": ms,
                     "n_agents": hw.n, "groups": len(hw.groups), "sizes": list(W.HETERO_SIZES), "K": ht["K"],
                     "block": ht["block"],
                     "roofline": {"bound": "alu", "achieved": FLOPS_PER_AGENT_STEP * hrate / 1e12, "peak": peak_tf,
                                  "unit": "TFLOP/s", "frac": FLOPS_PER_AGENT_STEP * hrate / 1e12 / peak_tf,
                                  "flops_per_agent_step": FLOPS_PER_AGENT_STEP,
                                  "note": "the quadrotor step's count; every group runs the same operations"}}
    hg.close()
    hs.close()

    # PID body-rate loop: 1e6 agents with 20-component states, tuned K, one graph
    pw = W.closed_loop_pid(n=N_AGENTS, nsteps=T_STEPS)
    ps = Sim(pw.groups, pw.n, pw.mode)
    px0 = planar(torch.from_numpy(pw.x0)).to(x0.device)
    pcmd = torch.from_numpy(pw.cmd).reshape(-1).to(x0.device)
    px = px0.clone()
    pt = autotune.tune_step(ps, px0, pcmd, DT, T_STEPS)
    pg = ps.graph(px, pcmd, DT, T_STEPS, K=pt["K"])
    preset = lambda: px.copy_(px0)  # noqa: E731
    timed_steps(pg.launch, 2, preset)
    t = timed_steps(pg.launch, reps, preset)
    ms = max_over_ranks(sum(t), world) / reps
    rate = pw.n * T_STEPS / (ms / 1e3)
    out["pid"] = {"value": world * rate, "unit": UNIT, "ms_per_step": ms, "n_agents": pw.n, "K": pt["K"],
                  "block": pt["block"],
                  "roofline": {"bound": "alu", "achieved": FLOPS_PER_AGENT_STEP_PID * rate / 1e12, "peak": peak_tf,
                               "unit": "TFLOP/s", "frac": FLOPS_PER_AGENT_STEP_PID * rate / 1e12 / peak_tf,
                               "flops_per_agent_step": FLOPS_PER_AGENT_STEP_PID}}
    pg.close()
    ps.close()
    del px, px0, pcmd

    # quadrotors, cars and fixed-wing drones (200,000 each) in one persistent launch
    mw = W.multi_type(nsteps=T_STEPS)
    ms_ = Sim(mw.groups, mw.n, mw.mode, gid=torch.from_numpy(mw.gid).to(x0.device))
    mx0 = planar(torch.from_numpy(mw.x0)).to(x0.device)
    mcmd = torch.from_numpy(mw.cmd).reshape(-1).to(x0.device)
    mx = mx0.clone()
    mt = autotune.tune_step(ms_, mx0, mcmd, DT, T_STEPS)
    mg = ms_.graph(mx, mcmd, DT, T_STEPS, K=mt["K"])
    mreset = lambda: mx.copy_(mx0)  # noqa: E731
    timed_steps(mg.launch, 2, mreset)
    t = timed_steps(mg.launch, reps, mreset)
    ms = max_over_ranks(sum(t), world) / reps
    sizes = W.MULTI_TYPE_SIZES
    flops = (sizes[0] * FLOPS_PER_AGENT_STEP + sizes[1] * FLOPS_PER_AGENT_STEP_CAR +
             sizes[2] * FLOPS_PER_AGENT_STEP_FIXED_WING) * T_STEPS / (ms / 1e3)
    out["multi_type"] = {"value": world * mw.n * T_STEPS / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                         "n_agents": mw.n, "sizes": {"quadrotor": sizes[0], "car": sizes[1], "fixed_wing": sizes[2]},
                         "K": mt["K"], "block": mt["block"],
                         "roofline": {"bound": "alu", "achieved": flops / 1e12, "peak": peak_tf, "unit": "TFLOP/s",
                                      "frac": flops / 1e12 / peak_tf,
                                      "note": "flops weighted by type; the drones' tan/atan2 are not counted"}}
    mg.close()
    ms_.close()
    del mx, mx0, mcmd

    # decision rounds: commands from pinned host memory every M steps, positions back after
    # each round, both overlapped with the physics (1000 steps per bench step)
    rounds = {}
    for M in (10, 100):
        R = T_STEPS // M
        h_cmds = torch.from_numpy(wl.cmd).reshape(1, -1).repeat(R, 1).contiguous().pin_memory()
        h_obs = torch.empty((R, 4 * N_AGENTS), dtype=torch.float32).pin_memory()
        cmd2 = torch.empty(8 * N_AGENTS, dtype=torch.float32, device=x0.device)
        obs2 = torch.empty(8 * N_AGENTS, dtype=torch.float32, device=x0.device)
        Kr = min(sim.launch()["K"], M)
        rrun = lambda: sim.run_rounds(x, h_cmds, M, DT, K=Kr, h_obs=h_obs, cmd2=cmd2, obs2=obs2)  # noqa: E731
        timed_steps(rrun, 2, reset)
        t = timed_steps(rrun, reps, reset)
        ms = max_over_ranks(sum(t), world) / reps
        rounds[f"M{M}"] = {"value": world * N_AGENTS * T_STEPS / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                           "rounds": R, "K": Kr, "h2d_bytes_per_round": 16 * N_AGENTS,
                           "d2h_bytes_per_round": 16 * N_AGENTS}
    out["decision_rounds"] = rounds

    # collision detection: 1e6 agents at 2 m mean spacing, 1 % planted near pairs
    cw = W.collision_field(N_AGENTS)
    cs = Sim(cw.groups, cw.n, cw.mode)
    cx = planar(torch.from_numpy(cw.x0)).to(x0.device)
    cws = torch.empty(max(cs.collide_workspace_bytes(), 1), dtype=torch.uint8, device=x0.device)
    crun = lambda: cs.collide(cx, 1.0, cws)  # noqa: E731
    timed_steps(crun, 2, cs.reset_status)
    t = timed_steps(crun, reps, cs.reset_status)
    ms = max_over_ranks(sum(t), world) / reps
    hits = int((cs.status() == 2).sum().item())
    out["collide"] = {"value": world * cw.n / (ms / 1e3), "unit": "agents/s", "ms_per_call": ms,
                      "n_agents": cw.n, "collided": hits, "table_and_lists_MB": cws.numel() / 1e6,
                      "method": "spatial hash, linked lists, 27-cell search"}
    cs.close()
    del cx, cws

    # scale sweep 1e3 .. 1e7 agents, 1000 closed-loop steps: plain K = 1, fused K = 10 and 100,
    # and fused at the tuned K
    sweep = []
    peak_tflops = sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    hbm = measured_peaks().get("hbm_gbs")
    for n in (1_000, 10_000, 100_000, 1_000_000, 10_000_000):
        sw = W.scale_sweep(n, nsteps=T_STEPS)
        ss = Sim(sw.groups, sw.n, sw.mode)
        sx0 = planar(torch.from_numpy(sw.x0)).to(x0.device)
        scmd = torch.from_numpy(sw.cmd).reshape(-1).to(x0.device)
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
                          "alu_frac": FLOPS_PER_AGENT_STEP * rate / 1e12 / peak_tflops}
            if k == 1:
                row[label]["hbm_gbs"] = BYTES_PER_AGENT_STEP_PLAIN * rate / 1e9
                row[label]["hbm_frac"] = (BYTES_PER_AGENT_STEP_PLAIN * rate / 1e9 / hbm) if hbm else None
            gr.close()
        ss.close()
        sweep.append(row)
        del sx0, sx, scmd
    out["sweep"] = sweep

    # the paper's own measurement point: 1000 quadrotors, per-round time (context only)
    pw = W.scale_sweep(1000, nsteps=T_STEPS)
    ps = Sim(pw.groups, pw.n, pw.mode)
    px0 = planar(torch.from_numpy(pw.x0)).to(x0.device)
    pcmd = torch.from_numpy(pw.cmd).reshape(-1).to(x0.device)
    px = px0.clone()
    pt = autotune.tune_step(ps, px0, pcmd, DT, T_STEPS)
    pg = ps.graph(px, pcmd, DT, T_STEPS, K=pt["K"])
    preset = lambda: px.copy_(px0)  # noqa: E731
    timed_steps(pg.launch, 2, preset)
    t = timed_steps(pg.launch, reps, preset)
    ms = sum(t) / reps
    out["n1000"] = {"value": 1000 * T_STEPS / (ms / 1e3), "unit": UNIT, "us_per_physics_step": ms,
                    "K": pt["K"], "note": "latency bound: 1000 agents fill 4 of the SMs",
                    "paper_context": PAPER_1000}
    pg.close()
    ps.close()
    return out


if __name__ == "__main__":
    main()
