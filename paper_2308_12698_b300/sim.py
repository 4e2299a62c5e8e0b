"""Python face of libquadsim.so: a handle class, a CUDA-graph wrapper and a
torch.autograd.Function over the hand-written adjoint.

PyTorch only provides device memory and the stream; every step of the
simulation runs in the library's kernels.  State tensors are flat float32
CUDA tensors in the planar layout of include/quadsim.h (17 N floats; 20 N in
the PID mode).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import SimError, check, group_struct, lib

THETA_FIELDS = (("kp", 0), ("kp", 1), ("kp", 2), ("kd", 0), ("kd", 1), ("kd", 2), ("katt", 0), ("katt", 1),
                ("katt", 2), ("krate", 0), ("krate", 1), ("krate", 2), ("m", None), ("Jxx", None), ("Jyy", None),
                ("Jzz", None))


def _ptr(t) -> ctypes.c_void_p | None:
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_f32(t: torch.Tensor, numel: int, name: str):
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == numel):
        raise SimError(f"{name}: expected a contiguous float32 CUDA tensor of {numel} elements")


def theta_of(group: dict) -> list[float]:
    """The 16 differentiable parameters of a group, in the library's order."""
    return [float(group[k][i] if i is not None else group[k]) for k, i in THETA_FIELDS]


def with_theta(group: dict, theta) -> dict:
    g = {k: (list(v) if isinstance(v, (list, tuple)) else v) for k, v in group.items()}
    for (k, i), v in zip(THETA_FIELDS, theta):
        if i is None:
            g[k] = float(v)
        else:
            g[k][i] = float(v)
    return g


class Sim:
    """One swarm: n agents, parameter groups, per-agent uint8 group ids.

    gid: a uint8 CUDA tensor of n ids (kept alive by the handle), or None
    for a single group.
    """

    def __init__(self, groups: list[dict], n: int, mode: int, gid: torch.Tensor | None = None):
        L = lib()
        self.groups = [dict(g) for g in groups]
        self.n = int(n)
        self.mode = int(mode)
        #: state components per agent: 20 with the PID rate loop's integral, else 17
        self.nx = 20 if self.mode == _lib.SIM_CLOSED_LOOP_PID else 17
        if gid is not None:
            if not (gid.is_cuda and gid.dtype == torch.uint8 and gid.is_contiguous() and gid.numel() == n):
                raise SimError("gid: expected a contiguous uint8 CUDA tensor of n elements")
        self.gid = gid
        arr = (_lib.GroupParams * len(groups))(*[group_struct(g) for g in groups])
        h = ctypes.c_void_p()
        rc = L.sim_create(arr, len(groups), self.n, _ptr(gid) if len(groups) > 1 else None, self.mode,
                          ctypes.byref(h))
        check(rc, "sim_create")
        self._h = h

    # -- lifecycle --
    def close(self):
        if getattr(self, "_h", None):
            lib().sim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def n_groups(self) -> int:
        return len(self.groups)

    # -- configuration --
    def set_params(self, groups: list[dict]):
        arr = (_lib.GroupParams * len(groups))(*[group_struct(g) for g in groups])
        check(lib().sim_set_params(self._h, arr, len(groups)), "sim_set_params")
        self.groups = [dict(g) for g in groups]

    def set_theta(self, theta: np.ndarray):
        """Replace the 16 differentiable parameters of every group ((G, 16) array)."""
        theta = np.asarray(theta, dtype=np.float64).reshape(self.n_groups, 16)
        self.set_params([with_theta(g, t) for g, t in zip(self.groups, theta)])

    def theta(self) -> np.ndarray:
        return np.array([theta_of(g) for g in self.groups], dtype=np.float32)

    def set_launch(self, block: int = 0, K: int = 0, C: int = 0, block_adj: int = 0):
        check(lib().sim_set_launch(self._h, int(block), int(block_adj), int(K), int(C)), "sim_set_launch")

    def launch(self) -> dict:
        """Current launch configuration: block, block_adj, K, C."""
        v = [ctypes.c_int() for _ in range(4)]
        check(lib().sim_get_launch(self._h, *[ctypes.byref(x) for x in v]), "sim_get_launch")
        return dict(zip(("block", "block_adj", "K", "C"), (x.value for x in v)))

    # -- forward --
    def step(self, state: torch.Tensor, cmd: torch.Tensor, dt: float, nsteps: int, K: int = 0, stream=None):
        _check_f32(state, self.nx * self.n, "state")
        _check_f32(cmd, 4 * self.n, "cmd")
        check(lib().sim_step(self._h, _ptr(state), _ptr(cmd), float(dt), int(nsteps), int(K), _stream(stream)),
              "sim_step")

    def step_host(self, h_state: torch.Tensor, h_cmd: torch.Tensor, d_state: torch.Tensor, d_cmd: torch.Tensor,
                  dt: float, nsteps: int, K: int = 0, stream=None):
        """Host-resident state: copy in, step, copy out, wait (pinned host tensors)."""
        for t, m in ((h_state, self.nx), (h_cmd, 4)):
            if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or t.numel() != m * self.n:
                raise SimError("host buffers: expected contiguous float32 CPU tensors")
        _check_f32(d_state, self.nx * self.n, "d_state")
        _check_f32(d_cmd, 4 * self.n, "d_cmd")
        check(lib().sim_step_host(self._h, _ptr(h_state), _ptr(h_cmd), _ptr(d_state), _ptr(d_cmd), float(dt),
                                  int(nsteps), int(K), _stream(stream)), "sim_step_host")

    def run_rounds(self, state: torch.Tensor, h_cmds: torch.Tensor, steps_per_round: int, dt: float, K: int = 0,
                   h_obs: torch.Tensor | None = None, cmd2: torch.Tensor | None = None,
                   obs2: torch.Tensor | None = None, stream=None):
        """Decision rounds: h_cmds (rounds, 4 N) pinned host commands, one set per round; the
        positions plane after each round lands in h_obs (rounds, 4 N) pinned host memory."""
        _check_f32(state, self.nx * self.n, "state")
        rounds = h_cmds.shape[0]
        if h_cmds.is_cuda or h_cmds.dtype != torch.float32 or not h_cmds.is_contiguous() or \
                h_cmds.numel() != rounds * 4 * self.n:
            raise SimError("h_cmds: expected a contiguous float32 CPU tensor (rounds, 4 N)")
        if h_obs is not None and (h_obs.is_cuda or h_obs.dtype != torch.float32 or not h_obs.is_contiguous() or
                                  h_obs.numel() != rounds * 4 * self.n):
            raise SimError("h_obs: expected a contiguous float32 CPU tensor (rounds, 4 N)")
        dev = state.device
        if cmd2 is None:
            cmd2 = torch.empty(8 * self.n, dtype=torch.float32, device=dev)
        if h_obs is not None and obs2 is None:
            obs2 = torch.empty(8 * self.n, dtype=torch.float32, device=dev)
        check(lib().sim_run_rounds(self._h, _ptr(state), _ptr(cmd2), _ptr(h_cmds), _ptr(obs2) if h_obs is not None
                                   else None, _ptr(h_obs), float(dt), int(steps_per_round), int(rounds), int(K),
                                   _stream(stream)), "sim_run_rounds")

    def launches(self, nsteps: int, K: int = 0) -> int:
        return int(lib().sim_step_launches(self._h, int(nsteps), int(K)))

    def n_segments(self, nsteps: int, C: int = 0) -> int:
        C = C or self.launch()["C"]
        return (int(nsteps) + C - 1) // C

    def ckpt_stride(self) -> int:
        """Floats from one checkpoint state to the next: nx N rounded up to a multiple of 4."""
        return (self.nx * self.n + 3) & ~3

    def ckpt_buffer(self, nsteps: int, C: int = 0, device=None) -> torch.Tensor:
        """An uninitialised checkpoint buffer: (S+1, nx N) rows, one planar state each, ckpt_stride()
        floats apart (contiguous when N is a multiple of 4)."""
        S = self.n_segments(nsteps, C)
        P = self.ckpt_stride()
        buf = torch.empty(S * P + self.nx * self.n, dtype=torch.float32, device=device)
        return buf.as_strided((S + 1, self.nx * self.n), (P, 1))

    def _check_ckpt(self, ckpt: torch.Tensor, nsteps: int, C: int):
        S = self.n_segments(nsteps, C)
        if not (ckpt.is_cuda and ckpt.dtype == torch.float32 and tuple(ckpt.shape) == (S + 1, self.nx * self.n)
                and (self.n == 0 or ckpt.stride() == (self.ckpt_stride(), 1))):
            raise SimError(f"ckpt: expected a float32 CUDA tensor ({S + 1}, {self.nx * self.n}) with row stride "
                           f"{self.ckpt_stride()} (see ckpt_buffer)")

    def rollout_forward(self, x0: torch.Tensor, cmd: torch.Tensor, dt: float, nsteps: int, C: int = 0,
                        ckpt: torch.Tensor | None = None, run_cost: torch.Tensor | None = None, stream=None):
        """Returns (ckpt, run_cost): ckpt is (S+1, nx N) rows of planar states (ckpt_buffer),
        ckpt[-1] the final state."""
        _check_f32(x0, self.nx * self.n, "x0")
        _check_f32(cmd, 4 * self.n, "cmd")
        if ckpt is None:
            ckpt = self.ckpt_buffer(nsteps, C, device=x0.device)
        self._check_ckpt(ckpt, nsteps, C)
        if run_cost is None:
            run_cost = torch.empty(self.n, dtype=torch.float32, device=x0.device)
        check(lib().sim_rollout_forward(self._h, _ptr(x0), _ptr(cmd), float(dt), int(nsteps), int(C), _ptr(ckpt),
                                        _ptr(run_cost), _stream(stream)), "sim_rollout_forward")
        return ckpt, run_cost

    # -- adjoint --
    def workspace_bytes(self, C: int = 0) -> int:
        return int(lib().sim_workspace_bytes(self._h, int(C)))

    def rollout_backward(self, ckpt: torch.Tensor, cmd: torch.Tensor, dt: float, nsteps: int, dL_dxT: torch.Tensor,
                         w_run: torch.Tensor | None = None, C: int = 0, per_agent: bool = False,
                         workspace: torch.Tensor | None = None, stream=None):
        """Returns (dL/dx0 planar, dL/dtheta (G, 16), per-agent (N, 16) or None)."""
        self._check_ckpt(ckpt, nsteps, C)
        _check_f32(dL_dxT, self.nx * self.n, "dL_dxT")
        if w_run is not None:
            _check_f32(w_run, self.n, "w_run")
        dev = ckpt.device
        ws = self.workspace_bytes(C)
        if workspace is None or workspace.numel() < ws:
            workspace = torch.empty(max(ws, 1), dtype=torch.uint8, device=dev)
        dx0 = torch.empty(self.nx * self.n, dtype=torch.float32, device=dev)
        dth = torch.empty((self.n_groups, 16), dtype=torch.float32, device=dev)
        dth_a = torch.empty((self.n, 16), dtype=torch.float32, device=dev) if per_agent else None
        check(lib().sim_rollout_backward(self._h, _ptr(ckpt), _ptr(cmd), float(dt), int(nsteps), int(C),
                                         _ptr(dL_dxT), _ptr(w_run), _ptr(dx0), _ptr(dth), _ptr(dth_a),
                                         _ptr(workspace), ws, _stream(stream)), "sim_rollout_backward")
        return dx0, dth, dth_a

    # -- collisions --
    def collide_workspace_bytes(self) -> int:
        return int(lib().sim_collide_workspace_bytes(self._h))

    def collide(self, state: torch.Tensor, radius_scale: float = 1.0, workspace: torch.Tensor | None = None,
                stream=None):
        """Marks agents closer than the sum of their arm lengths (x radius_scale) dead (status 2)."""
        _check_f32(state, self.nx * self.n, "state")
        ws = self.collide_workspace_bytes()
        if workspace is None or workspace.numel() < ws:
            workspace = torch.empty(max(ws, 1), dtype=torch.uint8, device=state.device)
        check(lib().sim_collide(self._h, _ptr(state), float(radius_scale), _ptr(workspace), ws, _stream(stream)),
              "sim_collide")

    def status(self, stream=None) -> torch.Tensor:
        """Per-agent status bytes (0 alive, 1 non-finite, 2 collided) as a uint8 CUDA tensor."""
        out = torch.empty(max(self.n, 0), dtype=torch.uint8, device=torch.device("cuda", torch.cuda.current_device()))
        check(lib().sim_copy_status(self._h, _ptr(out) if self.n else None, _stream(stream)), "sim_copy_status")
        return out

    def load_status(self, status: torch.Tensor, stream=None):
        """Replace the per-agent status bytes (uint8 CUDA tensor of n): with the state, a resume."""
        if not (status.is_cuda and status.dtype == torch.uint8 and status.is_contiguous() and
                status.numel() == self.n):
            raise SimError("status: expected a contiguous uint8 CUDA tensor of n elements")
        check(lib().sim_load_status(self._h, _ptr(status) if self.n else None, _stream(stream)), "sim_load_status")

    # -- status --
    def n_dead(self, timeout_ms: int = 60000, stream=None) -> int:
        v = ctypes.c_int64()
        check(lib().sim_status(self._h, ctypes.byref(v), int(timeout_ms), _stream(stream)), "sim_status")
        return int(v.value)

    def reset_status(self, stream=None):
        check(lib().sim_reset_status(self._h, _stream(stream)), "sim_reset_status")

    def group_stats(self, state: torch.Tensor, stream=None):
        """Per group: live, non-finite and collided counts and the live agents' mean position,
        as a (n_groups, 6) float64 numpy array (sim_group_stats)."""
        _check_f32(state, self.nx * self.n, "state")
        out = np.zeros((self.n_groups, 6), dtype=np.float64)
        check(lib().sim_group_stats(self._h, _ptr(state) if self.n else None,
                                    out.ctypes.data_as(ctypes.c_void_p), _stream(stream)), "sim_group_stats")
        return out

    def compact(self, stream=None):
        """Step only the live agents from now on (sim_compact); graphs captured before go stale."""
        check(lib().sim_compact(self._h, _stream(stream)), "sim_compact")

    # -- graphs --
    def graph(self, state: torch.Tensor, cmd: torch.Tensor, dt: float, nsteps: int, K: int = 0) -> "Graph":
        return Graph(self, state, cmd, dt, nsteps, K)


class Graph:
    """ceil(nsteps/K) sim_step launches captured once, replayed by launch()."""

    def __init__(self, sim: Sim, state: torch.Tensor, cmd: torch.Tensor, dt: float, nsteps: int, K: int = 0):
        _check_f32(state, sim.nx * sim.n, "state")
        _check_f32(cmd, 4 * sim.n, "cmd")
        self.sim = sim
        self._bufs = (state, cmd)
        self.launches_per_replay = sim.launches(nsteps, K)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        g = ctypes.c_void_p()
        check(lib().sim_graph_create(sim.handle, _ptr(state), _ptr(cmd), float(dt), int(nsteps), int(K),
                                     ctypes.c_void_p(side.cuda_stream), ctypes.byref(g)), "sim_graph_create")
        torch.cuda.current_stream().wait_stream(side)
        self._g = g

    def launch(self, stream=None):
        if not self.sim.handle:  # the graph's kernels use the handle's buffers: it must outlive the graph
            raise SimError("graph launch after its Sim was closed")
        check(lib().sim_graph_launch(self._g, _stream(stream)), "sim_graph_launch")

    def close(self):
        if getattr(self, "_g", None):
            lib().sim_graph_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class QuadRollout(torch.autograd.Function):
    """(theta (G, 16), x0 planar) -> (x_T planar, run_cost (N,)).

    theta = per group (kp[3], kd[3], katt[3], krate[3], m, Jxx, Jyy, Jzz);
    run_cost_a = sum_{n=1..T} sum_i Omega_{n,i}^2.  The backward pass is the
    library's discrete adjoint with checkpoints every C steps; it returns
    gradients for theta and x0.

    The adjoint recomputes the rollout from its checkpoints under the handle's
    parameters, so backward runs under the theta that forward used: if the
    handle's theta has changed since (sim.set_theta, or another forward with
    another theta on the same handle), backward puts the saved theta back for
    its own call and restores the newer one afterwards.  Parameter changes
    wait for the current stream (sim_set_params does not order itself against
    work in flight).
    """

    @staticmethod
    def forward(ctx, theta, x0, sim: Sim, cmd, dt: float, nsteps: int, C: int = 0):
        th = theta.detach().cpu().numpy().astype(np.float32)
        if not np.array_equal(th, sim.theta()):
            _set_theta_ordered(sim, th)
        ckpt, rc = sim.rollout_forward(x0.detach().contiguous(), cmd, dt, nsteps, C)
        ctx.sim, ctx.cmd, ctx.dt, ctx.nsteps, ctx.C = sim, cmd, dt, nsteps, C
        ctx.theta_device = theta.device
        ctx.theta = th
        ctx.save_for_backward(ckpt)
        return ckpt[-1].clone(), rc

    @staticmethod
    def backward(ctx, g_xT, g_rc):
        (ckpt,) = ctx.saved_tensors
        sim = ctx.sim
        if g_xT is None:
            g_xT = torch.zeros(sim.nx * sim.n, dtype=torch.float32, device=ckpt.device)
        w = None if g_rc is None else g_rc.contiguous().float()
        current = [dict(g) for g in sim.groups]
        swapped = not np.array_equal(sim.theta(), ctx.theta)
        if swapped:
            _set_theta_ordered(sim, ctx.theta)
        dx0, dth, _ = sim.rollout_backward(ckpt, ctx.cmd, ctx.dt, ctx.nsteps, g_xT.contiguous().float(), w, ctx.C)
        if swapped:
            torch.cuda.current_stream().synchronize()
            sim.set_params(current)
        return dth.to(ctx.theta_device), dx0, None, None, None, None, None


def _set_theta_ordered(sim: Sim, theta: np.ndarray):
    """sim.set_theta after the current stream's work (which may still read the old parameters)."""
    torch.cuda.current_stream().synchronize()
    sim.set_theta(theta)


def planar(x: torch.Tensor) -> torch.Tensor:
    """(N, 17) or (N, 20) -> flat planar layout (data movement only): planes of components
    0-3, 4-7, 8-11, 12-15, then the rest (16, or 16-19) interleaved per agent."""
    n, nx = x.shape
    if nx not in (17, 20):
        raise SimError("planar: states have 17 or 20 components")
    out = torch.empty(nx * n, dtype=x.dtype, device=x.device)
    for k in range(4):
        out[4 * k * n: 4 * k * n + 4 * n] = x[:, 4 * k:4 * k + 4].reshape(-1)
    out[16 * n:] = x[:, 16:].reshape(-1)
    return out


def unplanar(flat: torch.Tensor, n: int) -> torch.Tensor:
    """flat planar layout -> (N, 17) or (N, 20), from the size."""
    nx = flat.numel() // n if n else 17
    if nx not in (17, 20) or nx * n != flat.numel():
        raise SimError("unplanar: expected 17 N or 20 N floats")
    x = torch.empty((n, nx), dtype=flat.dtype, device=flat.device)
    for k in range(4):
        x[:, 4 * k:4 * k + 4] = flat[4 * k * n: 4 * k * n + 4 * n].reshape(n, 4)
    x[:, 16:] = flat[16 * n: nx * n].reshape(n, nx - 16)
    return x
