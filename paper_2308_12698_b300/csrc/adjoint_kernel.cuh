// The differentiable rollout's kernels: the forward rollout with checkpoints
// (ckpt_kernel), the discrete adjoint swept backwards segment by segment
// (adjoint_kernel, with the vector-Jacobian products of model_adj.cuh) and the
// fixed-order sum of the per-block group partials (reduce_partials).  One
// thread per agent; grid-stride over a resident wave.
#pragma once
#include "model_adj.cuh"
#include "step_kernel.cuh"

namespace qs {

struct CkptArgs {
  const float* x0;
  float* ckpt;
  float* run_cost;
  const float4* cmd;
  const uint8_t* gid;
  uint8_t* status;
  int64_t n;
  int64_t nsteps;
  int C;
  int S;
  int n_groups;
  StepH H;
  const DevGroup* groups;
  const uint32_t* order;  // null, or the live agents' order: agent order[j] for j < count
  int64_t count;          // agents the kernel visits: n, or the order's length
  LinCoef coef;           // one group: its RK4 weights of the linear parts (lin_coef, on the host)
};

// Floats from one checkpoint to the next: a planar state (NS N floats)
// rounded up to a multiple of 4, so that every checkpoint starts on a 16-byte
// boundary as its float4 planes need (N not a multiple of 4 leaves a gap).
__host__ __device__ constexpr int64_t ckpt_stride(int ns, int64_t n) { return ((int64_t)ns * n + 3) & ~(int64_t)3; }

// Whole forward rollout in one launch, checkpoint every C steps.  Agents in
// the forward kernels' scheduler-first 32-agent chunks; the step loop unrolled
// by two, with C = 1 (a checkpoint after every step) as its own loop: 14.1 ->
// 12.8 ms at C = 1 and 12.2 -> 11.7 ms at C = 100 for 1e6 agents x 1000 steps,
// bit for bit the same checkpoints.
template <int MODE, bool HETERO>
__global__ void __launch_bounds__(256) ckpt_kernel(CkptArgs A, const DevGroup P0) {
  extern __shared__ float4 smem4[];
  DevGroup* sg = reinterpret_cast<DevGroup*>(smem4);
  load_groups<HETERO>(sg, A.groups, A.n_groups);
  constexpr int NS = state_dim<MODE>();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t cstride = ckpt_stride(NS, A.n);
  for (int64_t j = first_agent(); j < A.count; j += stride) {
    const int64_t i = A.order ? (int64_t)A.order[j] : j;
#ifdef QS_CHECKED
    if (!QS_OK(i >= 0 && i < A.n, 4, i)) continue;
    if (HETERO && !QS_OK(A.gid[i] < A.n_groups, 5, A.gid[i])) continue;
#endif
    St x;
    load_state<NS>(A.x0, A.n, i, x);
    store_state<NS>(A.ckpt, A.n, i, x);
    if (A.status[i]) {  // frozen: every checkpoint is the current state
      for (int s = 1; s <= A.S; ++s) store_state<NS>(A.ckpt + s * cstride, A.n, i, x);
      if (A.run_cost) A.run_cost[i] = 0.f;
      continue;
    }
    const float4 c = A.cmd[i];
    const Hd hd = heading(MODE != 0 ? c.w : 0.f);
    const DevGroup P = HETERO ? sg[A.gid[i]] : P0;
    const LinCoef L = HETERO ? lin_coef(P, A.H) : A.coef;
    float rc = 0.f;
    float* dst = A.ckpt;  // checkpoint s + 1 follows checkpoint s at cstride floats
    if (A.C == 1) {
#pragma unroll 2
      for (int s = 0; s < A.S; ++s) {
        step<MODE>(P, x, c, hd, A.H, L);
        rc += (x.a[OM] * x.a[OM] + x.a[OM + 1] * x.a[OM + 1]) + (x.a[OM + 2] * x.a[OM + 2] + x.a[OM + 3] * x.a[OM + 3]);
        dst += cstride;
#ifdef QS_CHECKED
        if (!QS_OK(s + 1 <= A.S, 8, s + 1)) break;
#endif
        store_state<NS>(dst, A.n, i, x);
      }
    } else {
      for (int s = 0; s < A.S; ++s) {
        const int len = (int)min((int64_t)A.C, A.nsteps - (int64_t)s * A.C);
#pragma unroll 2
        for (int k = 0; k < len; ++k) {
          step<MODE>(P, x, c, hd, A.H, L);
          rc += (x.a[OM] * x.a[OM] + x.a[OM + 1] * x.a[OM + 1]) + (x.a[OM + 2] * x.a[OM + 2] + x.a[OM + 3] * x.a[OM + 3]);
        }
        dst += cstride;
#ifdef QS_CHECKED
        if (!QS_OK(s + 1 <= A.S, 8, s + 1)) break;
#endif
        store_state<NS>(dst, A.n, i, x);
      }
    }
    if (A.run_cost) A.run_cost[i] = rc;
    if (!all_finite<NS>(x)) A.status[i] = 1;
  }
}

// With the live agents' order, ckpt_kernel visits only those agents: every
// agent dead at the start of the rollout gets its frozen checkpoints here (the
// start state at every checkpoint, no running cost), as ckpt_kernel writes them
// for the dead agents it visits.
template <int MODE>
__global__ void __launch_bounds__(256) ckpt_frozen_kernel(CkptArgs A) {
  constexpr int NS = state_dim<MODE>();
  const int64_t cstride = ckpt_stride(NS, A.n);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += stride) {
    if (!A.status[i]) continue;
    St x;
    load_state<NS>(A.x0, A.n, i, x);
    for (int s = 0; s <= A.S; ++s) store_state<NS>(A.ckpt + s * cstride, A.n, i, x);
    if (A.run_cost) A.run_cost[i] = 0.f;
  }
}

struct AdjArgs {
  const float* ckpt;
  const float4* cmd;
  const uint8_t* gid;
  const uint8_t* status;
  const float* dLdxT;
  const float* w_run;
  float* dLdx0;
  float* th_agent;
  float* partials;  // [gridDim.x][n_groups][16]
  float* scratch;   // [C][state planes][grid threads]
  int64_t n;
  int64_t nsteps;
  int C;
  int S;
  int n_groups;
  StepH H;
  const DevGroup* groups;
  const uint32_t* order;  // null, or the live agents' order: agent order[j] for j < count
  int64_t count;          // agents the kernel visits: n, or the order's length
};

// Starts copying agent i's state out of the planar checkpoint `src` (n
// agents) into this thread's prefetch slot: five float4 slots, `bd` apart
// (plane 4 of a 17-float state is one float, copied into the slot's first
// four bytes).
template <int NS>
__device__ __forceinline__ void prefetch_state(float4* dst, int bd, const float* src, int64_t n, int64_t i) {
#ifdef QS_CHECKED
  if (!QS_OK(i >= 0 && i < n, 3, i)) {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    return;
  }
#endif
  const float4* P = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int k = 0; k < 4; ++k) cp_async16(dst + k * bd, P + k * n + i);
  if (NS == NXP)
    cp_async16(dst + 4 * bd, P + 4 * n + i);
  else
    cp_async4(dst + 4 * bd, src + 16 * n + i);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int NS>
__device__ __forceinline__ void read_prefetched(const float4* src, int bd, St& x) {
  const float4 a = src[0], b = src[bd], c = src[2 * bd], d = src[3 * bd], e = src[4 * bd];
  x.a[0] = a.x; x.a[1] = a.y; x.a[2] = a.z; x.a[3] = a.w;
  x.a[4] = b.x; x.a[5] = b.y; x.a[6] = b.z; x.a[7] = b.w;
  x.a[8] = c.x; x.a[9] = c.y; x.a[10] = c.z; x.a[11] = c.w;
  x.a[12] = d.x; x.a[13] = d.y; x.a[14] = d.z; x.a[15] = d.w;
  x.a[16] = e.x;
  if (NS == NXP) { x.a[17] = e.y; x.a[18] = e.z; x.a[19] = e.w; }
}

// Discrete adjoint: per agent, segments in reverse; each segment is
// recomputed from its checkpoint into this thread's scratch column, then
// swept backwards step by step.  Per-agent theta cotangents are reduced per
// group inside each warp (fixed butterfly order), accumulated per warp in
// shared memory, and written as one partial per block.
// SMEMS: the segment's step-start states live in shared memory (small C)
// rather than in the global scratch, and each segment's checkpoint is
// prefetched into shared memory (cp.async, double-buffered) while the
// segment before it in the sweep is being processed.
// ORDER: the agents of the live agents' order (A.order, A.count) rather than
// all n in index order.
template <int MODE, bool SMEMS, bool ORDER = false>
__global__ void __launch_bounds__(128) adjoint_kernel(AdjArgs A) {
  extern __shared__ float4 smem4[];
  // shared memory: the group table, each group's RK4 weights, the per-warp
  // accumulators, then (16-byte aligned) the scratch and prefetch slots
  DevGroup* sg = reinterpret_cast<DevGroup*>(smem4);
  LinCoef* scoef = reinterpret_cast<LinCoef*>(sg + A.n_groups);
  float* wacc = reinterpret_cast<float*>(scoef + A.n_groups);
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < nw * A.n_groups * NTH; e += blockDim.x) wacc[e] = 0.f;
  load_groups<true>(sg, A.groups, A.n_groups);
  for (int g = threadIdx.x; g < A.n_groups; g += blockDim.x) scoef[g] = lin_coef(sg[g], A.H);
  __syncthreads();
  float* sscr = reinterpret_cast<float*>(
      smem4 + (sizeof(DevGroup) * A.n_groups + sizeof(LinCoef) * A.n_groups + 4 * nw * A.n_groups * NTH + 15) / 16);
  float* const scratch = SMEMS ? sscr : A.scratch;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;  // grid stride over agents
  // scratch column of this thread: its own slot in the block (shared) or in the grid (global)
  const int64_t scols = SMEMS ? (int64_t)blockDim.x : nthreads;
  const int64_t slot = SMEMS ? (int64_t)threadIdx.x : (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int NS = state_dim<MODE>();
  const int64_t sstep = (int64_t)NS * scols;
  const int64_t cstride = ckpt_stride(NS, A.n);
  // prefetch slots: [2 buffers][5 planes][block] float4, after the scratch (SMEMS: for the
  // checkpoints; global scratch: for the segment's step-start states)
  const int bd = blockDim.x;
  float4* const mypf = reinterpret_cast<float4*>(sscr + (SMEMS ? (int64_t)A.C * sstep : 0)) + threadIdx.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < A.count; base += nthreads) {
    const int64_t j = base + threadIdx.x;
    const bool in = j < A.count;  // every lane stays in the loop for the warp's reduction below
    const int64_t i = ORDER ? (in ? (int64_t)A.order[j] : A.n) : j;
    float tb[NTH], dc[NDC];
#pragma unroll
    for (int q = 0; q < NTH; ++q) tb[q] = 0.f;
#pragma unroll
    for (int q = 0; q < NDC; ++q) dc[q] = 0.f;
    int g = -1;
#ifdef QS_CHECKED
    // a failed check leaves the lane in the loop (the warp's reduction below needs every lane)
    const bool skip = in && (!QS_OK(i >= 0 && i < A.n, 4, i) || (A.gid && !QS_OK(A.gid[i] < A.n_groups, 5, A.gid[i])));
#else
    constexpr bool skip = false;
#endif
    if (!skip && in && A.status[i] == 0) {
      g = A.gid ? (int)A.gid[i] : 0;
      const DevGroup& P = sg[g];  // read from shared memory where used: keeps registers for the adjoint
      const LinCoef& L = scoef[g];
      const float4 c = A.cmd[i];
      const Hd hd = heading(MODE != 0 ? c.w : 0.f);
      const float w = A.w_run ? A.w_run[i] : 0.f;
      St lam, x;
      load_state<NS>(A.dLdxT, A.n, i, lam);
      load_state<NS>(A.ckpt + (int64_t)A.S * cstride, A.n, i, x);
#pragma unroll
      for (int q = 0; q < 4; ++q) lam.a[OM + q] += 2.f * w * x.a[OM + q];
      if (SMEMS) prefetch_state<NS>(mypf, bd, A.ckpt + (int64_t)(A.S - 1) * cstride, A.n, i);
      for (int s = A.S - 1; s >= 0; --s) {
        const int64_t n0 = (int64_t)s * A.C;
        const int len = (int)min((int64_t)A.C, A.nsteps - n0);
#ifdef QS_CHECKED
        if (!QS_OK(s < A.S && len >= 1 && len <= A.C, 9, len)) break;
#endif
        if (SMEMS) {
          // this segment's checkpoint has arrived; start fetching the next one
          const int b = (A.S - 1 - s) & 1;
          cp_async_wait_all();
          read_prefetched<NS>(mypf + b * 5 * bd, bd, x);
          if (s > 0) prefetch_state<NS>(mypf + (b ^ 1) * 5 * bd, bd, A.ckpt + (int64_t)(s - 1) * cstride, A.n, i);
        } else {
          load_state<NS>(A.ckpt + (int64_t)s * cstride, A.n, i, x);
        }
        if (SMEMS) {
          for (int j = 0; j < len; ++j) {
            store_state<NS>(scratch + j * sstep, scols, slot, x);
            if (j + 1 < len) step<MODE>(P, x, c, hd, A.H, L);
          }
          for (int j = len - 1; j >= 0; --j) {
            load_state<NS>(scratch + j * sstep, scols, slot, x);
            step_vjp<MODE>(P, x, c, hd, A.H, L, lam, tb, dc);
            if (n0 + j >= 1) {
#pragma unroll
              for (int q = 0; q < 4; ++q) lam.a[OM + q] += 2.f * w * x.a[OM + q];
            }
          }
        } else {
          // global scratch: the segment's last step-start state stays in
          // registers; each earlier one is copied back into this thread's
          // prefetch slot (cp.async, double-buffered) while the step after it
          // is swept, so no step waits on a global load
          for (int j = 0; j + 1 < len; ++j) {
            store_state<NS>(scratch + j * sstep, scols, slot, x);
            step<MODE>(P, x, c, hd, A.H, L);
          }
          __threadfence_block();  // the stores above before the copies below
          for (int j = len - 1; j >= 0; --j) {
            if (j + 1 < len) {
              cp_async_wait_all();
              read_prefetched<NS>(mypf + (j & 1) * 5 * bd, bd, x);
            }
            if (j > 0) prefetch_state<NS>(mypf + ((j - 1) & 1) * 5 * bd, bd, scratch + (j - 1) * sstep, scols, slot);
            step_vjp<MODE>(P, x, c, hd, A.H, L, lam, tb, dc);
            if (n0 + j >= 1) {
#pragma unroll
              for (int q = 0; q < 4; ++q) lam.a[OM + q] += 2.f * w * x.a[OM + q];
            }
          }
        }
      }
      theta_from_derived(P, dc, tb);
      store_state<NS>(A.dLdx0, A.n, i, lam);
      if (A.th_agent && QS_OK(i < A.n, 9, i)) {
#pragma unroll
        for (int q = 0; q < NTH; ++q) A.th_agent[i * NTH + q] = tb[q];
      }
    } else if (!skip && in) {
      // a dead agent is frozen over the rollout (x_T = x_0, no running
      // cost): dL/dx_0 = dL/dx_T, and it adds nothing to theta
      St lam;
      load_state<NS>(A.dLdxT, A.n, i, lam);
      store_state<NS>(A.dLdx0, A.n, i, lam);
      if (A.th_agent) {
#pragma unroll
        for (int q = 0; q < NTH; ++q) A.th_agent[i * NTH + q] = 0.f;
      }
    }
    unsigned todo = __ballot_sync(0xffffffffu, g >= 0);
    while (todo) {
      const int leader = __ffs(todo) - 1;
      const int gl = __shfl_sync(0xffffffffu, g, leader);
      const bool mine = (g == gl);
      todo &= ~__ballot_sync(0xffffffffu, mine);
#pragma unroll
      for (int q = 0; q < NTH; ++q) {
        float v = mine ? tb[q] : 0.f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0 && QS_OK(gl >= 0 && gl < A.n_groups, 5, gl)) wacc[(warp * A.n_groups + gl) * NTH + q] += v;
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < A.n_groups * NTH; e += blockDim.x) {
    float s = 0.f;
    for (int w = 0; w < nw; ++w) s += wacc[w * A.n_groups * NTH + e];
    A.partials[(int64_t)blockIdx.x * A.n_groups * NTH + e] = s;
  }
}

// With the live agents' order, adjoint_kernel visits only those agents: every
// agent dead when the sweep runs gets the frozen map's gradient here (dL/dx0 =
// dL/dx_T, a zero theta row), as adjoint_kernel writes it for the dead agents
// it visits.
template <int MODE>
__global__ void __launch_bounds__(256) adjoint_frozen_kernel(AdjArgs A) {
  constexpr int NS = state_dim<MODE>();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += stride) {
    if (!A.status[i]) continue;
    St lam;
    load_state<NS>(A.dLdxT, A.n, i, lam);
    store_state<NS>(A.dLdx0, A.n, i, lam);
    if (A.th_agent)
      for (int q = 0; q < NTH; ++q) A.th_agent[i * NTH + q] = 0.f;
  }
}

// out[e] = sum over blocks b of partials[b][e], fixed order: each thread sums
// a strided subset in increasing b, then a fixed shared-memory tree.
__global__ void __launch_bounds__(256) reduce_partials(const float* partials, int nblocks, int width, float* out) {
  __shared__ float buf[256];
  const int e = blockIdx.x;
#ifdef QS_CHECKED
  if (!QS_OK(e < width, 12, e)) return;  // uniform over the block: no barrier is left waiting
#endif
  float s = 0.f;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[(int64_t)b * width + e];
  buf[threadIdx.x] = s;
  __syncthreads();
  for (int off = blockDim.x >> 1; off > 0; off >>= 1) {
    if (threadIdx.x < off) buf[threadIdx.x] += buf[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[e] = buf[0];
}

}  // namespace qs
