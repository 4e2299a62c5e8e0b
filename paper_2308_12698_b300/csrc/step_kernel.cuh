// The fused forward kernel: K RK4 steps per launch, one thread per agent,
// state in registers between steps and in HBM (planar float4 SoA) between
// launches; one parameter group in kernel parameters or several in shared
// memory indexed by a per-agent uint8 id; grid-stride over a resident wave.
// Agents with a nonzero status byte are skipped; an agent whose state turns
// non-finite keeps its last finite state, whatever K, and is marked (status
// 1): the plain form (K = 1) keeps the launch-start state; the fused form
// marks the agent kStatusDiverged without storing, and refreeze_kernel, run
// after the call's launches, steps the launch-start state again one step at
// a time.
#pragma once
#include "model_fwd.cuh"
#include "vehicles.cuh"

namespace qs {

struct StepArgs {
  float* state;
  const float4* cmd;
  const uint8_t* gid;
  uint8_t* status;
  int64_t n;      // agents in the buffers (the plane stride)
  int64_t first;  // this launch steps agents [first, first + count)
  int64_t count;
  int K;
  int n_groups;
  StepH H;
  const DevGroup* groups;  // device table (several groups)
  const uint32_t* order;   // group_kernel<..., ORDER>: agent at each group-sorted position
  LinCoef coef;            // one group: its RK4 weights of the linear parts (lin_coef, on the host)
};

// Asynchronous global -> shared copies (cp.async, sm_80 and later), each
// thread copying its own data; cp.async.wait_group 0 makes the thread's own
// copies visible to it.  No barrier is involved.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Status byte of an agent whose state went non-finite at some step of a
// launch of the fused form and is still at that launch's start state; within
// the same call refreeze_kernel turns it into 1 at the last finite state.
constexpr uint8_t kStatusDiverged = 3;

template <int NS = NX>
__device__ __forceinline__ bool all_finite(const St& x) {
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < NS; ++i) s += x.a[i];
  return isfinite(s);
}

// The grid's warps take 32-agent chunks: warp r takes chunks r, r + W, r + 2W,
// ... (W warps in the grid; a round of W chunks is one resident wave).  r
// numbers the warps scheduler-first: warp j of a block runs on scheduler
// j % 4 of its SM and consecutive blocks start on different SMs, so the
// first chunks of each round go one per scheduler.  A last round that the
// agents fill only partly is then spread over all schedulers instead of
// doubling the load of the first blocks' SMs.
__device__ __forceinline__ int64_t first_agent() {
  const int wpb = blockDim.x >> 5, j = threadIdx.x >> 5;
  const int q = (wpb & 3) == 0 ? 4 : (wpb & 1) == 0 ? 2 : 1;
  const int64_t r = ((int64_t)(j / q) * gridDim.x + blockIdx.x) * q + (j % q);
  return r * 32 + (threadIdx.x & 31);
}

template <bool HETERO>
__device__ __forceinline__ void load_groups(DevGroup* sg, const DevGroup* src, int n_groups) {
  if (HETERO) {
    const float4* s = reinterpret_cast<const float4*>(src);
    float4* d = reinterpret_cast<float4*>(sg);
    for (int i = threadIdx.x; i < n_groups * (int)(sizeof(DevGroup) / 16); i += blockDim.x) d[i] = s[i];
    __syncthreads();
  }
}

// Shared memory of the plain form: per thread two slots of six float4 (the
// state's five planes and the command).
constexpr int kPlainSlotF4 = 6;

// The plain form (K = 1, one 17-float group): each thread copies its next
// agent's state and command into its own shared-memory slot with cp.async
// while it steps the current agent (double-buffered), so every warp keeps a
// load in flight through its arithmetic.  Same arithmetic and results as the
// register path.
__device__ __forceinline__ void fetch_agent(float4* slot, int bd, const StepArgs& A, int64_t i) {
#ifdef QS_CHECKED
  if (!QS_OK(i >= 0 && i < A.n, 3, i)) {
    cp_async_commit();
    return;
  }
#endif
  const float4* P = reinterpret_cast<const float4*>(A.state);
#pragma unroll
  for (int k = 0; k < 4; ++k) cp_async16(slot + k * bd, P + k * A.n + i);
  cp_async4(slot + 4 * bd, A.state + 16 * A.n + i);
  cp_async16(slot + 5 * bd, A.cmd + i);
  cp_async_commit();
}

template <int MODE>
__device__ __forceinline__ void plain_loop(const StepArgs& A, const DevGroup& P0, float4* smem) {
  const int bd = blockDim.x;
  float4* const slot = smem + threadIdx.x;  // [2 buffers][kPlainSlotF4][bd]
  const int64_t stride = (int64_t)gridDim.x * bd;
  const int64_t end = A.first + A.count;
  const LinCoef& L = A.coef;
  int64_t i = A.first + first_agent();
  if (i < end) fetch_agent(slot, bd, A, i);
  for (int b = 0; i < end; i += stride, b ^= 1) {
    cp_async_wait_all();  // agent i has arrived in buffer b
    if (i + stride < end) fetch_agent(slot + (b ^ 1) * kPlainSlotF4 * bd, bd, A, i + stride);
#ifdef QS_CHECKED
    if (!QS_OK(i >= 0 && i < A.n, 4, i)) continue;
#endif
    if (A.status[i]) continue;  // dead agents are frozen
    const float4* s = slot + b * kPlainSlotF4 * bd;
    const float4 p0 = s[0], p1 = s[bd], p2 = s[2 * bd], p3 = s[3 * bd], c = s[5 * bd];
    St x;
    x.a[0] = p0.x; x.a[1] = p0.y; x.a[2] = p0.z; x.a[3] = p0.w;
    x.a[4] = p1.x; x.a[5] = p1.y; x.a[6] = p1.z; x.a[7] = p1.w;
    x.a[8] = p2.x; x.a[9] = p2.y; x.a[10] = p2.z; x.a[11] = p2.w;
    x.a[12] = p3.x; x.a[13] = p3.y; x.a[14] = p3.z; x.a[15] = p3.w;
    x.a[16] = s[4 * bd].x;
    const Hd hd = heading(MODE != 0 ? c.w : 0.f);
    step<MODE>(P0, x, c, hd, A.H, L);
    if (all_finite<NX>(x)) {
      store_state<NX>(A.state, A.n, i, x);
    } else {
      A.status[i] = 1;  // keep the last finite state
    }
  }
}

// K fused RK4 steps per launch; the state touches HBM once per launch.
// MULTI: some groups are cars or fixed-wing drones (closed loop only); each
// agent runs its group's model.  PLAIN (1 or 2): one step per launch (K =
// 1), where HBM bounds the kernel.  Registers are capped so that 3 blocks of
// 256 stay resident: the plain form keeps more loads in flight, and the fused
// one-group form fits in 80 without spilling (uncapped it takes 88 in the
// closed loop, the same speed, and the PID loop runs 3 % slower).  The
// heterogeneous form, which holds its group's constants in registers, is left
// uncapped: capped it spills.  PLAIN 2 prefetches each thread's next agent
// (plain_loop); the host takes it when the agents exceed one resident wave,
// PLAIN 1 (nothing to overlap) otherwise.
template <int MODE, bool HETERO, bool MULTI = false, int PLAIN = 0>
__global__ void __launch_bounds__(256, (PLAIN || !HETERO) ? 3 : 1) step_kernel(StepArgs A, const DevGroup P0) {
  extern __shared__ float4 smem4[];
  if (PLAIN == 2) {
    plain_loop<MODE>(A, P0, smem4);
    return;
  }
  DevGroup* sg = reinterpret_cast<DevGroup*>(smem4);
  load_groups<HETERO>(sg, A.groups, A.n_groups);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t end = A.first + A.count;
  const int K = PLAIN ? 1 : A.K;
  for (int64_t i = A.first + first_agent(); i < end; i += stride) {
#ifdef QS_CHECKED
    if (!QS_OK(i >= 0 && i < A.n, 4, i)) continue;
    if (HETERO && !QS_OK(A.gid[i] < A.n_groups, 5, A.gid[i])) continue;
#endif
    if (A.status[i]) continue;  // dead agents are frozen
    St x;
    load_state<state_dim<MODE>()>(A.state, A.n, i, x);
    const float4 c = A.cmd[i];
    const Hd hd = heading(MODE != 0 ? c.w : 0.f);
    if (MULTI && (HETERO ? sg[A.gid[i]].vt : P0.vt) != (float)TYPE_QUAD) {
      const DevGroup& P = HETERO ? sg[A.gid[i]] : P0;
      for (int k = 0; k < K; ++k) vehicle_step(P, x, c, A.H);
    } else if (HETERO) {
      const DevGroup P = sg[A.gid[i]];
      const LinCoef L = lin_coef(P, A.H);
      for (int k = 0; k < K; ++k) step<MODE>(P, x, c, hd, A.H, L);
    } else {
      const LinCoef& L = A.coef;
#pragma unroll 2
      for (int k = 0; k < K; ++k) step<MODE>(P0, x, c, hd, A.H, L);  // unrolled: +0.5-1 %
    }
    if (all_finite<state_dim<MODE>()>(x)) {
      store_state<state_dim<MODE>()>(A.state, A.n, i, x);
    } else {
      // the plain form (one step) keeps the launch-start state, the last finite
      // one; after a fused launch refreeze_kernel finds it
      A.status[i] = PLAIN ? 1 : kStatusDiverged;
    }
  }
}

// K fused RK4 steps for one range of one group: [A.first, A.first + A.count)
// of agent ids, or of positions in a group-sorted order of the agents
// (ORDER: A.order, for ids in which the groups interleave; a warp then still
// holds agents of one group, and of one agent type).  One agent per thread,
// one block per chunk (not persistent: the hardware scheduler evens out the
// last wave better than a resident grid taking whole chunks in turn).  The
// group's constants (P) and RK4 weights (A.coef) are kernel parameters at
// fixed offsets, which the step's operations read from the constant bank as
// operands.  The host launches one per range, each on a stream of its own, so
// that the ranges run side by side.  (One launch over a table of all ranges,
// indexed by a block-uniform range, spent 17 more thread instructions per
// agent-step reading the constants: 3-5 % slower.)  Same arithmetic, results
// and status marks as step_kernel's fused form.  VEH: the group is a car or
// fixed-wing group (vehicle_step).
template <int MODE, bool VEH = false, bool ORDER = false>
__global__ void __launch_bounds__(256, 3) group_kernel(StepArgs A, const DevGroup P) {
  const int64_t j = A.first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= A.first + A.count) return;
#ifdef QS_CHECKED
  if (!QS_OK(j >= 0 && j < A.n, 6, j)) return;
  if (ORDER && !QS_OK(A.order[j] < A.n, 7, A.order[j])) return;
#endif
  const int64_t i = ORDER ? (int64_t)A.order[j] : j;
  if (A.status[i]) return;  // dead agents are frozen
  constexpr int NS = state_dim<MODE>();
  St x;
  load_state<NS>(A.state, A.n, i, x);
  const float4 c = A.cmd[i];
  if (VEH) {
    for (int k = 0; k < A.K; ++k) vehicle_step(P, x, c, A.H);
  } else {
    const Hd hd = heading(MODE != 0 ? c.w : 0.f);
    const LinCoef& L = A.coef;
#pragma unroll 2
    for (int k = 0; k < A.K; ++k) step<MODE>(P, x, c, hd, A.H, L);
  }
  if (all_finite<NS>(x))
    store_state<NS>(A.state, A.n, i, x);
  else
    A.status[i] = kStatusDiverged;  // refreeze_kernel finds its last finite state
}

// After a call's K-step launches (same state, command and step size): each
// agent marked kStatusDiverged is still at the start state of the launch in
// which its state went non-finite.  That state is stepped again one step at a
// time, with the same arithmetic, and stored after every finite step; the
// replay meets the same non-finite step, within K steps, and stops there.
// The agent ends at its last finite state -- the bits that K = 1 launches
// keep -- and is marked non-finite (1).  A separate kernel, so that the hot
// loop's code is not touched; its cost is one read of the status bytes.
template <int MODE, bool MULTI = false>
__global__ void __launch_bounds__(256) refreeze_kernel(StepArgs A) {
  constexpr int NS = state_dim<MODE>();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t end = A.first + A.count;
  for (int64_t i = A.first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < end; i += stride) {
#ifdef QS_CHECKED
    if (!QS_OK(i >= 0 && i < A.n, 4, i)) continue;
    if (A.n_groups > 1 && !QS_OK(A.gid[i] < A.n_groups, 5, A.gid[i])) continue;
#endif
    if (A.status[i] != kStatusDiverged) continue;
    const DevGroup& P = A.groups[A.n_groups > 1 ? A.gid[i] : 0];
    const float4 c = A.cmd[i];
    const Hd hd = heading(MODE != 0 ? c.w : 0.f);
    const LinCoef L = lin_coef(P, A.H);
    St x;
    load_state<NS>(A.state, A.n, i, x);
    for (int k = 0; k < A.K; ++k) {
      if (MULTI && P.vt != (float)TYPE_QUAD)
        vehicle_step(P, x, c, A.H);
      else
        step<MODE>(P, x, c, hd, A.H, L);
      if (!all_finite<NS>(x)) break;
      store_state<NS>(A.state, A.n, i, x);
    }
    A.status[i] = 1;
  }
}

}  // namespace qs
