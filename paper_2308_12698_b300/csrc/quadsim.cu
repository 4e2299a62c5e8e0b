// libquadsim.so: the C ABI of include/quadsim.h and the sm_103a kernels
// behind it.  One thread per agent; state in planar float4 SoA; parameter
// groups in kernel parameters (one group) or shared memory (several groups,
// indexed by a per-agent uint8 id); grid-stride loops over a grid of one
// resident wave (blocks per SM x SMs).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/quadsim.h"
#include "adjoint_kernel.cuh"
#include "collide.cuh"
#include "compact.cuh"
#include "stats.cuh"
#include "model_fwd.cuh"
#include "step_kernel.cuh"

using namespace qs;

namespace {

// forward 128: the fused step of one group 1.7 % faster than at 256, the plain step and the
// per-range launches the same (1e6, 6e5 and 1e7 agents)
constexpr int kDefaultBlockFwd = 128;
constexpr int kDefaultBlockAdj = 128;

// Default threads per block for n agents on sms SMs: the largest of `largest`,
// largest/2, ... 32 that still gives every SM a block.  A swarm too small for
// that runs 32-thread blocks, one warp per SM, so that no scheduler holds two
// of its warps (4,096 agents: 128 single-warp blocks rather than 16 blocks of
// 256, whose eight warps share four schedulers on each of 16 SMs).
int spread_block(int64_t n, int sms, int largest) {
  int b = largest;
  while (b > 32 && (n + b - 1) / b < sms) b /= 2;
  return b;
}
constexpr int kDefaultK = 10;
constexpr int kDefaultC = 100;

// ----------------------------------------------------- utility kernels --
// (the step kernels are in step_kernel.cuh, the rollout and adjoint kernels
// in adjoint_kernel.cuh, collision detection in collide.cuh)

__global__ void max_gid_kernel(const uint8_t* gid, int64_t n, unsigned int* out) {
  unsigned int m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (unsigned int)gid[i]);
  for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void count_dead_kernel(const uint8_t* status, int64_t n, unsigned long long* out) {
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += status[i] != 0;
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// ------------------------------------------------------------ host side --

DevGroup derive(const sim_group_params_t& p) {
  DevGroup d;
  std::memset(&d, 0, sizeof(d));
  const double m = p.m, Jx = p.Jxx, Jy = p.Jyy, Jz = p.Jzz, kt = p.kt, kq = p.kq;
  const double Ls = (double)p.L * std::sin((double)p.alpha), Lc = (double)p.L * std::cos((double)p.alpha);
  const double om2 = (double)p.omega_max * p.omega_max;
  const double taumax[3] = {2.0 * Ls * kt * om2, 2.0 * Lc * kt * om2, 2.0 * kq * om2};
  const double mix[3] = {1.0 / (4.0 * kt * Ls), 1.0 / (4.0 * kt * Lc), 1.0 / (4.0 * kq)};
  d.T2c = (float)(2.0 * kt / m);
  d.cd_m = (float)(p.c_d / m);
  d.g = p.g;
  d.inv_tau = (float)(1.0 / p.tau_m);
  d.txc = (float)(kt * Ls / Jx);
  d.tyc = (float)(kt * Lc / Jy);
  d.tzc = (float)(kq / Jz);
  d.omax = p.omega_max;
  d.gx = (float)((Jy - Jz) / Jx);
  d.gy = (float)((Jz - Jx) / Jy);
  d.gz = (float)((Jx - Jy) / Jz);
  d.gxt = (float)((Jy - Jz) / (kt * Ls));  // the gyroscopic coefficients over the torque ones
  d.gyt = (float)((Jz - Jx) / (kt * Lc));
  d.gzt = (float)((Jx - Jy) / kq);
  d.m = p.m;
  for (int i = 0; i < 3; ++i) {
    d.kp[i] = p.kp[i];
    d.kd[i] = p.kd[i];
    // the mixer's constants in units of omega_max^2 (mix_i taumax_i / omega_max^2 = 1/2)
    d.qa[i] = (float)(mix[i] * p.krate[i] * taumax[i] * 2.0 * p.katt[i] / om2);
    d.wa[i] = (float)(mix[i] * p.krate[i] * taumax[i] / om2);
    d.krate[i] = p.krate[i];
    d.katt2[i] = (float)(2.0 * p.katt[i]);
    d.mt[i] = (float)(mix[i] * taumax[i] / om2);
    d.kic[i] = (float)(mix[i] * taumax[i] * p.kI[i] / om2);
    d.kdc[i] = (float)(mix[i] * taumax[i] * p.kD[i] / om2);
    d.xim[i] = p.xi_max[i];
  }
  d.vt = (float)p.type;
  if (p.type == SIM_TYPE_CAR) {
    d.vk[0] = (float)((double)p.veh[1] / p.veh[0]);  // largest curvature tan(delta_max) / L_w
    d.vk[1] = p.veh[2];
    d.vk[2] = p.veh[3];
    d.vk[3] = p.veh[4];
  } else if (p.type == SIM_TYPE_FIXED_WING) {
    for (int i = 0; i < 6; ++i) d.vk[i] = p.veh[i];
  }
  d.a_max = p.a_max;
  d.az_lo = (float)((double)p.g - p.a_max);  // the z clamp with gravity added: g -+ a_max
  d.az_hi = (float)((double)p.g + p.a_max);
  d.f0c = (float)(m / (2.0 * kt * om2));
  d.inv_m = (float)(1.0 / m);
  d.Jx = p.Jxx; d.Jy = p.Jyy; d.Jz = p.Jzz;
  d.iJx = (float)(1.0 / Jx); d.iJy = (float)(1.0 / Jy); d.iJz = (float)(1.0 / Jz);
  d.mix0 = (float)(1.0 / (4.0 * kt * om2));
  return d;
}

bool valid_vehicle(const sim_group_params_t& p) {
  if (!std::isfinite(p.g) || !(std::isfinite(p.L) && p.L > 0.f)) return false;
  const float* v = p.veh;
  if (p.type == SIM_TYPE_CAR)  // L_w > 0, tan(delta_max), a_max, k_v >= 0, l_min > 0
    return v[0] > 0.f && std::isfinite(v[0]) && v[1] >= 0.f && std::isfinite(v[1]) && v[2] >= 0.f &&
           std::isfinite(v[2]) && v[3] >= 0.f && std::isfinite(v[3]) && v[4] > 0.f && std::isfinite(v[4]);
  // fixed-wing: b_phi > 0, 0 < phi_max < pi/2, k_chi finite, b_hd, b_h, b_V >= 0
  return v[0] > 0.f && std::isfinite(v[0]) && v[1] > 0.f && v[1] < 1.5707f && std::isfinite(v[2]) &&
         v[3] >= 0.f && std::isfinite(v[3]) && v[4] >= 0.f && std::isfinite(v[4]) && v[5] >= 0.f &&
         std::isfinite(v[5]);
}

bool valid_params(const sim_group_params_t& p) {
  if (p.type == SIM_TYPE_CAR || p.type == SIM_TYPE_FIXED_WING) return valid_vehicle(p);
  if (p.type != SIM_TYPE_QUADROTOR) return false;
  const float pos[] = {p.m, p.Jxx, p.Jyy, p.Jzz, p.L, p.kt, p.kq, p.tau_m, p.omega_max};
  for (float v : pos)
    if (!(std::isfinite(v) && v > 0.f)) return false;
  if (!(std::isfinite(p.c_d) && p.c_d >= 0.f) || !std::isfinite(p.g)) return false;
  if (!(std::sin((double)p.alpha) > 0.0 && std::cos((double)p.alpha) > 0.0)) return false;
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(p.kp[i]) || !std::isfinite(p.kd[i]) || !std::isfinite(p.katt[i]) ||
        !std::isfinite(p.krate[i]) || !std::isfinite(p.kI[i]) || !std::isfinite(p.kD[i]) || !(p.xi_max[i] >= 0.f))
      return false;
  return p.a_max >= 0.f;  // +inf allowed (no clamp)
}

StepH make_h(float dt) {
  StepH H;
  H.h = dt;
  H.h2 = (float)(0.5 * (double)dt);
  H.h6 = (float)((double)dt / 6.0);
  H.hq = (float)(0.5 * (double)dt);
  H.h2q = (float)(0.25 * (double)dt);
  H.h6q = (float)((double)dt / 12.0);
  return H;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <class F>
int occupancy(F kernel, int block, size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, block, smem) != cudaSuccess) return 1;
  return std::max(nb, 1);
}

}  // namespace

// sim_step_host: at most kHostChunks chunks of at least kHostChunkMin agents.
// Only the first chunk's copy in and the last chunk's copy out are exposed.
// The chunks' steps go round kComputeStreams streams, so that several chunks'
// launches (each a fraction of a resident wave) fill the GPU together.  1e6
// agents x 1000 steps end to end: 16 chunks on 2 streams 12.66 ms, 32 (30 at
// this size) on 4 streams 12.52 ms, against 12.37 ms with the state on the device.
constexpr int kHostChunks = 32;
constexpr int kComputeStreams = 4;
constexpr int64_t kHostChunkMin = 32768;

// The host pipeline's chunks of n agents: m chunks of `chunk` agents (the last
// one shorter).  A function of n alone, so that the group-sorted order built at
// creation can keep each chunk's agents together.
static void host_chunks(int64_t n, int* m, int64_t* chunk) {
  *m = (int)std::max<int64_t>(1, std::min<int64_t>(kHostChunks, n / kHostChunkMin));
  *chunk = (n + *m - 1) / *m;
}

// Fused launches of K steps or more take the group-sorted order when the
// groups' ids interleave.  Measured on 8 quadrotor groups of 600,000 agents in
// random order: the order's scattered loads and stores cost 8.7 us per launch,
// and warps of one group gain 0.33 us per step (1000 steps at K = 1000: 7.44
// -> 7.11 ms; at K = 1: 16.2 -> 24.9 ms), so it pays from K ~ 26.  Swarms that
// mix agent types take it at any K: a warp of mixed types runs every type's
// model (200,000 each of quadrotors, cars and fixed-wing drones in random
// order: 13.1 -> 4.1 ms at K = 1000, 21.5 -> 19.9 ms at K = 1).
constexpr int kOrderMinK = 32;
// The live agents' order keeps each chunk's agents in index order, so its loads
// stay close together, and it pays from 2 fused steps on.  Half of 1e6 agents
// dead at random, 200 steps: one group 3.44 -> 2.10 ms at K = 2 and 2.56 ->
// 1.37 ms at K = 10; 8 interleaved groups 1.65 -> 0.91 ms at K = 10, but 3.25
// -> 3.71 ms at K = 1.
constexpr int kLiveMinK = 2;

struct sim_s {
  int device = 0;
  int sms = 1;
  int n_groups = 1;
  int64_t n = 0;
  int mode = SIM_CLOSED_LOOP;
  int nx = NX;                   // state floats per agent: 17, or 20 in the PID mode
  bool multi = false;            // some groups are cars or fixed-wing drones
  const uint8_t* gid = nullptr;  // borrowed
  uint8_t* status = nullptr;     // owned
  DevGroup* d_groups = nullptr;  // owned
  float* d_arm = nullptr;        // owned: arm length per group (collision radius)
  unsigned long long* d_count = nullptr;  // owned: counter for sim_status
  unsigned long long* h_count = nullptr;  // owned, pinned: its host copy (outlives a timed-out wait)
  float max_arm = 0.f;
  DevGroup host_group0;
  DevGroup host_groups[SIM_MAX_GROUPS];
  // each group's agents form one contiguous range [g_start, g_end) (found at
  // creation from the ids): the fused steps then run as group_kernel launches, one per range
  bool ranged = false;
  int64_t g_start[SIM_MAX_GROUPS] = {}, g_end[SIM_MAX_GROUPS] = {};
  // ids in which the groups interleave: the agents sorted by (group, host
  // pipeline chunk, index) in d_order (owned); the agents of group g and chunk
  // c sit at positions [g_off[g][c], g_off[g][c + 1]), and group_kernel steps
  // any run of whole chunks through it
  uint32_t* d_order = nullptr;
  int n_chunks = 1;
  int64_t chunk = 0;
  std::vector<int64_t> g_off;  // [n_groups][n_chunks + 1]
  // sim_compact: the live agents alone in the same (group, chunk, index) order
  // (d_live, owned; live_off as g_off), used while `live` holds; `epoch` counts
  // the changes of the agent order that graphs captured before must not outlive
  uint32_t* d_live = nullptr;
  bool live = false;
  std::vector<int64_t> live_off;
  unsigned int* d_live_cnt = nullptr;  // owned: the counting pass's output, and its pinned host copy
  unsigned int* h_live_cnt = nullptr;
  int64_t* d_live_off = nullptr;       // owned: the positions the scatter pass writes from, and theirs
  int64_t* h_live_off = nullptr;
  // sim_group_stats: per-block partial rows and the summed row (device, owned), its pinned copy
  double* d_stat = nullptr;
  double* h_stat = nullptr;
  int stat_blocks = 0;
  uint64_t epoch = 0;
  // host-buffer pipeline (sim_step_host): created on first use
  cudaStream_t s_h2d = nullptr, s_d2h = nullptr, s_comp[kComputeStreams] = {};
  cudaEvent_t ev_start = nullptr, ev_end = nullptr, ev_in[kHostChunks] = {}, ev_done[kHostChunks] = {};
  // decision rounds (sim_run_rounds): per command plane and observation plane
  cudaEvent_t ev_cmd[2] = {}, ev_cmd_free[2] = {}, ev_obs[2] = {}, ev_obs_free[2] = {};
  // several groups: a stream per group range of a fused launch (launch_ranged),
  // forked from the caller's stream and joined back to it; created with the handle
  cudaStream_t s_grp[SIM_MAX_GROUPS] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[SIM_MAX_GROUPS] = {};
  int block_fwd = kDefaultBlockFwd;
  int block_adj = kDefaultBlockAdj;
  int K = kDefaultK;
  int C = kDefaultC;
};

struct sim_graph_s {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const sim_s* h = nullptr;  // the handle it steps, and that handle's agent-order epoch at capture
  uint64_t epoch = 0;
};

namespace {

bool hetero(const sim_s* h) { return h->n_groups > 1; }

// Agents may come alive again: the live agents' order no longer covers them.
void drop_live(sim_s* h) {
  if (h->live) {
    h->live = false;
    ++h->epoch;
  }
}

size_t group_smem(const sim_s* h) { return hetero(h) ? sizeof(DevGroup) * h->n_groups : 0; }

// The plain form's per-thread prefetch slots: 2 x kPlainSlotF4 float4.
size_t plain_smem(const sim_s* h) { return (size_t)2 * kPlainSlotF4 * sizeof(float4) * h->block_fwd; }

// The plain (K = 1) instantiation for one quadrotor group, open or P closed loop.
bool plain_path(const sim_s* h, int K) {
  return K == 1 && !hetero(h) && !h->multi && h->mode != SIM_CLOSED_LOOP_PID;
}

int fwd_grid(const sim_s* h, size_t smem, int64_t count, bool plain = false) {
  // one resident wave of blocks, grid-stride over the agents
  int occ;
  if (plain)
    occ = h->mode == SIM_CLOSED_LOOP ? occupancy(step_kernel<1, false, false, 2>, h->block_fwd, smem)
                                     : occupancy(step_kernel<0, false, false, 2>, h->block_fwd, smem);
  else if (h->multi)
    occ = hetero(h) ? occupancy(step_kernel<1, true, true>, h->block_fwd, smem)
                    : occupancy(step_kernel<1, false, true>, h->block_fwd, smem);
  else if (h->mode == SIM_CLOSED_LOOP_PID)
    occ = hetero(h) ? occupancy(step_kernel<2, true>, h->block_fwd, smem)
                    : occupancy(step_kernel<2, false>, h->block_fwd, smem);
  else if (h->mode == SIM_CLOSED_LOOP)
    occ = hetero(h) ? occupancy(step_kernel<1, true>, h->block_fwd, smem)
                    : occupancy(step_kernel<1, false>, h->block_fwd, smem);
  else
    occ = hetero(h) ? occupancy(step_kernel<0, true>, h->block_fwd, smem)
                    : occupancy(step_kernel<0, false>, h->block_fwd, smem);
  const int64_t need = (count + h->block_fwd - 1) / h->block_fwd;
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)occ * h->sms));
}

// Shared-memory budget per block for the segment scratch (small C).
constexpr size_t kSmemScratchMax = 96 * 1024;

// Shared-memory scratch of one block: the segment's step-start states plus the
// double-buffered checkpoint prefetch slots (2 x 5 float4 per thread).
size_t adj_smem_scratch_bytes(const sim_s* h, int C) {
  return ((size_t)C * h->nx * sizeof(float) + 2 * 5 * sizeof(float4)) * h->block_adj;
}

bool adj_smem_scratch(const sim_s* h, int C) { return adj_smem_scratch_bytes(h, C) <= kSmemScratchMax; }

// Dynamic shared memory of one adjoint block: the group table, the groups'
// RK4 weights and the per-warp accumulators, then (16-byte aligned) the segment scratch with the
// checkpoint prefetch slots when they fit, else the prefetch slots alone
// (for the step-start states read back from the global scratch).
size_t adj_smem(const sim_s* h, int C) {
  size_t b = (sizeof(DevGroup) + sizeof(LinCoef)) * h->n_groups +
             (size_t)(h->block_adj / 32) * h->n_groups * NTH * sizeof(float);
  b = (b + 15) & ~(size_t)15;
  return b + (adj_smem_scratch(h, C) ? adj_smem_scratch_bytes(h, C) : 2 * 5 * sizeof(float4) * h->block_adj);
}

int adj_grid(const sim_s* h, int C) {
  const size_t smem = adj_smem(h, C);
  const bool sm = adj_smem_scratch(h, C);
  int occ;
  if (h->mode == SIM_CLOSED_LOOP_PID)
    occ = sm ? occupancy(adjoint_kernel<2, true>, h->block_adj, smem) : occupancy(adjoint_kernel<2, false>, h->block_adj, smem);
  else if (h->mode == SIM_CLOSED_LOOP)
    occ = sm ? occupancy(adjoint_kernel<1, true>, h->block_adj, smem) : occupancy(adjoint_kernel<1, false>, h->block_adj, smem);
  else
    occ = sm ? occupancy(adjoint_kernel<0, true>, h->block_adj, smem) : occupancy(adjoint_kernel<0, false>, h->block_adj, smem);
  const int64_t need = (h->n + h->block_adj - 1) / h->block_adj;
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)occ * h->sms));
}

// The agents a rollout kernel visits: the live agents' order after
// sim_compact, else all n in index order.
void live_visit(const sim_s* h, const uint32_t** order, int64_t* count) {
  *order = h->live ? h->d_live : nullptr;
  *count = h->live ? h->live_off.back() : h->n;
}

int launch_adjoint(const sim_s* h, const AdjArgs& A, int C, int grid, cudaStream_t st) {
  const size_t smem = adj_smem(h, C);
  const bool sm = adj_smem_scratch(h, C);
  if (A.order) {
    const int fgrid = (int)std::max<int64_t>(1, std::min<int64_t>((h->n + 255) / 256, (int64_t)h->sms * 8));
    if (h->mode == SIM_CLOSED_LOOP_PID) adjoint_frozen_kernel<2><<<fgrid, 256, 0, st>>>(A);
    else if (h->mode == SIM_CLOSED_LOOP) adjoint_frozen_kernel<1><<<fgrid, 256, 0, st>>>(A);
    else adjoint_frozen_kernel<0><<<fgrid, 256, 0, st>>>(A);
  }
  const bool o = A.order != nullptr;
  if (h->mode == SIM_CLOSED_LOOP_PID) {
    if (sm) o ? adjoint_kernel<2, true, true><<<grid, h->block_adj, smem, st>>>(A)
              : adjoint_kernel<2, true><<<grid, h->block_adj, smem, st>>>(A);
    else o ? adjoint_kernel<2, false, true><<<grid, h->block_adj, smem, st>>>(A)
           : adjoint_kernel<2, false><<<grid, h->block_adj, smem, st>>>(A);
  } else if (h->mode == SIM_CLOSED_LOOP) {
    if (sm) o ? adjoint_kernel<1, true, true><<<grid, h->block_adj, smem, st>>>(A)
              : adjoint_kernel<1, true><<<grid, h->block_adj, smem, st>>>(A);
    else o ? adjoint_kernel<1, false, true><<<grid, h->block_adj, smem, st>>>(A)
           : adjoint_kernel<1, false><<<grid, h->block_adj, smem, st>>>(A);
  } else {
    if (sm) o ? adjoint_kernel<0, true, true><<<grid, h->block_adj, smem, st>>>(A)
              : adjoint_kernel<0, true><<<grid, h->block_adj, smem, st>>>(A);
    else o ? adjoint_kernel<0, false, true><<<grid, h->block_adj, smem, st>>>(A)
           : adjoint_kernel<0, false><<<grid, h->block_adj, smem, st>>>(A);
  }
  return cudaGetLastError() == cudaSuccess ? SIM_OK : SIM_ERR_CUDA;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t scratch_bytes(const sim_s* h, int C, int grid) {
  if (adj_smem_scratch(h, C)) return 0;
  return align256((size_t)C * h->nx * sizeof(float) * (size_t)grid * h->block_adj);
}

int wait_stream(cudaStream_t st, int timeout_ms);

// The agents whose status byte is 0, sorted by (group, host-pipeline chunk,
// index), written to out (n entries) by the two passes of live_order_kernel,
// with off[g][c] the first position of (group g, chunk c).  Ordered after
// earlier work on st; returns after the order is written (bounded waits).
int order_live(sim_s* h, cudaStream_t st, uint32_t* out, std::vector<int64_t>& off) {
  const int nc = h->n_chunks, G = h->n_groups;
  const size_t ncnt = (size_t)G * nc, noff = (size_t)G * (nc + 1);
  // each buffer on its own, so that a failed call leaves none half-made
  if ((!h->d_live_cnt && cudaMalloc(&h->d_live_cnt, sizeof(unsigned int) * ncnt) != cudaSuccess) ||
      (!h->d_live_off && cudaMalloc(&h->d_live_off, sizeof(int64_t) * noff) != cudaSuccess) ||
      (!h->h_live_cnt && cudaMallocHost(&h->h_live_cnt, sizeof(unsigned int) * ncnt) != cudaSuccess) ||
      (!h->h_live_off && cudaMallocHost(&h->h_live_off, sizeof(int64_t) * noff) != cudaSuccess))
    return SIM_ERR_CUDA;
  LiveArgs A;
  A.status = h->status;
  A.gid = G > 1 ? h->gid : nullptr;
  A.n = h->n;
  A.chunk = h->chunk;
  A.n_groups = G;
  A.n_chunks = nc;
  A.counts = h->d_live_cnt;
  A.off = h->d_live_off;
  A.order = out;
  // pass 1: live agents per (group, chunk), back to the host
  live_order_kernel<false><<<nc, kLiveBlock, 0, st>>>(A);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(h->h_live_cnt, h->d_live_cnt, sizeof(unsigned int) * ncnt, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess)
    return SIM_ERR_CUDA;
  int rc = wait_stream(st, 600000);
  if (rc != SIM_OK) return rc;
  int64_t pos = 0;
  for (int g = 0; g < G; ++g)
    for (int c = 0; c <= nc; ++c) {
      h->h_live_off[(size_t)g * (nc + 1) + c] = pos;
      if (c < nc) pos += h->h_live_cnt[(size_t)g * nc + c];
    }
  // pass 2: each agent's index at its position
  if (cudaMemcpyAsync(h->d_live_off, h->h_live_off, sizeof(int64_t) * noff, cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return SIM_ERR_CUDA;
  live_order_kernel<true><<<nc, kLiveBlock, 0, st>>>(A);
  if (cudaGetLastError() != cudaSuccess) return SIM_ERR_CUDA;
  rc = wait_stream(st, 600000);
  if (rc != SIM_OK) return rc;
  off.assign(h->h_live_off, h->h_live_off + noff);
  return SIM_OK;
}

// How the fused steps reach the groups, decided once at creation from the
// caller's id buffer (read synchronously; the handle's contract keeps it
// unchanged): contiguous ranges, one per group (sorted ids, or contiguous
// blocks in any order: a group_kernel launch per range), a group-sorted order
// (interleaved ids), or neither (one group).
int plan_groups(sim_s* h) {
  h->ranged = false;
  host_chunks(h->n, &h->n_chunks, &h->chunk);
  // one group: its fused launches are group_kernel over the whole range, its
  // constants in the kernel's parameters (faster than the persistent grid of
  // step_kernel: 9.93 against 10.25 ms for 1e6 agents x 1000 steps)
  if (h->n_groups == 1) return SIM_OK;
  if (h->n == 0) return SIM_OK;
  std::vector<uint8_t> ids((size_t)h->n);
  if (cudaMemcpy(ids.data(), h->gid, (size_t)h->n, cudaMemcpyDeviceToHost) != cudaSuccess) return SIM_ERR_CUDA;
  int64_t first[SIM_MAX_GROUPS], last[SIM_MAX_GROUPS], cnt[SIM_MAX_GROUPS] = {};
  for (int g = 0; g < SIM_MAX_GROUPS; ++g) first[g] = -1, last[g] = -1;
  for (int64_t i = 0; i < h->n; ++i) {
    const int g = ids[(size_t)i];
    if (g >= h->n_groups) return SIM_ERR_GROUP;
    if (first[g] < 0) first[g] = i;
    last[g] = i;
    ++cnt[g];
  }
  bool split = false;
  for (int g = 0; g < h->n_groups; ++g) split = split || (cnt[g] && last[g] - first[g] + 1 != cnt[g]);
  if (!split) {
    for (int g = 0; g < h->n_groups; ++g) {
      h->g_start[g] = cnt[g] ? first[g] : 0;
      h->g_end[g] = cnt[g] ? last[g] + 1 : 0;
    }
    h->ranged = true;
    return SIM_OK;
  }
  // the groups interleave: the agents sorted by (group, chunk, index), every
  // status byte being 0 at creation; positions fit 32 bits (more agents keep
  // the persistent kernel)
  if (h->n > (int64_t)UINT32_MAX) return SIM_OK;
  if (cudaMalloc(&h->d_order, sizeof(uint32_t) * (size_t)h->n) != cudaSuccess) return SIM_ERR_CUDA;
  return order_live(h, 0, h->d_order, h->g_off);
}

// Whether [first, first + count) is a run of whole host-pipeline chunks, the
// launches the group-sorted order can serve.
bool whole_chunks(const sim_s* h, int64_t first, int64_t count) {
  const int64_t end = first + count;
  return h->chunk > 0 && first % h->chunk == 0 && (end == h->n || end % h->chunk == 0);
}

// How a fused launch runs: the persistent kernel, one launch per group range
// of contiguous groups, or one per group range of the group-sorted order or of
// the live agents' order.
enum RangeMode { kPersistent, kContiguous, kGroupOrder, kLiveOrder };

template <bool ORDER>
void launch_group(const sim_s* h, const StepArgs& A, const DevGroup& P, int grid, cudaStream_t s) {
  const int bd = h->block_fwd;
  if (P.vt != (float)TYPE_QUAD) group_kernel<1, true, ORDER><<<grid, bd, 0, s>>>(A, P);
  else if (h->mode == SIM_CLOSED_LOOP_PID) group_kernel<2, false, ORDER><<<grid, bd, 0, s>>>(A, P);
  else if (h->mode == SIM_CLOSED_LOOP) group_kernel<1, false, ORDER><<<grid, bd, 0, s>>>(A, P);
  else group_kernel<0, false, ORDER><<<grid, bd, 0, s>>>(A, P);
}

// The fused steps of several groups as group_kernel launches, one per group
// range clipped to [first, first + count), or, with an order (a run of whole
// chunks), one per group over its positions in the order for those chunks.
// With more than one range each runs on its group's stream, forked from st
// and joined back to it (the same form inside a graph capture: parallel
// branches).  The ranges' launches then run side by side; a small group's
// launch, whose blocks each take K whole steps, overlaps the large ones.
int launch_ranged(sim_s* h, StepArgs A, cudaStream_t st, int64_t first, int64_t count, RangeMode mode) {
  const bool ordered = mode != kContiguous;
  A.order = mode == kLiveOrder ? h->d_live : h->d_order;
  const std::vector<int64_t>& offs = mode == kLiveOrder ? h->live_off : h->g_off;
  const int64_t ca = ordered ? first / h->chunk : 0;
  const int64_t cb = ordered ? (first + count == h->n ? h->n_chunks : (first + count) / h->chunk) : 0;
  int gs[SIM_MAX_GROUPS];
  int64_t ra[SIM_MAX_GROUPS], rb[SIM_MAX_GROUPS];
  int nr = 0;
  for (int g = 0; g < h->n_groups; ++g) {
    const int64_t* off = ordered ? &offs[(size_t)g * (h->n_chunks + 1)] : nullptr;
    const int64_t a = ordered ? off[ca] : std::max(h->g_start[g], first);
    const int64_t b = ordered ? off[cb] : std::min(h->g_end[g], first + count);
    if (b <= a) continue;
    if ((b - a + h->block_fwd - 1) / h->block_fwd > INT32_MAX) return SIM_ERR_ARG;
    gs[nr] = g;
    ra[nr] = a;
    rb[nr] = b;
    ++nr;
  }
  if (nr == 0) return SIM_OK;
  const bool fork = nr > 1;
  if (fork && cudaEventRecord(h->ev_fork, st) != cudaSuccess) return SIM_ERR_CUDA;
  int rc = SIM_OK;
  for (int r = 0; r < nr; ++r) {
    const int g = gs[r];
    const cudaStream_t s = fork ? h->s_grp[g] : st;
    if (fork && cudaStreamWaitEvent(s, h->ev_fork, 0) != cudaSuccess) {
      rc = SIM_ERR_CUDA;
      break;  // nothing launched on s: nothing to join
    }
    const DevGroup& P = h->host_groups[g];
    A.first = ra[r];
    A.count = rb[r] - ra[r];
    A.coef = lin_coef(P, A.H);
    const int grid = (int)((A.count + h->block_fwd - 1) / h->block_fwd);
    if (ordered) launch_group<true>(h, A, P, grid, s);
    else launch_group<false>(h, A, P, grid, s);
    if (cudaGetLastError() != cudaSuccess) rc = SIM_ERR_CUDA;
    // join even after a failed launch: a capture must get every forked stream back
    if (fork && (cudaEventRecord(h->ev_join[g], s) != cudaSuccess ||
                 cudaStreamWaitEvent(st, h->ev_join[g], 0) != cudaSuccess))
      rc = SIM_ERR_CUDA;
  }
  return rc;
}

// How a fused launch of K steps over [first, first + count) runs.  An order
// serves runs of whole chunks, for mixed agent types at any K and for one type
// from kOrderMinK steps: the live agents' order after sim_compact, else the
// group-sorted order of interleaved ids.  Contiguous groups take the range
// kernel directly; everything else the persistent kernel.
RangeMode range_mode(const sim_s* h, int K, int64_t first, int64_t count) {
  const bool whole = whole_chunks(h, first, count);
  if (h->live && whole && (h->multi || K >= kLiveMinK)) return kLiveOrder;
  const bool order_pays = (h->multi || K >= kOrderMinK) && whole;
  if (h->ranged) return kContiguous;
  if (h->d_order && order_pays) return kGroupOrder;
  return kPersistent;
}

int launch_step(sim_s* h, float* d_state, const float* d_cmd, StepH H, int K, cudaStream_t st, int64_t first,
                int64_t count) {
  StepArgs A;
  A.state = d_state;
  A.cmd = reinterpret_cast<const float4*>(d_cmd);
  A.gid = h->gid;
  A.status = h->status;
  A.n = h->n;
  A.first = first;
  A.count = count;
  A.K = K;
  A.n_groups = h->n_groups;
  A.H = H;
  A.groups = h->d_groups;
  A.order = nullptr;
  A.coef = lin_coef(h->host_group0, H);
  const bool plain = plain_path(h, K);
  const RangeMode rm = plain ? kPersistent : range_mode(h, K, first, count);
  if (rm != kPersistent) return launch_ranged(h, A, st, first, count, rm);
  // one group: group_kernel over the whole range, one block per chunk, its
  // constants as kernel parameters (3 % faster than step_kernel's persistent
  // grid, which now runs only the plain form and several groups that no range
  // or order serves; its fused one-group form still sizes the checkpointed
  // rollout's grid)
  if (!plain && h->n_groups == 1) {
    const int64_t blocks = (count + h->block_fwd - 1) / h->block_fwd;
    if (blocks > INT32_MAX) return SIM_ERR_ARG;
    if (blocks > 0) launch_group<false>(h, A, h->host_group0, (int)blocks, st);
    return cudaGetLastError() == cudaSuccess ? SIM_OK : SIM_ERR_CUDA;
  }
  const size_t smem = plain ? plain_smem(h) : group_smem(h);
  const int grid = fwd_grid(h, smem, count, plain);
  const DevGroup& P0 = h->host_group0;
  if (plain && count > (int64_t)grid * h->block_fwd) {  // several agents per thread: prefetch
    if (h->mode == SIM_CLOSED_LOOP) step_kernel<1, false, false, 2><<<grid, h->block_fwd, smem, st>>>(A, P0);
    else step_kernel<0, false, false, 2><<<grid, h->block_fwd, smem, st>>>(A, P0);
  } else if (plain) {
    if (h->mode == SIM_CLOSED_LOOP) step_kernel<1, false, false, 1><<<grid, h->block_fwd, 0, st>>>(A, P0);
    else step_kernel<0, false, false, 1><<<grid, h->block_fwd, 0, st>>>(A, P0);
  } else if (h->multi) {  // several groups that no range or order serves: the table in shared memory
    step_kernel<1, true, true><<<grid, h->block_fwd, smem, st>>>(A, P0);
  } else if (h->mode == SIM_CLOSED_LOOP_PID) {
    step_kernel<2, true><<<grid, h->block_fwd, smem, st>>>(A, P0);
  } else if (h->mode == SIM_CLOSED_LOOP) {
    step_kernel<1, true><<<grid, h->block_fwd, smem, st>>>(A, P0);
  } else {
    step_kernel<0, true><<<grid, h->block_fwd, smem, st>>>(A, P0);
  }
  return cudaGetLastError() == cudaSuccess ? SIM_OK : SIM_ERR_CUDA;
}

// After the launches of one call over agents [first, first + count) with one
// command plane, at most kmax steps each: replays the agents whose state went
// non-finite in a launch of the fused form to their last finite state
// (refreeze_kernel).  Nothing to do when every launch was of the plain form.
int launch_refreeze(sim_s* h, float* d_state, const float* d_cmd, StepH H, int64_t kmax, cudaStream_t st,
                    int64_t first, int64_t count) {
  if (count <= 0 || plain_path(h, (int)kmax)) return SIM_OK;
  StepArgs A;
  A.state = d_state;
  A.cmd = reinterpret_cast<const float4*>(d_cmd);
  A.gid = h->gid;
  A.status = h->status;
  A.n = h->n;
  A.first = first;
  A.count = count;
  A.K = (int)kmax;
  A.n_groups = h->n_groups;
  A.H = H;
  A.groups = h->d_groups;
  A.order = nullptr;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, (int64_t)h->sms * 4));
  if (h->multi) refreeze_kernel<1, true><<<grid, 256, 0, st>>>(A);
  else if (h->mode == SIM_CLOSED_LOOP_PID) refreeze_kernel<2><<<grid, 256, 0, st>>>(A);
  else if (h->mode == SIM_CLOSED_LOOP) refreeze_kernel<1><<<grid, 256, 0, st>>>(A);
  else refreeze_kernel<0><<<grid, 256, 0, st>>>(A);
  return cudaGetLastError() == cudaSuccess ? SIM_OK : SIM_ERR_CUDA;
}

// Library-owned streams and events of the host pipelines, created on first use.
int pipeline_streams(sim_s* h) {
  if (h->s_h2d) return SIM_OK;
  for (cudaStream_t* p : {&h->s_h2d, &h->s_d2h})
    if (cudaStreamCreateWithFlags(p, cudaStreamNonBlocking) != cudaSuccess) return SIM_ERR_CUDA;
  for (cudaStream_t& sc : h->s_comp)
    if (cudaStreamCreateWithFlags(&sc, cudaStreamNonBlocking) != cudaSuccess) return SIM_ERR_CUDA;
  for (cudaEvent_t* e : {&h->ev_start, &h->ev_end})
    if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return SIM_ERR_CUDA;
  for (int c = 0; c < kHostChunks; ++c)
    if (cudaEventCreateWithFlags(&h->ev_in[c], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_done[c], cudaEventDisableTiming) != cudaSuccess)
      return SIM_ERR_CUDA;
  for (int b = 0; b < 2; ++b)
    for (cudaEvent_t* e : {&h->ev_cmd[b], &h->ev_cmd_free[b], &h->ev_obs[b], &h->ev_obs_free[b]})
      if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return SIM_ERR_CUDA;
  return SIM_OK;
}

int wait_stream(cudaStream_t st, int timeout_ms) {
  cudaEvent_t ev;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return SIM_ERR_CUDA;
  if (cudaEventRecord(ev, st) != cudaSuccess) {
    cudaEventDestroy(ev);
    return SIM_ERR_CUDA;
  }
  const auto t0 = std::chrono::steady_clock::now();
  int rc = SIM_OK;
  for (;;) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) {
      rc = SIM_ERR_CUDA;
      break;
    }
    const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
    if (timeout_ms >= 0 && ms.count() > timeout_ms) {
      rc = SIM_ERR_TIMEOUT;
      break;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  cudaEventDestroy(ev);
  return rc;
}


}  // namespace

extern "C" {

int sim_bounds_checks(uint64_t* first_failure) {
  if (!first_failure) return SIM_ERR_ARG;
  *first_failure = 0;
#ifdef QS_CHECKED
  unsigned long long w = 0, zero = 0;
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpyFromSymbol(&w, g_check_word, sizeof(w)) != cudaSuccess ||
      cudaMemcpyToSymbol(g_check_word, &zero, sizeof(zero)) != cudaSuccess)
    return SIM_ERR_CUDA;
  *first_failure = w;
  return 1;
#else
  return 0;
#endif
}

const char* sim_error_string(int code) {
  switch (code) {
    case SIM_OK: return "ok";
    case SIM_ERR_ARG: return "invalid argument";
    case SIM_ERR_CUDA: return "CUDA runtime error";
    case SIM_ERR_WORKSPACE: return "workspace too small";
    case SIM_ERR_TIMEOUT: return "timed out waiting for the stream";
    case SIM_ERR_GROUP: return "group id out of range";
    case SIM_ERR_STALE: return "graph captured before the agent order changed (capture it again)";
    default: return "unknown error";
  }
}

int sim_create(const sim_group_params_t* groups, int n_groups, int64_t n_agents, const uint8_t* d_group_id, int mode,
               sim_handle_t* out) {
  if (!out) return SIM_ERR_ARG;
  *out = nullptr;
  if (!groups || n_groups < 1 || n_groups > SIM_MAX_GROUPS || n_agents < 0) return SIM_ERR_ARG;
  if (mode != SIM_OPEN_LOOP && mode != SIM_CLOSED_LOOP && mode != SIM_CLOSED_LOOP_PID) return SIM_ERR_ARG;
  if (n_groups > 1 && !d_group_id && n_agents > 0) return SIM_ERR_ARG;
  bool multi = false;
  for (int g = 0; g < n_groups; ++g) {
    if (!valid_params(groups[g])) return SIM_ERR_ARG;
    multi = multi || groups[g].type != SIM_TYPE_QUADROTOR;
  }
  if (multi && mode != SIM_CLOSED_LOOP) return SIM_ERR_ARG;  // vehicles run closed loop only
  sim_s* h = new (std::nothrow) sim_s();
  if (!h) return SIM_ERR_ARG;
  h->n_groups = n_groups;
  h->n = n_agents;
  h->mode = mode;
  h->nx = mode == SIM_CLOSED_LOOP_PID ? NXP : NX;
  h->multi = multi;
  h->gid = d_group_id;
  h->host_group0 = derive(groups[0]);
  int rc = SIM_OK;
  DevGroup tbl[SIM_MAX_GROUPS];
  float arm[SIM_MAX_GROUPS];
  for (int g = 0; g < n_groups; ++g) {
    tbl[g] = derive(groups[g]);
    h->host_groups[g] = tbl[g];
    arm[g] = groups[g].L;
    h->max_arm = std::max(h->max_arm, arm[g]);
  }
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
      cudaMalloc(&h->d_groups, sizeof(DevGroup) * n_groups) != cudaSuccess ||
      cudaMemcpy(h->d_groups, tbl, sizeof(DevGroup) * n_groups, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMalloc(&h->d_arm, sizeof(float) * n_groups) != cudaSuccess ||
      cudaMalloc(&h->d_count, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMallocHost(&h->h_count, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemcpy(h->d_arm, arm, sizeof(float) * n_groups, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMalloc(&h->status, std::max<int64_t>(n_agents, 1)) != cudaSuccess ||
      cudaMemset(h->status, 0, std::max<int64_t>(n_agents, 1)) != cudaSuccess) {
    rc = SIM_ERR_CUDA;
  }
  if (rc == SIM_OK) {
    h->block_fwd = spread_block(n_agents, h->sms, kDefaultBlockFwd);
    h->block_adj = spread_block(n_agents, h->sms, kDefaultBlockAdj);
  }
  if (rc == SIM_OK && n_groups > 1 && n_agents > 0) {
    unsigned int* d_max = nullptr;
    unsigned int mx = 0;
    if (cudaMalloc(&d_max, sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(d_max, 0, sizeof(unsigned int)) != cudaSuccess) {
      rc = SIM_ERR_CUDA;
    } else {
      max_gid_kernel<<<std::min<int64_t>((n_agents + 255) / 256, 4096), 256>>>(d_group_id, n_agents, d_max);
      if (cudaGetLastError() != cudaSuccess ||
          cudaMemcpy(&mx, d_max, sizeof(unsigned int), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = SIM_ERR_CUDA;
      else if ((int)mx >= n_groups)
        rc = SIM_ERR_GROUP;
    }
    if (d_max) cudaFree(d_max);
  }
  if (rc == SIM_OK) rc = plan_groups(h);
  if (rc == SIM_OK && n_groups > 1) {
    if (cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess) rc = SIM_ERR_CUDA;
    for (int g = 0; g < n_groups && rc == SIM_OK; ++g)
      if (cudaStreamCreateWithFlags(&h->s_grp[g], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->ev_join[g], cudaEventDisableTiming) != cudaSuccess)
        rc = SIM_ERR_CUDA;
  }
  if (rc == SIM_OK) {
    // allow the shared-memory scratch variant of the adjoint its full size
    const int big = (int)(kSmemScratchMax + 64 * 1024);
    if (cudaFuncSetAttribute(adjoint_kernel<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big) != cudaSuccess ||
        cudaFuncSetAttribute(adjoint_kernel<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big) != cudaSuccess ||
        cudaFuncSetAttribute(adjoint_kernel<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big) != cudaSuccess ||
        cudaFuncSetAttribute(adjoint_kernel<2, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big) !=
            cudaSuccess ||
        cudaFuncSetAttribute(adjoint_kernel<1, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big) !=
            cudaSuccess ||
        cudaFuncSetAttribute(adjoint_kernel<0, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big) !=
            cudaSuccess)
      rc = SIM_ERR_CUDA;
  }
  if (rc != SIM_OK) {
    sim_destroy(h);
    return rc;
  }
  *out = h;
  return SIM_OK;
}

int sim_set_params(sim_handle_t h, const sim_group_params_t* groups, int n_groups) {
  if (!h || !groups || n_groups != h->n_groups) return SIM_ERR_ARG;
  DevGroup tbl[SIM_MAX_GROUPS];
  float arm[SIM_MAX_GROUPS];
  float max_arm = 0.f;
  bool multi = false;
  for (int g = 0; g < n_groups; ++g) {
    if (!valid_params(groups[g])) return SIM_ERR_ARG;
    multi = multi || groups[g].type != SIM_TYPE_QUADROTOR;
  }
  if (multi && h->mode != SIM_CLOSED_LOOP) return SIM_ERR_ARG;
  for (int g = 0; g < n_groups; ++g) {
    tbl[g] = derive(groups[g]);
    arm[g] = groups[g].L;
    max_arm = std::max(max_arm, arm[g]);
  }
  // the host copies change only once the device copies have succeeded
  if (cudaMemcpy(h->d_groups, tbl, sizeof(DevGroup) * n_groups, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->d_arm, arm, sizeof(float) * n_groups, cudaMemcpyHostToDevice) != cudaSuccess)
    return SIM_ERR_CUDA;
  h->max_arm = max_arm;
  h->host_group0 = tbl[0];
  for (int g = 0; g < n_groups; ++g) h->host_groups[g] = tbl[g];
  h->multi = multi;
  return SIM_OK;
}

int sim_set_launch(sim_handle_t h, int block_fwd, int block_adj, int K, int C) {
  if (!h || block_fwd < 0 || block_adj < 0 || K < 0 || C < 0) return SIM_ERR_ARG;
  if (block_fwd && (block_fwd % 32 || block_fwd > 256)) return SIM_ERR_ARG;
  if (block_adj && (block_adj % 32 || block_adj > 128)) return SIM_ERR_ARG;
  if (block_fwd) h->block_fwd = block_fwd;
  if (block_adj) h->block_adj = block_adj;
  if (K) h->K = K;
  if (C) h->C = C;
  return SIM_OK;
}

int sim_get_launch(sim_handle_t h, int* block_fwd, int* block_adj, int* K, int* C) {
  if (!h) return SIM_ERR_ARG;
  if (block_fwd) *block_fwd = h->block_fwd;
  if (block_adj) *block_adj = h->block_adj;
  if (K) *K = h->K;
  if (C) *C = h->C;
  return SIM_OK;
}

int64_t sim_step_launches(sim_handle_t h, int64_t nsteps, int substeps_K) {
  if (!h || nsteps <= 0 || h->n == 0) return 0;
  const int64_t K = substeps_K > 0 ? substeps_K : h->K;
  // a fused launch over several groups' ranges is one launch per range (at most one per group)
  const int64_t per = h->n_groups > 1 && range_mode(h, (int)std::min(K, nsteps), 0, h->n) != kPersistent
                          ? h->n_groups : 1;
  const bool plain = plain_path(h, (int)std::min(K, nsteps));
  return (nsteps + K - 1) / K * (plain ? 1 : per) + (plain ? 0 : 1);  // + the refreeze pass
}

int sim_step(sim_handle_t h, float* d_state, const float* d_cmd, float dt, int64_t nsteps, int substeps_K,
             void* stream) {
  if (!h || nsteps < 0 || substeps_K < 0 || !(dt > 0.f) || !std::isfinite(dt)) return SIM_ERR_ARG;
  if (h->n == 0 || nsteps == 0) return SIM_OK;
  if (!d_state || !d_cmd || !aligned16(d_state) || !aligned16(d_cmd)) return SIM_ERR_ARG;
  const int K = substeps_K > 0 ? substeps_K : h->K;
  const StepH H = make_h(dt);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int64_t done = 0;
  while (done < nsteps) {
    const int k = (int)std::min<int64_t>(K, nsteps - done);
    const int rc = launch_step(h, d_state, d_cmd, H, k, st, 0, h->n);
    if (rc != SIM_OK) return rc;
    done += k;
  }
  return launch_refreeze(h, d_state, d_cmd, H, std::min<int64_t>(K, nsteps), st, 0, h->n);
}

int sim_step_host(sim_handle_t h, float* h_state, const float* h_cmd, float* d_state, float* d_cmd, float dt,
                  int64_t nsteps, int substeps_K, void* stream) {
  if (!h || !h_state || !h_cmd || !d_state || !d_cmd || nsteps < 0 || substeps_K < 0 || !(dt > 0.f) ||
      !std::isfinite(dt))
    return SIM_ERR_ARG;
  if (!aligned16(d_state) || !aligned16(d_cmd)) return SIM_ERR_ARG;
  const int64_t n = h->n;
  if (n == 0) return SIM_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (pipeline_streams(h) != SIM_OK) return SIM_ERR_CUDA;
  // Chunks of agents flow through H2D copy -> steps -> D2H copy on separate
  // streams, so the copies of one chunk overlap the steps of the others, and
  // the compute streams run several chunks' launches at once.
  int m;
  int64_t chunk;
  host_chunks(n, &m, &chunk);
  const int K = substeps_K > 0 ? substeps_K : h->K;
  const StepH H = make_h(dt);
  const size_t fs = sizeof(float);
  if (cudaEventRecord(h->ev_start, st) != cudaSuccess) return SIM_ERR_CUDA;
  for (cudaStream_t s2 : {h->s_h2d, h->s_d2h})
    if (cudaStreamWaitEvent(s2, h->ev_start, 0) != cudaSuccess) return SIM_ERR_CUDA;
  for (cudaStream_t s2 : h->s_comp)
    if (cudaStreamWaitEvent(s2, h->ev_start, 0) != cudaSuccess) return SIM_ERR_CUDA;
  auto copy_planes = [&](float* dst, const float* src, int64_t a0, int64_t cnt, cudaMemcpyKind kind,
                         cudaStream_t s2) -> bool {
    for (int k = 0; k < 4; ++k) {
      const size_t off = (size_t)4 * k * n + (size_t)4 * a0;
      if (cudaMemcpyAsync(dst + off, src + off, (size_t)4 * cnt * fs, kind, s2) != cudaSuccess) return false;
    }
    const size_t r = h->mode == SIM_CLOSED_LOOP_PID ? 4 : 1;  // components in plane 4
    const size_t off = (size_t)16 * n + r * (size_t)a0;
    return cudaMemcpyAsync(dst + off, src + off, r * (size_t)cnt * fs, kind, s2) == cudaSuccess;
  };
  for (int c = 0; c < m; ++c) {
    const int64_t a0 = c * chunk, cnt = std::min<int64_t>(chunk, n - a0);
    if (cnt <= 0) break;
    if (!copy_planes(d_state, h_state, a0, cnt, cudaMemcpyHostToDevice, h->s_h2d) ||
        cudaMemcpyAsync(d_cmd + 4 * a0, h_cmd + 4 * a0, (size_t)4 * cnt * fs, cudaMemcpyHostToDevice, h->s_h2d) !=
            cudaSuccess ||
        cudaEventRecord(h->ev_in[c], h->s_h2d) != cudaSuccess)
      return SIM_ERR_CUDA;
    cudaStream_t sc = h->s_comp[c % kComputeStreams];
    if (cudaStreamWaitEvent(sc, h->ev_in[c], 0) != cudaSuccess) return SIM_ERR_CUDA;
    for (int64_t done = 0; done < nsteps;) {
      const int k = (int)std::min<int64_t>(K, nsteps - done);
      const int rc = launch_step(h, d_state, d_cmd, H, k, sc, a0, cnt);
      if (rc != SIM_OK) return rc;
      done += k;
    }
    if (launch_refreeze(h, d_state, d_cmd, H, std::min<int64_t>(K, nsteps), sc, a0, cnt) != SIM_OK)
      return SIM_ERR_CUDA;
    if (cudaEventRecord(h->ev_done[c], sc) != cudaSuccess ||
        cudaStreamWaitEvent(h->s_d2h, h->ev_done[c], 0) != cudaSuccess ||
        !copy_planes(h_state, d_state, a0, cnt, cudaMemcpyDeviceToHost, h->s_d2h))
      return SIM_ERR_CUDA;
  }
  if (cudaEventRecord(h->ev_end, h->s_d2h) != cudaSuccess || cudaStreamWaitEvent(st, h->ev_end, 0) != cudaSuccess)
    return SIM_ERR_CUDA;
  return wait_stream(st, 600000);
}

int sim_run_rounds(sim_handle_t h, float* d_state, float* d_cmd2, const float* h_cmds, float* d_obs2, float* h_obs,
                   float dt, int64_t steps_per_round, int64_t rounds, int substeps_K, void* stream) {
  if (!h || !d_state || !d_cmd2 || !h_cmds || steps_per_round < 1 || rounds < 0 || substeps_K < 0 ||
      !(dt > 0.f) || !std::isfinite(dt))
    return SIM_ERR_ARG;
  if ((h_obs == nullptr) != (d_obs2 == nullptr)) return SIM_ERR_ARG;
  if (!aligned16(d_state) || !aligned16(d_cmd2) || (d_obs2 && !aligned16(d_obs2))) return SIM_ERR_ARG;
  const int64_t n = h->n;
  if (n == 0 || rounds == 0) return SIM_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (pipeline_streams(h) != SIM_OK) return SIM_ERR_CUDA;
  const size_t plane = (size_t)4 * n;  // floats in one command or observation plane
  const StepH H = make_h(dt);
  const int K = substeps_K > 0 ? substeps_K : h->K;
  if (cudaEventRecord(h->ev_start, st) != cudaSuccess || cudaStreamWaitEvent(h->s_h2d, h->ev_start, 0) != cudaSuccess ||
      cudaStreamWaitEvent(h->s_d2h, h->ev_start, 0) != cudaSuccess)
    return SIM_ERR_CUDA;
  auto push = [&](int64_t r) -> bool {  // commands of round r into plane r % 2
    const int b = (int)(r & 1);
    float* dst = d_cmd2 + b * plane;
    if (r >= 2 && cudaStreamWaitEvent(h->s_h2d, h->ev_cmd_free[b], 0) != cudaSuccess) return false;
    return cudaMemcpyAsync(dst, h_cmds + (size_t)r * plane, plane * sizeof(float), cudaMemcpyHostToDevice,
                           h->s_h2d) == cudaSuccess &&
           cudaEventRecord(h->ev_cmd[b], h->s_h2d) == cudaSuccess;
  };
  if (!push(0)) return SIM_ERR_CUDA;
  for (int64_t r = 0; r < rounds; ++r) {
    const int b = (int)(r & 1);
    if (r + 1 < rounds && !push(r + 1)) return SIM_ERR_CUDA;
    if (cudaStreamWaitEvent(st, h->ev_cmd[b], 0) != cudaSuccess) return SIM_ERR_CUDA;
    const float* cmd = d_cmd2 + b * plane;
    for (int64_t done = 0; done < steps_per_round;) {
      const int k = (int)std::min<int64_t>(K, steps_per_round - done);
      const int rc = launch_step(h, d_state, cmd, H, k, st, 0, n);
      if (rc != SIM_OK) return rc;
      done += k;
    }
    if (launch_refreeze(h, d_state, cmd, H, std::min<int64_t>(K, steps_per_round), st, 0, n) != SIM_OK)
      return SIM_ERR_CUDA;
    if (cudaEventRecord(h->ev_cmd_free[b], st) != cudaSuccess) return SIM_ERR_CUDA;
    if (d_obs2) {
      float* snap = d_obs2 + b * plane;
      if (r >= 2 && cudaStreamWaitEvent(st, h->ev_obs_free[b], 0) != cudaSuccess) return SIM_ERR_CUDA;
      if (cudaMemcpyAsync(snap, d_state, plane * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
          cudaEventRecord(h->ev_obs[b], st) != cudaSuccess ||
          cudaStreamWaitEvent(h->s_d2h, h->ev_obs[b], 0) != cudaSuccess ||
          cudaMemcpyAsync(h_obs + (size_t)r * plane, snap, plane * sizeof(float), cudaMemcpyDeviceToHost, h->s_d2h) !=
              cudaSuccess ||
          cudaEventRecord(h->ev_obs_free[b], h->s_d2h) != cudaSuccess)
        return SIM_ERR_CUDA;
    }
  }
  if (cudaEventRecord(h->ev_end, h->s_d2h) != cudaSuccess || cudaStreamWaitEvent(st, h->ev_end, 0) != cudaSuccess)
    return SIM_ERR_CUDA;
  // the copy stream may still hold the last command copies' completion: order them too
  if (cudaEventRecord(h->ev_start, h->s_h2d) != cudaSuccess || cudaStreamWaitEvent(st, h->ev_start, 0) != cudaSuccess)
    return SIM_ERR_CUDA;
  return wait_stream(st, 600000);
}

int sim_rollout_forward(sim_handle_t h, const float* d_state0, const float* d_cmd, float dt, int64_t nsteps,
                        int ckpt_C, float* d_ckpt, float* d_run_cost, void* stream) {
  if (!h || nsteps < 1 || ckpt_C < 0 || !(dt > 0.f) || !std::isfinite(dt)) return SIM_ERR_ARG;
  if (h->multi) return SIM_ERR_ARG;  // rollouts and the adjoint cover quadrotor groups
  if (h->n == 0) return SIM_OK;
  if (!d_state0 || !d_cmd || !d_ckpt || !aligned16(d_state0) || !aligned16(d_cmd) || !aligned16(d_ckpt))
    return SIM_ERR_ARG;
  const int C = ckpt_C > 0 ? ckpt_C : h->C;
  CkptArgs A;
  A.x0 = d_state0;
  A.ckpt = d_ckpt;
  A.run_cost = d_run_cost;
  A.cmd = reinterpret_cast<const float4*>(d_cmd);
  A.gid = h->gid;
  A.status = h->status;
  A.n = h->n;
  A.nsteps = nsteps;
  A.C = C;
  A.S = (int)((nsteps + C - 1) / C);
  A.n_groups = h->n_groups;
  A.H = make_h(dt);
  A.groups = h->d_groups;
  live_visit(h, &A.order, &A.count);
  A.coef = lin_coef(h->host_group0, A.H);
  const size_t smem = group_smem(h);
  const int grid = fwd_grid(h, smem, h->n);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const DevGroup& P0 = h->host_group0;
  if (A.order) {
    // the agents dead at the start first: ckpt_kernel marks the ones that die on the way
    const int fgrid = (int)std::max<int64_t>(1, std::min<int64_t>((h->n + 255) / 256, (int64_t)h->sms * 8));
    if (h->mode == SIM_CLOSED_LOOP_PID) ckpt_frozen_kernel<2><<<fgrid, 256, 0, st>>>(A);
    else if (h->mode == SIM_CLOSED_LOOP) ckpt_frozen_kernel<1><<<fgrid, 256, 0, st>>>(A);
    else ckpt_frozen_kernel<0><<<fgrid, 256, 0, st>>>(A);
  }
  if (h->mode == SIM_CLOSED_LOOP_PID) {
    if (hetero(h)) ckpt_kernel<2, true><<<grid, h->block_fwd, smem, st>>>(A, P0);
    else ckpt_kernel<2, false><<<grid, h->block_fwd, smem, st>>>(A, P0);
  } else if (h->mode == SIM_CLOSED_LOOP) {
    if (hetero(h)) ckpt_kernel<1, true><<<grid, h->block_fwd, smem, st>>>(A, P0);
    else ckpt_kernel<1, false><<<grid, h->block_fwd, smem, st>>>(A, P0);
  } else {
    if (hetero(h)) ckpt_kernel<0, true><<<grid, h->block_fwd, smem, st>>>(A, P0);
    else ckpt_kernel<0, false><<<grid, h->block_fwd, smem, st>>>(A, P0);
  }
  return cudaGetLastError() == cudaSuccess ? SIM_OK : SIM_ERR_CUDA;
}

size_t sim_workspace_bytes(sim_handle_t h, int ckpt_C) {
  if (!h || ckpt_C < 0) return 0;
  const int C = ckpt_C > 0 ? ckpt_C : h->C;
  const int grid = adj_grid(h, C);
  return scratch_bytes(h, C, grid) + align256((size_t)grid * h->n_groups * NTH * sizeof(float));
}

int sim_rollout_backward(sim_handle_t h, const float* d_ckpt, const float* d_cmd, float dt, int64_t nsteps,
                         int ckpt_C, const float* d_dL_dxT, const float* d_w_run, float* d_dL_dx0,
                         float* d_dL_dtheta, float* d_dL_dtheta_agent, void* d_workspace, size_t ws_bytes,
                         void* stream) {
  if (!h || nsteps < 1 || ckpt_C < 0 || !(dt > 0.f) || !std::isfinite(dt)) return SIM_ERR_ARG;
  if (!d_dL_dtheta || h->multi) return SIM_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (h->n == 0) {
    return cudaMemsetAsync(d_dL_dtheta, 0, sizeof(float) * h->n_groups * NTH, st) == cudaSuccess ? SIM_OK
                                                                                                : SIM_ERR_CUDA;
  }
  if (!d_ckpt || !d_cmd || !d_dL_dxT || !d_dL_dx0 || !d_workspace) return SIM_ERR_ARG;
  if (!aligned16(d_ckpt) || !aligned16(d_cmd) || !aligned16(d_dL_dxT) || !aligned16(d_dL_dx0) ||
      (reinterpret_cast<uintptr_t>(d_workspace) & 255u))
    return SIM_ERR_ARG;
  const int C = ckpt_C > 0 ? ckpt_C : h->C;
  const int grid = adj_grid(h, C);
  const size_t sbytes = scratch_bytes(h, C, grid);
  const size_t need = sbytes + align256((size_t)grid * h->n_groups * NTH * sizeof(float));
  if (ws_bytes < need) return SIM_ERR_WORKSPACE;
  AdjArgs A;
  A.ckpt = d_ckpt;
  A.cmd = reinterpret_cast<const float4*>(d_cmd);
  A.gid = h->n_groups > 1 ? h->gid : nullptr;
  A.status = h->status;
  A.dLdxT = d_dL_dxT;
  A.w_run = d_w_run;
  A.dLdx0 = d_dL_dx0;
  A.th_agent = d_dL_dtheta_agent;
  A.scratch = static_cast<float*>(d_workspace);
  A.partials = reinterpret_cast<float*>(static_cast<char*>(d_workspace) + sbytes);
  A.n = h->n;
  A.nsteps = nsteps;
  A.C = C;
  A.S = (int)((nsteps + C - 1) / C);
  A.n_groups = h->n_groups;
  A.H = make_h(dt);
  A.groups = h->d_groups;
  live_visit(h, &A.order, &A.count);
  if (launch_adjoint(h, A, C, grid, st) != SIM_OK) return SIM_ERR_CUDA;
  reduce_partials<<<h->n_groups * NTH, 256, 0, st>>>(A.partials, grid, h->n_groups * NTH, d_dL_dtheta);
  return cudaGetLastError() == cudaSuccess ? SIM_OK : SIM_ERR_CUDA;
}

}  // extern "C"

// ------------------------------------------------ workspace-free adjoint --
// Scratch for sim_rollout_backward_noalloc: a fixed array in the module's own
// device memory, present on every GPU that loads the library until exit.
// Device code could name it directly; host code needs its device address,
// which cudaGetSymbolAddress returns per device (the host-side symbol is only
// a stand-in).  Every call shares it: scratch is written before it is read
// and the per-block partials are written in full, so nothing is cleared.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SIM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device`, looked up once per device
// with that device current.
int noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return SIM_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return SIM_ERR_CUDA;
    if (cur != device && cudaSetDevice(device) != cudaSuccess) return SIM_ERR_CUDA;
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (cur != device) cudaSetDevice(cur);
    if (e != cudaSuccess || !p) return SIM_ERR_CUDA;
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return SIM_OK;
}

}  // namespace

extern "C" {

int sim_rollout_backward_noalloc(sim_handle_t h, const float* d_ckpt, const float* d_cmd, float dt, int64_t nsteps,
                                 int ckpt_C, const float* d_dL_dxT, const float* d_w_run, float* d_dL_dx0,
                                 float* d_dL_dtheta, float* d_dL_dtheta_agent, void* stream) {
  if (!h || nsteps < 1 || ckpt_C < 0 || !(dt > 0.f) || !std::isfinite(dt)) return SIM_ERR_ARG;
  if (!d_dL_dtheta || h->multi) return SIM_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (h->n == 0) {
    return cudaMemsetAsync(d_dL_dtheta, 0, sizeof(float) * h->n_groups * NTH, st) == cudaSuccess ? SIM_OK
                                                                                                : SIM_ERR_CUDA;
  }
  if (!d_ckpt || !d_cmd || !d_dL_dxT || !d_dL_dx0) return SIM_ERR_ARG;
  if (!aligned16(d_ckpt) || !aligned16(d_cmd) || !aligned16(d_dL_dxT) || !aligned16(d_dL_dx0)) return SIM_ERR_ARG;
  const int C = ckpt_C > 0 ? ckpt_C : h->C;
  // as many resident blocks as the usual grid, but no more than the fixed
  // scratch holds: per block, C step-start states per thread plus one partial
  const size_t per_block = (adj_smem_scratch(h, C) ? 0 : (size_t)C * h->nx * sizeof(float) * h->block_adj) +
                           (size_t)h->n_groups * NTH * sizeof(float);
  const size_t fit = (SIM_NOALLOC_SCRATCH_BYTES - 512) / per_block;
  if (fit < 1) return SIM_ERR_WORKSPACE;
  const int grid = (int)std::min<size_t>((size_t)adj_grid(h, C), fit);
  const size_t sbytes = scratch_bytes(h, C, grid);
  if (sbytes + align256((size_t)grid * h->n_groups * NTH * sizeof(float)) > SIM_NOALLOC_SCRATCH_BYTES)
    return SIM_ERR_WORKSPACE;
  void* base = nullptr;
  const int rc = noalloc_scratch(h->device, &base);
  if (rc != SIM_OK) return rc;
  AdjArgs A;
  A.ckpt = d_ckpt;
  A.cmd = reinterpret_cast<const float4*>(d_cmd);
  A.gid = h->n_groups > 1 ? h->gid : nullptr;
  A.status = h->status;
  A.dLdxT = d_dL_dxT;
  A.w_run = d_w_run;
  A.dLdx0 = d_dL_dx0;
  A.th_agent = d_dL_dtheta_agent;
  A.scratch = static_cast<float*>(base);
  A.partials = reinterpret_cast<float*>(static_cast<char*>(base) + sbytes);
  A.n = h->n;
  A.nsteps = nsteps;
  A.C = C;
  A.S = (int)((nsteps + C - 1) / C);
  A.n_groups = h->n_groups;
  A.H = make_h(dt);
  A.groups = h->d_groups;
  live_visit(h, &A.order, &A.count);
  if (launch_adjoint(h, A, C, grid, st) != SIM_OK) return SIM_ERR_CUDA;
  reduce_partials<<<h->n_groups * NTH, 256, 0, st>>>(A.partials, grid, h->n_groups * NTH, d_dL_dtheta);
  return cudaGetLastError() == cudaSuccess ? SIM_OK : SIM_ERR_CUDA;
}

}  // extern "C"

namespace {

// Buckets of the collision hash: a power of two >= 4 n (few unrelated agents
// share a bucket: 0.25 per bucket on average).
uint32_t collide_table(int64_t n) {
  uint64_t t = 1024;
  while (t < (uint64_t)(4 * n) && t < (1ull << 30)) t <<= 1;
  return (uint32_t)t;
}

// Workspace: the bucket heads, one 32-byte record per agent, one hit byte per agent.
size_t collide_bytes(const sim_s* h) {
  return align256((size_t)collide_table(h->n) * sizeof(int)) + align256((size_t)h->n * sizeof(CollRec)) +
         align256((size_t)h->n);
}

}  // namespace

extern "C" {

size_t sim_collide_workspace_bytes(sim_handle_t h) { return h ? collide_bytes(h) : 0; }

int sim_collide(sim_handle_t h, const float* d_state, float radius_scale, void* d_workspace, size_t ws_bytes,
                void* stream) {
  if (!h || !(radius_scale > 0.f) || !std::isfinite(radius_scale)) return SIM_ERR_ARG;
  if (h->n == 0) return SIM_OK;
  if (h->n > (int64_t)INT32_MAX) return SIM_ERR_ARG;
  if (!d_state || !aligned16(d_state) || !d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u))
    return SIM_ERR_ARG;
  if (ws_bytes < collide_bytes(h)) return SIM_ERR_WORKSPACE;
  const uint32_t table = collide_table(h->n);
  char* w = static_cast<char*>(d_workspace);
  CollArgs A;
  A.pos = reinterpret_cast<const float4*>(d_state);
  A.gid = h->n_groups > 1 ? h->gid : nullptr;
  A.status = h->status;
  A.arm = h->d_arm;
  A.scale = radius_scale;
  // cells 1 % wider than twice the largest contact distance 2 max_arm scale: a
  // pair in contact is less than half a cell apart on every axis, so each
  // agent searches 2 x 2 x 2 cells
  A.inv_cell = 1.0 / (4.0 * (double)h->max_arm * radius_scale * 1.01);
  A.mask = table - 1;
  A.head = reinterpret_cast<int*>(w);
  A.rec = reinterpret_cast<CollRec*>(w + align256((size_t)table * sizeof(int)));
  A.hit = reinterpret_cast<uint8_t*>(w + align256((size_t)table * sizeof(int)) +
                                     align256((size_t)h->n * sizeof(CollRec)));
  A.n = h->n;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(A.head, 0xff, (size_t)table * sizeof(int), st) != cudaSuccess) return SIM_ERR_CUDA;
  const int grid = (int)std::min<int64_t>((h->n + 255) / 256, (int64_t)h->sms * 8);
  collide_insert<<<grid, 256, 0, st>>>(A);
  collide_query<<<grid, 256, 0, st>>>(A);
  collide_apply<<<grid, 256, 0, st>>>(A);
  return cudaGetLastError() == cudaSuccess ? SIM_OK : SIM_ERR_CUDA;
}

int sim_copy_status(sim_handle_t h, uint8_t* d_status_out, void* stream) {
  if (!h) return SIM_ERR_ARG;
  if (h->n == 0) return SIM_OK;
  if (!d_status_out) return SIM_ERR_ARG;
  return cudaMemcpyAsync(d_status_out, h->status, (size_t)h->n, cudaMemcpyDeviceToDevice,
                         reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? SIM_OK
             : SIM_ERR_CUDA;
}

int sim_load_status(sim_handle_t h, const uint8_t* d_status_in, void* stream) {
  if (!h) return SIM_ERR_ARG;
  if (h->n == 0) return SIM_OK;
  if (!d_status_in) return SIM_ERR_ARG;
  drop_live(h);
  return cudaMemcpyAsync(h->status, d_status_in, (size_t)h->n, cudaMemcpyDeviceToDevice,
                         reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? SIM_OK
             : SIM_ERR_CUDA;
}

int sim_status(sim_handle_t h, int64_t* n_dead, int timeout_ms, void* stream) {
  if (!h || !n_dead) return SIM_ERR_ARG;
  *n_dead = 0;
  if (h->n == 0) return SIM_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the count lands in the handle's pinned word: a copy still in flight after
  // a timed-out wait writes there, not into a dead stack frame
  if (cudaMemsetAsync(h->d_count, 0, sizeof(unsigned long long), st) != cudaSuccess) return SIM_ERR_CUDA;
  count_dead_kernel<<<std::min<int64_t>((h->n + 255) / 256, 4096), 256, 0, st>>>(h->status, h->n, h->d_count);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(h->h_count, h->d_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return SIM_ERR_CUDA;
  const int rc = wait_stream(st, timeout_ms);
  if (rc == SIM_OK) *n_dead = (int64_t)*h->h_count;
  return rc;
}

int sim_reset_status(sim_handle_t h, void* stream) {
  if (!h) return SIM_ERR_ARG;
  if (h->n == 0) return SIM_OK;
  drop_live(h);
  return cudaMemsetAsync(h->status, 0, h->n, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? SIM_OK
                                                                                                   : SIM_ERR_CUDA;
}

int sim_group_stats(sim_handle_t h, const float* d_state, double* h_out, void* stream) {
  if (!h || !h_out) return SIM_ERR_ARG;
  const int G = h->n_groups, width = G * kStatFields;
  for (int e = 0; e < width; ++e) h_out[e] = 0.0;
  if (h->n == 0) return SIM_OK;
  if (!d_state || !aligned16(d_state)) return SIM_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((h->n + kStatBlock - 1) / kStatBlock,
                                                                 (int64_t)h->sms * 8));
  if (!h->d_stat) {
    h->stat_blocks = std::max(blocks, h->sms * 8);
    if (cudaMalloc(&h->d_stat, sizeof(double) * (size_t)(h->stat_blocks + 1) * width) != cudaSuccess) {
      h->d_stat = nullptr;
      return SIM_ERR_CUDA;
    }
  }
  if (!h->h_stat && cudaMallocHost(&h->h_stat, sizeof(double) * width) != cudaSuccess) {
    h->h_stat = nullptr;
    return SIM_ERR_CUDA;
  }
  StatArgs A;
  A.pos = reinterpret_cast<const float4*>(d_state);
  A.status = h->status;
  A.gid = G > 1 ? h->gid : nullptr;
  A.n = h->n;
  A.n_groups = G;
  A.partials = h->d_stat;
  double* sums = h->d_stat + (size_t)h->stat_blocks * width;
  group_stats_kernel<<<blocks, kStatBlock, 0, st>>>(A);
  group_stats_finish<<<1, 256, 0, st>>>(h->d_stat, blocks, width, sums);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(h->h_stat, sums, sizeof(double) * width, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return SIM_ERR_CUDA;
  const int rc = wait_stream(st, 600000);
  if (rc != SIM_OK) return rc;
  for (int g = 0; g < G; ++g) {
    const double* r = h->h_stat + g * kStatFields;
    double* o = h_out + g * kStatFields;
    o[0] = r[0];
    o[1] = r[1];
    o[2] = r[2];
    for (int k = 3; k < 6; ++k) o[k] = r[0] > 0 ? r[k] / r[0] : 0.0;
  }
  return SIM_OK;
}

int sim_compact(sim_handle_t h, void* stream) {
  if (!h) return SIM_ERR_ARG;
  if (h->n == 0 || h->n > (int64_t)UINT32_MAX) return SIM_OK;
  if (!h->d_live && cudaMalloc(&h->d_live, sizeof(uint32_t) * (size_t)h->n) != cudaSuccess) return SIM_ERR_CUDA;
  // returns with the order in place, so that launches on any stream may use it
  const int rc = order_live(h, reinterpret_cast<cudaStream_t>(stream), h->d_live, h->live_off);
  if (rc != SIM_OK) {
    drop_live(h);
    return rc;
  }
  h->live = true;
  ++h->epoch;
  return SIM_OK;
}

int sim_graph_create(sim_handle_t h, float* d_state, const float* d_cmd, float dt, int64_t nsteps, int substeps_K,
                     void* stream, sim_graph_t* out) {
  if (!h || !out || !stream) return SIM_ERR_ARG;
  *out = nullptr;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  sim_graph_s* g = new (std::nothrow) sim_graph_s();
  if (!g) return SIM_ERR_ARG;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    delete g;
    return SIM_ERR_CUDA;
  }
  const int rc = sim_step(h, d_state, d_cmd, dt, nsteps, substeps_K, stream);
  const cudaError_t e = cudaStreamEndCapture(st, &g->graph);
  if (rc != SIM_OK || e != cudaSuccess) {
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return rc != SIM_OK ? rc : SIM_ERR_CUDA;
  }
  if (cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) {
    cudaGraphDestroy(g->graph);
    delete g;
    return SIM_ERR_CUDA;
  }
  g->h = h;
  g->epoch = h->epoch;
  *out = g;
  return SIM_OK;
}

int sim_graph_launch(sim_graph_t g, void* stream) {
  if (!g) return SIM_ERR_ARG;
  if (g->h->epoch != g->epoch) return SIM_ERR_STALE;  // the agent order it captured has changed
  return cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? SIM_OK : SIM_ERR_CUDA;
}

void sim_graph_destroy(sim_graph_t g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

void sim_destroy(sim_handle_t h) {
  if (!h) return;
  for (cudaStream_t st : {h->s_h2d, h->s_d2h})
    if (st) cudaStreamDestroy(st);
  for (cudaStream_t st : h->s_comp)
    if (st) cudaStreamDestroy(st);
  for (cudaStream_t st : h->s_grp)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t e : h->ev_join)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : {h->ev_start, h->ev_end, h->ev_fork})
    if (e) cudaEventDestroy(e);
  for (int c = 0; c < kHostChunks; ++c) {
    if (h->ev_in[c]) cudaEventDestroy(h->ev_in[c]);
    if (h->ev_done[c]) cudaEventDestroy(h->ev_done[c]);
  }
  for (int b = 0; b < 2; ++b)
    for (cudaEvent_t e : {h->ev_cmd[b], h->ev_cmd_free[b], h->ev_obs[b], h->ev_obs_free[b]})
      if (e) cudaEventDestroy(e);
  if (h->status) cudaFree(h->status);
  if (h->d_groups) cudaFree(h->d_groups);
  if (h->d_arm) cudaFree(h->d_arm);
  if (h->d_count) cudaFree(h->d_count);
  if (h->h_count) cudaFreeHost(h->h_count);
  if (h->d_order) cudaFree(h->d_order);
  if (h->d_live) cudaFree(h->d_live);
  if (h->d_stat) cudaFree(h->d_stat);
  if (h->h_stat) cudaFreeHost(h->h_stat);
  if (h->d_live_cnt) cudaFree(h->d_live_cnt);
  if (h->d_live_off) cudaFree(h->d_live_off);
  if (h->h_live_cnt) cudaFreeHost(h->h_live_cnt);
  if (h->h_live_off) cudaFreeHost(h->h_live_off);
  delete h;
}

}  // extern "C"
