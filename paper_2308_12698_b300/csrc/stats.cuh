// Per-group diagnostics of a swarm (sim_group_stats): for every parameter
// group the number of live agents, of agents frozen non-finite and of agents
// marked collided, and the mean position of the live agents.  One thread per
// agent over a grid-stride loop; inside a warp the agents of each group are
// summed by a segmented butterfly (the group of the lowest remaining lane
// first), per warp into shared memory, per block into a partial row; a second
// kernel adds the rows in block order.  FP64 sums, no atomics: the same
// result on every run.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "checks.cuh"

namespace qs {

constexpr int kStatBlock = 256;
constexpr int kStatFields = 6;  // live, non-finite, collided, sum px, sum py, sum pz

struct StatArgs {
  const float4* pos;      // plane 0 of the planar state: (px, py, pz, vx)
  const uint8_t* status;
  const uint8_t* gid;     // null for one group
  int64_t n;
  int n_groups;
  double* partials;       // [gridDim.x][n_groups][kStatFields]
};

__global__ void __launch_bounds__(kStatBlock) group_stats_kernel(StatArgs A) {
  __shared__ double acc[kStatBlock / 32][32][kStatFields];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < (kStatBlock / 32) * 32 * kStatFields; e += blockDim.x) (&acc[0][0][0])[e] = 0.0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // every lane runs the same number of rounds, so the warp's shuffles see all 32 lanes
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < A.n; base += stride) {
    const int64_t i = base + threadIdx.x;
    int g = -1;
    double v[kStatFields] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (i < A.n) {
      g = A.gid ? (int)A.gid[i] : 0;
      if (!QS_OK(g < A.n_groups, 5, g) || g >= A.n_groups) g = -1;  // off the hot path: guarded in every build
    }
    if (g >= 0) {
      const uint8_t s = A.status[i];
      if (s == 0) {
        const float4 p = A.pos[i];
        v[0] = 1.0;
        v[3] = p.x;
        v[4] = p.y;
        v[5] = p.z;
      } else if (s == 2) {
        v[2] = 1.0;
      } else {
        v[1] = 1.0;
      }
    }
    unsigned todo = __ballot_sync(0xffffffffu, g >= 0);
    while (todo) {
      const int leader = __ffs(todo) - 1;
      const int gl = __shfl_sync(0xffffffffu, g, leader);
      const bool mine = g == gl;
      todo &= ~__ballot_sync(0xffffffffu, mine);
#pragma unroll
      for (int q = 0; q < kStatFields; ++q) {
        double t = mine ? v[q] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0) acc[warp][gl][q] += t;
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < A.n_groups * kStatFields; e += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < kStatBlock / 32; ++w) t += acc[w][e / kStatFields][e % kStatFields];
    A.partials[(int64_t)blockIdx.x * A.n_groups * kStatFields + e] = t;
  }
}

// out[e] = sum of partials[b][e] over the blocks b in increasing order, one
// thread per entry (at most 32 groups x 6 fields); means from the sums.
__global__ void group_stats_finish(const double* partials, int nblocks, int width, double* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= width) return;
  double t = 0.0;
  for (int b = 0; b < nblocks; ++b) t += partials[(int64_t)b * width + e];
  out[e] = t;
}

}  // namespace qs
