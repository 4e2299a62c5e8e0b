// The live agents' order for sim_compact, built on the device in two passes
// over the status bytes: live_order_kernel<false> counts the live agents of
// every (group, host-pipeline chunk), the host turns the counts into
// positions, and live_order_kernel<true> writes each live agent's index at its
// position.  One block of 1024 threads per chunk walks the chunk's agents in
// index order, 1024 at a time, so that the order is sorted by (group, chunk,
// index): the same order a host-side counting sort gives.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "checks.cuh"

namespace qs {

constexpr int kLiveBlock = 1024;  // threads of live_order_kernel: 32 warps
constexpr int kLiveGroups = 32;   // the most groups a handle has

struct LiveArgs {
  const uint8_t* status;  // n status bytes: 0 = live
  const uint8_t* gid;     // n group ids, or null for one group
  int64_t n;
  int64_t chunk;          // agents per host-pipeline chunk (the last one shorter)
  int n_groups;
  int n_chunks;
  unsigned int* counts;   // pass 1: [n_groups][n_chunks] live agents
  const int64_t* off;     // pass 2: [n_groups][n_chunks + 1] first position of each (group, chunk)
  uint32_t* order;        // pass 2: agent index at each position
};

template <bool SCATTER>
__global__ void __launch_bounds__(kLiveBlock) live_order_kernel(LiveArgs A) {
  __shared__ unsigned int wcnt[kLiveBlock / 32][kLiveGroups];  // live agents per warp and group, this round
  __shared__ int64_t next[kLiveGroups];                        // next position (or running count) per group
  const int c = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t a0 = (int64_t)c * A.chunk, a1 = a0 + A.chunk < A.n ? a0 + A.chunk : A.n;
  if (threadIdx.x < A.n_groups) next[threadIdx.x] = SCATTER ? A.off[threadIdx.x * (A.n_chunks + 1) + c] : 0;
  for (int64_t r0 = a0; r0 < a1; r0 += kLiveBlock) {
    for (int k = threadIdx.x; k < (kLiveBlock / 32) * kLiveGroups; k += kLiveBlock) (&wcnt[0][0])[k] = 0;
    __syncthreads();
    const int64_t i = r0 + threadIdx.x;
    int g = 0;
    bool live = i < a1 && A.status[i] == 0;
    if (live && A.gid) g = A.gid[i];
    live = live && g < A.n_groups;
    // lanes of this warp holding live agents of the same group; rank = how many sit below
    const unsigned peers = __match_any_sync(0xffffffffu, live ? g : -1);
    const unsigned below = peers & ((1u << lane) - 1u);
    if (live && below == 0) wcnt[w][g] = __popc(peers);
    __syncthreads();
    if (SCATTER && live) {
      int64_t pos = next[g] + __popc(below);
      for (int v = 0; v < w; ++v) pos += wcnt[v][g];
      // the bucket's end bounds the write even if the status changed between the passes
      if (pos < A.off[g * (A.n_chunks + 1) + c + 1] && QS_OK(pos >= 0 && pos < A.n, 11, pos))
        A.order[pos] = (uint32_t)i;
    }
    __syncthreads();
    if (threadIdx.x < A.n_groups) {
      unsigned int t = 0;
      for (int v = 0; v < kLiveBlock / 32; ++v) t += wcnt[v][threadIdx.x];
      next[threadIdx.x] += t;
    }
    __syncthreads();  // the sums have read wcnt before the next round clears it
  }
  __syncthreads();
  if (!SCATTER && threadIdx.x < A.n_groups) A.counts[threadIdx.x * A.n_chunks + c] = (unsigned int)next[threadIdx.x];
}

}  // namespace qs
