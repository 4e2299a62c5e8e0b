// Collision detection between live agents (Sec. III-A: colliding agents are
// marked dead): a spatial hash of the agents' cells with one linked list per
// bucket (collide_insert), a 27-cell neighbour search per agent deciding
// d^2 < (r_i + r_j)^2 in FP32 with every operation rounded on its own
// (collide_query), then the marks (collide_apply), so that the outcome does
// not depend on the order of the lists.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace qs {

struct CollArgs {
  const float4* pos;      // plane 0 of the planar state: (px, py, pz, vx)
  const uint8_t* gid;
  uint8_t* status;
  const float* arm;
  float scale;
  float inv_cell;
  uint32_t mask;          // table size - 1 (power of two)
  int* head;              // [table] first agent of each bucket, -1 if empty
  int* next;              // [n] next agent in the same bucket, -1 at the end
  uint8_t* hit;           // [n]
  int64_t n;
};

// Spatial hash of an integer cell (Teschner et al., 2003).
__device__ __forceinline__ uint32_t cell_key(int cx, int cy, int cz, uint32_t mask) {
  return (((uint32_t)cx * 73856093u) ^ ((uint32_t)cy * 19349663u) ^ ((uint32_t)cz * 83492791u)) & mask;
}

__device__ __forceinline__ int cell_of(float v, float inv_cell) { return (int)floorf(v * inv_cell); }

__global__ void __launch_bounds__(256) collide_insert(CollArgs A) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += stride) {
    if (A.status[i]) continue;
    const float4 p = A.pos[i];
    const uint32_t k = cell_key(cell_of(p.x, A.inv_cell), cell_of(p.y, A.inv_cell), cell_of(p.z, A.inv_cell), A.mask);
    A.next[i] = atomicExch(&A.head[k], (int)i);
  }
}

// FP32 pair test with every operation rounded separately (no contraction).
__device__ __forceinline__ bool pair_hit(float4 pi, float ri, float4 pj, float rj) {
  const float dx = __fsub_rn(pj.x, pi.x), dy = __fsub_rn(pj.y, pi.y), dz = __fsub_rn(pj.z, pi.z);
  const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
  const float rs = __fadd_rn(ri, rj);
  return d2 < __fmul_rn(rs, rs);
}

__global__ void __launch_bounds__(256) collide_query(CollArgs A) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += stride) {
    uint8_t h = 0;
    if (A.status[i] == 0) {
      const float4 pi = A.pos[i];
      const float ri = __fmul_rn(A.arm[A.gid ? A.gid[i] : 0], A.scale);
      const int cx = cell_of(pi.x, A.inv_cell), cy = cell_of(pi.y, A.inv_cell), cz = cell_of(pi.z, A.inv_cell);
      int64_t budget = A.n + 27;  // a list never holds more than n agents
      for (int dz = -1; dz <= 1 && !h; ++dz)
        for (int dy = -1; dy <= 1 && !h; ++dy)
          for (int dx = -1; dx <= 1 && !h; ++dx) {
            int j = A.head[cell_key(cx + dx, cy + dy, cz + dz, A.mask)];
            while (j >= 0 && budget-- > 0) {
              if ((int64_t)j != i) {
                const float rj = __fmul_rn(A.arm[A.gid ? A.gid[j] : 0], A.scale);
                if (pair_hit(pi, ri, A.pos[j], rj)) {
                  h = 1;
                  break;
                }
              }
              j = A.next[j];
            }
          }
    }
    A.hit[i] = h;
  }
}

__global__ void __launch_bounds__(256) collide_apply(CollArgs A) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += stride)
    if (A.hit[i] && A.status[i] == 0) A.status[i] = 2;
}

}  // namespace qs
