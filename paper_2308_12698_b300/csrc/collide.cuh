// Collision detection between live agents (Sec. III-A: colliding agents are
// marked dead).  Cells of side s >= 2 x (the largest contact distance) are
// hashed into a power-of-two table with one linked list per bucket
// (collide_insert); a pair in contact is then less than s / 2 apart on every
// axis, so each agent searches only the 2 x 2 x 2 block of cells on the side
// of its own cell that it lies nearer to on each axis (collide_query), deciding
// d^2 < (r_i + r_j)^2 in FP32 with every operation rounded on its own; the
// marks come last (collide_apply), so that the outcome does not depend on the
// order of the lists.
//
// Each agent's list entry is one 32-byte record (position, contact radius,
// link): a step of a walk reads one L2 sector.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "checks.cuh"

namespace qs {

struct __align__(32) CollRec {
  float4 p;     // x, y, z, contact radius r = arm length of its group x radius_scale
  int next;     // next agent in the same bucket, -1 at the end
  int pad[3];
};

struct CollArgs {
  const float4* pos;      // plane 0 of the planar state: (px, py, pz, vx)
  const uint8_t* gid;
  uint8_t* status;
  const float* arm;
  float scale;
  double inv_cell;        // 1 / cell side
  uint32_t mask;          // table size - 1 (power of two)
  int* head;              // [table] first agent of each bucket, -1 if empty
  CollRec* rec;           // [n] the agents' records (live agents only)
  uint8_t* hit;           // [n]
  int64_t n;
};

// Spatial hash of an integer cell (Teschner et al., 2003).
__device__ __forceinline__ uint32_t cell_key(int cx, int cy, int cz, uint32_t mask) {
  return (((uint32_t)cx * 73856093u) ^ ((uint32_t)cy * 19349663u) ^ ((uint32_t)cz * 83492791u)) & mask;
}

// Cell coordinate of v in FP64 (an FP32 position is exact in FP64, and the
// product's rounding is far below the half-cell margin at any cell count
// an int holds), and which neighbour (-1 or +1) lies nearer.
__device__ __forceinline__ int cell_of(float v, double inv_cell, int* side) {
  const double t = (double)v * inv_cell;
  const double c = floor(t);
  *side = (t - c) < 0.5 ? -1 : 1;
  return (int)c;
}

__device__ __forceinline__ float contact_radius(const CollArgs& A, int64_t i) {
  return __fmul_rn(A.arm[A.gid ? A.gid[i] : 0], A.scale);
}

__global__ void __launch_bounds__(256) collide_insert(CollArgs A) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += stride) {
    if (A.status[i]) continue;
    const float4 p = A.pos[i];
    int s;
    const uint32_t k = cell_key(cell_of(p.x, A.inv_cell, &s), cell_of(p.y, A.inv_cell, &s),
                                cell_of(p.z, A.inv_cell, &s), A.mask);
    A.rec[i].p = make_float4(p.x, p.y, p.z, contact_radius(A, i));
    A.rec[i].next = atomicExch(&A.head[k], (int)i);
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
      const float4 pi = A.rec[i].p;
      int sx, sy, sz;
      const int cx = cell_of(pi.x, A.inv_cell, &sx), cy = cell_of(pi.y, A.inv_cell, &sy),
                cz = cell_of(pi.z, A.inv_cell, &sz);
      int64_t budget = A.n + 8;  // a list never holds more than n agents
      for (int b = 0; b < 8 && !h; ++b) {
        int j = A.head[cell_key(cx + ((b & 1) ? sx : 0), cy + ((b & 2) ? sy : 0), cz + ((b & 4) ? sz : 0), A.mask)];
        while (j >= 0 && budget-- > 0) {
#ifdef QS_CHECKED
          if (!QS_OK(j < A.n, 10, j)) break;
#endif
          const float4* r4 = reinterpret_cast<const float4*>(A.rec + j);
          const float4 pj = r4[0];
          const int nj = __float_as_int(r4[1].x);
          if ((int64_t)j != i && pair_hit(pi, pi.w, pj, pj.w)) {
            h = 1;
            break;
          }
          j = nj;
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
