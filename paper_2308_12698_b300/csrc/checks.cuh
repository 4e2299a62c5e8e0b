// Device-side bounds checks for the checked build (QS_CHECKED defined): every
// instrumented access first tests its index against the extent of the buffer
// it reads or writes.  A failed test records the first failure in a device
// word -- site << 48 | (index & (2^48 - 1)) -- and the access is skipped; the
// kernel goes on (no trap, no assert), so the context stays usable and the
// host reads the word (sim_bounds_checks).  Without QS_CHECKED the tests
// compile to nothing and the kernels are the product kernels.
//
// Sites:
//   1 load_state      agent index outside [0, n) of a planar state
//   2 store_state     agent index outside [0, n) of a planar state
//   3 prefetch_state  agent index outside [0, n) of a planar state (cp.async)
//   4 step kernels    agent index outside [0, n) (status, command, group id)
//   5 group tables    group id outside [0, n_groups)
//   6 group_kernel    position outside [0, n)
//   7 group_kernel    order[position] outside [0, n)
//   8 checkpoints     checkpoint index outside [0, S]
//   9 adjoint         scratch step outside [0, C), or per-agent theta row outside [0, n)
//  10 collisions      bucket outside the table, record outside [0, n)
//  11 live order      position outside [0, n), or (group, chunk) outside the count table
//  12 partial sums    partial slot outside [0, blocks x groups x 16)
#pragma once
#include <stdint.h>

namespace qs {

#ifdef QS_CHECKED
__device__ unsigned long long g_check_word;

__device__ __forceinline__ bool check_ok(bool ok, unsigned long long site, int64_t index) {
  if (!ok) atomicCAS(&g_check_word, 0ull, (site << 48) | ((unsigned long long)index & 0xffffffffffffull));
  return ok;
}
#define QS_OK(cond, site, index) ::qs::check_ok((cond), (site), (int64_t)(index))
#else
#define QS_OK(cond, site, index) true
#endif

}  // namespace qs
