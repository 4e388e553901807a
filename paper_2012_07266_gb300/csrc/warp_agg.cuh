// Warp-aggregated atomic addition.  Lanes of a warp that add to the same
// address are grouped (__match_any_sync); the group's lowest lane sums the
// group's values through shared memory and issues a single atomic.  Clustered
// particles come from a compact Lagrangian patch, i.e. from consecutive lanes,
// so in dense regions this turns up to 32 same-address atomics into one.
// All 32 lanes of the warp must call it together (inactive work adds 0).
#pragma once

#include <cuda_runtime.h>

namespace pmlens {

template <typename T, typename I>
__device__ __forceinline__ void warp_agg_add(T* base, I idx, T v, T* wsm /* 32 per warp */) {
  const int lane = threadIdx.x & 31;
  unsigned peers;
  if constexpr (sizeof(I) <= 4) peers = __match_any_sync(0xffffffffu, (unsigned)idx);
  else peers = __match_any_sync(0xffffffffu, (unsigned long long)idx);
  wsm[lane] = v;
  __syncwarp();
  if (lane == __ffs(peers) - 1) {
    T s = v;
    unsigned m = peers & (peers - 1);  // the other lanes of the group
    while (m) {
      s += wsm[__ffs(m) - 1];
      m &= m - 1;
    }
    atomicAdd(base + idx, s);
  }
  __syncwarp();
}

}  // namespace pmlens
