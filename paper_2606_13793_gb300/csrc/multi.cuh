// Multi-item launches: one launch runs the same kernel body over many
// independent items (the fields of a batched solve), each with its own grid
// of blocks.  Block b of the launch belongs to the item i whose block range
// [start_i, start_i + gx gy gz) holds it; the body sees the item's virtual
// block index and grid extents instead of blockIdx / gridDim.
#pragma once

#include "fmm_internal.h"

namespace fmmgb {

struct VBlock {
  unsigned x, y, z;     // block index inside the item's grid
  unsigned gx, gy, gz;  // the item's grid
};

__device__ __forceinline__ VBlock native_vblock() {
  VBlock v;
  v.x = blockIdx.x, v.y = blockIdx.y, v.z = blockIdx.z;
  v.gx = gridDim.x, v.gy = gridDim.y, v.gz = gridDim.z;
  return v;
}

// The item of this block: the last one whose first block is <= blockIdx.x
// (items are sorted by their first block; n >= 1).
__device__ __forceinline__ int multi_item(const MultiGrid* __restrict__ g, int n) {
  const long long b = blockIdx.x;
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (g[mid].start <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ VBlock multi_vblock(const MultiGrid& g) {
  const long long l = (long long)blockIdx.x - g.start;
  VBlock v;
  v.gx = g.gx, v.gy = g.gy, v.gz = g.gz;
  v.x = (unsigned)(l % g.gx);
  v.y = (unsigned)((l / g.gx) % g.gy);
  v.z = (unsigned)(l / ((long long)g.gx * g.gy));
  return v;
}

}  // namespace fmmgb
