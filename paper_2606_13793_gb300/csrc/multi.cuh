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

// The item of launch block b: the last one whose first block is <= b (items
// are sorted by their first block; n >= 1).  Host callable for the checks of
// the batch's tables.
__host__ __device__ __forceinline__ int multi_item_at(const MultiGrid* __restrict__ g, int n, long long b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (g[mid].start <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Block b of the launch as a block of item g's own grid.
__host__ __device__ __forceinline__ VBlock multi_vblock_at(const MultiGrid& g, long long b) {
  const long long l = b - g.start;
  VBlock v;
  v.gx = g.gx, v.gy = g.gy, v.gz = g.gz;
  v.x = (unsigned)(l % g.gx);
  v.y = (unsigned)((l / g.gx) % g.gy);
  v.z = (unsigned)(l / ((long long)g.gx * g.gy));
  return v;
}

__device__ __forceinline__ int multi_item(const MultiGrid* __restrict__ g, int n) {
  return multi_item_at(g, n, (long long)blockIdx.x);
}

__device__ __forceinline__ VBlock multi_vblock(const MultiGrid& g) { return multi_vblock_at(g, (long long)blockIdx.x); }

}  // namespace fmmgb
