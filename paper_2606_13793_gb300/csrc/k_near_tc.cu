// Near field of leaf-4 boxes on the 5th-generation tensor cores (tcgen05,
// sm_103a), bf16x3.
//
// The near field (Sec. 2.3, eq. direct) over the 27 neighbour leaf boxes is
// the contraction
//   C[P][t] = sum_{d in 27 neighbours} sum_{s < 64} rho[P + d][s] * W_d[s][t],
// P a leaf box, s / t its 4^3 source / target cells, W_d[s][t] = g(x_t - x_s)
// for the source box at offset d (g = -1/r, g(0) = -1/dx in cell units).
// Every box has the same 27 x 64 x 64 weights (442 KB as bf16 hi + lo), too
// many for shared memory, so they stream from L2.  The general tensor-core
// schedules stream them per row tile in many small pieces, and measurement
// showed the near field bound by those copies' round trips rather than by
// bytes or MMAs.  This kernel moves fewer, larger copies:
//
//   * a work item is 4 row tiles of 128 boxes (8 x 16 x 1 each);
//   * for each of the 9 neighbour columns (dx, dz), one 48 KB bulk copy brings
//     the weights of its three dy neighbours, which serve all 4 tiles;
//   * per (tile, column) one TMA box of 8 x 18 x 1 rows (hi and lo planes,
//     128-byte swizzle) whose one-row y halo serves the three dy neighbours
//     through the descriptor start address; rows past the domain are
//     zero-filled by TMA, which is the isolated boundary.
//
// Products: hi*lo and lo*hi first, then hi*hi (12 + 12 + 12 MMAs of
// M = 128, N = 64, K = 16 per tile and column), into one accumulator per tile.
// The tensor cores add into FP32 accumulators by truncation, which on these
// same-signed sums biases each MMA's addition by up to an ulp; so every
// neighbour column is a segment of its own: the accumulators of the 4 tiles
// (256 TMEM columns) are drained after each column into registers of the
// epilogue warps, which add the 9 segments in order with rounding to nearest,
// while the MMAs of the next column fill the other 256 columns.  The small
// correction products go first, while the accumulator is small.
//
// Roles (20 warps): warp 0 lane 0 loads the activation boxes, warp 1 lane 0
// the weight groups, warps 2 and 3 (lane 0) issue the MMAs of tiles 0-1 and
// 2-3, warps 4..19 drain tensor memory (warp w: tile (w - 4) / 4, TMEM lanes
// 32 (w mod 4) ..).  A CTA per SM walks items blockIdx.x, + gridDim.x, ...
//
// Every wait is bounded (2 s): on time-out the CTA records FMM_ERR_TIMEOUT
// and the wait site in the plan's flag, lets its copies and MMAs land, frees
// tensor memory and exits; a CTA that sees the flag set by another gives up.
#include <cuda.h>

#include "fmm_internal.h"
#include "tc_ptx.cuh"

namespace fmmgb {
namespace {

constexpr int kNtTiles = 4;                     // row tiles per work item
constexpr int kNtEpiWarps = 4 * kNtTiles;       // one per (tile, TMEM lane quarter)
constexpr int kNtWarps = 4 + kNtEpiWarps;       // A producer, W producer, 2 issuers, epilogue
constexpr int kNtThreads = 32 * kNtWarps;       // 640
constexpr int kNtAPlane = kTcAPlaneBytes;       // 8 x 18 rows x 128 B
constexpr int kNtAStage = 2 * kNtAPlane;        // hi + lo planes
constexpr int kNtAStages = 3;
constexpr int kNtPlane = 64 * 128;              // 64 target-cell rows of 128 B (64 bf16 source cells)
constexpr int kNtWGroup = 3 * kNtPieceBytes;    // the three dy neighbours of a column
constexpr int kNtCols = 64;                     // accumulator columns per tile
constexpr int kNtSetCols = kNtTiles * kNtCols;  // 256: two sets fill the 512 TMEM columns
constexpr int kNtSmem = 1024 /*barriers*/ + kNtAStages * kNtAStage + 2 * kNtWGroup + 1024 /*alignment*/;
static_assert(kNtPieceBytes == 2 * kNtPlane, "weight piece: hi plane then lo plane");
static_assert(kNtSmem <= 227 * 1024, "shared memory of the near-field kernel");
static_assert(kNtAPlane % 1024 == 0 && kNtPlane % 1024 == 0, "operands keep the 1 KB swizzle alignment");

__device__ __forceinline__ void tile_origin(int tile, int ntx, int nty, int& ox, int& oy, int& oz) {
  ox = (tile % ntx) * kTcTileX;
  oy = ((tile / ntx) % nty) * kTcTileY;
  oz = (tile / (ntx * nty)) * kTcTileZ;
}

__global__ void __launch_bounds__(kNtThreads, 1)
    near_tc_kernel(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
                   const __grid_constant__ NearTcLaunch P) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base);  // first 1 KB
  uint64_t* a_full = bars;                             // [3]
  uint64_t* a_empty = bars + kNtAStages;               // [3]
  uint64_t* w_full = bars + 2 * kNtAStages;            // [2]
  uint64_t* w_empty = w_full + 2;                      // [2]
  uint64_t* acc_full = w_empty + 2;                    // [2]
  uint64_t* acc_empty = acc_full + 2;                  // [2]
  uint64_t* fin = acc_empty + 2;                       // [2] one per issuer
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 2);
  unsigned char* a_ring = base + 1024;
  unsigned char* w_ring = a_ring + kNtAStages * kNtAStage;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntx = (P.grid[0] + kTcTileX - 1) / kTcTileX, nty = (P.grid[1] + kTcTileY - 1) / kTcTileY;
  const int ntiles = ntx * nty * ((P.grid[2] + kTcTileZ - 1) / kTcTileZ);
  const int nitems = (ntiles + kNtTiles - 1) / kNtTiles;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kNtAStages; ++i) {
      mbar_init(&a_full[i], 1);
      mbar_init(&a_empty[i], 1);  // the issuer of the box's tile
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&w_full[i], 1);
      mbar_init(&w_empty[i], 2);  // both issuers
      mbar_init(&acc_full[i], 2);
      mbar_init(&acc_empty[i], kNtEpiWarps);
      mbar_init(&fin[i], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    __syncwarp();  // tcgen05.alloc is warp-collective: reconverge after thread 0's block
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2u * kNtSetCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- activation boxes: (item, column, tile) order ----------------
    uint32_t ai = 0;
    bool ok = !(*reinterpret_cast<volatile int*>(P.err) & 2);
    for (int item = blockIdx.x; ok && item < nitems; item += gridDim.x)
      for (int g = 0; ok && g < 9; ++g) {
        const int dx = g % 3 - 1, dz = g / 3 - 1;
        for (int t = 0; ok && t < kNtTiles; ++t) {
          const int tile = item * kNtTiles + t;
          if (tile >= ntiles) break;
          int ox, oy, oz;
          tile_origin(tile, ntx, nty, ox, oy, oz);
          const uint32_t sa = ai % kNtAStages;
          if (!(ok = wait_fast(&a_empty[sa], ((ai / kNtAStages) & 1) ^ 1, P.err, W_PROD_A))) break;
          unsigned char* dst = a_ring + sa * kNtAStage;
          mbar_expect_tx(&a_full[sa], kNtAStage);
          tma_load_4d(dst, &map_hi, &a_full[sa], 0, ox + dx, oy - 1, oz + dz);
          tma_load_4d(dst + kNtAPlane, &map_lo, &a_full[sa], 0, ox + dx, oy - 1, oz + dz);
          ++ai;
        }
      }
    if (!ok)  // drain: never leave the CTA with copies in flight
      for (uint32_t i = (ai > kNtAStages ? ai - kNtAStages : 0); i < ai; ++i)
        mbar_wait_drain(&a_full[i % kNtAStages], (i / kNtAStages) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---------------- weight groups: (item, column) order ----------------
    uint32_t gi = 0;
    bool ok = !(*reinterpret_cast<volatile int*>(P.err) & 2);
    for (int item = blockIdx.x; ok && item < nitems; item += gridDim.x)
      for (int g = 0; ok && g < 9; ++g, ++gi) {
        const int dx = g % 3 - 1, dz = g / 3 - 1;
        const uint32_t wb = gi & 1;
        if (!(ok = wait_fast(&w_empty[wb], ((gi >> 1) & 1) ^ 1, P.err, W_PROD_B))) break;
        mbar_expect_tx(&w_full[wb], kNtWGroup);
        for (int dy = 0; dy < 3; ++dy) {
          const int d = (dx + 1) + 3 * dy + 9 * (dz + 1);
          bulk_load(w_ring + wb * kNtWGroup + dy * kNtPieceBytes, P.W + (size_t)d * kNtPieceBytes, kNtPieceBytes,
                    &w_full[wb]);
        }
      }
    if (!ok)
      for (uint32_t i = (gi > 2 ? gi - 2 : 0); i < gi; ++i) mbar_wait_drain(&w_full[i & 1], (i >> 1) & 1);
  } else if ((warp == 2 || warp == 3) && lane == 0) {
    // ---------------- MMA issuers: tiles 2q, 2q + 1 of every item ----------------
    const int q = warp - 2;
    const uint64_t a_desc0 = sw128_desc(smem_u32(a_ring));
    const uint64_t w_desc0 = sw128_desc(smem_u32(w_ring));
    uint32_t ai = 0, gi = 0;
    bool ok = !(*reinterpret_cast<volatile int*>(P.err) & 2);
    for (int item = blockIdx.x; ok && item < nitems; item += gridDim.x)
      for (int g = 0; ok && g < 9; ++g, ++gi) {
        const uint32_t set = gi & 1, use = gi >> 1;
        // the set's previous segment has been drained by every epilogue warp
        if (!(ok = wait_fast(&acc_empty[set], (use & 1) ^ 1, P.err, W_MMA_ACC))) break;
        const uint32_t wb = gi & 1;
        if (!(ok = wait_fast(&w_full[wb], (gi >> 1) & 1, P.err, W_MMA_B))) break;
        tc_fence_after();
        const uint64_t wg = w_desc0 + (uint64_t)((wb * kNtWGroup) >> 4);
        for (int t = 0; ok && t < kNtTiles; ++t) {
          if (item * kNtTiles + t >= ntiles) break;
          if ((t >> 1) == q) {
            const uint32_t sa = ai % kNtAStages;
            if (!(ok = wait_fast(&a_full[sa], (ai / kNtAStages) & 1, P.err, W_MMA_A))) break;
            tc_fence_after();
            const uint64_t a_hi = a_desc0 + (uint64_t)((sa * kNtAStage) >> 4);
            const uint64_t a_lo = a_hi + (uint64_t)(kNtAPlane >> 4);
            const uint32_t d = tmem + set * kNtSetCols + (uint32_t)(t * kNtCols);
            uint32_t acc = 0;  // the first MMA of the segment overwrites the accumulator
            // corrections hi*lo and lo*hi, then hi*hi; dy = window of rows 8 dy ..
#pragma unroll
            for (int pr = 0; pr < 3; ++pr)
#pragma unroll
              for (int dy = 0; dy < 3; ++dy) {
                const uint64_t aw = (pr == 1 ? a_lo : a_hi) + (uint64_t)(dy * (kTcTileX * 128 / 16));
                const uint64_t bw = wg + (uint64_t)((dy * kNtPieceBytes + (pr == 0 ? kNtPlane : 0)) >> 4);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                  mma_f16(d, aw + 2ull * k, bw + 2ull * k, P.idesc, acc);
                  acc = 1u;
                }
              }
            mma_commit(&a_empty[sa]);  // the box is free once these MMAs have read it
          }
          ++ai;
        }
        if (!ok) break;
        mma_commit(&w_empty[wb]);
        mma_commit(&acc_full[set]);  // fires when this issuer's MMAs of the segment have completed
      }
    mma_commit(&fin[q]);
    mbar_wait_drain(&fin[q], 0);  // every MMA of this issuer has landed before tensor memory is freed
  } else if (warp >= 4) {
    // ---------------- epilogue: 9 segments per item, added in order ----------------
    const int t = (warp - 4) >> 2, wq = warp & 3;
    const int r = wq * 32 + lane;  // tile row = TMEM lane
    const uint32_t lane_base = (uint32_t)(wq * 32) << 16;
    uint32_t gi = 0;
    bool live = true;
    for (int item = blockIdx.x; live && item < nitems; item += gridDim.x) {
      const int tile = item * kNtTiles + t;
      const bool has = tile < ntiles;  // warp-uniform
      float acc[kNtCols];
#pragma unroll
      for (int c = 0; c < kNtCols; ++c) acc[c] = 0.f;
      for (int g = 0; g < 9; ++g, ++gi) {
        const uint32_t set = gi & 1, use = gi >> 1;
        int done = 0;
        if (lane == 0) done = mbar_wait(&acc_full[set], use & 1, P.err, W_EPI) ? 1 : 0;
        done = __shfl_sync(0xffffffffu, done, 0);
        if (!done) {
          live = false;
          break;
        }
        tc_fence_after();
        if (has) {
          const uint32_t tb = tmem + lane_base + set * kNtSetCols + (uint32_t)(t * kNtCols);
#pragma unroll
          for (int c = 0; c < kNtCols; c += 16) {
            float v[16];
            tmem_ld16(tb + (uint32_t)c, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[c + i] += v[i];
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[set]);
      }
      if (!live || !has) continue;
      int ox, oy, oz;
      tile_origin(tile, ntx, nty, ox, oy, oz);
      const int x = ox + (r & 7), y = oy + (r >> 3), z = oz;
      if (x < P.grid[0] && y < P.grid[1] && z < P.grid[2]) {
        float4* o = reinterpret_cast<float4*>(P.C + (((long long)z * P.grid[1] + y) * P.grid[0] + x) * kNtCols);
#pragma unroll
        for (int c = 0; c < kNtCols; c += 4) o[c >> 2] = make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2u * kNtSetCols));
  }
}

}  // namespace

cudaError_t launch_near_tc4(const NearTcLaunch& L, const void* map_hi, const void* map_lo, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(near_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kNtSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int ntx = (L.grid[0] + kTcTileX - 1) / kTcTileX, nty = (L.grid[1] + kTcTileY - 1) / kTcTileY,
            ntz = (L.grid[2] + kTcTileZ - 1) / kTcTileZ;
  const long long items = ((long long)ntx * nty * ntz + kNtTiles - 1) / kNtTiles;
  if (items <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 148;
  const unsigned ctas = (unsigned)std::min<long long>(items, sms);  // persistent: one CTA per SM
  near_tc_kernel<<<ctas, kNtThreads, kNtSmem, s>>>(*reinterpret_cast<const CUtensorMap*>(map_hi),
                                                  *reinterpret_cast<const CUtensorMap*>(map_lo), L);
  return cudaGetLastError();
}

}  // namespace fmmgb
