// M2L on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The uniform grid makes every level's M2L (Sec. 2.3, eq. M2L, over the fixed
// interaction list of Sec. 2.2) the same translation-invariant contraction,
//   L[P][n] += sum_{d in 27 neighbours} sum_{k < K(n)} M[P + d][k] * W_d[k][n],
// with P a parent box, k = (alpha, source child) and n = (beta, target child).
// One CTA computes 128 parents (an 8x16x1 block) for one "pass" of output
// columns:
//   * A (M = 128 rows): the neighbour-shifted parent rows, one 128-byte chunk
//     of the reduction at a time, loaded by TMA from a 4-D tensor map as an
//     8x18x1 box whose one-row y halo serves the three dy neighbours; rows
//     past the domain are zero-filled by TMA, which is the isolated boundary.
//   * B: a weight tile per (neighbour, chunk, column group), stored
//     pre-swizzled (128-byte swizzle) so one bulk copy lands it ready for the
//     MMA.  Column groups are order-sorted so the truncation
//     |alpha|+|beta| <= p is a per-group prefix of the reduction: only the
//     chunks a group needs are multiplied.
//   * D: FP32 accumulators in tensor memory, one column range per group.
// Precisions: kind::tf32 on the FP32 rows (one product), or bf16 hi/lo planes
// with three products hi*hi + hi*lo + lo*hi (kind::f16, BF16 inputs).
// Roles (13 warps): lane 0 of warp 0 loads the activation boxes all issuers
// read; the accumulators of a pass are shared out between four MMA issuers
// (lane 0 of warps 5..8), which write disjoint tensor-memory columns; issuer
// q has its own weight ring, filled by its own producer (lane 0 of warp
// 1 + q).  A single issuing thread cannot keep the tensor pipe busy with the
// narrow low-order spans; four can.  The activation loads have a thread of
// their own so that a full weight ring never delays the next box.  The rings
// are byte-granular (1 KB units), so small spans do not hold a slot sized for
// the largest.  Warps 9..12 drain tensor memory (warp w reads TMEM lanes
// 32 (w mod 4) ..).
//
// Persistent tiles: a CTA takes row tiles blockIdx.x, blockIdx.x + gridDim.x,
// ... of pass blockIdx.y, so the rings keep streaming from one tile to the
// next; when two accumulator sets fit in tensor memory the epilogue of a tile
// overlaps the MMAs of the next (acc_full / acc_empty barriers per set).  Every wait is bounded:
// on time-out the kernel sets the plan's error flag (FMM_ERR_TIMEOUT) and
// unwinds; a CTA that sees the flag set by another gives up at once.
#include <cuda.h>

#include <algorithm>

#include "fmm_internal.h"
#include "tc_ptx.cuh"

namespace fmmgb {
namespace {

constexpr int kAPlane = kTcAPlaneBytes;                  // 144 rows x 128 B, a multiple of 1024
constexpr int kRingE = 16;                               // spans in flight per weight ring
constexpr int kEpiWarps = 4;                             // one per TMEM lane quarter
constexpr int kThreads = 32 * (1 + 2 * kTcIssuers + kEpiWarps);  // producers, issuers, epilogue
constexpr int kSmemBytes = kTcSmemUsable + 1024 /*alignment*/;
static_assert((2 * kTcMaxAStages + 2 * kTcIssuers * kRingE + 4) * 8 + 4 <= 2048, "barrier region");
static_assert(kSmemBytes <= 227 * 1024, "shared memory of the tensor-core kernel");
static_assert(kAPlane % 1024 == 0, "activation planes keep the 1 KB swizzle alignment");

// Issues the MMAs of one span: KS K steps of 32 bytes each (descriptor start
// address + 2 per step), three products per step for bf16x3.
template <int KIND, int KS>
__device__ __forceinline__ void issue_span(uint32_t d, uint64_t a, uint64_t a_lo, uint64_t b, uint64_t b_lo,
                                           uint32_t idesc, uint32_t acc0) {
#pragma unroll
  for (int k = 0; k < KS; ++k) {
    const uint64_t o = 2ull * k;
    if (KIND == TC_BF16X3) {
      mma_f16(d, a + o, b + o, idesc, k == 0 ? acc0 : 1u);
      mma_f16(d, a + o, b_lo + o, idesc, 1u);
      mma_f16(d, a_lo + o, b + o, idesc, 1u);
    } else {
      mma_tf32(d, a + o, b + o, idesc, k == 0 ? acc0 : 1u);
    }
  }
}

// One product per K step (a product-split span): A (hi or lo plane) x B.
template <int KS>
__device__ __forceinline__ void issue_span1(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc0) {
#pragma unroll
  for (int k = 0; k < KS; ++k) mma_f16(d, a + 2ull * k, b + 2ull * k, idesc, k == 0 ? acc0 : 1u);
}

// 72 registers a thread (13 warps: 29,952 of the SM's 65,536): the FP64
// levels' blocks running beside it keep the rest (512^3 bf16x3: their
// concurrent span 3.9 -> 3.0 ms, the step 8.59 -> 8.45 ms with the tree
// kernels' register bounds).
template <int KIND>
__global__ void __maxnreg__(72)
    m2l_tc_kernel(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
                  const __grid_constant__ TcLaunch P) {
  constexpr bool split = KIND == TC_BF16X3;
  constexpr int chunk_elems = split ? 64 : 32;
  constexpr uint32_t planes = split ? 2 : 1;
  constexpr int NQ = kTcIssuers;
  constexpr uint32_t kAStage = planes * kAPlane;
  const uint32_t nA = (uint32_t)P.a_stages;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* a_full = reinterpret_cast<uint64_t*>(base);  // barriers: first 2 KB
  unsigned char* a_ring = base + 2048;
  unsigned char* b_rings = a_ring + nA * kAStage;
  uint64_t* a_empty = a_full + kTcMaxAStages;
  uint64_t* b_full = a_empty + kTcMaxAStages;  // [NQ][kRingE]
  uint64_t* b_empty = b_full + NQ * kRingE;    // [NQ][kRingE]
  uint64_t* acc_full = b_empty + NQ * kRingE;  // [2]
  uint64_t* acc_empty = acc_full + 2;          // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);

  const TcPass& pass = P.pass[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntx = (P.grid[0] + kTcTileX - 1) / kTcTileX, nty = (P.grid[1] + kTcTileY - 1) / kTcTileY;
  const int ntiles = ntx * nty * ((P.grid[2] + kTcTileZ - 1) / kTcTileZ);
  const uint32_t nbuf = 2 * pass.tmem_cols <= 512 ? 2u : 1u;  // accumulator sets
  const int seg = pass.seg_xz >= 1 && pass.seg_xz <= 9 ? pass.seg_xz : 9;  // neighbour columns per segment

  {
    // one barrier per thread: a_full, a_empty (every issuer releases a
    // stage), the ring barriers, acc_full (every issuer commits) and
    // acc_empty (every epilogue warp releases)
    constexpr int kBars = 2 * kTcMaxAStages + 2 * NQ * kRingE + 4;
    static_assert(kBars <= kThreads, "barrier initialisation");
    const int i = threadIdx.x;
    if (i < kBars) {
      uint32_t count = 1;
      if (i >= kTcMaxAStages && i < 2 * kTcMaxAStages) count = NQ;      // a_empty
      if (i == kBars - 4 || i == kBars - 3) count = NQ;                 // acc_full
      if (i == kBars - 2 || i == kBars - 1) count = kEpiWarps;          // acc_empty
      mbar_init(a_full + i, count);  // the barriers are contiguous from a_full on
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  if (warp == 0) {
    __syncwarp();  // tcgen05.alloc is warp-collective: reconverge after thread 0's block
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)pass.tmem_cols * nbuf));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const unsigned char* wpass = P.W + pass.w_base;

  if (warp == 0 && lane == 0) {
    // ---------------- activation producer ----------------
    // One box per (tile, neighbour column (dx, dz), chunk j): rows y-1 .. y+16
    // of the shifted x/z column, which serve the three dy neighbours.
    uint32_t ai = 0;
    bool ok = !(*reinterpret_cast<volatile int*>(P.err) & 2);
    for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
      const int ox = (tile % ntx) * kTcTileX, oy = ((tile / ntx) % nty) * kTcTileY;
      const int oz = (tile / (ntx * nty)) * kTcTileZ;
      for (int xz = 0; ok && xz < 9; ++xz) {
        const int dx = xz % 3 - 1, dz = xz / 3 - 1;
        for (int j = 0; ok && j < pass.nchunks; ++j) {
          const uint32_t sa = ai % nA;
          if (!(ok = wait_fast(&a_empty[sa], ((ai / nA) & 1) ^ 1, P.err, W_PROD_A))) break;
          unsigned char* adst = a_ring + sa * kAStage;
          mbar_expect_tx(&a_full[sa], split ? 2 * kAPlane : kAPlane);
          tma_load_4d(adst, &map_hi, &a_full[sa], j * chunk_elems, ox + dx, oy - 1, oz + dz);
          if (split)
            tma_load_4d(adst + kAPlane, &map_lo, &a_full[sa], j * chunk_elems, ox + dx, oy - 1, oz + dz);
          ++ai;
        }
      }
    }
    if (!ok)  // drain: never leave the CTA with copies in flight
      for (uint32_t i = (ai > nA ? ai - nA : 0); i < ai; ++i)
        mbar_wait_drain(&a_full[i % nA], (i / nA) & 1);
  } else if (warp >= 1 && warp <= NQ && lane == 0) {
    // ---------------- weight producers ----------------
    // Ring q = warp - 1, in the order its issuer consumes: tile, neighbour
    // column (dx, dz), chunk j, then dy and the issuer's spans of the chunk.
    const int q = warp - 1;
    const uint32_t RB = (uint32_t)pass.ring_bytes[q];
    uint32_t rbase = 0;
    for (int t = 0; t < q; ++t) rbase += (uint32_t)pass.ring_bytes[t];
    unsigned char* ring = b_rings + rbase;
    uint64_t* full = b_full + q * kRingE;
    uint64_t* empty = b_empty + q * kRingE;
    // Byte ring in virtual positions: v = start of the next span, last =
    // end of the last span written, freed = end of the spans released so far.
    // A span that does not fit before the end of the ring starts at offset 0;
    // it may be written once the live data [freed, last) no longer overlaps
    // its physical range, i.e. freed >= min(last, v + bytes - RB).
    uint32_t end_v[kRingE];
    uint32_t e = 0, tail = 0, v = 0, off = 0, freed = 0, last = 0;
    bool ok = !(*reinterpret_cast<volatile int*>(P.err) & 2);
    for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
      for (int xz = 0; ok && xz < 9; ++xz) {
        const int dx = xz % 3 - 1, dz = xz / 3 - 1;
        for (int j = 0; ok && j < pass.nchunks; ++j) {
          const int s0 = pass.span_idx[j][q], s1 = pass.span_idx[j][q + 1];
          for (int dy = 0; ok && dy < 3; ++dy) {
            const unsigned char* wd = wpass + (long long)((dx + 1) + 3 * dy + 9 * (dz + 1)) * pass.bytes_per_d;
            for (int si = s0; si < s1; ++si) {
              const uint32_t bytes = (uint32_t)pass.span[si].n * 128u * (pass.span[si].prod ? 1u : planes);
              if (off + bytes > RB) v += RB - off, off = 0;  // a span never wraps
              const uint32_t need = v + bytes > RB ? min(last, v + bytes - RB) : 0u;
              while (freed < need || e - tail >= (uint32_t)kRingE) {  // release the oldest span
                if (!(ok = wait_fast(&empty[tail % kRingE], (tail / kRingE) & 1, P.err, W_PROD_B))) break;
                freed = end_v[tail % kRingE];
                ++tail;
              }
              if (!ok) break;
              mbar_expect_tx(&full[e % kRingE], bytes);
              bulk_load(ring + off, wd + pass.span[si].w_off, bytes, &full[e % kRingE]);
              end_v[e % kRingE] = v + bytes;
              v += bytes;
              last = v;
              off += bytes;
              ++e;
            }
          }
        }
      }
    }
    if (!ok)  // drain: never leave the CTA with copies in flight
      for (uint32_t i = tail; i < e; ++i) mbar_wait_drain(&full[i % kRingE], (i / kRingE) & 1);
  } else if (warp > NQ && warp <= 2 * NQ && lane == 0) {
    // ---------------- MMA issuers ----------------
    const int q = warp - 1 - NQ;
    const uint32_t RB = (uint32_t)pass.ring_bytes[q];
    uint32_t rbase = 0;
    for (int t = 0; t < q; ++t) rbase += (uint32_t)pass.ring_bytes[t];
    const uint64_t ring_desc = sw128_desc(smem_u32(b_rings + rbase));
    uint64_t* full = b_full + q * kRingE;
    uint64_t* empty = b_empty + q * kRingE;
    uint32_t ai = 0, e = 0, off = 0, it = 0;
    bool ok = !(*reinterpret_cast<volatile int*>(P.err) & 2);
    // one accumulation segment (seg neighbour columns of a tile) per accumulator set
    for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x)
     for (int xz0 = 0; ok && xz0 < 9; xz0 += seg, ++it) {
      const uint32_t buf = it % nbuf, use = it / nbuf;
      // this accumulator set must have been drained by the epilogue
      if (!(ok = wait_fast(&acc_empty[buf], (use & 1) ^ 1, P.err, W_MMA_ACC))) break;
      tc_fence_after();
      const uint32_t tbase = tmem + buf * (uint32_t)pass.tmem_cols;
      for (int xz = xz0; ok && xz < xz0 + seg && xz < 9; ++xz) {
        for (int j = 0; ok && j < pass.nchunks; ++j) {
          const uint32_t sa = ai % nA;
          if (!(ok = wait_fast(&a_full[sa], (ai / nA) & 1, P.err, W_MMA_A))) break;
          tc_fence_after();
          const uint64_t a_desc = sw128_desc(smem_u32(a_ring + sa * kAStage));
          const int s0 = pass.span_idx[j][q], s1 = pass.span_idx[j][q + 1];
          for (int dy = 0; ok && dy < 3; ++dy) {
            const uint64_t a = a_desc + (uint64_t)(dy * (kTcTileX * 128 / 16));  // 128-row window
            const uint64_t a_lo = a + (uint64_t)(kAPlane / 16);
            for (int si = s0; si < s1; ++si) {
              const TcSpan& S = pass.span[si];
              const uint32_t plane = (uint32_t)S.n * 128u;
              const uint32_t bytes = plane * (S.prod ? 1u : planes);
              if (off + bytes > RB) off = 0;
              if (!(ok = wait_fast(&full[e % kRingE], (e / kRingE) & 1, P.err, W_MMA_B))) break;
              tc_fence_after();
              const uint64_t b = ring_desc + (uint64_t)(off >> 4);
              const uint64_t b_lo = b + (uint64_t)(plane >> 4);
              const uint32_t d = tbase + (uint32_t)S.tmem_col;
              const uint32_t acc0 = (xz == xz0 && dy == 0 && j == S.first) ? 0u : 1u;  // the first step opens
              if (KIND == TC_BF16X3 && S.prod) {
                const uint64_t as = S.prod == 3 ? a_lo : a;
                switch (S.ksteps) {
                  case 1: issue_span1<1>(d, as, b, S.idesc, acc0); break;
                  case 2: issue_span1<2>(d, as, b, S.idesc, acc0); break;
                  case 3: issue_span1<3>(d, as, b, S.idesc, acc0); break;
                  default: issue_span1<4>(d, as, b, S.idesc, acc0); break;
                }
              } else {
                switch (S.ksteps) {
                  case 1: issue_span<KIND, 1>(d, a, a_lo, b, b_lo, S.idesc, acc0); break;
                  case 2: issue_span<KIND, 2>(d, a, a_lo, b, b_lo, S.idesc, acc0); break;
                  case 3: issue_span<KIND, 3>(d, a, a_lo, b, b_lo, S.idesc, acc0); break;
                  default: issue_span<KIND, 4>(d, a, a_lo, b, b_lo, S.idesc, acc0); break;
                }
              }
              mma_commit(&empty[e % kRingE]);
              off += bytes;
              ++e;
            }
          }
          mma_commit(&a_empty[sa]);
          ++ai;
        }
      }
      mma_commit(&acc_full[buf]);  // fires when every MMA of this segment has completed
    }
  } else if (warp > 2 * NQ) {
    // ---------------- epilogue: TMEM -> registers -> C ----------------
    const int wq = warp & 3;
    const int r = wq * 32 + lane;  // tile row = TMEM lane
    const uint32_t lane_base = (uint32_t)(wq * 32) << 16;
    uint32_t it = 0;
    bool live = true;
    for (int tile = blockIdx.x; live && tile < ntiles; tile += gridDim.x)
     for (int xz0 = 0; live && xz0 < 9; xz0 += seg, ++it) {
      const uint32_t buf = it % nbuf, use = it / nbuf;
      int done = 0;
      if (lane == 0) done = mbar_wait(&acc_full[buf], use & 1, P.err, W_EPI) ? 1 : 0;
      done = __shfl_sync(0xffffffffu, done, 0);  // warp-uniform: tcgen05.ld is warp-collective
      if (!done) {
        live = false;
        break;
      }
      tc_fence_after();
      const int ox = (tile % ntx) * kTcTileX, oy = ((tile / ntx) % nty) * kTcTileY;
      const int oz = (tile / (ntx * nty)) * kTcTileZ;
      const int x = ox + (r & 7), y = oy + (r >> 3), z = oz;
      const bool valid = x < P.grid[0] && y < P.grid[1] && z < P.grid[2];
      // later segments add to what this thread stored for the earlier ones
      const bool add = P.accumulate || xz0 > 0;
      float* crow = P.C + ((((long long)z * P.grid[1] + y) * P.grid[0] + x) * P.n_cols);
      const uint32_t tbase = tmem + buf * (uint32_t)pass.tmem_cols;
      for (int g = 0; g < pass.ng; ++g) {
        const int n_mma = pass.out_nmma[g], ncols = pass.out_ncols[g], col0 = pass.out_col0[g];
        const int t2 = pass.out_tmem2[g], t3 = pass.out_tmem3[g], t4 = pass.out_tmem4[g];
        for (int c = 0; c < n_mma; c += 16) {
          float vv[16];
          __syncwarp();  // tcgen05.ld is warp-collective: reconverge after the masked stores
          tmem_ld16(tbase + lane_base + (uint32_t)(pass.out_tmem[g] + c), vv);
          if (t2 >= 0) {  // split group: accumulators added in a fixed order
            float w2[16];
            tmem_ld16(tbase + lane_base + (uint32_t)(t2 + c), w2);
#pragma unroll
            for (int i = 0; i < 16; ++i) vv[i] += w2[i];
          }
          if (t3 >= 0) {
            float w3[16];
            tmem_ld16(tbase + lane_base + (uint32_t)(t3 + c), w3);
#pragma unroll
            for (int i = 0; i < 16; ++i) vv[i] += w3[i];
          }
          if (t4 >= 0) {
            float w4[16];
            tmem_ld16(tbase + lane_base + (uint32_t)(t4 + c), w4);
#pragma unroll
            for (int i = 0; i < 16; ++i) vv[i] += w4[i];
          }
          if (valid) {  // out_col0 and out_ncols are multiples of 8: whole float4s
#pragma unroll
            for (int jj = 0; jj < 16; jj += 4)
              if (c + jj < ncols) {
                int col = col0 + c + jj;
                if (P.col_mapped) col = (int)P.col_map[col >> 3] * 8 + (col & 7);
                float4* o = reinterpret_cast<float4*>(crow + col);
                float4 q4 = make_float4(vv[jj], vv[jj + 1], vv[jj + 2], vv[jj + 3]);
                if (add) {
                  const float4 old = *o;
                  q4.x += old.x, q4.y += old.y, q4.z += old.z, q4.w += old.w;
                }
                *o = q4;
              }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);  // this warp's reads of the set are done
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)pass.tmem_cols * nbuf));
  }
}

}  // namespace

cudaError_t make_row_map(void* map_out, const void* base, int row_len, int elem_bytes, const int grid[3],
                         int box_inner) {
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<EncodeFn>(fn);
  }
  const cuuint64_t dims[4] = {(cuuint64_t)row_len, (cuuint64_t)grid[0], (cuuint64_t)grid[1], (cuuint64_t)grid[2]};
  const cuuint64_t row_bytes = (cuuint64_t)row_len * elem_bytes;
  const cuuint64_t strides[3] = {row_bytes, row_bytes * grid[0], row_bytes * grid[0] * grid[1]};
  const cuuint32_t box[4] = {(cuuint32_t)box_inner, kTcTileX, kTcBoxY, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = encode(reinterpret_cast<CUtensorMap*>(map_out),
                      elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                      const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_m2l_tc(const TcLaunch& L, const void* map_hi, const void* map_lo, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(m2l_tc_kernel<TC_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemBytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(m2l_tc_kernel<TC_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int ntx = (L.grid[0] + kTcTileX - 1) / kTcTileX, nty = (L.grid[1] + kTcTileY - 1) / kTcTileY,
            ntz = (L.grid[2] + kTcTileZ - 1) / kTcTileZ;
  const int tiles = ntx * nty * ntz;
  // single-pass launches run persistent CTAs (one per SM, shared memory allows
  // no more); with several passes each CTA takes one tile, so that the light
  // passes do not leave SMs idle while the heavy pass finishes
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 148;
  const int ctas = L.npass == 1 ? std::min(tiles, sms) : tiles;
  dim3 grid((unsigned)ctas, (unsigned)L.npass);
  if (L.kind == TC_BF16X3)
    m2l_tc_kernel<TC_BF16X3><<<grid, kThreads, kSmemBytes, s>>>(*reinterpret_cast<const CUtensorMap*>(map_hi),
                                                           *reinterpret_cast<const CUtensorMap*>(map_lo), L);
  else
    m2l_tc_kernel<TC_TF32><<<grid, kThreads, kSmemBytes, s>>>(*reinterpret_cast<const CUtensorMap*>(map_hi),
                                                         *reinterpret_cast<const CUtensorMap*>(map_lo), L);
  return cudaGetLastError();
}


}  // namespace fmmgb
