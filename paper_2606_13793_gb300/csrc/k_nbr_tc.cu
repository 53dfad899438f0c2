// Neighbour contraction on the 5th-generation tensor cores, prefix schedule
// (tcgen05, sm_103a).
//
// The M2L of a level (Sec. 2.3, eq. M2L, over the interaction list of Sec.
// 2.2), the paper's final-stage M2P (Sec. 4) and the near field (Sec. 2.3,
// eq. direct) are the same translation-invariant contraction over a 3-D grid
// of rows,
//   C[P][n] (+)= sum_{d in 27 neighbours} sum_{k < K(n)} A[P + d][k] W_d[k][n],
// with K(n) non-increasing in n (the order truncation |alpha| + |beta| <= p
// when the columns run over orders from 0 up).  Every K step of 16 bf16 (or 8
// TF32) reduction values is therefore needed by a prefix [0, N_s) of the
// columns.  A tile of 128 rows (an 8 x 16 x 1 block) keeps all the columns
// of its pass in one set of tensor-memory accumulators and multiplies each
// K step with one MMA per product over that whole prefix (N <= 256 per
// instruction): few, wide MMAs.  An MMA costs the tensor pipe at least ~40
// cycles whatever its N, and a thread issues one every ~55 cycles at best, so
// narrow per-order MMAs left the pipe idle.
//
// Operands.  A: the neighbour-shifted rows, one 128-byte chunk of the
// reduction at a time, loaded by TMA as an 8 x 18 x 1 box (128-byte swizzle)
// whose one-row y halo serves the three dy neighbours; rows past the domain
// are zero-filled by TMA, which is the isolated boundary.  B: per K step the
// pre-swizzled weight blocks (32-byte rows, 32-byte swizzle) of the plan,
// streamed in pieces of up to 16 KB in the order the MMAs read them.
//
// Accumulators (per set): E (reversed hi*lo of the "fused" narrow K steps),
// D (every column) and L2 (the late K steps), summed by the epilogue in that
// fixed order; see TpPass.  Every set is zeroed by the epilogue after it is
// drained, so every MMA accumulates.
//
// Roles (13 warps):
//   warp 0, lanes 0..3  activation boxes (a lane per plane and slot group:
//                       TMA copies issued by one thread complete in order,
//                       ~0.9 us each, so the copies are spread over threads);
//   warps 1..4          weight pieces, one warp per issuer ("owner"), each
//                       into a ring of 16 KB slots of its own;
//   warps 5..8, lane 0  MMA issuers: each owns a set of accumulator columns
//                       and reads only the weight pieces of its columns, so
//                       every column sums its products in one fixed order;
//   warps 9..12         epilogue: tensor memory -> registers -> C, then zero.
// Work items are (pass, row tile) pairs, pass-major; a CTA per SM walks items
// blockIdx.x, blockIdx.x + gridDim.x, ...  Two accumulator sets, when they
// fit in the 512 columns, let a tile's epilogue overlap the next tile's MMAs.
//
// Every wait is bounded (2 s): on time-out the CTA records FMM_ERR_TIMEOUT
// and the wait site in the plan's flag, lets its copies and MMAs land, frees
// tensor memory and exits; a CTA that sees the flag set by another gives up.
#include <cuda.h>

#include <algorithm>

#include "fmm_internal.h"
#include "tc_ptx.cuh"

namespace fmmgb {
namespace {

constexpr int kAPlane = kTcAPlaneBytes;  // 144 rows x 128 B
constexpr int kEpiWarps = 4;
constexpr int kWarpA = 0, kWarpW0 = 1, kWarpI0 = 1 + kTpIssuers, kWarpE0 = 1 + 2 * kTpIssuers;
constexpr int kThreads = 32 * (kWarpE0 + kEpiWarps);
constexpr int kSmemBytes = kTcSmemUsable + 1024 /*alignment*/;
constexpr int kBars = 2 * kTpMaxAStages + 2 * kTpMaxSlots + 4 + kTpIssuers;
static_assert(kBars * 8 + 8 <= 2048, "barrier region");
static_assert(kBars <= kThreads, "barrier initialisation");
static_assert(kSmemBytes <= 227 * 1024, "shared memory of the tensor-core kernel");
static_assert(kAPlane % 1024 == 0, "activation planes keep the 1 KB swizzle alignment");
static_assert(kTpWLanes <= 32 && kTpALanes <= 32, "producer lanes");
static_assert(kThreads == 32 * 13, "warp roles");

// Work item -> (pass, tile origin) of the 8 x 16 x 1 row tiles.
struct Tile {
  int pass, ox, oy, oz;
};
__device__ __forceinline__ Tile item_tile(int item, int ntiles, int ntx, int nty) {
  Tile t;
  t.pass = item / ntiles;
  const int tile = item - t.pass * ntiles;
  t.ox = (tile % ntx) * kTcTileX;
  t.oy = ((tile / ntx) % nty) * kTcTileY;
  t.oz = tile / (ntx * nty);
  return t;
}

// Accumulator set of each work item: passes with two sets alternate them.
struct AccSeq {
  uint32_t uses[2] = {0, 0};
  uint32_t flip = 0;
  __device__ __forceinline__ void next(int nbuf, uint32_t& buf, uint32_t& phase) {
    buf = nbuf == 2 ? (flip++ & 1u) : 0u;
    phase = uses[buf]++ & 1u;
  }
};

template <int KIND>
__global__ void __maxnreg__(96)
    nbr_tc_kernel(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
                  const __grid_constant__ TpLaunch P) {
  constexpr bool split = KIND == TC_BF16X3;
  constexpr int planes = split ? 2 : 1;
  constexpr int chunk_elems = split ? 64 : 32;
  constexpr uint32_t kAStage = planes * kAPlane;
  constexpr int Q = kTpIssuers;
  const uint32_t nA = (uint32_t)P.a_stages;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* a_full = reinterpret_cast<uint64_t*>(base);  // barriers: first 2 KB
  uint64_t* a_empty = a_full + kTpMaxAStages;
  uint64_t* w_full = a_empty + kTpMaxAStages;
  uint64_t* w_empty = w_full + kTpMaxSlots;
  uint64_t* acc_full = w_empty + kTpMaxSlots;  // [2]
  uint64_t* acc_empty = acc_full + 2;          // [2]
  uint64_t* fin = acc_empty + 2;               // [Q]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + Q);
  unsigned char* a_ring = base + 2048;
  unsigned char* w_ring = a_ring + nA * kAStage;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntx = (P.grid[0] + kTcTileX - 1) / kTcTileX, nty = (P.grid[1] + kTcTileY - 1) / kTcTileY;
  const int ntiles = ntx * nty * P.grid[2];
  const int nitems = ntiles * P.npass;
  uint32_t tmem_need = 32;
  for (int ps = 0; ps < P.npass; ++ps) {
    const uint32_t c = (uint32_t)(P.pass[ps].tmem_cols * P.pass[ps].nbuf);
    while (tmem_need < c) tmem_need *= 2;
  }

  {
    const int i = threadIdx.x;
    if (i < kBars) {
      uint32_t count = 1;
      if (i < kTpMaxAStages) count = planes;                                               // a_full
      else if (i < 2 * kTpMaxAStages) count = Q;                                           // a_empty
      else if (i >= 2 * kTpMaxAStages + 2 * kTpMaxSlots && i < 2 * kTpMaxAStages + 2 * kTpMaxSlots + 2)
        count = Q;                                                                         // acc_full
      else if (i >= 2 * kTpMaxAStages + 2 * kTpMaxSlots + 2 && i < 2 * kTpMaxAStages + 2 * kTpMaxSlots + 4)
        count = kEpiWarps;                                                                 // acc_empty
      mbar_init(a_full + i, count);  // the barriers are contiguous from a_full on
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  if (warp == 0) {
    __syncwarp();  // tcgen05.alloc is warp-collective
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tmem_need));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == kWarpA) {
    // ---------------- activation producer ----------------
    // Stage t (tile, neighbour column (dx, dz), chunk j): an 8 x 18 box per
    // plane, rows y-1 .. y+16 of the shifted column, serving the three dy.
    // Every slot has its own lanes (one per plane: lane l serves the slots s
    // with s mod G = l / planes), which fill it in sequence order: a parity
    // wait is only meaningful one phase ahead, so two lanes must never take
    // turns on one slot.
    constexpr int G = kTpALanes / planes;
    const int my_g = lane / planes, my_plane = lane % planes;
    const bool active = lane < kTpALanes;
    bool ok = !(*reinterpret_cast<volatile int*>(P.err) & 2);
    uint32_t t = 0, done = 0;  // done: 1 + the last stage this lane issued
    for (int item = blockIdx.x; ok && item < nitems; item += gridDim.x) {
      const Tile T = item_tile(item, ntiles, ntx, nty);
      const int nch = P.pass[T.pass].nchunks;
      for (int xz = 0; ok && xz < 9; ++xz) {
        const int dx = xz % 3 - 1, dz = xz / 3 - 1;
        for (int j = 0; ok && j < nch; ++j, ++t) {
          const uint32_t sa = t % nA;
          if (!active || (int)(sa % G) != my_g) continue;
          if (P.skip_first_a && t == 0) continue;  // test hook: nothing is copied, nothing waits on a copy
          if (!(ok = wait_fast(&a_empty[sa], ((t / nA) & 1) ^ 1, P.err, W_PROD_A))) break;
          unsigned char* dst = a_ring + sa * kAStage + my_plane * kAPlane;
          mbar_expect_tx(&a_full[sa], kAPlane);
          tma_load_4d(dst, my_plane ? static_cast<const void*>(&map_lo) : static_cast<const void*>(&map_hi),
                      &a_full[sa], j * chunk_elems, T.ox + dx, T.oy - 1, T.oz + dz);
          done = t + 1;
        }
      }
    }
    if (!ok && active)  // let this lane's copies land before the CTA exits
      for (uint32_t i = (done > nA ? done - nA : 0); i < done; ++i)
        if ((int)((i % nA) % G) == my_g && !(P.skip_first_a && i == 0)) mbar_wait_drain(&a_full[i % nA], (i / nA) & 1);
  } else if (warp < kWarpI0) {
    // ---------------- weight producers: one warp per owner ----------------
    // Owner q's pieces, in its reading order, go round-robin through its own
    // slots; the warp scans the pieces uniformly (one lane waits at a time,
    // so no lane spins while another must issue) and spreads the copies over
    // kTpWLanes lanes, whose copies then overlap (bulk copies issued by one
    // thread complete one after another).  Every slot therefore has a single
    // filling sequence and a single reader: each parity wait is exact.
    const int q = warp - kWarpW0;
    const uint32_t s0 = (uint32_t)P.owner_slot0[q], ns = (uint32_t)P.owner_nslots[q];
    bool ok = !(*reinterpret_cast<volatile int*>(P.err) & 2) && ns > 0;
    constexpr int kRec = kTpMaxSlots + 1;
    uint32_t rec = 0, nrec = 0;  // this lane's last issued owner-local piece index + 1, and how many
    uint32_t li = 0;             // owner-local index of the next piece
    for (int item = blockIdx.x; ok && item < nitems; item += gridDim.x) {
      const Tile T = item_tile(item, ntiles, ntx, nty);
      const TpPass& pass = P.pass[T.pass];
      const int np = pass.npieces;
      const unsigned char* wsrc = P.W + pass.w_base;
      for (int xz = 0; ok && xz < 9; ++xz) {
        for (int k = 0; ok && k < np; ++k) {
          if (pass.piece_owner[k] != q) continue;
          const uint32_t l = li++, slot = s0 + l % ns;
          if ((int)(l % kTpWLanes) == lane) {
            if (!(ok = wait_fast(&w_empty[slot], ((l / ns) & 1) ^ 1, P.err, W_PROD_B))) {
              ok = false;
            } else {
              const uint32_t bytes = (uint32_t)pass.piece_len16[k] * 16u;
              mbar_expect_tx(&w_full[slot], bytes);
              bulk_load(w_ring + (size_t)slot * kTpPieceBytes, wsrc + ((long long)xz * np + k) * kTpPieceBytes,
                        bytes, &w_full[slot]);
              rec = l + 1;
              ++nrec;
            }
          }
          ok = __all_sync(0xffffffffu, ok);  // the warp stays uniform
        }
      }
    }
    (void)kRec;
    // after a time-out: this lane's pieces among the owner's last ns issued
    // (one per slot) land before the CTA exits
    const uint32_t top = __reduce_max_sync(0xffffffffu, rec);
    if (!ok && ns > 0 && nrec > 0)
      for (uint32_t l = (top > ns ? top - ns : 0); l < top; ++l)
        if ((int)(l % kTpWLanes) == lane && l < rec) mbar_wait_drain(&w_full[s0 + l % ns], (l / ns) & 1);
  } else if (warp < kWarpE0) {
    // ---------------- MMA issuers ----------------
    if (lane == 0) {
      const int q = warp - kWarpI0;
      const uint32_t s0 = (uint32_t)P.owner_slot0[q], ns = (uint32_t)P.owner_nslots[q];
      uint32_t li = 0;  // owner-local index of the next own piece (the producer's numbering)
      const uint32_t ab = split ? 1u : 2u;  // BF16 : TF32 operands, FP32 accumulate, K-major, M = 128
      const uint32_t idesc0 = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(128 >> 4) << 24);
      AccSeq acc;
      uint32_t t = 0;
      bool ok = !(*reinterpret_cast<volatile int*>(P.err) & 2);
      for (int item = blockIdx.x; ok && item < nitems; item += gridDim.x) {
        const Tile T = item_tile(item, ntiles, ntx, nty);
        const TpPass& pass = P.pass[T.pass];
        uint32_t buf, phase;
        acc.next(pass.nbuf, buf, phase);
        if (!(ok = wait_fast(&acc_empty[buf], phase, P.err, W_MMA_ACC))) break;
        tc_fence_after();
        const uint32_t tbase = tmem + buf * (uint32_t)pass.tmem_cols;
        for (int xz = 0; ok && xz < 9; ++xz) {
          for (int j = 0; ok && j < pass.nchunks; ++j, ++t) {
            const uint32_t sa = t % nA;
            if (!(ok = wait_fast(&a_full[sa], (t / nA) & 1, P.err, W_MMA_A))) break;
            tc_fence_after();
            const uint64_t a_desc = sw128_desc(smem_u32(a_ring + sa * kAStage));
            const uint64_t a_hi0 = a_desc, a_lo0 = a_desc + (uint64_t)(kAPlane >> 4);
            for (int k = pass.chunk_piece[j]; ok && k < pass.chunk_piece[j + 1]; ++k) {
              if (pass.piece_owner[k] != q) continue;  // another issuer's accumulators
              const uint32_t l = li++, slot = s0 + l % ns;
              if (!(ok = wait_fast(&w_full[slot], (l / ns) & 1, P.err, W_MMA_B))) break;
              tc_fence_after();
              const uint64_t b_desc = sw32_desc(smem_u32(w_ring + (size_t)slot * kTpPieceBytes));
              const int u1 = pass.piece_unit[k + 1];
              for (int u = pass.piece_unit[k]; u < u1; ++u) {
                const uint32_t w = pass.unit[u];
                const uint32_t aoff = ((w >> 7) & 3u) * (uint32_t)(kTcTileX * 128 >> 4) + ((w >> 5) & 3u) * 2u;
                const uint64_t b = b_desc + (uint64_t)((w & 31u) << 5);
                const uint32_t d = tbase + (((w >> 11) & 31u) << 4);
                const uint32_t n16 = (w >> 16) & 31u;
                const uint32_t form = (w >> 9) & 3u;
                if (split) {
                  if (form == 0) {  // hi rows then lo rows: hi*hi, lo*hi, hi*lo
                    const uint32_t idesc = idesc0 | (n16 << 18);
                    const uint64_t b_lo = b + (uint64_t)(n16 * 32u);  // n rows of 32 B, in 16-byte units
                    mma_f16_acc(d, a_hi0 + aoff, b, idesc);
                    mma_f16_acc(d, a_lo0 + aoff, b, idesc);
                    mma_f16_acc(d, a_hi0 + aoff, b_lo, idesc);
                  } else {  // lo rows reversed, then hi rows: hi*[lo; hi] over 2N columns, then lo*hi
                    mma_f16_acc(d, a_hi0 + aoff, b, idesc0 | (n16 << 19));
                    mma_f16_acc(tbase + (((w >> 21) & 31u) << 4), a_lo0 + aoff, b + (uint64_t)(n16 * 32u),
                                idesc0 | (n16 << 18));
                  }
                } else {
                  mma_tf32_acc(d, a_hi0 + aoff, b, idesc0 | (n16 << 18));
                }
              }
              mma_commit(&w_empty[slot]);  // the slot is free once this owner's MMAs have read it
            }
            mma_commit(&a_empty[sa]);
          }
        }
        if (ok) mma_commit(&acc_full[buf]);  // fires when every MMA of the tile has completed
      }
      // every MMA of this issuer completes before tensor memory is freed
      mma_commit(&fin[q]);
      mbar_wait_drain(&fin[q], 0);
    }
  } else {
    // ---------------- epilogue: TMEM -> registers -> C, then zero ----------------
    const int wq = warp & 3;
    const int r = wq * 32 + lane;  // tile row = TMEM lane
    const uint32_t lane_base = (uint32_t)(wq * 32) << 16;
    // every accumulator set starts at zero
    for (uint32_t c = 0; c < tmem_need; c += 16) tmem_st16_zero(tmem + lane_base + c);
    tmem_st_wait();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&acc_empty[0]);
      mbar_arrive(&acc_empty[1]);
    }
    AccSeq acc;
    bool live = true;
    for (int item = blockIdx.x; live && item < nitems; item += gridDim.x) {
      const Tile T = item_tile(item, ntiles, ntx, nty);
      const TpPass& pass = P.pass[T.pass];
      uint32_t buf, phase;
      acc.next(pass.nbuf, buf, phase);
      int ready = 0;
      if (lane == 0) ready = mbar_wait(&acc_full[buf], phase, P.err, W_EPI) ? 1 : 0;
      ready = __shfl_sync(0xffffffffu, ready, 0);  // warp-uniform: tcgen05.ld is warp-collective
      if (!ready) {
        live = false;
        break;
      }
      tc_fence_after();
      const int x = T.ox + (r & 7), y = T.oy + (r >> 3), z = T.oz;
      const bool valid = x < P.grid[0] && y < P.grid[1] && z < P.grid[2];
      float* crow = P.C + ((((long long)z * P.grid[1] + y) * P.grid[0] + x) * P.n_cols);
      const uint32_t tb = tmem + buf * (uint32_t)pass.tmem_cols + lane_base;
      for (int gi = 0; gi < pass.ngroups; ++gi) {
        uint32_t rd[16], re[16], rl[16];
        const int ge = pass.grp_e[gi], gl = pass.grp_l2[gi];
        __syncwarp();  // tcgen05.ld is warp-collective: reconverge after the masked stores
        tmem_ld16_nowait(tb + (uint32_t)pass.grp_d[gi], rd);
        if (ge >= 0) tmem_ld16_nowait(tb + (uint32_t)ge, re);
        if (gl >= 0) tmem_ld16_nowait(tb + (uint32_t)gl, rl);
        tmem_ld_wait();
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(rd[i]);
        if (ge >= 0) {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] += __uint_as_float(re[15 - i]);
        }
        if (gl >= 0) {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] += __uint_as_float(rl[i]);
        }
        if (valid) {
          const int c0 = 16 * gi;
#pragma unroll
          for (int jj = 0; jj < 16; jj += 4)
            if (c0 + jj < pass.ncols) {
              int col = pass.col0 + c0 + jj;
              if (P.col_mapped) col = (int)P.col_map[col >> 3] * 8 + (col & 7);
              float4* o = reinterpret_cast<float4*>(crow + col);
              float4 q4 = make_float4(v[jj], v[jj + 1], v[jj + 2], v[jj + 3]);
              if (P.accumulate) {
                const float4 old = *o;
                q4.x += old.x, q4.y += old.y, q4.z += old.z, q4.w += old.w;
              }
              *o = q4;
            }
        }
      }
      __syncwarp();
      for (uint32_t c = 0; c < (uint32_t)pass.tmem_cols; c += 16)
        tmem_st16_zero(tmem + buf * (uint32_t)pass.tmem_cols + lane_base + c);
      tmem_st_wait();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);  // this warp's lanes of the set are drained and zeroed
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_need));
  }
}

}  // namespace

cudaError_t launch_nbr_tc(const TpLaunch& L, const void* map_hi, const void* map_lo, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(nbr_tc_kernel<TC_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemBytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(nbr_tc_kernel<TC_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (L.npass < 1 || L.npass > kTpMaxPasses || L.a_stages < 2 || L.a_stages > kTpMaxAStages || L.w_slots < 1 ||
      L.w_slots > kTpMaxSlots)
    return cudaErrorInvalidValue;
  for (int q = 0, s0 = 0; q < kTpIssuers; ++q) {  // the owner rings tile the slots
    if (L.owner_slot0[q] != s0 || L.owner_nslots[q] < 0) return cudaErrorInvalidValue;
    s0 += L.owner_nslots[q];
    if (q == kTpIssuers - 1 && s0 != L.w_slots) return cudaErrorInvalidValue;
  }
  const int planes = L.kind == TC_BF16X3 ? 2 : 1;
  if (2048 + L.a_stages * planes * kAPlane + L.w_slots * kTpPieceBytes > kTcSmemUsable) return cudaErrorInvalidValue;
  const int ntx = (L.grid[0] + kTcTileX - 1) / kTcTileX, nty = (L.grid[1] + kTcTileY - 1) / kTcTileY;
  const long long items = (long long)ntx * nty * L.grid[2] * L.npass;
  if (items <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 148;
  const int ctas = (int)std::min<long long>(items, sms);
  if (L.kind == TC_BF16X3)
    nbr_tc_kernel<TC_BF16X3><<<ctas, kThreads, kSmemBytes, s>>>(*reinterpret_cast<const CUtensorMap*>(map_hi),
                                                                 *reinterpret_cast<const CUtensorMap*>(map_lo), L);
  else
    nbr_tc_kernel<TC_TF32><<<ctas, kThreads, kSmemBytes, s>>>(*reinterpret_cast<const CUtensorMap*>(map_hi),
                                                               *reinterpret_cast<const CUtensorMap*>(map_lo), L);
  return cudaGetLastError();
}

}  // namespace fmmgb
