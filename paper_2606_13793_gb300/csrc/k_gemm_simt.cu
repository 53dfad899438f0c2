// Neighbour contraction on the CUDA cores (FP32 / FP64).
//
// Both translation-invariant steps of the solve are the same contraction over
// a 3-D grid of "rows" and their 27 neighbours:
//
//   C[r][n] (+)= sum_{d in {-1,0,1}^3} sum_{k < K(n)} A[r + d][k] * W_d[k][n]
//
//  * M2L (Sec. 2.3, eq. M2L) at level l: a row is a parent box of level l-1,
//    A[r] its children's scaled multipoles [coef][child], n = (beta, target
//    child) and W_d the unit-box translation operator restricted to the
//    interaction list (Sec. 2.2: source children at Chebyshev distance >= 2
//    from the target child).  Ordering coefficients by total order makes
//    the truncation |alpha| + |beta| <= p a prefix K(n) of the reduction.
//  * P2P (Sec. 2.3, eq. direct): a row is a leaf box, A[r] its b^3 cell
//    masses and W_d[s][t] = g(x_t - x_s) for the neighbour box d.
//
// A neighbour outside the grid contributes zero: that is the isolated
// boundary.  Tile: 64 rows (a 4x4x4 block of the row grid) x 32 columns,
// 64 threads, each thread an 8x4 register tile.  A work item is one (row
// tile, column tile, neighbour) combination; a launch may cap its CTAs, each
// then looping over items (a few persistent CTAs that share SMs with other
// kernels instead of flooding them).
#include "fmm_internal.h"
#include "multi.cuh"

namespace fmmgb {
namespace {

constexpr int kRows = 64;
constexpr int kPad = 1;

// Reduction values per stage: 32 (FP32) or 16 (FP64), i.e. 12.4 KB of shared
// memory for FP64, small enough to sit beside a tensor-core block.
template <typename T>
constexpr int kChunkOf = sizeof(T) == 8 ? kKChunk / 2 : kKChunk;

template <typename T>
__device__ __forceinline__ void nbr_gemm_simt_body(const NbrGemm& g, const VBlock vb) {
  constexpr int KC = kChunkOf<T>;
  __shared__ T As[KC][kRows + kPad];
  __shared__ T Bs[KC][kNTile];
  const int tx = threadIdx.x;
  const int rg = tx & 7;   // rows rg*8 .. rg*8+7
  const int cg = tx >> 3;  // cols cg*4 .. cg*4+3
  const int ntx = (g.grid[0] + 3) >> 2, nty = (g.grid[1] + 3) >> 2, ntz = (g.grid[2] + 3) >> 2;
  const long long tiles = (long long)ntx * nty * ntz;
  const long long items = tiles * g.ntiles * (g.dsplit > 1 ? 27 : 1);
  for (long long w = vb.x; w < items; w += vb.gx) {
    const int bt = (int)(w % tiles);
    const int tile = (int)((w / tiles) % g.ntiles);
    const int dgrp = (int)(w / (tiles * g.ntiles));
    const int ox = (bt % ntx) * 4, oy = ((bt / ntx) % nty) * 4, oz = (bt / (ntx * nty)) * 4;
    const int K = g.tile_k[tile];
    const T* W0 = static_cast<const T*>(g.W) + g.tile_w[tile];
    const T* A = static_cast<const T*>(g.A);

    T acc[8][4];
  #pragma unroll
    for (int i = 0; i < 8; ++i)
  #pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    const int d0 = g.dsplit > 1 ? dgrp : 0;  // dsplit is 1 or 27 here
    const int d1 = g.dsplit > 1 ? d0 + 1 : 27;
    for (int d = d0; d < d1; ++d) {
      if (d == 13 && g.skip_center) continue;  // the centre block is zero
      const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
      const T* Wd = W0 + (long long)d * K * kNTile;
      for (int kc = 0; kc < K; kc += KC) {
        const int kn = min(KC, K - kc);
        for (int e = tx; e < kRows * KC; e += 64) {
          const int r = e / KC, k = e % KC;
          T v = T(0);
          if (k < kn) {
            const int x = ox + (r & 3) + dx, y = oy + ((r >> 2) & 3) + dy, z = oz + (r >> 4) + dz;
            if (x >= 0 && y >= 0 && z >= 0 && x < g.grid[0] && y < g.grid[1] && z < g.grid[2])
              v = A[(((long long)z * g.grid[1] + y) * g.grid[0] + x) * g.row_len + kc + k];
          }
          As[k][r] = v;
        }
        for (int e = tx; e < KC * kNTile; e += 64) {
          const int k = e / kNTile, n = e % kNTile;
          Bs[k][n] = (k < kn) ? Wd[(long long)(kc + k) * kNTile + n] : T(0);
        }
        __syncthreads();
        for (int k = 0; k < kn; ++k) {
          T a[8], b[4];
  #pragma unroll
          for (int i = 0; i < 8; ++i) a[i] = As[k][rg * 8 + i];
  #pragma unroll
          for (int j = 0; j < 4; ++j) b[j] = Bs[k][cg * 4 + j];
  #pragma unroll
          for (int i = 0; i < 8; ++i)
  #pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
      }
    }

    T* C = static_cast<T*>(g.C);
    const long long rows = (long long)g.grid[0] * g.grid[1] * g.grid[2];
    T* Pz = g.dsplit > 1 ? static_cast<T*>(g.partial) + (long long)dgrp * rows * g.n_cols : nullptr;
  #pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = rg * 8 + i;
      const int x = ox + (r & 3), y = oy + ((r >> 2) & 3), z = oz + (r >> 4);
      if (x >= g.grid[0] || y >= g.grid[1] || z >= g.grid[2]) continue;
      const long long row = ((long long)z * g.grid[1] + y) * g.grid[0] + x;
  #pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = tile * kNTile + cg * 4 + j;
        if (n >= g.n_cols) continue;
        if (Pz) {
          Pz[row * g.n_cols + n] = acc[i][j];
        } else {
          T* dst = C + row * g.n_cols + n;
          *dst = g.accumulate ? (*dst + acc[i][j]) : acc[i][j];
        }
      }
    }
  }  // work items
}

template <typename T>
__global__ void __launch_bounds__(64) nbr_gemm_simt_kernel(NbrGemm g) {
  nbr_gemm_simt_body<T>(g, native_vblock());
}

template <typename T>
__global__ void __launch_bounds__(64) nbr_gemm_simt_multi_kernel(const NbrGemm* __restrict__ gs,
                                                                 const MultiGrid* __restrict__ grids, int n) {
  __shared__ NbrGemm g;  // the item's description, read by the body from shared memory
  const int i = multi_item(grids, n);
  if (threadIdx.x == 0) g = gs[i];
  __syncthreads();
  nbr_gemm_simt_body<T>(g, multi_vblock(grids[i]));
}

// Column-per-lane variant (shape 3), for the FP64 levels: every lane owns one
// output column and R consecutive rows of its warp, so a block is 4 warps x
// 32 columns x R rows with no shared memory.  The 64-bit FMA pipe of an SM is
// narrow (a warp instruction occupies it for many cycles), so what counts is
// that every row computed is a real row, that the work comes in many small
// blocks spread over all SMs and their four sub-partitions, and that no block
// carries a long reduction alone; loads (one coalesced weight row per k, one
// broadcast activation per row) are cheap beside the FMAs.
constexpr int kColRows = 4;  // rows per warp

template <typename T>
__device__ __forceinline__ void nbr_gemm_col_body(const NbrGemm& g, const VBlock vb) {
  constexpr int R = kColRows;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long rows = (long long)g.grid[0] * g.grid[1] * g.grid[2];
  const int tile = vb.y;
  const int d0 = g.dsplit > 1 ? (int)vb.z : 0;  // dsplit is 1 or 27 here
  const int d1 = g.dsplit > 1 ? d0 + 1 : 27;
  const int K = g.tile_k[tile];
  const T* W0 = static_cast<const T*>(g.W) + g.tile_w[tile] + lane;
  const T* A = static_cast<const T*>(g.A);
  long long row[R];
  int rx[R], ry[R], rz[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    row[i] = ((long long)vb.x * 4 + warp) * R + i;
    const long long rr = row[i] < rows ? row[i] : 0;
    rx[i] = (int)(rr % g.grid[0]);
    ry[i] = (int)((rr / g.grid[0]) % g.grid[1]);
    rz[i] = (int)(rr / ((long long)g.grid[0] * g.grid[1]));
  }
  T acc[R];
#pragma unroll
  for (int i = 0; i < R; ++i) acc[i] = T(0);
  for (int d = d0; d < d1; ++d) {
    if (d == 13 && g.skip_center) continue;  // the centre block is zero
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    const T* ap[R];
    bool av[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int x = rx[i] + dx, y = ry[i] + dy, z = rz[i] + dz;
      av[i] = row[i] < rows && x >= 0 && y >= 0 && z >= 0 && x < g.grid[0] && y < g.grid[1] && z < g.grid[2];
      ap[i] = A + (av[i] ? (((long long)z * g.grid[1] + y) * g.grid[0] + x) * g.row_len : 0);
    }
    const T* w = W0 + (long long)d * K * kNTile;
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      const T wk = __ldg(w + (long long)k * kNTile);
#pragma unroll
      for (int i = 0; i < R; ++i) acc[i] = fma(av[i] ? __ldg(ap[i] + k) : T(0), wk, acc[i]);
    }
  }
  const int col = tile * kNTile + lane;
  if (col >= g.n_cols) return;
  T* Pz = g.dsplit > 1 ? static_cast<T*>(g.partial) + (long long)d0 * rows * g.n_cols : nullptr;
  T* C = static_cast<T*>(g.C);
#pragma unroll
  for (int i = 0; i < R; ++i) {
    if (row[i] >= rows) continue;
    if (Pz) {
      Pz[row[i] * g.n_cols + col] = acc[i];
    } else {
      T* dst = C + row[i] * g.n_cols + col;
      *dst = g.accumulate ? (*dst + acc[i]) : acc[i];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(128) nbr_gemm_col_kernel(NbrGemm g) {
  nbr_gemm_col_body<T>(g, native_vblock());
}

template <typename T>
__global__ void __launch_bounds__(128) nbr_gemm_col_multi_kernel(const NbrGemm* __restrict__ gs,
                                                                 const MultiGrid* __restrict__ grids, int n) {
  __shared__ NbrGemm g;  // the item's description, read by the body from shared memory
  const int i = multi_item(grids, n);
  if (threadIdx.x == 0) g = gs[i];
  __syncthreads();
  nbr_gemm_col_body<T>(g, multi_vblock(grids[i]));
}

// Grids of at most 64 rows (4 x 4 x 4, the coarse levels of small fields):
// one block per column tile, a thread taking two rows and four columns and
// summing over the in-grid neighbours only.  The level's useful
// multiply-adds are few; the general tiles would spend most of theirs on
// padded rows and out-of-grid neighbours, and their staged reduction chunks
// (two barriers each) would set a long latency for little work.  No shared
// memory: the rows and weights of such a level stay in L1 / L2.
// The reduction is split into kTinyKS parts over as many groups of 256
// threads, added in part order at the end: the blocks are latency-bound, and
// this divides their length.
constexpr int kTinyRows = 64;
constexpr int kTinyKS = 4;
constexpr int kTinyThreads = 256 * kTinyKS;  // per part: 32 row pairs x 8 column groups of 4

template <typename T>
__device__ __forceinline__ void nbr_gemm_tiny_body(const NbrGemm& g, const VBlock vb) {
  __shared__ T part[(kTinyKS > 1 ? kTinyKS - 1 : 1) * 256 * 8];
  const int tile = vb.x;
  const int kp = threadIdx.x >> 8, tl = threadIdx.x & 255;  // reduction part, thread in the part
  const int cq = tl & 7, r0 = tl >> 3;
  const int R = g.grid[0] * g.grid[1] * g.grid[2];
  const int Kt = g.tile_k[tile];
  const int Kq = (Kt + kTinyKS - 1) / kTinyKS;
  const int k0 = kp * Kq, k1 = min(Kt, k0 + Kq);
  const T* W0 = static_cast<const T*>(g.W) + g.tile_w[tile] + cq * 4;
  const T* A = static_cast<const T*>(g.A);
  T acc[2][4];
  int rx[2], ry[2], rz[2];
  bool live[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int r = r0 + 32 * i;
    live[i] = r < R;
    const int rr = live[i] ? r : 0;
    rx[i] = rr % g.grid[0];
    ry[i] = (rr / g.grid[0]) % g.grid[1];
    rz[i] = rr / (g.grid[0] * g.grid[1]);
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[i][c] = T(0);
  }
  for (int d = 0; d < 27; ++d) {
    if (d == 13 && g.skip_center) continue;  // the centre block is zero
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    bool v[2];
    const T* ap[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int x = rx[i] + dx, y = ry[i] + dy, z = rz[i] + dz;
      v[i] = live[i] && x >= 0 && y >= 0 && z >= 0 && x < g.grid[0] && y < g.grid[1] && z < g.grid[2];
      ap[i] = A + (v[i] ? ((long long)(z * g.grid[1] + y) * g.grid[0] + x) * g.row_len : 0);
    }
    if (!v[0] && !v[1]) continue;
    const T* w = W0 + (long long)d * Kt * kNTile;
    for (int k = k0; k < k1; ++k) {
      const T* wk = w + (long long)k * kNTile;
      const T w0 = __ldg(wk), w1 = __ldg(wk + 1), w2 = __ldg(wk + 2), w3 = __ldg(wk + 3);
      const T a0 = v[0] ? __ldg(ap[0] + k) : T(0), a1 = v[1] ? __ldg(ap[1] + k) : T(0);
      acc[0][0] = fma(a0, w0, acc[0][0]);
      acc[0][1] = fma(a0, w1, acc[0][1]);
      acc[0][2] = fma(a0, w2, acc[0][2]);
      acc[0][3] = fma(a0, w3, acc[0][3]);
      acc[1][0] = fma(a1, w0, acc[1][0]);
      acc[1][1] = fma(a1, w1, acc[1][1]);
      acc[1][2] = fma(a1, w2, acc[1][2]);
      acc[1][3] = fma(a1, w3, acc[1][3]);
    }
  }
  if (kTinyKS > 1) {  // parts 1 .. KS-1 hand their sums to part 0, which adds them in order
    if (kp > 0) {
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) part[((kp - 1) * 256 + tl) * 8 + i * 4 + c] = acc[i][c];
    }
    __syncthreads();
    if (kp > 0) return;
    for (int q = 1; q < kTinyKS; ++q)
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] += part[((q - 1) * 256 + tl) * 8 + i * 4 + c];
  }
  T* C = static_cast<T*>(g.C);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    if (!live[i]) continue;
    const long long row = r0 + 32 * i;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int col = tile * kNTile + cq * 4 + c;
      if (col >= g.n_cols) continue;
      T* dst = C + row * g.n_cols + col;
      *dst = g.accumulate ? (*dst + acc[i][c]) : acc[i][c];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kTinyThreads) nbr_gemm_tiny_multi_kernel(const NbrGemm* __restrict__ gs,
                                                                           const MultiGrid* __restrict__ grids,
                                                                           int n) {
  __shared__ NbrGemm g;  // the item's description, read by the body from shared memory
  const int i = multi_item(grids, n);
  if (threadIdx.x == 0) g = gs[i];
  __syncthreads();
  nbr_gemm_tiny_body<T>(g, multi_vblock(grids[i]));
}

// C (+)= sum over the neighbour-group partials, in group order.
template <typename T>
__global__ void reduce_partials_kernel(const T* __restrict__ part, int nparts, long long count, T* __restrict__ C,
                                       int accumulate) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    T s = accumulate ? C[i] : T(0);
    for (int d = 0; d < nparts; ++d) s += part[d * count + i];
    C[i] = s;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_reduce_partials(const T* part, int nparts, long long count, T* C, int accumulate, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  long long blocks = (count + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  reduce_partials_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(part, nparts, count, C, accumulate);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_nbr_gemm_col(const NbrGemm& g, cudaStream_t s) {
  const long long rows = (long long)g.grid[0] * g.grid[1] * g.grid[2];
  const long long blocks = (rows + 4 * kColRows - 1) / (4 * kColRows);
  if (blocks <= 0 || g.ntiles <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL || g.ntiles > 65535) return cudaErrorInvalidConfiguration;
  nbr_gemm_col_kernel<T><<<dim3((unsigned)blocks, (unsigned)g.ntiles, g.dsplit > 1 ? 27u : 1u), 128, 0, s>>>(g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || g.dsplit <= 1) return e;
  return launch_reduce_partials<T>(static_cast<const T*>(g.partial), g.dsplit, rows * g.n_cols,
                                   static_cast<T*>(g.C), g.accumulate, s);
}

template <typename T>
cudaError_t launch_nbr_gemm(const NbrGemm& g, cudaStream_t s) {
  if (g.shape == 3) return launch_nbr_gemm_col<T>(g, s);
  return g.shape == 0 ? launch_nbr_gemm_simt<T>(g, s) : launch_nbr_gemm_zrun<T>(g, g.shape - 1, s);
}

template <typename T>
cudaError_t launch_nbr_gemm_simt(const NbrGemm& g, cudaStream_t s) {
  const long long tiles = (long long)((g.grid[0] + 3) / 4) * ((g.grid[1] + 3) / 4) * ((g.grid[2] + 3) / 4);
  if (tiles <= 0 || g.ntiles <= 0) return cudaSuccess;
  long long items = tiles * g.ntiles * (g.dsplit > 1 ? 27 : 1);
  if (g.max_blocks > 0 && items > g.max_blocks) items = g.max_blocks;
  if (items > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  nbr_gemm_simt_kernel<T><<<(unsigned)items, 64, 0, s>>>(g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || g.dsplit <= 1) return e;
  return launch_reduce_partials<T>(static_cast<const T*>(g.partial), g.dsplit,
                                   (long long)g.grid[0] * g.grid[1] * g.grid[2] * g.n_cols, static_cast<T*>(g.C),
                                   g.accumulate, s);
}

// Multi-item forms: shapes 0 and 3 (z-run shapes in k_gemm_zrun.cu).
template <typename T>
cudaError_t launch_nbr_gemm_simt_multi(const NbrGemm* gs, const MultiGrid* grids, int n, long long blocks,
                                       cudaStream_t s) {
  if (n <= 0 || blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  nbr_gemm_simt_multi_kernel<T><<<(unsigned)blocks, 64, 0, s>>>(gs, grids, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_nbr_gemm_col_multi(const NbrGemm* gs, const MultiGrid* grids, int n, long long blocks,
                                      cudaStream_t s) {
  if (n <= 0 || blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  nbr_gemm_col_multi_kernel<T><<<(unsigned)blocks, 128, 0, s>>>(gs, grids, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_nbr_gemm_tiny_multi(const NbrGemm* gs, const MultiGrid* grids, int n, long long blocks,
                                       cudaStream_t s) {
  if (n <= 0 || blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  nbr_gemm_tiny_multi_kernel<T><<<(unsigned)blocks, kTinyThreads, 0, s>>>(gs, grids, n);
  return cudaGetLastError();
}

bool nbr_gemm_tiny_fits(const NbrGemm& g) { return (long long)g.grid[0] * g.grid[1] * g.grid[2] <= kTinyRows; }

template <typename T>
void nbr_gemm_simt_col_grid(const NbrGemm& g, unsigned out[3]) {
  const unsigned nd = g.dsplit > 1 ? 27u : 1u;
  if (g.shape == 3) {
    const long long rows = (long long)g.grid[0] * g.grid[1] * g.grid[2];
    out[0] = (unsigned)((rows + 4 * kColRows - 1) / (4 * kColRows));
    out[1] = (unsigned)g.ntiles;
    out[2] = nd;
  } else {
    const long long tiles = (long long)((g.grid[0] + 3) / 4) * ((g.grid[1] + 3) / 4) * ((g.grid[2] + 3) / 4);
    out[0] = (unsigned)(tiles * g.ntiles * nd);
    out[1] = out[2] = 1;
  }
}

template cudaError_t launch_nbr_gemm_simt_multi<float>(const NbrGemm*, const MultiGrid*, int, long long, cudaStream_t);
template cudaError_t launch_nbr_gemm_simt_multi<double>(const NbrGemm*, const MultiGrid*, int, long long, cudaStream_t);
template cudaError_t launch_nbr_gemm_col_multi<float>(const NbrGemm*, const MultiGrid*, int, long long, cudaStream_t);
template cudaError_t launch_nbr_gemm_col_multi<double>(const NbrGemm*, const MultiGrid*, int, long long, cudaStream_t);
template cudaError_t launch_nbr_gemm_tiny_multi<float>(const NbrGemm*, const MultiGrid*, int, long long, cudaStream_t);
template cudaError_t launch_nbr_gemm_tiny_multi<double>(const NbrGemm*, const MultiGrid*, int, long long, cudaStream_t);
template void nbr_gemm_simt_col_grid<float>(const NbrGemm&, unsigned[3]);
template void nbr_gemm_simt_col_grid<double>(const NbrGemm&, unsigned[3]);
template cudaError_t launch_nbr_gemm_simt<float>(const NbrGemm&, cudaStream_t);
template cudaError_t launch_nbr_gemm_simt<double>(const NbrGemm&, cudaStream_t);
template cudaError_t launch_nbr_gemm<float>(const NbrGemm&, cudaStream_t);
template cudaError_t launch_nbr_gemm<double>(const NbrGemm&, cudaStream_t);
template cudaError_t launch_reduce_partials<float>(const float*, int, long long, float*, int, cudaStream_t);
template cudaError_t launch_reduce_partials<double>(const double*, int, long long, double*, int, cudaStream_t);

}  // namespace fmmgb
