// Internal declarations of the GB300 FMM library: plan layout, level arena,
// device tables and the kernel launchers shared between translation units.
//
// Data layout in HBM (one arena per plan):
//  * Level l (2 <= l <= L) expansions are stored "parent-blocked": for each
//    box of the parent grid (level l-1, x fastest), the 8 children's
//    coefficients as [coef][child] with child = cx + 2 cy + 4 cz fastest.
//    A parent block is 8*nc contiguous values, so every neighbour-block read
//    of the M2L contraction is a contiguous row, and an order prefix
//    (coefficients of order <= k) is a contiguous prefix of the row.
//  * Children past the level's extent ("phantom" boxes of the round-up
//    hierarchy) hold zeros: the arena is cleared once at plan time and those
//    slots are never written.
//  * Scaled variables: at a level of box side h (cells),
//      Mt_alpha = M_alpha / h^|alpha|,   Lt_beta = h^(1+|beta|) L_beta / beta!
//    so the M2L translation operator is the same for every level, the
//    M2M/L2L shifts are pure numbers, and values stay O(mass).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/fmm.h"

namespace fmmgb {

constexpr int kMaxOrder = 8;
constexpr int kMaxCoef = 165;  // C(8+3, 3)
constexpr int kMaxLevels = 24;
constexpr int kNTile = 32;     // output columns per SIMT GEMM tile
constexpr int kKChunk = 32;    // reduction values per SIMT GEMM stage

// Pair lists of the M2M / L2L shifts.  Entry: coefficient index `src`,
// magnitude `coef`, and `mask`: bit q set when the shift exponent along
// axis q is odd (its sign then depends on which side of the parent the
// child sits).
struct ShiftEntry {
  double coef;   // FP64 copy (FP64 levels)
  float coef_f;  // FP32 copy (FP32 levels: no FP64 arithmetic there)
  int src;
  int mask;
};

struct Level {
  int n[3];        // boxes per axis at this level
  int np[3];       // boxes per axis of the parent grid (level l-1)
  long long nbox;
  long long npar;  // product of np
  int f64;         // expansions of this level kept in FP64
  size_t m_off;    // byte offset of the multipoles in the arena
  size_t l_off;    // byte offset of the local expansions in the arena
  size_t bytes;    // bytes of one of the two arrays
  int tc;          // M2L of this level on the tensor cores
  size_t hi_off, lo_off;  // bf16 hi / lo planes of the multipoles (tensor-core bf16x3 levels)
  // CUDA-core harmonic M2L: folded multipoles and the M2L's c <= 1 locals,
  // rows of 8 (p+1)^2 values in the level's type (0: none)
  size_t fold_off, lred_off;
};

// One item of a multi-item launch (multi.cuh): its grid of blocks and the
// first flat block of the launch that belongs to it.
struct MultiGrid {
  unsigned gx, gy, gz, pad;
  long long start;
};

// Neighbour-contraction ("implicit GEMM") description for the SIMT kernel:
//   C[row][n] (+)= sum_{d in 27 neighbours} sum_{k < K(tile(n))} A[row + d][k] * W_d[k][n]
// rows live on a 3-D grid; a neighbour outside the grid contributes zero.
struct NbrGemm {
  const void* A;       // [rows][row_len]
  int row_len;
  int grid[3];         // row grid extents
  const void* W;       // weights, see plan.cu (tile-major, then neighbour)
  const int* tile_k;   // device [ntiles]: reduction length of each column tile
  const long long* tile_w;  // device [ntiles]: offset of the tile's neighbour-0 block
  void* C;             // [rows][n_cols]
  int n_cols;
  int ntiles;
  int accumulate;      // 1: C += result, 0: C = result
  int dsplit;          // CTAs sharing the 27 neighbours of a row tile (partial sums reduced in a fixed order):
                       // shapes 0, 3: 1 or 27; shapes 1, 2: 1, 3 or 9
  void* partial;       // [dsplit][rows][n_cols] scratch when dsplit > 1
  int shape = 0;       // 0: 4x4x4 rows per CTA, 3: one column per lane (k_gemm_simt.cu);
                       // 1, 2: z-run tiles (k_gemm_zrun.cu)
  int max_blocks = 0;  // shape 0: at most this many CTAs, each looping over work items (0: one per item)
  int skip_center = 0; // 1: W_d of the centre neighbour (d = 13) is all zero (the M2L: a parent's
                       // children are each other's near neighbours), and the kernels skip it
};

template <typename T>
cudaError_t launch_nbr_gemm_simt(const NbrGemm& g, cudaStream_t s);
// z-run tiles: shape 0 = 8x4x8 (FP32) / 8x4x4 (FP64) rows per CTA, shape 1 = 8x4x4 / 8x4x2
template <typename T>
cudaError_t launch_nbr_gemm_zrun(const NbrGemm& g, int shape, cudaStream_t s);
// Whether the z-run kernel handles this contraction (reduction lengths and
// column counts multiples of 8, dsplit 1, 3 or 9).
bool zrun_eligible(const NbrGemm& g, const int* tile_k_host, int ntiles);
// Dispatch on g.shape.
template <typename T>
cudaError_t launch_nbr_gemm(const NbrGemm& g, cudaStream_t s);
// Multi-item forms (multi.cuh) for items of one shape with dsplit 1 (no
// partial sums): gs / grids are device arrays of n items; *_grid gives an
// item's grid (shape 0 / 3: nbr_gemm_simt_col_grid, shapes 1 / 2:
// nbr_gemm_zrun_grid with shape - 1).
template <typename T>
cudaError_t launch_nbr_gemm_simt_multi(const NbrGemm* gs, const MultiGrid* grids, int n, long long blocks,
                                       cudaStream_t s);
template <typename T>
cudaError_t launch_nbr_gemm_col_multi(const NbrGemm* gs, const MultiGrid* grids, int n, long long blocks,
                                      cudaStream_t s);
// shape here: 0 / 1 as launch_nbr_gemm_zrun, 2 = a z run of 6 rows (FP32; 3 in FP64)
template <typename T>
cudaError_t launch_nbr_gemm_zrun_multi(int shape, const NbrGemm* gs, const MultiGrid* grids, int n, long long blocks,
                                       cudaStream_t s);
template <typename T>
void nbr_gemm_simt_col_grid(const NbrGemm& g, unsigned out[3]);
// Grids of at most 64 rows (nbr_gemm_tiny_fits): one block per column tile
// (an item's grid is ntiles x 1 x 1), in-grid neighbours only.
bool nbr_gemm_tiny_fits(const NbrGemm& g);
template <typename T>
cudaError_t launch_nbr_gemm_tiny_multi(const NbrGemm* gs, const MultiGrid* grids, int n, long long blocks,
                                       cudaStream_t s);
template <typename T>
void nbr_gemm_zrun_grid(const NbrGemm& g, int shape, unsigned out[3]);
// C (+)= sum over nparts partial arrays of count values, in part order.
template <typename T>
cudaError_t launch_reduce_partials(const T* part, int nparts, long long count, T* C, int accumulate, cudaStream_t s);

// Upward pass.
struct TreeTables {
  const int8_t* mi;          // [nc][3] multi-indices (canonical order)
  const int* m2m_start;      // [nc+1] CSR over output alpha
  const ShiftEntry* m2m;     // entries (src = beta)
  const int* l2l_start;      // [nc+1] CSR over output beta
  const ShiftEntry* l2l;     // entries (src = gamma)
  int p, nc, b;
};

// P2M: Mleaf always; rho_box (FP32/FP64 near field) and the bf16 hi/lo planes
// (Mhi/Mlo for a tensor-core leaf level, rho_hi/rho_lo for the tensor-core
// near field) when non-NULL.  Sets bit 0 of *flag for a non-finite density.
// harm = 1: the planes hold the harmonic ((p+1)^2, c <= 1) components of the
// folded multipoles (tree_common.cuh), rows of 8 (p+1)^2 values per parent.
// Mfold (nullable, with harm): the folded components in the level's type,
// rows of 8 (p+1)^2 values (the CUDA-core harmonic M2L reads them).
// dip (nullable): dipole sources [3][cells], weights v_q adding v_q d/de_q (e^alpha)
// (box units) per cell -- the transpose of the analytic force's L2P gradient.
template <typename T>
cudaError_t launch_p2m(const TreeTables& t, const T* rho, const int dims[3], const Level& leaf, T* Mleaf, T* rho_box,
                       void* Mhi, void* Mlo, void* rho_hi, void* rho_lo, int* flag, int harm, T* Mfold,
                       cudaStream_t s, const T* dip = nullptr);
// M2M into the parent level; Mhi/Mlo (bf16 planes of the parent, harmonic
// components when harm = 1) when non-NULL.
template <typename Tc, typename Tp>
cudaError_t launch_m2m(const TreeTables& t, const Level& child, const Tc* Mc, const Level& par, Tp* Mp, void* Mhi,
                       void* Mlo, int harm, Tp* Mfold, cudaStream_t s);
template <typename Tp, typename Tc>
// accumulate = 1: child locals += shifted parent locals (after the level's M2L wrote them);
// harm = 1: that M2L wrote only the harmonic components, the rest are rebuilt;
// Lp = NULL: no parent locals (only the rebuild); Lred (nullable): the
// M2L's c <= 1 locals in compact rows [parent][reduced coef][child] instead
// of in the full rows
cudaError_t launch_l2l(const TreeTables& t, const Level& par, const Tp* Lp, const Level& child, Tc* Lc, int accumulate,
                       int harm, const Tc* Lred, cudaStream_t s);
// Near field of leaf-4 boxes on the tensor cores, bf16x3 (k_near_tc.cu):
// W holds, per neighbour d = (dx+1) + 3 (dy+1) + 9 (dz+1), the 64 x 64
// weights W_d[source cell][target cell] as the B operand's shared-memory
// image: 64 rows (target cells) of 128 B (64 bf16 source cells), 16-byte
// chunks swizzled by (row mod 8); the hi plane, then the lo plane.
constexpr int kNtPieceBytes = 2 * 64 * 128;
struct NearTcLaunch {
  const unsigned char* W;  // device, 27 x kNtPieceBytes
  float* C;                // device [leaf boxes][64], written (not accumulated)
  int grid[3];             // leaf boxes per axis
  int* err;                // plan flag: FMM_ERR_TIMEOUT bit and wait site
  uint32_t idesc;          // MMA instruction descriptor, M = 128, N = 64, bf16 in, FP32 out
};
// map_hi / map_lo: the bf16 hi / lo density rows (64 values per leaf box),
// box 64 x 8 x 18 x 1 with 128-byte swizzle (make_row_map).
cudaError_t launch_near_tc4(const NearTcLaunch& L, const void* map_hi, const void* map_lo, cudaStream_t s);

// Multi-item forms (batched solves, multi.cuh): args and grids are device
// arrays of n items sorted by first block; blocks = the launch's total, bs
// the block size every item's grid was computed with.
// P2M of one leaf level (launch_p2m's arguments; boxes of kThreads / 2 per
// block: grid = ceil(npar * 16 / kThreads) blocks of kThreads).
struct P2mArgs {
  const void* rho;
  int nx, ny, b;
  Level leaf;
  void* Mleaf;
  void* Mhi;
  void* Mlo;
  void* rho_box;
  void* rho_hi;
  void* rho_lo;
  int* flag;
  int harm;
  void* Mfold;
  long long ncell;
};
// harm_rows: 1 when any item stages folded rows (harm with Mhi or Mfold)
template <typename T>
cudaError_t launch_p2m_multi(int p, const P2mArgs* args, const MultiGrid* grids, int n, long long blocks,
                             int harm_rows, cudaStream_t s);
// Leaf evaluation (launch_leaf_finish's arguments; one thread per leaf box:
// grid = ceil(npar * 8 / kThreads) blocks of kThreads).
struct LeafArgs {
  Level leaf;
  const void* Lleaf;
  const void* near_box;
  int near_stride;
  const void* m2p;
  int nx, ny, b;
  double scale;
  void* phi;
  // the last L2L in the leaf kernel (launch_leaf_finish's `down`; Lp NULL: none)
  Level par;
  const void* Lp;
  int harm;
  const void* Lred;
};
template <typename T>
cudaError_t launch_leaf_finish_multi(int p, const LeafArgs* args, const MultiGrid* grids, int n, long long blocks,
                                     cudaStream_t s);
// The 5-point stencil of App. C on FP32 rows of a multiple of four cells,
// 16-byte aligned; fd_multi_grid gives an item's grid (blocks of 32 x 8).
struct FdArgs {
  const void* phi;
  int nx, ny, nz;
  double inv_dx;
  void* accel;
};
cudaError_t launch_fd_accel_multi(const FdArgs* args, const MultiGrid* grids, int n, long long blocks,
                                  cudaStream_t s);
void fd_multi_grid(const int dims[3], unsigned g[3]);
struct M2mArgs {
  Level child;
  const void* Mc;
  Level par;
  void* Mp;
  void* Mhi;
  void* Mlo;
  int harm;
  void* Mfold;
};
template <typename Tc, typename Tp>
cudaError_t launch_m2m_multi(int p, const M2mArgs* args, const MultiGrid* grids, int n, long long blocks, int bs,
                             cudaStream_t s);
struct L2lArgs {
  Level par;
  const void* Lp;
  Level child;
  void* Lc;
  int accumulate;
  int harm;
  const void* Lred;
};
template <typename Tp, typename Tc>
cudaError_t launch_l2l_multi(int p, const L2lArgs* args, const MultiGrid* grids, int n, long long blocks, int bs,
                             cudaStream_t s);
template <typename T>
cudaError_t launch_zero(T* p, size_t count, cudaStream_t s);
// dst = sc * src (count values)
template <typename T>
cudaError_t launch_scaled_copy(const T* src, size_t count, double sc, T* dst, cudaStream_t s);
// Copy of a cell grid in the leaf level's parent-blocked box order
// [parent][child][b^3] (phantom boxes zero).
template <typename T>
cudaError_t launch_cells_to_parent_blocks(const T* src, const int dims[3], const Level& leaf, int b, T* dst,
                                          cudaStream_t s);
// [w, sc g_x, sc g_y, sc g_z] x b^3 per leaf box (g nullable: zeros), boxes in
// grid order (parent_blocked = 0) or [parent][child] order (1).
template <typename T>
cudaError_t launch_cells_to_boxes4(const T* w, const T* g, double sc, const int dims[3], const Level& leaf, int b,
                                   int parent_blocked, T* dst, cudaStream_t s);
// near_box rows hold near_stride values per leaf box, the potential sums first.
// m2p (nullable): final-stage M2P potentials, parent-blocked [parent][child][b^3], in the
// leaf level's scaled units (multiplied by 1/b like the L2P term).
// down (nullable): the last L2L (level L - 1 -> leaf, accumulate) done by the
// leaf kernel in registers, with launch_l2l's arguments for that level pair
// (type T on both); Lleaf then holds only the leaf level's M2L locals (full
// rows, or the c <= 1 ones in Lleaf / in down->Lred with harm) and is not
// written.
template <typename T>
struct LeafDownArgs {
  Level par;
  const T* Lp = nullptr;
  int harm = 0;
  const T* Lred = nullptr;
};
template <typename T>
cudaError_t launch_leaf_finish(const TreeTables& t, const Level& leaf, const T* Lleaf, const T* near_box,
                               int near_stride, const T* m2p, const int dims[3], double scale, T* phi, cudaStream_t s,
                               const LeafDownArgs<T>* down = nullptr);
// With the analytic acceleration: near_box rows are [potential, d/dx, d/dy,
// d/dz] x b^3; accel = ascale (far gradient + near gradient).  m2p (nullable):
// the final-stage M2P's [parent][child][potential, d/dx, d/dy, d/dz][b^3],
// box units like the local expansion's terms.
template <typename T>
cudaError_t launch_leaf_finish_grad(const TreeTables& t, const Level& leaf, const T* Lleaf, const T* near_box,
                                    const T* m2p, const int dims[3], double scale, double ascale, T* phi, T* accel,
                                    cudaStream_t s);
template <typename T>
cudaError_t launch_fd_accel(const T* phi, const int dims[3], double inv_dx, T* accel, cudaStream_t s);
template <typename T>
cudaError_t launch_adjoint_source(const T* gphi, const T* gaccel, const int dims[3], double inv_dx, T* out,
                                  cudaStream_t s);
template <typename T>
cudaError_t launch_check_finite(const T* x, size_t count, int* flag, cudaStream_t s);
// Level copy into the canonical [box][coef] double layout with the
// scaling undone (debug export).
template <typename T>
cudaError_t launch_export_level(const T* src, const Level& lv, int what, double h, const int8_t* mi, int nc,
                                double* dst, cudaStream_t s);

// ---------------------------------------------------------------------------
// Tensor-core M2L (k_m2l_tc.cu).  The contraction of k_gemm_simt.cu with a
// tile of 128 parent boxes as the MMA M dimension, the output columns split
// into "groups" (one MMA N each, order-sorted so each group has one reduction
// prefix) and the reduction streamed as 128-byte chunks of one neighbour's
// row.  A operand: TMA tile of the (shifted) parent rows; B operand: a
// pre-swizzled weight tile per (neighbour, chunk, group).
constexpr int kTcMaxPasses = 4;        // passes of one launch (kernel parameter space)
constexpr int kTcMaxNearLaunches = 4;  // near-field launches of a plan
// 128 rows per tile as 8 (x) x 16 (y) x 1 (z): the activation stage is an
// 8 x 18 x 1 box (y halo of one row each side), in which the three y-shifts
// of a neighbour column are contiguous 128-row windows.
constexpr int kTcTileX = 8, kTcTileY = 16, kTcTileZ = 1;
constexpr int kTcBoxY = kTcTileY + 2;
constexpr int kTcMaxGroupN = 128;                         // B tile <= 128 rows

enum TcKind { TC_BF16X3 = 0, TC_TF32 = 1 };

constexpr int kTcIssuers = 4;       // MMA-issuing threads per CTA, each with its own weight ring
constexpr int kTcMaxGroups = 12;    // output column groups per pass
constexpr int kTcMaxChunks = 48;    // 128-byte reduction chunks per neighbour
constexpr int kTcMaxSpans = 128;    // MMA spans per pass (all chunks)
constexpr int kTcMaxSpanN = 128;    // columns of one span (one MMA instruction)
constexpr int kTcMaxColMap = 96;    // reduced coefficients of a column map ((p+1)^2, p <= 8)
// Shared memory of the tensor-core kernel: barriers (2 KB), then the
// activation stages (one 144-row box per plane, 18 KB a plane), then the
// weight rings, which take what the stages leave.  4 KB short of the SM's
// 228 KB so that CUDA-core blocks of the concurrent FP64 levels (no shared
// memory, 1 KB reserved each) fit beside a tensor-core CTA: its 13 warps
// leave half the register file and the DFMA units idle (8.6 vs 9.8 ms per
// 512^3 bf16x3 step against 226 KB).
constexpr int kTcSmemUsable = 222 * 1024;
constexpr int kTcMaxAStages = 8;
constexpr int kTcAPlaneBytes = kTcTileX * kTcBoxY * 128;
inline int tc_ring_budget(int kind, int a_stages) {
  return kTcSmemUsable - 2048 - a_stages * kTcAPlaneBytes * (kind == 0 ? 2 : 1);
}

// One MMA instruction shape of a chunk: adjacent column groups that use the
// chunk with the same number of K steps, merged so that each tcgen05.mma
// carries as many columns as possible (an MMA costs at least ~55 issue
// cycles, i.e. the math of N = 110 bf16 columns).
struct TcSpan {
  int tmem_col;    // first TMEM column
  int n;           // MMA N (rows of the weight tile per plane)
  int ksteps;      // MMA K steps in this chunk (1..4)
  int w_off;       // byte offset of the tile inside the neighbour block
  uint32_t idesc;  // instruction descriptor (kind, N, M = 128)
  int first;       // chunk in which the span's accumulators open (first MMA overwrites)
  int prod;        // bf16x3 products: 0 all three (hi and lo weight planes in the tile);
                   // 1 A_hi x B (B = hi plane), 2 A_hi x B (B = lo plane), 3 A_lo x B (B = hi plane);
                   // 4 A_hi x [B_hi; B_lo]: one MMA of N = n over n/2 hi rows then n/2 lo rows
};

// One pass of the schedule, passed by value (kernel parameter space), so the
// producer and MMA threads never wait on a global load for their next step.
// Weight tiles: offset(d, span) = w_base + d * bytes_per_d + span.w_off; one
// tile = n rows x 128 B per plane (bf16 hi plane, then lo plane).
struct TcPass {
  int ng, nchunks, tmem_cols, bytes_per_d;
  // neighbour columns (dx, dz) per accumulation segment (1..9): after each
  // segment the epilogue drains the accumulators into C (FP32, rounded to
  // nearest) and the next segment reopens them
  int seg_xz;
  long long w_base;
  int out_tmem[kTcMaxGroups];   // epilogue: TMEM column of the group's accumulator
  int out_tmem2[kTcMaxGroups];  // second accumulator (reduction- or product-split group), or -1
  int out_tmem3[kTcMaxGroups];  // third accumulator (product-split group), or -1
  int out_tmem4[kTcMaxGroups];  // second half of a product-split group's hi*hi reduction, or -1
  int out_col0[kTcMaxGroups];   // first output column (beta*8 + child)
  int out_ncols[kTcMaxGroups];  // real output columns
  int out_nmma[kTcMaxGroups];   // TMEM columns of the group (multiple of 16)
  // Accumulators are shared out between kTcIssuers MMA issuers (disjoint TMEM
  // columns).  Spans of issuer q in chunk j: span[span_idx[j][q] ..
  // span_idx[j][q + 1]); span_idx[j][kTcIssuers] == span_idx[j + 1][0].
  int span_idx[kTcMaxChunks + 1][kTcIssuers + 1];
  int ring_bytes[kTcIssuers];   // weight ring of each issuer (multiples of 1024, sum <= the ring budget)
  TcSpan span[kTcMaxSpans];
};
struct TcLaunch {
  TcPass pass[kTcMaxPasses];
  int npass;
  int a_stages;    // activation stages in flight (2 .. kTcMaxAStages)
  const unsigned char* W;
  float* C;        // [parents][n_cols]
  int n_cols;
  int accumulate;  // 1: C += result, 0: C = result
  int grid[3];     // parent grid
  int kind;
  int* err;
  // col_mapped = 1: output column n (a reduced coefficient r = n / 8, child
  // n % 8) lands in C column col_map[r] * 8 + n % 8 (harmonic M2L: the full
  // local rows receive the c <= 1 components)
  int col_mapped;
  int16_t col_map[kTcMaxColMap];
};

// Builds a 4-D TMA map over one level's parent-blocked rows (one plane).
cudaError_t make_row_map(void* map_out /* CUtensorMap */, const void* base, int row_len, int elem_bytes,
                         const int grid[3], int box_inner);
cudaError_t launch_m2l_tc(const TcLaunch& L, const void* map_hi, const void* map_lo, cudaStream_t s);

// ---------------------------------------------------------------------------
// Prefix-schedule tensor-core contraction (k_nbr_tc.cu): the same neighbour
// contraction, with output columns ordered so that every K step of the
// reduction (16 bf16 or 8 TF32 values) is needed by a prefix of them.  One
// tile (128 rows) keeps all its output columns in one accumulator set, so a
// K step is one MMA per product and 128-column chunk of that prefix instead
// of one per column group:
//   * D: the accumulators of every output column (hi*hi, lo*hi, hi*lo);
//   * E (TMEM columns [0, e), before D): "fused" K steps with a narrow
//     prefix issue hi*hi and hi*lo as one MMA of 2N columns over a weight
//     block [lo rows reversed; hi rows], whose first N columns land in E
//     (E column c holds output column e - 1 - c) and the last N in D;
//   * L2: the K steps from a split point on accumulate in a region of their
//     own (or, with no such split, the fused steps' lo*hi), so that no FP32
//     accumulator takes more than about half of the long low-order sums (the
//     tensor cores add with truncation).
// The epilogue adds D, E and L2 in a fixed order.  Every accumulator column
// has one issuing thread ("owner": 128-column chunks of D, E with the first
// chunk, L2 apart), so each column sums its products in a fixed order and
// results are bit-reproducible.  Weights stream as pieces (<= 16 KB, never
// across a reduction chunk, each read by one owner only) copied by
// kTpWLanes threads: bulk copies issued by one thread complete one after
// another.
constexpr int kTpMaxPasses = 4;
constexpr int kTpMaxChunks = 48;
constexpr int kTpMaxPieces = 256;
constexpr int kTpMaxUnits = 1024;
constexpr int kTpMaxGroups = 48;
constexpr int kTpIssuers = 4;
constexpr int kTpWLanes = 4;  // copy lanes of one owner's producer warp
constexpr int kTpALanes = 4;
constexpr int kTpPieceBytes = 16384;
constexpr int kTpMaxSlots = 16;
constexpr int kTpMaxAStages = 4;

// One unit of a column program: the MMAs that read one weight block of one
// K step, 32 bits:
//   bits 0-4    block offset in its piece / 512
//   bits 5-6    K step in the activation chunk
//   bits 7-8    dy (activation window)
//   bits 9-10   form: 0 three products (hi rows, then lo rows: hi*hi, lo*hi,
//               hi*lo into columns tcol..), 1 fused (lo rows reversed, then
//               hi rows: hi*[lo; hi] over 2N columns from tcol, then lo*hi
//               into tcol2), 2 one product (TF32)
//   bits 11-15  TMEM column / 16 of the (first) MMA
//   bits 16-20  N / 16
//   bits 21-25  form 1: TMEM column / 16 of the lo*hi MMA
inline constexpr uint32_t tp_unit(int b_off, int ks, int dy, int form, int tcol, int n, int tcol2) {
  return (uint32_t)(b_off >> 9) | ((uint32_t)ks << 5) | ((uint32_t)dy << 7) | ((uint32_t)form << 9) |
         ((uint32_t)(tcol >> 4) << 11) | ((uint32_t)(n >> 4) << 16) | ((uint32_t)(tcol2 >> 4) << 21);
}

struct TpPass {
  int nchunks;        // 128-byte activation chunks per neighbour row
  int npieces;        // weight pieces per (dx, dz) neighbour column
  int tmem_cols;      // TMEM columns of one accumulator set (E + D + L2, multiple of 16)
  int nbuf;           // accumulator sets (2 when they fit in 512 columns)
  int ngroups;        // 16-column output groups
  int col0, ncols;    // output columns [col0, col0 + ncols) of the full row
  long long w_base;   // bytes: pieces of this pass, [dx, dz column][piece] x kTpPieceBytes
  int16_t chunk_piece[kTpMaxChunks + 1];  // pieces of chunk j: [chunk_piece[j], chunk_piece[j + 1])
  int16_t piece_unit[kTpMaxPieces + 1];   // units of piece k: [piece_unit[k], piece_unit[k + 1])
  uint16_t piece_len16[kTpMaxPieces];     // bytes of piece k / 16
  int8_t piece_owner[kTpMaxPieces];       // issuer that reads piece k
  // epilogue: group g = output columns col0 + 16 g ..: TMEM column of its D
  // accumulators, of its reversed E accumulators (column grp_e[g] + 15 - i
  // holds column 16 g + i) and of its L2 accumulators; -1 when absent
  int16_t grp_d[kTpMaxGroups], grp_e[kTpMaxGroups], grp_l2[kTpMaxGroups];
  uint32_t unit[kTpMaxUnits];
};

struct TpLaunch {
  TpPass pass[kTpMaxPasses];
  int npass;
  int a_stages;   // activation stages (2 .. kTpMaxAStages)
  int w_slots;    // weight ring slots of kTpPieceBytes (<= kTpMaxSlots)
  // each issuer ("owner") has a ring of its own: slots [owner_slot0[q],
  // owner_slot0[q] + owner_nslots[q]), the same for every pass, filled by a
  // producer warp of its own in the owner's piece order
  int8_t owner_slot0[kTpIssuers], owner_nslots[kTpIssuers];
  const unsigned char* W;
  float* C;       // [rows][n_cols]
  int n_cols;
  int accumulate; // 1: C += result, 0: C = result
  int grid[3];    // row grid
  int kind;       // TC_BF16X3 or TC_TF32
  int* err;
  int col_mapped; // as TcLaunch
  int skip_first_a; // test hook: every CTA leaves its first activation stage unloaded (its waits time out)
  int16_t col_map[kTcMaxColMap];
};

// Shared memory of the prefix-schedule kernel for a stage count / kind.
inline int tp_smem_budget() { return kTcSmemUsable; }
inline int tp_w_slots(int kind, int a_stages) {
  const int left = kTcSmemUsable - 2048 - a_stages * kTcAPlaneBytes * (kind == 0 ? 2 : 1);
  const int s = left / kTpPieceBytes;
  return s > kTpMaxSlots ? kTpMaxSlots : s;
}
cudaError_t launch_nbr_tc(const TpLaunch& L, const void* map_hi, const void* map_lo, cudaStream_t s);

}  // namespace fmmgb
