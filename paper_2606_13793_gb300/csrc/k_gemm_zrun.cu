// Neighbour contraction on the CUDA cores, register z-run variant.
//
// Same contraction as k_gemm_simt.cu (M2L of Sec. 2.3 and the near-field
// P2P sum, both as C[r][n] (+)= sum_d sum_k A[r+d][k] W_d[k][n] over the 27
// neighbours d of a 3-D row grid), organised so that one load of A feeds the
// three neighbours that differ only in dz:
//
//  * a CTA covers BX x BY x RZ rows (BX = 8 lanes along x, BY = 4 warps along
//    y, RZ rows along z held by every thread) and one 32-column weight tile;
//    each thread owns RZ rows (a z-run) x 8 columns of the output;
//  * per reduction stage of 8 values the CTA stages the A halo
//    (BX+2) x (BY+2) x (RZ+2) once, and the weights of the neighbours it
//    handles; for each (dx, dy) the thread reads RZ+2 halo values along z
//    and applies them to the dz = -1, 0, +1 weights, i.e. 3 * RZ * 8 FMAs per
//    RZ + 2 scalar and 6 vector shared-memory loads;
//  * the nine (dx, dy) pairs may be split over 3 or 9 CTAs (blockIdx.z) that
//    write partial sums, reduced afterwards in a fixed order.
//
// A neighbour row outside the grid reads zero: the isolated boundary.
#include "fmm_internal.h"
#include "multi.cuh"

namespace fmmgb {
namespace {

constexpr int kZrKC = 8;       // reduction values per stage
constexpr int kZrThreads = 128;
constexpr int kZrCT = 8;       // output columns per thread
constexpr int kZrCG = kNTile / kZrCT;  // column groups (4)
constexpr int kZrBX = 32 / kZrCG;      // x extent of a warp (8)
constexpr int kZrBY = kZrThreads / 32; // y extent of the CTA (4 warps)

template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec<double> {
  using type = double2;
  static constexpr int n = 2;
};

// Packed FP32 multiply-add (two lanes of IEEE fma, round to nearest: the
// same results as two scalar fmaf): one instruction for two products halves
// the issue slots of the FP32 kernel, which the scalar form spent almost
// entirely on FMAs and shared-memory loads.
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long f2_splat(float a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}

template <int RZ>
struct ZrHalo {
  static constexpr int hx = kZrBX + 2, hy = kZrBY + 2, hz = RZ + 2;
  static constexpr int rows = hx * hy * hz;
  static constexpr int stride = ((rows + 7) / 8) * 8 + 4;  // per reduction value, staggers the stage stores
};

template <typename T, int RZ>
constexpr size_t zrun_smem_bytes() {
  return sizeof(T) * ((size_t)kZrKC * ZrHalo<RZ>::stride + (size_t)27 * kZrKC * kNTile);
}

template <typename T, int RZ>
__device__ __forceinline__ void nbr_gemm_zrun_body(const NbrGemm& g, const VBlock vb) {
  using H = ZrHalo<RZ>;
  using V = typename Vec<T>::type;
  constexpr int VN = Vec<T>::n;
  extern __shared__ __align__(16) unsigned char zr_smem[];
  T* As = reinterpret_cast<T*>(zr_smem);  // [kZrKC][H::stride]
  T* Ws = As + kZrKC * H::stride;          // [3 * nxy][kZrKC][kNTile]

  const int t = threadIdx.x;
  const int cg = t % kZrCG, xr = (t / kZrCG) % kZrBX, yr = t / 32;
  const int ntx = (g.grid[0] + kZrBX - 1) / kZrBX, nty = (g.grid[1] + kZrBY - 1) / kZrBY;
  const int bt = vb.x;
  const int ox = (bt % ntx) * kZrBX, oy = ((bt / ntx) % nty) * kZrBY, oz = (bt / (ntx * nty)) * RZ;
  const int tile = vb.y;
  const int K = g.tile_k[tile];
  const T* W0 = static_cast<const T*>(g.W) + g.tile_w[tile];
  const T* A = static_cast<const T*>(g.A);
  const int nxy = 9 / g.dsplit;  // (dx, dy) pairs of this CTA
  const int xy0 = (g.dsplit > 1 ? (int)vb.z : 0) * nxy;

  constexpr bool kPacked = sizeof(T) == 4;  // FP32: column pairs in packed registers
  T acc[RZ][kZrCT];
  unsigned long long acc2[kPacked ? RZ : 1][kZrCT / 2];
#pragma unroll
  for (int z = 0; z < RZ; ++z)
#pragma unroll
    for (int c = 0; c < kZrCT; ++c) acc[z][c] = T(0);
#pragma unroll
  for (int z = 0; z < (kPacked ? RZ : 1); ++z)
#pragma unroll
    for (int c = 0; c < kZrCT / 2; ++c) acc2[z][c] = 0ull;  // +0.0f in both lanes

  for (int kc = 0; kc < K; kc += kZrKC) {
    // A halo, one vector of VN reduction values per load
    constexpr int PER_ROW = kZrKC / VN;
    for (int e = t; e < H::rows * PER_ROW; e += kZrThreads) {
      const int h = e / PER_ROW, q = e % PER_ROW;
      const int hx = h % H::hx, hy = (h / H::hx) % H::hy, hz = h / (H::hx * H::hy);
      const int x = ox + hx - 1, y = oy + hy - 1, z = oz + hz - 1;
      V v;
      T* pv = reinterpret_cast<T*>(&v);
#pragma unroll
      for (int i = 0; i < VN; ++i) pv[i] = T(0);
      if (x >= 0 && y >= 0 && z >= 0 && x < g.grid[0] && y < g.grid[1] && z < g.grid[2] && kc + q * VN < K)
        v = __ldg(reinterpret_cast<const V*>(A + (((long long)z * g.grid[1] + y) * g.grid[0] + x) * g.row_len +
                                             kc + q * VN));
#pragma unroll
      for (int i = 0; i < VN; ++i) As[(q * VN + i) * H::stride + h] = pv[i];
    }
    // weights of neighbours d = dz * 9 + xy for this CTA's (dx, dy) pairs
    constexpr int BLK = kZrKC * kNTile / VN;
    for (int e = t; e < 3 * nxy * BLK; e += kZrThreads) {
      const int blk = e / BLK, w = e % BLK;
      const int d = (blk % 3) * 9 + xy0 + blk / 3;
      reinterpret_cast<V*>(Ws)[e] =
          __ldg(reinterpret_cast<const V*>(W0 + (long long)d * K * kNTile + (long long)kc * kNTile) + w);
    }
    __syncthreads();
    for (int j = 0; j < nxy; ++j) {
      const int xy = xy0 + j;
      const int dxo = xy % 3, dyo = xy / 3;  // offsets + 1
      const T* Ab = As + (yr + dyo) * H::hx + (xr + dxo);
      const T* Wb = Ws + (j * 3) * kZrKC * kNTile + cg * kZrCT;
#pragma unroll 2
      for (int k = 0; k < kZrKC; ++k) {
        T a[RZ + 2];
#pragma unroll
        for (int zz = 0; zz < RZ + 2; ++zz) a[zz] = Ab[k * H::stride + zz * H::hx * H::hy];
        if constexpr (kPacked) {
          unsigned long long a2[RZ + 2];
#pragma unroll
          for (int zz = 0; zz < RZ + 2; ++zz) a2[zz] = f2_splat(a[zz]);
#pragma unroll
          for (int dz = 0; dz < 3; ++dz) {
            if (dz == 1 && xy == 4 && g.skip_center) continue;  // the centre block is zero
            const ulonglong2* wv = reinterpret_cast<const ulonglong2*>(Wb + (dz * kZrKC + k) * kNTile);
            const ulonglong2 w0 = wv[0], w1 = wv[1];  // columns (0,1) (2,3) | (4,5) (6,7)
            const unsigned long long b2[4] = {w0.x, w0.y, w1.x, w1.y};
#pragma unroll
            for (int z = 0; z < RZ; ++z)
#pragma unroll
              for (int c = 0; c < kZrCT / 2; ++c) acc2[z][c] = f2_fma(a2[z + dz], b2[c], acc2[z][c]);
          }
        } else {
#pragma unroll
          for (int dz = 0; dz < 3; ++dz) {
            if (dz == 1 && xy == 4 && g.skip_center) continue;  // the centre block is zero
            T b[kZrCT];
            const V* wv = reinterpret_cast<const V*>(Wb + (dz * kZrKC + k) * kNTile);
#pragma unroll
            for (int i = 0; i < kZrCT / VN; ++i) *reinterpret_cast<V*>(&b[i * VN]) = wv[i];
#pragma unroll
            for (int z = 0; z < RZ; ++z)
#pragma unroll
              for (int c = 0; c < kZrCT; ++c) acc[z][c] = fma(a[z + dz], b[c], acc[z][c]);
          }
        }
      }
    }
    __syncthreads();
  }

  if constexpr (kPacked) {
#pragma unroll
    for (int z = 0; z < RZ; ++z)
#pragma unroll
      for (int c = 0; c < kZrCT / 2; ++c) {
        const float2 v = f2_unpack(acc2[z][c]);
        acc[z][2 * c] = v.x;
        acc[z][2 * c + 1] = v.y;
      }
  }
  const int col0 = tile * kNTile + cg * kZrCT;
  if (col0 >= g.n_cols) return;
  const int x = ox + xr, y = oy + yr;
  if (x >= g.grid[0] || y >= g.grid[1]) return;
  const long long rows = (long long)g.grid[0] * g.grid[1] * g.grid[2];
  T* Pz = g.dsplit > 1 ? static_cast<T*>(g.partial) + (long long)vb.z * rows * g.n_cols : nullptr;
  T* C = static_cast<T*>(g.C);
#pragma unroll
  for (int z = 0; z < RZ; ++z) {
    const int zz = oz + z;
    if (zz >= g.grid[2]) break;
    const long long row = ((long long)zz * g.grid[1] + y) * g.grid[0] + x;
    V* dst = reinterpret_cast<V*>((Pz ? Pz : C) + row * g.n_cols + col0);
#pragma unroll
    for (int i = 0; i < kZrCT / VN; ++i) {
      V v;
      T* pv = reinterpret_cast<T*>(&v);
      if (!Pz && g.accumulate) v = dst[i];
#pragma unroll
      for (int q = 0; q < VN; ++q) pv[q] = (!Pz && g.accumulate) ? pv[q] + acc[z][i * VN + q] : acc[z][i * VN + q];
      dst[i] = v;
    }
  }
}

template <typename T, int RZ>
__global__ void __launch_bounds__(kZrThreads, 4) nbr_gemm_zrun_kernel(NbrGemm g) {
  nbr_gemm_zrun_body<T, RZ>(g, native_vblock());
}

template <typename T, int RZ>
__global__ void __launch_bounds__(kZrThreads, 4) nbr_gemm_zrun_multi_kernel(const NbrGemm* __restrict__ gs,
                                                                         const MultiGrid* __restrict__ grids, int n) {
  __shared__ NbrGemm g;  // the item's description, read by the body from shared memory
  const int i = multi_item(grids, n);
  if (threadIdx.x == 0) g = gs[i];
  __syncthreads();
  nbr_gemm_zrun_body<T, RZ>(g, multi_vblock(grids[i]));
}

template <typename T, int RZ>
cudaError_t launch_rz_multi(const NbrGemm* gs, const MultiGrid* grids, int n, long long blocks, cudaStream_t s) {
  constexpr size_t smem = zrun_smem_bytes<T, RZ>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(nbr_gemm_zrun_multi_kernel<T, RZ>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (n <= 0 || blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  nbr_gemm_zrun_multi_kernel<T, RZ><<<(unsigned)blocks, kZrThreads, smem, s>>>(gs, grids, n);
  return cudaGetLastError();
}

template <typename T, int RZ>
cudaError_t launch_rz(const NbrGemm& g, cudaStream_t s) {
  constexpr size_t smem = zrun_smem_bytes<T, RZ>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(nbr_gemm_zrun_kernel<T, RZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const long long tiles = (long long)((g.grid[0] + kZrBX - 1) / kZrBX) * ((g.grid[1] + kZrBY - 1) / kZrBY) *
                          ((g.grid[2] + RZ - 1) / RZ);
  if (tiles <= 0 || g.ntiles <= 0) return cudaSuccess;
  if (tiles > 0x7fffffffLL || g.ntiles > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)tiles, (unsigned)g.ntiles, (unsigned)g.dsplit);
  nbr_gemm_zrun_kernel<T, RZ><<<grid, kZrThreads, smem, s>>>(g);
  return cudaGetLastError();
}

}  // namespace

// z-run lengths of the two tile shapes per precision
template <typename T>
constexpr int zrun_rz(int which);
template <>
constexpr int zrun_rz<float>(int which) {
  return which == 0 ? 8 : which == 1 ? 4 : 6;
}
template <>
constexpr int zrun_rz<double>(int which) {
  return which == 0 ? 4 : which == 1 ? 2 : 3;
}

bool zrun_eligible(const NbrGemm& g, const int* tile_k_host, int ntiles) {
  if (g.row_len % kZrKC != 0 || g.n_cols % kZrCT != 0) return false;
  if (g.dsplit != 1 && g.dsplit != 3 && g.dsplit != 9) return false;
  for (int i = 0; i < ntiles; ++i)
    if (tile_k_host[i] % kZrKC != 0) return false;
  return true;
}

template <typename T>
cudaError_t launch_nbr_gemm_zrun(const NbrGemm& g, int shape, cudaStream_t s) {
  cudaError_t e = shape == 0 ? launch_rz<T, zrun_rz<T>(0)>(g, s) : launch_rz<T, zrun_rz<T>(1)>(g, s);
  if (e != cudaSuccess || g.dsplit <= 1) return e;
  return launch_reduce_partials<T>(static_cast<const T*>(g.partial), g.dsplit,
                                   (long long)g.grid[0] * g.grid[1] * g.grid[2] * g.n_cols, static_cast<T*>(g.C),
                                   g.accumulate, s);
}

template <typename T>
void nbr_gemm_zrun_grid(const NbrGemm& g, int shape, unsigned out[3]) {
  const int rz = zrun_rz<T>(shape);
  out[0] = (unsigned)((long long)((g.grid[0] + kZrBX - 1) / kZrBX) * ((g.grid[1] + kZrBY - 1) / kZrBY) *
                      ((g.grid[2] + rz - 1) / rz));
  out[1] = (unsigned)g.ntiles;
  out[2] = (unsigned)g.dsplit;
}

template <typename T>
cudaError_t launch_nbr_gemm_zrun_multi(int shape, const NbrGemm* gs, const MultiGrid* grids, int n, long long blocks,
                                       cudaStream_t s) {
  return shape == 0   ? launch_rz_multi<T, zrun_rz<T>(0)>(gs, grids, n, blocks, s)
         : shape == 1 ? launch_rz_multi<T, zrun_rz<T>(1)>(gs, grids, n, blocks, s)
                      : launch_rz_multi<T, zrun_rz<T>(2)>(gs, grids, n, blocks, s);
}

template void nbr_gemm_zrun_grid<float>(const NbrGemm&, int, unsigned[3]);
template void nbr_gemm_zrun_grid<double>(const NbrGemm&, int, unsigned[3]);
template cudaError_t launch_nbr_gemm_zrun_multi<float>(int, const NbrGemm*, const MultiGrid*, int, long long,
                                                       cudaStream_t);
template cudaError_t launch_nbr_gemm_zrun_multi<double>(int, const NbrGemm*, const MultiGrid*, int, long long,
                                                        cudaStream_t);
template cudaError_t launch_nbr_gemm_zrun<float>(const NbrGemm&, int, cudaStream_t);
template cudaError_t launch_nbr_gemm_zrun<double>(const NbrGemm&, int, cudaStream_t);

}  // namespace fmmgb
