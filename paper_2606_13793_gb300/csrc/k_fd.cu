// Force by finite differences (App. C): a = -grad(phi) with the 4th-order
// 5-point central stencil, 2nd-order central one cell from an edge and
// 2nd-order one-sided at an edge; and the transpose of that map for the
// adjoint solve.  HBM-bound.  The force kernels walk z through tiles of the
// x-y plane (z neighbours in registers, x-y neighbours from a shared-memory
// tile with a 2-cell halo): fd_accel_vec4_kernel for FP32 rows with 16-byte
// alignment (four x-cells a thread), fd_accel_tiled_kernel otherwise, and a
// plain one-thread-per-cell kernel for grids past the launch limits.  The
// adjoint source kernel is one thread per cell, x fastest.
#include "fmm_internal.h"
#include "multi.cuh"

namespace fmmgb {
namespace {

// Weight of f[j + off] in the cell-unit derivative at index j of a line of
// n, in the arithmetic type of the data (no FP64 work on FP32 data).
template <typename T>
__device__ __forceinline__ T fd_weight(int j, int off, int n) {
  if (n <= 1) return T(0);
  if (n == 2) {  // f[1] - f[0] at both points
    const int m = j + off;
    return m == 1 ? T(1) : (m == 0 ? T(-1) : T(0));
  }
  if (j >= 2 && j <= n - 3) {
    switch (off) {
      case 2: return T(-1) / T(12);
      case 1: return T(8) / T(12);
      case -1: return T(-8) / T(12);
      case -2: return T(1) / T(12);
      default: return T(0);
    }
  }
  if (j >= 1 && j <= n - 2) return off == 1 ? T(0.5) : (off == -1 ? T(-0.5) : T(0));
  if (j == 0) return off == 0 ? T(-1.5) : (off == 1 ? T(2) : (off == 2 ? T(-0.5) : T(0)));
  return off == 0 ? T(1.5) : (off == -1 ? T(-2) : (off == -2 ? T(0.5) : T(0)));  // j == n-1
}

constexpr int kFdTX = 32, kFdTY = 8, kFdZC = 32;

// 32 x 8 columns of cells per block, walking kFdZC cells along z: the z
// neighbours come from a 5-value register window per column, the x-y
// neighbours from a shared-memory tile with a 2-cell halo whose centre is the
// window's middle value (only the halo is read from memory); the tile is
// double-buffered, so one barrier per plane.
template <typename T>
__global__ void __launch_bounds__(kFdTX* kFdTY) fd_accel_tiled_kernel(const T* __restrict__ phi, int nx, int ny,
                                                                      int nz, T inv_dx, T* __restrict__ accel) {
  constexpr int HX = kFdTX + 4, HY = kFdTY + 4;
  constexpr int kHalo = HX * HY - kFdTX * kFdTY;  // 176 halo cells per plane
  __shared__ T tile[2][HY][HX];
  const long long n = (long long)nx * ny * nz;
  const long long plane = (long long)nx * ny;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * kFdTX + tx;
  const int x0 = blockIdx.x * kFdTX, y0 = blockIdx.y * kFdTY, z0 = blockIdx.z * kFdZC;
  const int x = x0 + tx, y = y0 + ty;
  const bool inside = x < nx && y < ny;
  const long long col = (long long)y * nx + x;
  // halo cell of this thread (threads 0 .. kHalo-1): the tile's two-cell frame
  int hx = 0, hy = 0;
  long long hoff = -1;
  if (tid < kHalo) {
    int r = tid;
    if (r < 2 * HX) {
      hy = r / HX, hx = r % HX;  // top two rows
    } else if ((r -= 2 * HX) < 2 * HX) {
      hy = HY - 2 + r / HX, hx = r % HX;  // bottom two rows
    } else {
      r -= 2 * HX;  // side columns of the middle rows: 4 per row
      hy = 2 + r / 4;
      const int c = r % 4;
      hx = c < 2 ? c : kFdTX + c;
    }
    const int gx = x0 - 2 + hx, gy = y0 - 2 + hy;
    if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) hoff = (long long)gy * nx + gx;
  }
  T wx[5], wy[5];
#pragma unroll
  for (int o = -2; o <= 2; ++o) {
    wx[o + 2] = fd_weight<T>(x, o, nx);
    wy[o + 2] = fd_weight<T>(y, o, ny);
  }
  T w[5];  // phi at z-2 .. z+2 of this column
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int zz = z0 - 2 + q;
    w[q + 1] = (inside && zz >= 0 && zz < nz) ? phi[(long long)zz * plane + col] : T(0);
  }
  const int z1 = min(z0 + kFdZC, nz);
  for (int z = z0; z < z1; ++z) {
    const int buf = (z - z0) & 1;
#pragma unroll
    for (int q = 0; q < 4; ++q) w[q] = w[q + 1];
    w[4] = (inside && z + 2 < nz) ? phi[(long long)(z + 2) * plane + col] : T(0);
    tile[buf][ty + 2][tx + 2] = w[2];
    if (tid < kHalo) tile[buf][hy][hx] = hoff >= 0 ? phi[(long long)z * plane + hoff] : T(0);
    __syncthreads();
    if (inside) {
      T dx = T(0), dy = T(0), dz = T(0);
#pragma unroll
      for (int o = -2; o <= 2; ++o) {
        dx = fma(wx[o + 2], tile[buf][ty + 2][tx + 2 + o], dx);
        dy = fma(wy[o + 2], tile[buf][ty + 2 + o][tx + 2], dy);
        dz = fma(fd_weight<T>(z, o, nz), w[o + 2], dz);
      }
      const long long c = (long long)z * plane + col;
      accel[c] = -dx * inv_dx;
      accel[n + c] = -dy * inv_dx;
      accel[2 * n + c] = -dz * inv_dx;
    }
    // the next plane writes the other buffer; the one after this waits for
    // the barrier above of the next iteration
  }
}

// FP32 with nx % 4 == 0: the same walk with four x-cells a thread (16-byte
// loads and stores, a 128 x 8 tile), and every global load issued one plane
// ahead of its use (the column's next z value and this thread's share of the
// next plane's halo), so each warp keeps several loads in flight instead of
// waiting on one per plane.  Halo: the two rows above and below the tile
// (float4, no corners: the stencil is a cross) and two cells left and right
// of each tile row.
constexpr int kFd4TX = 4 * kFdTX;  // cells per tile row
__device__ __forceinline__ void fd_accel_vec4_body(const float* __restrict__ phi, int nx, int ny, int nz,
                                                  float inv_dx, float* __restrict__ accel, const VBlock& vb) {
  constexpr int HX = kFd4TX + 8, HY = kFdTY + 4, C0 = 4;  // tile row: halo at C0-2, C0-1 and C0+128, C0+129
  __shared__ __align__(16) float tile[2][HY][HX];
  const long long n = (long long)nx * ny * nz;
  const long long plane = (long long)nx * ny;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * kFdTX + tx;
  const int x0 = vb.x * kFd4TX, y0 = vb.y * kFdTY, z0 = vb.z * kFdZC;
  const int x = x0 + 4 * tx, y = y0 + ty;
  const bool inside = x < nx && y < ny;  // nx % 4 == 0: all four cells
  const long long col = (long long)y * nx + x;
  // halo role: tid < 128 one float4 of a halo row, 128 <= tid < 160 one side cell
  int hr = -1, hc = 0;
  long long hoff = -1;
  if (tid < 4 * kFdTX) {
    const int r = tid / kFdTX, cx = 4 * (tid % kFdTX);
    const int gy = r < 2 ? y0 - 2 + r : y0 + kFdTY + (r - 2);
    hr = r < 2 ? r : kFdTY + r;
    hc = C0 + cx;
    if (gy >= 0 && gy < ny && x0 + cx < nx) hoff = (long long)gy * nx + x0 + cx;
  } else if (tid < 4 * kFdTX + 4 * kFdTY) {
    const int r = tid - 4 * kFdTX, row = r / 4, c = r % 4;
    const int gx = c < 2 ? x0 - 2 + c : x0 + kFd4TX + (c - 2), gy = y0 + row;
    hr = row + 2;
    hc = c < 2 ? C0 - 2 + c : C0 + kFd4TX + (c - 2);
    if (gx >= 0 && gx < nx && gy < ny) hoff = (long long)gy * nx + gx;
  }
  const bool hvec = tid < 4 * kFdTX;
  float wx[4][5], wy[5];
#pragma unroll
  for (int o = -2; o <= 2; ++o) {
    wy[o + 2] = fd_weight<float>(y, o, ny);
#pragma unroll
    for (int q = 0; q < 4; ++q) wx[q][o + 2] = fd_weight<float>(x + q, o, nx);
  }
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  auto load_col = [&](int zz) {
    return (inside && zz >= 0 && zz < nz) ? __ldg(reinterpret_cast<const float4*>(phi + (long long)zz * plane + col))
                                          : zero4;
  };
  auto load_halo = [&](int zz, float4& v4, float& v1) {
    v4 = zero4;
    v1 = 0.f;
    if (hoff < 0 || zz >= nz) return;
    if (hvec)
      v4 = __ldg(reinterpret_cast<const float4*>(phi + (long long)zz * plane + hoff));
    else
      v1 = __ldg(phi + (long long)zz * plane + hoff);
  };
  float4 w[5];  // z-2 .. z+2 of this thread's four columns
#pragma unroll
  for (int q = 0; q < 4; ++q) w[q + 1] = load_col(z0 - 2 + q);
  float4 nxt = load_col(z0 + 2);  // value for the window's top at the first plane
  float4 h4;
  float h1;
  load_halo(z0, h4, h1);
  const int z1 = min(z0 + kFdZC, nz);
  for (int z = z0; z < z1; ++z) {
    const int buf = (z - z0) & 1;
#pragma unroll
    for (int q = 0; q < 4; ++q) w[q] = w[q + 1];
    w[4] = nxt;
    nxt = load_col(z + 3);  // one plane ahead
    *reinterpret_cast<float4*>(&tile[buf][ty + 2][C0 + 4 * tx]) = w[2];
    if (hr >= 0) {
      if (hvec)
        *reinterpret_cast<float4*>(&tile[buf][hr][hc]) = h4;
      else
        tile[buf][hr][hc] = h1;
    }
    load_halo(z + 1, h4, h1);  // next plane's halo, in flight across the barrier
    __syncthreads();
    if (inside) {
      float wz[5];
#pragma unroll
      for (int o = -2; o <= 2; ++o) wz[o + 2] = fd_weight<float>(z, o, nz);
      const float wc[4][5] = {{w[0].x, w[1].x, w[2].x, w[3].x, w[4].x},
                              {w[0].y, w[1].y, w[2].y, w[3].y, w[4].y},
                              {w[0].z, w[1].z, w[2].z, w[3].z, w[4].z},
                              {w[0].w, w[1].w, w[2].w, w[3].w, w[4].w}};
      float ax[4], ay[4], az[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float dx = 0.f, dy = 0.f, dz = 0.f;
#pragma unroll
        for (int o = -2; o <= 2; ++o) {
          dx = fmaf(wx[q][o + 2], tile[buf][ty + 2][C0 + 4 * tx + q + o], dx);
          dy = fmaf(wy[o + 2], tile[buf][ty + 2 + o][C0 + 4 * tx + q], dy);
          dz = fmaf(wz[o + 2], wc[q][o + 2], dz);
        }
        ax[q] = -dx * inv_dx, ay[q] = -dy * inv_dx, az[q] = -dz * inv_dx;
      }
      const long long c = (long long)z * plane + col;
      *reinterpret_cast<float4*>(accel + c) = make_float4(ax[0], ax[1], ax[2], ax[3]);
      *reinterpret_cast<float4*>(accel + n + c) = make_float4(ay[0], ay[1], ay[2], ay[3]);
      *reinterpret_cast<float4*>(accel + 2 * n + c) = make_float4(az[0], az[1], az[2], az[3]);
    }
  }
}

__global__ void __launch_bounds__(kFdTX* kFdTY, 3) fd_accel_vec4_kernel(const float* __restrict__ phi, int nx, int ny,
                                                                     int nz, float inv_dx,
                                                                     float* __restrict__ accel) {
  fd_accel_vec4_body(phi, nx, ny, nz, inv_dx, accel, native_vblock());
}

// The stencils of many solves in one launch (batched solves; FP32 rows of a
// multiple of four cells, 16-byte aligned).
__global__ void __launch_bounds__(kFdTX* kFdTY, 3) fd_accel_vec4_multi_kernel(const FdArgs* __restrict__ a,
                                                                           const MultiGrid* __restrict__ g, int n) {
  __shared__ FdArgs x;  // the item's arguments, read by the body from shared memory
  const int i = multi_item(g, n);
  if (threadIdx.x == 0 && threadIdx.y == 0) x = a[i];
  __syncthreads();
  fd_accel_vec4_body(static_cast<const float*>(x.phi), x.nx, x.ny, x.nz, (float)x.inv_dx, static_cast<float*>(x.accel),
                     multi_vblock(g[i]));
}

// Grid: x blocks over a row, y = row index, z = slice (32-bit indexing).
template <typename T>
__global__ void fd_accel_kernel(const T* __restrict__ phi, int nx, int ny, int nz, T inv_dx, T* __restrict__ accel) {
  const long long n = (long long)nx * ny * nz;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= nx) return;
  const long long c = ((long long)z * ny + y) * nx + x;
  {
    const int pos[3] = {x, y, z};
    const int len[3] = {nx, ny, nz};
    const long long stride[3] = {1, nx, (long long)nx * ny};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      T d = T(0);
#pragma unroll
      for (int off = -2; off <= 2; ++off) {
        const int m = pos[q] + off;
        if (m < 0 || m >= len[q]) continue;
        const T w = fd_weight<T>(pos[q], off, len[q]);
        if (w != T(0)) d = fma(w, phi[c + off * stride[q]], d);
      }
      accel[q * n + c] = -d * inv_dx;
    }
  }
}

// w = gphi - inv_dx * FD^T(gaccel) (gather form of the transpose): the
// adjoint source of the loss through accel = -inv_dx FD phi.
template <typename T>
__global__ void adjoint_source_kernel(const T* __restrict__ gphi, const T* __restrict__ gacc, int nx, int ny, int nz,
                                      T inv_dx, T* __restrict__ out) {
  const long long n = (long long)nx * ny * nz;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= nx) return;
  const long long c = ((long long)z * ny + y) * nx + x;
  {
    T v = gphi ? gphi[c] : T(0);
    if (gacc) {
      const int pos[3] = {x, y, z};
      const int len[3] = {nx, ny, nz};
      const long long stride[3] = {1, nx, (long long)nx * ny};
      T t = T(0);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
#pragma unroll
        for (int off = -2; off <= 2; ++off) {
          const int j = pos[q] + off;  // stencil centre whose derivative reads this cell
          if (j < 0 || j >= len[q]) continue;
          const T w = fd_weight<T>(j, -off, len[q]);
          if (w != T(0)) t = fma(w, gacc[q * n + c + off * stride[q]], t);
        }
      }
      v = fma(-inv_dx, t, v);
    }
    out[c] = v;
  }
}

template <typename T>
__global__ void check_finite_kernel(const T* __restrict__ x, size_t n, int* flag) {
  int bad = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

unsigned blocks_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 16) b = 152LL * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

dim3 row_grid(const int dims[3], int threads) {
  return dim3((unsigned)((dims[0] + threads - 1) / threads), (unsigned)dims[1], (unsigned)dims[2]);
}

template <typename T>
cudaError_t launch_fd_accel(const T* phi, const int dims[3], double inv_dx, T* accel, cudaStream_t s) {
  if (dims[1] > 65535 * kFdTY || dims[2] > 65535 * kFdZC) {
    const int th = dims[0] >= 256 ? 256 : ((dims[0] + 31) / 32) * 32;
    fd_accel_kernel<T><<<row_grid(dims, th), th, 0, s>>>(phi, dims[0], dims[1], dims[2], (T)inv_dx, accel);
    return cudaGetLastError();
  }
  if (sizeof(T) == 4 && dims[0] % 4 == 0 && (reinterpret_cast<uintptr_t>(phi) & 15) == 0 &&
      (reinterpret_cast<uintptr_t>(accel) & 15) == 0) {
    dim3 grid((unsigned)((dims[0] + kFd4TX - 1) / kFd4TX), (unsigned)((dims[1] + kFdTY - 1) / kFdTY),
              (unsigned)((dims[2] + kFdZC - 1) / kFdZC));
    fd_accel_vec4_kernel<<<grid, dim3(kFdTX, kFdTY), 0, s>>>(reinterpret_cast<const float*>(phi), dims[0], dims[1],
                                                             dims[2], (float)inv_dx, reinterpret_cast<float*>(accel));
    return cudaGetLastError();
  }
  dim3 grid((unsigned)((dims[0] + kFdTX - 1) / kFdTX), (unsigned)((dims[1] + kFdTY - 1) / kFdTY),
            (unsigned)((dims[2] + kFdZC - 1) / kFdZC));
  fd_accel_tiled_kernel<T><<<grid, dim3(kFdTX, kFdTY), 0, s>>>(phi, dims[0], dims[1], dims[2], (T)inv_dx, accel);
  return cudaGetLastError();
}

cudaError_t launch_fd_accel_multi(const FdArgs* args, const MultiGrid* grids, int n, long long blocks,
                                  cudaStream_t s) {
  if (n == 0 || blocks == 0) return cudaSuccess;
  fd_accel_vec4_multi_kernel<<<(unsigned)blocks, dim3(kFdTX, kFdTY), 0, s>>>(args, grids, n);
  return cudaGetLastError();
}

void fd_multi_grid(const int dims[3], unsigned g[3]) {
  g[0] = (unsigned)((dims[0] + kFd4TX - 1) / kFd4TX);
  g[1] = (unsigned)((dims[1] + kFdTY - 1) / kFdTY);
  g[2] = (unsigned)((dims[2] + kFdZC - 1) / kFdZC);
}

template <typename T>
cudaError_t launch_adjoint_source(const T* gphi, const T* gaccel, const int dims[3], double inv_dx, T* out,
                                  cudaStream_t s) {
  const int th = dims[0] >= 256 ? 256 : ((dims[0] + 31) / 32) * 32;
  adjoint_source_kernel<T><<<row_grid(dims, th), th, 0, s>>>(gphi, gaccel, dims[0], dims[1], dims[2], (T)inv_dx, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_check_finite(const T* x, size_t count, int* flag, cudaStream_t s) {
  check_finite_kernel<T><<<blocks_for((long long)count), 256, 0, s>>>(x, count, flag);
  return cudaGetLastError();
}

template cudaError_t launch_fd_accel<float>(const float*, const int*, double, float*, cudaStream_t);
template cudaError_t launch_fd_accel<double>(const double*, const int*, double, double*, cudaStream_t);
template cudaError_t launch_adjoint_source<float>(const float*, const float*, const int*, double, float*, cudaStream_t);
template cudaError_t launch_adjoint_source<double>(const double*, const double*, const int*, double, double*,
                                                   cudaStream_t);
template cudaError_t launch_check_finite<float>(const float*, size_t, int*, cudaStream_t);
template cudaError_t launch_check_finite<double>(const double*, size_t, int*, cudaStream_t);

}  // namespace fmmgb
