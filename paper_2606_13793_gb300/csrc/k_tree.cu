// Upward/downward tree kernels on the CUDA cores: P2M, M2M, L2L and the leaf
// evaluation (L2P plus the near-field sum, scaled to physical units).
//
// One warp owns one box of the parent grid and its 8 children, so the
// parent-blocked arrays ([coef][child], 8*nc contiguous values) are read or
// written by a whole warp at once.  P2M and L2P are separable in x, y, z
// (the monomial (x-c)^alpha factorises per axis), which cuts their cost from
// b^3 * nc to about b^3 * (p+1) * 3 multiply-adds per box.
#include "fmm_internal.h"

namespace fmmgb {
namespace {

constexpr int kWarpsPerBlock = 4;

// Index of multi-index (a, b, c) in the canonical order (total order n, then
// a descending, then b descending).
__device__ __forceinline__ int coef_index(int a, int b, int c) {
  const int n = a + b + c;
  return n * (n + 1) * (n + 2) / 6 + (n - a) * (n - a + 1) / 2 + (n - a - b);
}

// True when the shift term of parity `mask` changes sign for this child
// (an odd power of a negative half-offset).
__device__ __forceinline__ bool shift_neg(int mask, int child) { return __popc(mask & ~child & 7) & 1; }

template <typename T>
__device__ __forceinline__ T coef_of(const ShiftEntry& e);
template <>
__device__ __forceinline__ float coef_of<float>(const ShiftEntry& e) {
  return e.coef_f;
}
template <>
__device__ __forceinline__ double coef_of<double>(const ShiftEntry& e) {
  return e.coef;
}

// P2M (Sec. 2.1, eq. multipole) about each leaf-box centre, in scaled form
// Mt_alpha = sum_cells m ((x - c)/b)^alpha.  Also writes the box-blocked copy
// of the density the near-field contraction reads, and flags non-finite input.
template <typename T>
__global__ void p2m_kernel(TreeTables t, const T* __restrict__ rho, int nx, int ny, int nz, Level leaf,
                           T* __restrict__ Mleaf, T* __restrict__ rho_box) {
  extern __shared__ unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = t.b, p = t.p, nc = t.nc, P1 = p + 1, b3 = b * b * b;
  const long long par = (long long)blockIdx.x * kWarpsPerBlock + warp;
  const int per_warp = b3 + b * b * P1 + b * P1 * P1 + 8 * nc + b * P1;
  T* cells = reinterpret_cast<T*>(smem_raw) + (size_t)warp * per_warp;
  T* T1 = cells + b3;       // [k][j][a]
  T* T2 = T1 + b * b * P1;  // [k][a][bb]
  T* out = T2 + b * P1 * P1;
  T* xp = out + 8 * nc;     // [i][a] = ((i + 1/2)/b - 1/2)^a
  if (par >= leaf.npar) return;
  for (int e = lane; e < b * P1; e += 32) {
    const int i = e / P1, a = e % P1;
    const T x = (T(i) + T(0.5)) / T(b) - T(0.5);
    T v = T(1);
    for (int q = 0; q < a; ++q) v *= x;
    xp[e] = v;
  }
  const int px = (int)(par % leaf.np[0]);
  const int py = (int)((par / leaf.np[0]) % leaf.np[1]);
  const int pz = (int)(par / ((long long)leaf.np[0] * leaf.np[1]));
  __syncwarp();
  for (int c = 0; c < 8; ++c) {
    const int bx = 2 * px + (c & 1), by = 2 * py + ((c >> 1) & 1), bz = 2 * pz + (c >> 2);
    if (bx >= leaf.n[0] || by >= leaf.n[1] || bz >= leaf.n[2]) {
      for (int e = lane; e < nc; e += 32) out[e * 8 + c] = T(0);
      continue;
    }
    const long long box = ((long long)bz * leaf.n[1] + by) * leaf.n[0] + bx;
    for (int e = lane; e < b3; e += 32) {
      const int i = e % b, j = (e / b) % b, k = e / (b * b);
      const T v = rho[((long long)(bz * b + k) * ny + (by * b + j)) * nx + (bx * b + i)];
      cells[e] = v;
      rho_box[box * b3 + e] = v;
    }
    __syncwarp();
    for (int e = lane; e < b * b * P1; e += 32) {
      const int a = e % P1, jk = e / P1;  // jk = k*b + j
      T s = T(0);
      for (int i = 0; i < b; ++i) s = fma(cells[jk * b + i], xp[i * P1 + a], s);
      T1[e] = s;
    }
    __syncwarp();
    for (int e = lane; e < b * P1 * P1; e += 32) {
      const int bb = e % P1, a = (e / P1) % P1, k = e / (P1 * P1);
      T s = T(0);
      if (a + bb <= p)
        for (int j = 0; j < b; ++j) s = fma(T1[(k * b + j) * P1 + a], xp[j * P1 + bb], s);
      T2[e] = s;
    }
    __syncwarp();
    for (int e = lane; e < nc; e += 32) {
      const int a = t.mi[3 * e], bb = t.mi[3 * e + 1], cc = t.mi[3 * e + 2];
      T s = T(0);
      for (int k = 0; k < b; ++k) s = fma(T2[(k * P1 + a) * P1 + bb], xp[k * P1 + cc], s);
      out[e * 8 + c] = s;
    }
    __syncwarp();
  }
  T* dst = Mleaf + par * 8 * nc;
  for (int e = lane; e < 8 * nc; e += 32) dst[e] = out[e];
}

// M2M (Sec. 2.1, eq. M2M_general, child centre -> parent centre), scaled:
//   Mt_alpha(P) = sum_children sum_{beta <= alpha} C(alpha,beta) 2^-|alpha| (+-1/2)^(alpha-beta) Mt_beta(C)
template <typename Tc, typename Tp>
__global__ void m2m_kernel(TreeTables t, Level child, const Tc* __restrict__ Mc, Level par, Tp* __restrict__ Mp) {
  extern __shared__ unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nc = t.nc;
  const long long P = (long long)blockIdx.x * kWarpsPerBlock + warp;
  Tc* Ms = reinterpret_cast<Tc*>(smem_raw) + (size_t)warp * 8 * nc;
  if (P >= par.nbox) return;
  const Tc* src = Mc + P * 8 * nc;
  for (int e = lane; e < 8 * nc; e += 32) Ms[e] = src[e];
  __syncwarp();
  const int px = (int)(P % par.n[0]);
  const int py = (int)((P / par.n[0]) % par.n[1]);
  const int pz = (int)(P / ((long long)par.n[0] * par.n[1]));
  const long long gp = ((long long)(pz >> 1) * par.np[1] + (py >> 1)) * par.np[0] + (px >> 1);
  const int cp = (px & 1) | ((py & 1) << 1) | ((pz & 1) << 2);
  for (int a = lane; a < nc; a += 32) {
    Tp s = Tp(0);
    for (int q = t.m2m_start[a]; q < t.m2m_start[a + 1]; ++q) {
      const ShiftEntry& en = t.m2m[q];
      const Tc* m = Ms + en.src * 8;
      Tp part = Tp(0);
#pragma unroll
      for (int c = 0; c < 8; ++c) part += shift_neg(en.mask, c) ? -Tp(m[c]) : Tp(m[c]);
      s = fma(coef_of<Tp>(en), part, s);
    }
    Mp[(gp * nc + a) * 8 + cp] = s;
  }
}

// L2L (Sec. 2.3, eq. L2L, parent centre -> child centre), scaled:
//   Lt_beta(C) = sum_{gamma >= beta} C(gamma,beta) 2^(-1-|gamma|) (+-1/2)^(gamma-beta) Lt_gamma(P)
// Writes (overwrites) the children's block; the M2L contraction of the
// level then accumulates into it.
template <typename Tp, typename Tc>
__global__ void l2l_kernel(TreeTables t, Level par, const Tp* __restrict__ Lp, Level child, Tc* __restrict__ Lc) {
  extern __shared__ unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nc = t.nc;
  const long long P = (long long)blockIdx.x * kWarpsPerBlock + warp;
  Tp* Ls = reinterpret_cast<Tp*>(smem_raw) + (size_t)warp * nc;
  if (P >= par.nbox) return;
  const int px = (int)(P % par.n[0]);
  const int py = (int)((P / par.n[0]) % par.n[1]);
  const int pz = (int)(P / ((long long)par.n[0] * par.n[1]));
  const long long gp = ((long long)(pz >> 1) * par.np[1] + (py >> 1)) * par.np[0] + (px >> 1);
  const int cp = (px & 1) | ((py & 1) << 1) | ((pz & 1) << 2);
  for (int g = lane; g < nc; g += 32) Ls[g] = Lp[(gp * nc + g) * 8 + cp];
  __syncwarp();
  Tc* dst = Lc + P * 8 * nc;
  for (int o = lane; o < 8 * nc; o += 32) {
    const int be = o >> 3, c = o & 7;
    Tp s = Tp(0);
    for (int q = t.l2l_start[be]; q < t.l2l_start[be + 1]; ++q) {
      const ShiftEntry& en = t.l2l[q];
      const Tp cf = coef_of<Tp>(en);
      s = fma(shift_neg(en.mask, c) ? -cf : cf, Ls[en.src], s);
    }
    dst[o] = Tc(s);
  }
}

// Leaf evaluation (Sec. 2.3): phi = G dx^2 [ h^-1 sum_beta Lt_beta ((x-c)/h)^beta + near ].
// near_box holds the near-field sums per leaf box ([box][b^3] cells).
template <typename T>
__global__ void leaf_finish_kernel(TreeTables t, Level leaf, const T* __restrict__ Lleaf,
                                   const T* __restrict__ near_box, int nx, int ny, int nz, T scale,
                                   T* __restrict__ phi) {
  extern __shared__ unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = t.b, p = t.p, nc = t.nc, P1 = p + 1, b3 = b * b * b;
  const long long par = (long long)blockIdx.x * kWarpsPerBlock + warp;
  const int per_warp = 8 * nc + P1 * P1 * b + P1 * b * b + b * P1;
  T* Ls = reinterpret_cast<T*>(smem_raw) + (size_t)warp * per_warp;
  T* U2 = Ls + 8 * nc;       // [a][bb][k]
  T* U1 = U2 + P1 * P1 * b;  // [a][j][k]
  T* xp = U1 + P1 * b * b;
  if (par >= leaf.npar) return;
  for (int e = lane; e < b * P1; e += 32) {
    const int i = e / P1, a = e % P1;
    const T x = (T(i) + T(0.5)) / T(b) - T(0.5);
    T v = T(1);
    for (int q = 0; q < a; ++q) v *= x;
    xp[e] = v;
  }
  const T* src = Lleaf + par * 8 * nc;
  for (int e = lane; e < 8 * nc; e += 32) Ls[e] = src[e];
  const int px = (int)(par % leaf.np[0]);
  const int py = (int)((par / leaf.np[0]) % leaf.np[1]);
  const int pz = (int)(par / ((long long)leaf.np[0] * leaf.np[1]));
  const T inv_h = T(1) / T(b);
  __syncwarp();
  for (int c = 0; c < 8; ++c) {
    const int bx = 2 * px + (c & 1), by = 2 * py + ((c >> 1) & 1), bz = 2 * pz + (c >> 2);
    if (bx >= leaf.n[0] || by >= leaf.n[1] || bz >= leaf.n[2]) continue;
    const long long box = ((long long)bz * leaf.n[1] + by) * leaf.n[0] + bx;
    for (int e = lane; e < P1 * P1 * b; e += 32) {
      const int k = e % b, bb = (e / b) % P1, a = e / (b * P1);
      T s = T(0);
      for (int cc = 0; a + bb + cc <= p; ++cc) s = fma(Ls[coef_index(a, bb, cc) * 8 + c], xp[k * P1 + cc], s);
      U2[e] = s;
    }
    __syncwarp();
    for (int e = lane; e < P1 * b * b; e += 32) {
      const int k = e % b, j = (e / b) % b, a = e / (b * b);
      T s = T(0);
      for (int bb = 0; a + bb <= p; ++bb) s = fma(U2[(a * P1 + bb) * b + k], xp[j * P1 + bb], s);
      U1[e] = s;
    }
    __syncwarp();
    for (int e = lane; e < b3; e += 32) {
      const int i = e % b, j = (e / b) % b, k = e / (b * b);
      T s = T(0);
      for (int a = 0; a <= p; ++a) s = fma(U1[(a * b + j) * b + k], xp[i * P1 + a], s);
      const T v = scale * fma(s, inv_h, near_box[box * b3 + e]);
      phi[((long long)(bz * b + k) * ny + (by * b + j)) * nx + (bx * b + i)] = v;
    }
    __syncwarp();
  }
}

template <typename T>
__global__ void zero_kernel(T* p, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    p[i] = T(0);
}

// Debug export: parent-blocked scaled level -> canonical [box][coef] doubles
// in cell units (M_alpha = Mt h^|alpha|, L_beta = Lt beta! / h^(1+|beta|)).
template <typename T>
__global__ void export_level_kernel(const T* __restrict__ src, Level lv, int what, double h,
                                    const int8_t* __restrict__ mi, int nc, double* __restrict__ dst) {
  const long long total = lv.nbox * nc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long box = e / nc;
    const int k = (int)(e % nc);
    const int x = (int)(box % lv.n[0]);
    const int y = (int)((box / lv.n[0]) % lv.n[1]);
    const int z = (int)(box / ((long long)lv.n[0] * lv.n[1]));
    const long long pbox = ((long long)(z >> 1) * lv.np[1] + (y >> 1)) * lv.np[0] + (x >> 1);
    const int c = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
    const int a = mi[3 * k], b = mi[3 * k + 1], cc = mi[3 * k + 2];
    const int n = a + b + cc;
    double v = (double)src[(pbox * nc + k) * 8 + c];
    double hp = 1.0;
    for (int q = 0; q < n; ++q) hp *= h;
    if (what == 0) {
      v *= hp;
    } else {
      double f = 1.0;
      for (int q = 2; q <= a; ++q) f *= q;
      for (int q = 2; q <= b; ++q) f *= q;
      for (int q = 2; q <= cc; ++q) f *= q;
      v = v * f / (hp * h);
    }
    dst[e] = v;
  }
}

size_t grid_for(long long warps) { return (size_t)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock); }

}  // namespace

template <typename T>
cudaError_t launch_p2m(const TreeTables& t, const T* rho, const int dims[3], const Level& leaf, T* Mleaf, T* rho_box,
                       cudaStream_t s) {
  const int P1 = t.p + 1, b = t.b;
  const size_t per = (size_t)b * b * b + b * b * P1 + b * P1 * P1 + 8 * t.nc + b * P1;
  const size_t smem = per * sizeof(T) * kWarpsPerBlock;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(p2m_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const size_t blocks = grid_for(leaf.npar);
  if (blocks == 0) return cudaSuccess;
  p2m_kernel<T><<<(unsigned)blocks, 32 * kWarpsPerBlock, smem, s>>>(t, rho, dims[0], dims[1], dims[2], leaf, Mleaf,
                                                                     rho_box);
  return cudaGetLastError();
}

template <typename Tc, typename Tp>
cudaError_t launch_m2m(const TreeTables& t, const Level& child, const Tc* Mc, const Level& par, Tp* Mp, cudaStream_t s) {
  const size_t smem = (size_t)8 * t.nc * sizeof(Tc) * kWarpsPerBlock;
  const size_t blocks = grid_for(par.nbox);
  if (blocks == 0) return cudaSuccess;
  m2m_kernel<Tc, Tp><<<(unsigned)blocks, 32 * kWarpsPerBlock, smem, s>>>(t, child, Mc, par, Mp);
  return cudaGetLastError();
}

template <typename Tp, typename Tc>
cudaError_t launch_l2l(const TreeTables& t, const Level& par, const Tp* Lp, const Level& child, Tc* Lc, cudaStream_t s) {
  const size_t smem = (size_t)t.nc * sizeof(Tp) * kWarpsPerBlock;
  const size_t blocks = grid_for(par.nbox);
  if (blocks == 0) return cudaSuccess;
  l2l_kernel<Tp, Tc><<<(unsigned)blocks, 32 * kWarpsPerBlock, smem, s>>>(t, par, Lp, child, Lc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zero(T* p, size_t count, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  size_t blocks = (count + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  zero_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(p, count);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_leaf_finish(const TreeTables& t, const Level& leaf, const T* Lleaf, const T* near_box,
                               const int dims[3], double scale, T* phi, cudaStream_t s) {
  const int P1 = t.p + 1, b = t.b;
  const size_t per = (size_t)8 * t.nc + P1 * P1 * b + P1 * b * b + b * P1;
  const size_t smem = per * sizeof(T) * kWarpsPerBlock;
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(leaf_finish_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const size_t blocks = grid_for(leaf.npar);
  if (blocks == 0) return cudaSuccess;
  leaf_finish_kernel<T><<<(unsigned)blocks, 32 * kWarpsPerBlock, smem, s>>>(t, leaf, Lleaf, near_box, dims[0],
                                                                             dims[1], dims[2], (T)scale, phi);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_export_level(const T* src, const Level& lv, int what, double h, const int8_t* mi, int nc,
                                double* dst, cudaStream_t s) {
  export_level_kernel<T><<<256, 256, 0, s>>>(src, lv, what, h, mi, nc, dst);
  return cudaGetLastError();
}

template cudaError_t launch_p2m<float>(const TreeTables&, const float*, const int*, const Level&, float*, float*,
                                       cudaStream_t);
template cudaError_t launch_p2m<double>(const TreeTables&, const double*, const int*, const Level&, double*, double*,
                                        cudaStream_t);
template cudaError_t launch_m2m<float, float>(const TreeTables&, const Level&, const float*, const Level&, float*,
                                              cudaStream_t);
template cudaError_t launch_m2m<double, double>(const TreeTables&, const Level&, const double*, const Level&,
                                                double*, cudaStream_t);
template cudaError_t launch_m2m<float, double>(const TreeTables&, const Level&, const float*, const Level&, double*,
                                               cudaStream_t);
template cudaError_t launch_l2l<float, float>(const TreeTables&, const Level&, const float*, const Level&, float*,
                                              cudaStream_t);
template cudaError_t launch_l2l<double, double>(const TreeTables&, const Level&, const double*, const Level&,
                                                double*, cudaStream_t);
template cudaError_t launch_l2l<double, float>(const TreeTables&, const Level&, const double*, const Level&, float*,
                                               cudaStream_t);
template cudaError_t launch_zero<float>(float*, size_t, cudaStream_t);
template cudaError_t launch_zero<double>(double*, size_t, cudaStream_t);
template cudaError_t launch_leaf_finish<float>(const TreeTables&, const Level&, const float*, const float*,
                                               const int*, double, float*, cudaStream_t);
template cudaError_t launch_leaf_finish<double>(const TreeTables&, const Level&, const double*, const double*,
                                                const int*, double, double*, cudaStream_t);
template cudaError_t launch_export_level<float>(const float*, const Level&, int, double, const int8_t*, int, double*,
                                                cudaStream_t);
template cudaError_t launch_export_level<double>(const double*, const Level&, int, double, const int8_t*, int,
                                                 double*, cudaStream_t);

}  // namespace fmmgb
