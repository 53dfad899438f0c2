// Leaf evaluation (L2P + near sum + scaling) on the CUDA cores (see tree_common.cuh).
#include <cuda_bf16.h>

#include "multi.cuh"
#include "tree_common.cuh"

namespace fmmgb {
namespace {
using namespace tree;

// ---------------------------------------------------------------------------
// Leaf evaluation (Sec. 2.3):
//   phi = G dx^2 [ h^-1 sum_beta Lt_beta ((x - c)/h)^beta + near ]
// near_box holds the near-field sums per leaf box ([box][b^3] cells).
// near_box rows have near_stride values per box (the potential first).
// m2p (nullable): final-stage M2P potentials [parent][child][b^3], added to
// the L2P sum before its 1/h scaling.  Two blocks per SM for FP32 at p <= 6
// (128 registers, a few bytes spilled; 0.44 -> 0.37 ms at 512^3 against 169
// registers and one block).
template <int P, typename T>
__device__ __forceinline__ void leaf_finish_body(const Level& leaf, const T* __restrict__ Lleaf,
                                                 const T* __restrict__ near_box, int near_stride,
                                                 const T* __restrict__ m2p, int nx, int ny, int b, T scale,
                                                 T* __restrict__ phi, const VBlock& vb, const LeafDownArgs<T>& down) {
  constexpr int NC = ncoef_c(P);
  const long long t = (long long)vb.x * kThreads + threadIdx.x;
  const Box B = box_of(leaf, t);
  if (!B.real) return;
  T L[NC];
  const T* src = Lleaf + B.par * 8 * NC + B.c;
  if (down.Lp) {  // the last L2L, as its kernel computes it (the box's parent = B.par)
    l2l_child<P, T, T>(L, down.par, down.Lp, B.par, B.c, 1, down.harm, src, down.Lred);
  } else {
#pragma unroll
    for (int k = 0; k < NC; ++k) L[k] = src[k * 8];
  }
  const T inv_b = T(1) / T(b);
  const long long box = ((long long)B.z * leaf.n[1] + B.y) * leaf.n[0] + B.x;
  const T* mp = m2p ? m2p + (B.par * 8 + B.c) * (long long)(b * b * b) : nullptr;
  for (int k = 0; k < b; ++k) {
    T zpow[P + 1];
    powers<P, T>((T(k) + T(0.5)) * inv_b - T(0.5), zpow);
    T u2[(P + 1) * (P + 2) / 2];  // (a, bb) with a + bb <= P
#pragma unroll
    for (int a = 0; a <= P; ++a)
#pragma unroll
      for (int bb = 0; a + bb <= P; ++bb) {
        T s = T(0);
#pragma unroll
        for (int cc = 0; a + bb + cc <= P; ++cc) s = fma(L[cidx(a, bb, cc)], zpow[cc], s);
        u2[(a + bb) * (a + bb + 1) / 2 + bb] = s;
      }
    if (sizeof(T) == 4 && b == 4) {
      // the plane's four near rows in flight at once; 16-byte loads and stores
      float4 nr[4];
#pragma unroll
      for (int j = 0; j < 4; ++j)
        nr[j] = __ldg(reinterpret_cast<const float4*>(near_box + box * near_stride + (k * 4 + j) * 4));
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        T ypow[P + 1];
        powers<P, T>((T(j) + T(0.5)) * inv_b - T(0.5), ypow);
        T u1[P + 1];
#pragma unroll
        for (int a = 0; a <= P; ++a) {
          T s = T(0);
#pragma unroll
          for (int bb = 0; a + bb <= P; ++bb) s = fma(u2[(a + bb) * (a + bb + 1) / 2 + bb], ypow[bb], s);
          u1[a] = s;
        }
        float out[4];
        const float nv[4] = {nr[j].x, nr[j].y, nr[j].z, nr[j].w};
        float mv[4] = {0.f, 0.f, 0.f, 0.f};
        if (mp) {
          const float4 m4 = __ldg(reinterpret_cast<const float4*>(mp + (k * 4 + j) * 4));
          mv[0] = m4.x, mv[1] = m4.y, mv[2] = m4.z, mv[3] = m4.w;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const T xi = (T(i) + T(0.5)) * inv_b - T(0.5);
          T s = u1[P];
#pragma unroll
          for (int a = P - 1; a >= 0; --a) s = fma(s, xi, u1[a]);  // Horner in x
          out[i] = (float)(scale * fma(s + (T)mv[i], inv_b, (T)nv[i]));
        }
        *reinterpret_cast<float4*>(phi + ((long long)(B.z * 4 + k) * ny + (B.y * 4 + j)) * nx + (long long)B.x * 4) =
            make_float4(out[0], out[1], out[2], out[3]);
      }
      continue;
    }
    for (int j = 0; j < b; ++j) {
      T ypow[P + 1];
      powers<P, T>((T(j) + T(0.5)) * inv_b - T(0.5), ypow);
      T u1[P + 1];
#pragma unroll
      for (int a = 0; a <= P; ++a) {
        T s = T(0);
#pragma unroll
        for (int bb = 0; a + bb <= P; ++bb) s = fma(u2[(a + bb) * (a + bb + 1) / 2 + bb], ypow[bb], s);
        u1[a] = s;
      }
      T* row = phi + ((long long)(B.z * b + k) * ny + (B.y * b + j)) * nx + (long long)B.x * b;
      const T* nrow = near_box + box * near_stride + (k * b + j) * b;
      for (int i = 0; i < b; ++i) {
        const T xi = (T(i) + T(0.5)) * inv_b - T(0.5);
        T s = u1[P];
#pragma unroll
        for (int a = P - 1; a >= 0; --a) s = fma(s, xi, u1[a]);  // Horner in x
        if (mp) s += mp[(k * b + j) * b + i];
        row[i] = scale * fma(s, inv_b, nrow[i]);
      }
    }
  }
}

template <int P, typename T>
__global__ void __launch_bounds__(kThreads, (P <= 6 && sizeof(T) == 4) ? 2 : 1)
    leaf_finish_kernel(Level leaf, const T* __restrict__ Lleaf, const T* __restrict__ near_box, int near_stride,
                       const T* __restrict__ m2p, int nx, int ny, int b, T scale, T* __restrict__ phi,
                       const LeafDownArgs<T> down) {
  leaf_finish_body<P, T>(leaf, Lleaf, near_box, near_stride, m2p, nx, ny, b, scale, phi, native_vblock(), down);
}

// The leaf levels of many solves in one launch (batched solves).
template <int P, typename T>
__global__ void __launch_bounds__(kThreads, (P <= 6 && sizeof(T) == 4) ? 2 : 1)
    leaf_finish_multi_kernel(const LeafArgs* __restrict__ a, const MultiGrid* __restrict__ g, int n) {
  __shared__ LeafArgs x;  // the item's arguments, read by the body from shared memory
  const int i = multi_item(g, n);
  if (threadIdx.x == 0 && threadIdx.y == 0) x = a[i];
  __syncthreads();
  LeafDownArgs<T> down;
  down.par = x.par;
  down.Lp = static_cast<const T*>(x.Lp);
  down.harm = x.harm;
  down.Lred = static_cast<const T*>(x.Lred);
  leaf_finish_body<P, T>(x.leaf, static_cast<const T*>(x.Lleaf), static_cast<const T*>(x.near_box), x.near_stride,
                         static_cast<const T*>(x.m2p), x.nx, x.ny, x.b, (T)x.scale, static_cast<T*>(x.phi),
                         multi_vblock(g[i]), down);
}

// Leaf evaluation with the analytic acceleration: also the gradient of the
// local expansion (derivatives of the separable powers) and the near-field
// force columns (near_box row = potential, then d/dx, d/dy, d/dz sums of
// b^3 values each):
//   accel_q = -G dx [ h^-2 sum_beta Lt_beta d/dxi_q ((x - c)/h)^beta + near_q ]
template <int P, typename T>
__global__ void __launch_bounds__(kThreads) leaf_finish_grad_kernel(Level leaf, const T* __restrict__ Lleaf,
                                                                    const T* __restrict__ near_box,
                                                                    const T* __restrict__ m2p, int nx, int ny,
                                                                    int nz, int b, T scale, T ascale,
                                                                    T* __restrict__ phi, T* __restrict__ accel) {
  constexpr int NC = ncoef_c(P);
  constexpr int N2 = (P + 1) * (P + 2) / 2;
  const long long t = (long long)blockIdx.x * kThreads + threadIdx.x;
  const Box B = box_of(leaf, t);
  if (!B.real) return;
  T L[NC];
  const T* src = Lleaf + B.par * 8 * NC + B.c;
#pragma unroll
  for (int k = 0; k < NC; ++k) L[k] = src[k * 8];
  const T inv_b = T(1) / T(b);
  const long long ncell = (long long)nx * ny * nz;
  const long long box = ((long long)B.z * leaf.n[1] + B.y) * leaf.n[0] + B.x;
  const int b3 = b * b * b;
  const T* nb = near_box + box * 4 * b3;
  // final-stage M2P: the leaf interaction list's potential and its gradient
  // at the cell centres, in box units like the local expansion's ([comp][b^3])
  const T* mp = m2p ? m2p + (B.par * 8 + B.c) * (long long)(4 * b3) : nullptr;
  for (int k = 0; k < b; ++k) {
    const T zk = (T(k) + T(0.5)) * inv_b - T(0.5);
    T zpow[P + 1], dzpow[P + 1];
    powers<P, T>(zk, zpow);
    dzpow[0] = T(0);
#pragma unroll
    for (int c = 1; c <= P; ++c) dzpow[c] = T(c) * zpow[c - 1];
    T u2[N2], u2z[N2];  // (a, bb) with a + bb <= P: sums over c of L zk^c and of L d/dz zk^c
#pragma unroll
    for (int a = 0; a <= P; ++a)
#pragma unroll
      for (int bb = 0; a + bb <= P; ++bb) {
        T s = T(0), sz = T(0);
#pragma unroll
        for (int cc = 0; a + bb + cc <= P; ++cc) {
          s = fma(L[cidx(a, bb, cc)], zpow[cc], s);
          sz = fma(L[cidx(a, bb, cc)], dzpow[cc], sz);
        }
        u2[(a + bb) * (a + bb + 1) / 2 + bb] = s;
        u2z[(a + bb) * (a + bb + 1) / 2 + bb] = sz;
      }
    if (sizeof(T) == 4 && b == 4 && !mp) {
      // 16-byte loads of the four near columns and 16-byte stores of the
      // potential and the three force rows; the plane unrolled so the loads
      // of one row issue ahead of the previous row's arithmetic
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int e0 = (k * 4 + j) * 4;
        const float4 n0 = __ldg(reinterpret_cast<const float4*>(nb + e0));
        const float4 n1 = __ldg(reinterpret_cast<const float4*>(nb + 64 + e0));
        const float4 n2 = __ldg(reinterpret_cast<const float4*>(nb + 128 + e0));
        const float4 n3 = __ldg(reinterpret_cast<const float4*>(nb + 192 + e0));
        const T yj = (T(j) + T(0.5)) * inv_b - T(0.5);
        T ypow[P + 1], dypow[P + 1];
        powers<P, T>(yj, ypow);
        dypow[0] = T(0);
#pragma unroll
        for (int c = 1; c <= P; ++c) dypow[c] = T(c) * ypow[c - 1];
        T u1[P + 1], u1y[P + 1], u1z[P + 1];
#pragma unroll
        for (int a = 0; a <= P; ++a) {
          T sv = T(0), sy = T(0), sz = T(0);
#pragma unroll
          for (int bb = 0; a + bb <= P; ++bb) {
            const int q = (a + bb) * (a + bb + 1) / 2 + bb;
            sv = fma(u2[q], ypow[bb], sv);
            sy = fma(u2[q], dypow[bb], sy);
            sz = fma(u2z[q], ypow[bb], sz);
          }
          u1[a] = sv, u1y[a] = sy, u1z[a] = sz;
        }
        const float nv0[4] = {n0.x, n0.y, n0.z, n0.w}, nv1[4] = {n1.x, n1.y, n1.z, n1.w};
        const float nv2[4] = {n2.x, n2.y, n2.z, n2.w}, nv3[4] = {n3.x, n3.y, n3.z, n3.w};
        float o0[4], o1[4], o2[4], o3[4];
        const T ib2 = inv_b * inv_b;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const T xi = (T(i) + T(0.5)) * inv_b - T(0.5);
          T sv = u1[P], sx = T(0), sy = u1y[P], sz = u1z[P];
#pragma unroll
          for (int a = P - 1; a >= 0; --a) {
            sx = fma(sx, xi, sv);
            sv = fma(sv, xi, u1[a]);
            sy = fma(sy, xi, u1y[a]);
            sz = fma(sz, xi, u1z[a]);
          }
          o0[i] = (float)(scale * fma(sv, inv_b, (T)nv0[i]));
          o1[i] = (float)(ascale * fma(sx, ib2, (T)nv1[i]));
          o2[i] = (float)(ascale * fma(sy, ib2, (T)nv2[i]));
          o3[i] = (float)(ascale * fma(sz, ib2, (T)nv3[i]));
        }
        const long long row = ((long long)(B.z * 4 + k) * ny + (B.y * 4 + j)) * nx + (long long)B.x * 4;
        *reinterpret_cast<float4*>(phi + row) = make_float4(o0[0], o0[1], o0[2], o0[3]);
        *reinterpret_cast<float4*>(accel + row) = make_float4(o1[0], o1[1], o1[2], o1[3]);
        *reinterpret_cast<float4*>(accel + ncell + row) = make_float4(o2[0], o2[1], o2[2], o2[3]);
        *reinterpret_cast<float4*>(accel + 2 * ncell + row) = make_float4(o3[0], o3[1], o3[2], o3[3]);
      }
      continue;
    }
    for (int j = 0; j < b; ++j) {
      const T yj = (T(j) + T(0.5)) * inv_b - T(0.5);
      T ypow[P + 1], dypow[P + 1];
      powers<P, T>(yj, ypow);
      dypow[0] = T(0);
#pragma unroll
      for (int c = 1; c <= P; ++c) dypow[c] = T(c) * ypow[c - 1];
      T u1[P + 1], u1y[P + 1], u1z[P + 1];
#pragma unroll
      for (int a = 0; a <= P; ++a) {
        T s = T(0), sy = T(0), sz = T(0);
#pragma unroll
        for (int bb = 0; a + bb <= P; ++bb) {
          const int q = (a + bb) * (a + bb + 1) / 2 + bb;
          s = fma(u2[q], ypow[bb], s);
          sy = fma(u2[q], dypow[bb], sy);
          sz = fma(u2z[q], ypow[bb], sz);
        }
        u1[a] = s, u1y[a] = sy, u1z[a] = sz;
      }
      const long long row = ((long long)(B.z * b + k) * ny + (B.y * b + j)) * nx + (long long)B.x * b;
      const int e0 = (k * b + j) * b;
      for (int i = 0; i < b; ++i) {
        const T xi = (T(i) + T(0.5)) * inv_b - T(0.5);
        // Horner in x for the value, the x-derivative and the y/z-derivative polynomials
        T s = u1[P], sx = T(0), sy = u1y[P], sz = u1z[P];
#pragma unroll
        for (int a = P - 1; a >= 0; --a) {
          sx = fma(sx, xi, s);
          s = fma(s, xi, u1[a]);
          sy = fma(sy, xi, u1y[a]);
          sz = fma(sz, xi, u1z[a]);
        }
        if (mp) {
          s += mp[e0 + i];
          sx += mp[b3 + e0 + i];
          sy += mp[2 * b3 + e0 + i];
          sz += mp[3 * b3 + e0 + i];
        }
        phi[row + i] = scale * fma(s, inv_b, nb[e0 + i]);
        const T ib2 = inv_b * inv_b;
        accel[row + i] = ascale * fma(sx, ib2, nb[b3 + e0 + i]);
        accel[ncell + row + i] = ascale * fma(sy, ib2, nb[2 * b3 + e0 + i]);
        accel[2 * ncell + row + i] = ascale * fma(sz, ib2, nb[3 * b3 + e0 + i]);
      }
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_leaf_finish_grad(const TreeTables& t, const Level& leaf, const T* Lleaf, const T* near_box,
                                    const T* m2p, const int dims[3], double scale, double ascale, T* phi, T* accel,
                                    cudaStream_t s) {
  const long long threads = leaf.npar * 8;
  if (threads == 0) return cudaSuccess;
  FMM_ORDER_SWITCH(t.p, (leaf_finish_grad_kernel<PP, T><<<grid_threads(threads), kThreads, 0, s>>>(
                            leaf, Lleaf, near_box, m2p, dims[0], dims[1], dims[2], t.b, (T)scale, (T)ascale, phi,
                            accel)));
  return cudaGetLastError();
}

template cudaError_t launch_leaf_finish_grad<float>(const TreeTables&, const Level&, const float*, const float*,
                                                    const float*, const int*, double, double, float*, float*,
                                                    cudaStream_t);
template cudaError_t launch_leaf_finish_grad<double>(const TreeTables&, const Level&, const double*, const double*,
                                                     const double*, const int*, double, double, double*, double*,
                                                     cudaStream_t);

template <typename T>
cudaError_t launch_leaf_finish(const TreeTables& t, const Level& leaf, const T* Lleaf, const T* near_box,
                               int near_stride, const T* m2p, const int dims[3], double scale, T* phi, cudaStream_t s,
                               const LeafDownArgs<T>* down) {
  const long long threads = leaf.npar * 8;
  if (threads == 0) return cudaSuccess;
  const LeafDownArgs<T> none{};
  FMM_ORDER_SWITCH(t.p, (leaf_finish_kernel<PP, T><<<grid_threads(threads), kThreads, 0, s>>>(
                            leaf, Lleaf, near_box, near_stride, m2p, dims[0], dims[1], t.b, (T)scale, phi,
                            down ? *down : none)));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_leaf_finish_multi(int p, const LeafArgs* args, const MultiGrid* grids, int n, long long blocks,
                                     cudaStream_t s) {
  if (n == 0 || blocks == 0) return cudaSuccess;
  FMM_ORDER_SWITCH(p, (leaf_finish_multi_kernel<PP, T><<<(unsigned)blocks, kThreads, 0, s>>>(args, grids, n)));
  return cudaGetLastError();
}
template cudaError_t launch_leaf_finish_multi<float>(int, const LeafArgs*, const MultiGrid*, int, long long,
                                                     cudaStream_t);
template cudaError_t launch_leaf_finish_multi<double>(int, const LeafArgs*, const MultiGrid*, int, long long,
                                                      cudaStream_t);

template cudaError_t launch_leaf_finish<float>(const TreeTables&, const Level&, const float*, const float*, int,
                                               const float*, const int*, double, float*, cudaStream_t,
                                               const LeafDownArgs<float>*);
template cudaError_t launch_leaf_finish<double>(const TreeTables&, const Level&, const double*, const double*, int,
                                                const double*, const int*, double, double*, cudaStream_t,
                                                const LeafDownArgs<double>*);

// Cells of every leaf box in parent-blocked order, [parent][child][b^3]
// (phantom boxes zero): the rows of the final-stage M2P's transpose.
template <typename T>
__global__ void cells_to_parent_blocks_kernel(const T* __restrict__ src, int nx, int ny, Level leaf, int b,
                                              T* __restrict__ dst) {
  const long long b3 = (long long)b * b * b;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= leaf.npar * 8 * b3) return;
  const Box B = box_of(leaf, i / b3);
  const int cell = (int)(i % b3);
  T v = T(0);
  if (B.real) {
    const int x = B.x * b + cell % b, y = B.y * b + (cell / b) % b, z = B.z * b + cell / (b * b);
    v = src[((long long)z * ny + y) * nx + x];
  }
  dst[i] = v;
}

template <typename T>
cudaError_t launch_cells_to_parent_blocks(const T* src, const int dims[3], const Level& leaf, int b, T* dst,
                                          cudaStream_t s) {
  const long long n = leaf.npar * 8 * (long long)b * b * b;
  if (n == 0) return cudaSuccess;
  cells_to_parent_blocks_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dims[0], dims[1], leaf, b, dst);
  return cudaGetLastError();
}
template cudaError_t launch_cells_to_parent_blocks<float>(const float*, const int*, const Level&, int, float*,
                                                          cudaStream_t);
template cudaError_t launch_cells_to_parent_blocks<double>(const double*, const int*, const Level&, int, double*,
                                                           cudaStream_t);

// The four input columns of the analytic force's transposed near field and
// final-stage P2L, per leaf box: [w, sc g_x, sc g_y, sc g_z] x b^3 (g, the
// force's adjoint input [3][cells], may be NULL: zeros).  parent_blocked = 0:
// boxes in grid order (the near-field rows); 1: [parent][child] order, phantom
// children zero (the P2L rows).
template <typename T>
__global__ void cells_to_boxes4_kernel(const T* __restrict__ w, const T* __restrict__ g, T sc, int nx, int ny, int nz,
                                       Level leaf, int b, int parent_blocked, T* __restrict__ dst) {
  const long long b3 = (long long)b * b * b;
  const long long nbox = parent_blocked ? leaf.npar * 8 : (long long)leaf.n[0] * leaf.n[1] * leaf.n[2];
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbox * b3) return;
  const long long bi = i / b3;
  const int cell = (int)(i % b3);
  int bx, by, bz;
  bool real = true;
  if (parent_blocked) {
    const Box B = box_of(leaf, bi);
    bx = B.x, by = B.y, bz = B.z, real = B.real;
  } else {
    bx = (int)(bi % leaf.n[0]), by = (int)((bi / leaf.n[0]) % leaf.n[1]), bz = (int)(bi / ((long long)leaf.n[0] * leaf.n[1]));
  }
  T v[4] = {T(0), T(0), T(0), T(0)};
  if (real) {
    const int x = bx * b + cell % b, y = by * b + (cell / b) % b, z = bz * b + cell / (b * b);
    const long long c = ((long long)z * ny + y) * nx + x, n = (long long)nx * ny * nz;
    v[0] = w[c];
    if (g)
      for (int q = 0; q < 3; ++q) v[1 + q] = sc * g[q * n + c];
  }
  T* o = dst + bi * 4 * b3 + cell;
  for (int q = 0; q < 4; ++q) o[q * b3] = v[q];
}

template <typename T>
cudaError_t launch_cells_to_boxes4(const T* w, const T* g, double sc, const int dims[3], const Level& leaf, int b,
                                   int parent_blocked, T* dst, cudaStream_t s) {
  const long long nbox = parent_blocked ? leaf.npar * 8 : (long long)leaf.n[0] * leaf.n[1] * leaf.n[2];
  const long long n = nbox * b * b * b;
  if (n == 0) return cudaSuccess;
  cells_to_boxes4_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w, g, (T)sc, dims[0], dims[1], dims[2], leaf,
                                                                        b, parent_blocked, dst);
  return cudaGetLastError();
}
template cudaError_t launch_cells_to_boxes4<float>(const float*, const float*, double, const int*, const Level&, int,
                                                   int, float*, cudaStream_t);
template cudaError_t launch_cells_to_boxes4<double>(const double*, const double*, double, const int*, const Level&,
                                                    int, int, double*, cudaStream_t);

}  // namespace fmmgb
