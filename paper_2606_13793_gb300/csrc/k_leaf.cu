// Leaf evaluation (L2P + near sum + scaling) on the CUDA cores (see tree_common.cuh).
#include <cuda_bf16.h>

#include "tree_common.cuh"

namespace fmmgb {
namespace {
using namespace tree;

// ---------------------------------------------------------------------------
// Leaf evaluation (Sec. 2.3):
//   phi = G dx^2 [ h^-1 sum_beta Lt_beta ((x - c)/h)^beta + near ]
// near_box holds the near-field sums per leaf box ([box][b^3] cells).
template <int P, typename T>
__global__ void __launch_bounds__(kThreads) leaf_finish_kernel(Level leaf, const T* __restrict__ Lleaf,
                                                               const T* __restrict__ near_box, int nx, int ny, int b,
                                                               T scale, T* __restrict__ phi) {
  constexpr int NC = ncoef_c(P);
  const long long t = (long long)blockIdx.x * kThreads + threadIdx.x;
  const Box B = box_of(leaf, t);
  if (!B.real) return;
  T L[NC];
  const T* src = Lleaf + B.par * 8 * NC + B.c;
#pragma unroll
  for (int k = 0; k < NC; ++k) L[k] = src[k * 8];
  const T inv_b = T(1) / T(b);
  const long long box = ((long long)B.z * leaf.n[1] + B.y) * leaf.n[0] + B.x;
  const int b3 = b * b * b;
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
      for (int j = 0; j < 4; ++j) nr[j] = __ldg(reinterpret_cast<const float4*>(near_box + box * 64 + (k * 4 + j) * 4));
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
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const T xi = (T(i) + T(0.5)) * inv_b - T(0.5);
          T s = u1[P];
#pragma unroll
          for (int a = P - 1; a >= 0; --a) s = fma(s, xi, u1[a]);  // Horner in x
          out[i] = (float)(scale * fma(s, inv_b, (T)nv[i]));
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
      const T* nrow = near_box + box * b3 + (k * b + j) * b;
      for (int i = 0; i < b; ++i) {
        const T xi = (T(i) + T(0.5)) * inv_b - T(0.5);
        T s = u1[P];
#pragma unroll
        for (int a = P - 1; a >= 0; --a) s = fma(s, xi, u1[a]);  // Horner in x
        row[i] = scale * fma(s, inv_b, nrow[i]);
      }
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_leaf_finish(const TreeTables& t, const Level& leaf, const T* Lleaf, const T* near_box,
                               const int dims[3], double scale, T* phi, cudaStream_t s) {
  const long long threads = leaf.npar * 8;
  if (threads == 0) return cudaSuccess;
  FMM_ORDER_SWITCH(t.p, (leaf_finish_kernel<PP, T><<<grid_threads(threads), kThreads, 0, s>>>(
                            leaf, Lleaf, near_box, dims[0], dims[1], t.b, (T)scale, phi)));
  return cudaGetLastError();
}

template cudaError_t launch_leaf_finish<float>(const TreeTables&, const Level&, const float*, const float*,
                                               const int*, double, float*, cudaStream_t);
template cudaError_t launch_leaf_finish<double>(const TreeTables&, const Level&, const double*, const double*,
                                                const int*, double, double*, cudaStream_t);

}  // namespace fmmgb
