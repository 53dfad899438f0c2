// P2M on the CUDA cores (see tree_common.cuh for the layout and conventions).
#include <cuda_bf16.h>

#include "tree_common.cuh"

namespace fmmgb {
namespace {
using namespace tree;

// ---------------------------------------------------------------------------
// P2M (Sec. 2.1, eq. multipole) about each leaf-box centre, scaled:
//   Mt_alpha = sum_cells m ((x - c)/b)^alpha
// plus the box-blocked copy of the density for the near field.
template <int P, typename T>
__global__ void __launch_bounds__(kThreads) p2m_kernel(const T* __restrict__ rho, int nx, int ny, int b, Level leaf,
                                                       T* __restrict__ Mleaf, __nv_bfloat16* __restrict__ Mhi,
                                                       __nv_bfloat16* __restrict__ Mlo, T* __restrict__ rho_box,
                                                       __nv_bfloat16* __restrict__ rhi,
                                                       __nv_bfloat16* __restrict__ rlo, int* __restrict__ flag) {
  constexpr int NC = ncoef_c(P);
  const long long t = (long long)blockIdx.x * kThreads + threadIdx.x;
  const Box B = box_of(leaf, t);
  if (B.par >= leaf.npar) return;
  T acc[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) acc[k] = T(0);
  bool bad = false;  // non-finite density (reported through the plan's flag)
  if (B.real) {
    const T inv_b = T(1) / T(b);
    const long long box = ((long long)B.z * leaf.n[1] + B.y) * leaf.n[0] + B.x;
    const int b3 = b * b * b;
    for (int k = 0; k < b; ++k) {
      const T zk = (T(k) + T(0.5)) * inv_b - T(0.5);
      T t2[(P + 1) * (P + 2) / 2];
#pragma unroll
      for (int q = 0; q < (P + 1) * (P + 2) / 2; ++q) t2[q] = T(0);
      for (int j = 0; j < b; ++j) {
        const T yj = (T(j) + T(0.5)) * inv_b - T(0.5);
        const T* row = rho + ((long long)(B.z * b + k) * ny + (B.y * b + j)) * nx + (long long)B.x * b;
        const long long e0 = box * b3 + (k * b + j) * b;  // first cell of this row in the box-blocked copy
        T m[8];
        if (sizeof(T) == 4 && b == 4) {  // one 16-byte load, packed stores
          const float4 v = *reinterpret_cast<const float4*>(row);
          m[0] = v.x, m[1] = v.y, m[2] = v.z, m[3] = v.w;
          if (rho_box) *reinterpret_cast<float4*>(rho_box + e0) = v;
          if (rhi) {
            __nv_bfloat16 h[4], l[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              h[i] = __float2bfloat16_rn((float)m[i]);
              l[i] = __float2bfloat16_rn((float)m[i] - __bfloat162float(h[i]));
            }
            *reinterpret_cast<uint2*>(rhi + e0) = *reinterpret_cast<const uint2*>(h);
            *reinterpret_cast<uint2*>(rlo + e0) = *reinterpret_cast<const uint2*>(l);
          }
        } else {
          for (int i = 0; i < b; ++i) {
            m[i] = row[i];
            if (rho_box) rho_box[e0 + i] = m[i];
            if (rhi) store_split(rhi, rlo, (size_t)(e0 + i), m[i]);
          }
        }
        T t1[P + 1];
#pragma unroll
        for (int a = 0; a <= P; ++a) t1[a] = T(0);
        for (int i = 0; i < b; ++i) {
          bad |= !isfinite(m[i]);
          const T xi = (T(i) + T(0.5)) * inv_b - T(0.5);
          T w = m[i];
#pragma unroll
          for (int a = 0; a <= P; ++a) {
            t1[a] += w;
            w *= xi;
          }
        }
        // t2[(a, bb)] += t1[a] * yj^bb, packed by (a + bb) blocks
        T ypow[P + 1];
        powers<P, T>(yj, ypow);
#pragma unroll
        for (int a = 0; a <= P; ++a)
#pragma unroll
          for (int bb = 0; a + bb <= P; ++bb) t2[(a + bb) * (a + bb + 1) / 2 + bb] += t1[a] * ypow[bb];
      }
      T zpow[P + 1];
      powers<P, T>(zk, zpow);
#pragma unroll
      for (int a = 0; a <= P; ++a)
#pragma unroll
        for (int bb = 0; a + bb <= P; ++bb)
#pragma unroll
          for (int cc = 0; a + bb + cc <= P; ++cc)
            acc[cidx(a, bb, cc)] = fma(t2[(a + bb) * (a + bb + 1) / 2 + bb], zpow[cc], acc[cidx(a, bb, cc)]);
    }
  }
  if (bad) atomicOr(flag, 1);
  T* dst = Mleaf + B.par * 8 * NC + B.c;
#pragma unroll
  for (int k = 0; k < NC; ++k) dst[k * 8] = acc[k];
  if (Mhi) {
    const size_t base = (size_t)B.par * 8 * NC + B.c;
#pragma unroll
    for (int k = 0; k < NC; ++k) store_split(Mhi, Mlo, base + (size_t)k * 8, acc[k]);
  }
}

}  // namespace

template <typename T>
cudaError_t launch_p2m(const TreeTables& t, const T* rho, const int dims[3], const Level& leaf, T* Mleaf, T* rho_box,
                       void* Mhi, void* Mlo, void* rho_hi, void* rho_lo, int* flag, cudaStream_t s) {
  const long long threads = leaf.npar * 8;
  if (threads == 0) return cudaSuccess;
  FMM_ORDER_SWITCH(t.p, (p2m_kernel<PP, T><<<grid_threads(threads), kThreads, 0, s>>>(
                            rho, dims[0], dims[1], t.b, leaf, Mleaf, static_cast<__nv_bfloat16*>(Mhi),
                            static_cast<__nv_bfloat16*>(Mlo), rho_box, static_cast<__nv_bfloat16*>(rho_hi),
                            static_cast<__nv_bfloat16*>(rho_lo), flag)));
  return cudaGetLastError();
}

template cudaError_t launch_p2m<float>(const TreeTables&, const float*, const int*, const Level&, float*, float*,
                                       void*, void*, void*, void*, int*, cudaStream_t);
template cudaError_t launch_p2m<double>(const TreeTables&, const double*, const int*, const Level&, double*, double*,
                                        void*, void*, void*, void*, int*, cudaStream_t);

}  // namespace fmmgb
