// M2M on the CUDA cores (see tree_common.cuh for the layout and conventions).
#include <cuda_bf16.h>

#include "multi.cuh"
#include "tree_common.cuh"

namespace fmmgb {
namespace {
using namespace tree;

// ---------------------------------------------------------------------------
// M2M (Sec. 2.1, eq. M2M_general, child centre -> parent centre), scaled:
//   Mt_alpha(P) = 2^-|alpha| sum_children sum_{beta <= alpha} C(alpha,beta) (+-1/2)^(alpha-beta) Mt_beta(C)
// Each thread shifts one child; the 8 siblings are summed with shuffles.
// Two blocks per SM for FP32 at p <= 6 (<= 128 registers, no spills): the
// harmonic fold would otherwise take it to 153 registers and one block.
template <int P, typename Tc, typename Tp>
__device__ __forceinline__ void m2m_body(const Level& child, const Tc* __restrict__ Mc, const Level& par,
                                         Tp* __restrict__ Mp, __nv_bfloat16* __restrict__ Mhi,
                                         __nv_bfloat16* __restrict__ Mlo, int harm, Tp* __restrict__ Mfold,
                                         const VBlock& vb) {
  constexpr int NC = ncoef_c(P);
  const long long t = (long long)vb.x * blockDim.x + threadIdx.x;
  const long long p = t >> 3;
  const int c = (int)(t & 7);
  const bool live = p < child.npar;  // child.npar == par.nbox
  Tp M[NC];
  const Tc* src = Mc + (live ? p : 0) * 8 * NC + c;
#pragma unroll
  for (int k = 0; k < NC; ++k) M[k] = live ? Tp(src[k * 8]) : Tp(0);
  Tp dp[P + 1];
  powers<P, Tp>(half_offset<Tp>(c, 0), dp);
  shift_up<P, 0, Tp>(M, dp);
  powers<P, Tp>(half_offset<Tp>(c, 1), dp);
  shift_up<P, 1, Tp>(M, dp);
  powers<P, Tp>(half_offset<Tp>(c, 2), dp);
  shift_up<P, 2, Tp>(M, dp);
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    Tp v = M[k];
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    M[k] = v;
  }
  if (!live) return;
  // box p of the parent level, inside its own parent block
  const int px = (int)(p % par.n[0]);
  const int py = (int)((p / par.n[0]) % par.n[1]);
  const int pz = (int)(p / ((long long)par.n[0] * par.n[1]));
  const long long gp = ((long long)(pz >> 1) * par.np[1] + (py >> 1)) * par.np[0] + (px >> 1);
  const int cp = (px & 1) | ((py & 1) << 1) | ((pz & 1) << 2);
  Tp* dst = Mp + gp * 8 * NC + cp;
  const bool fold = harm && (Mhi || Mfold);
  if (!fold) {
    // sibling lanes share the writes: lane c stores coefficients c, c+8, ...
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      if ((k & 7) != c) continue;
      const int n = (k >= 1) + (k >= 4) + (k >= 10) + (k >= 20) + (k >= 35) + (k >= 56) + (k >= 84) + (k >= 120);
      const Tp v = M[k] * Tp(1.0 / (double)(1 << n));  // 2^-|alpha|
      dst[k * 8] = v;
      if (Mhi) store_split(Mhi, Mlo, (size_t)(gp * 8 * NC + cp + k * 8), v);
    }
    return;
  }
  // harmonic rows: every lane scales and folds the whole expansion, then
  // stores its share of the full row and of the (p+1)^2 folded components
  // ([parent][reduced coef][child]) as bf16 planes and / or in the level's type
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const int n = (k >= 1) + (k >= 4) + (k >= 10) + (k >= 20) + (k >= 35) + (k >= 56) + (k >= 84) + (k >= 120);
    M[k] *= Tp(1.0 / (double)(1 << n));  // 2^-|alpha|
    if ((k & 7) == c) dst[k * 8] = M[k];
  }
  constexpr int NR = nred_c(P);
  harmonic_fold<P, Tp>(M);
  int r = 0;
#pragma unroll
  for (int n = 0; n <= P; ++n)
#pragma unroll
    for (int s = 0; s <= n; ++s)
#pragma unroll
      for (int cc = 0; cc <= 1 && cc <= s; ++cc) {
        if ((r & 7) == c) {
          const size_t o = (size_t)(gp * 8 * NR + cp + r * 8);
          if (Mhi) store_split(Mhi, Mlo, o, M[cidx(n - s, s - cc, cc)]);
          if (Mfold) Mfold[o] = M[cidx(n - s, s - cc, cc)];
        }
        ++r;
      }
}

template <int P, typename Tc, typename Tp>
__global__ void __launch_bounds__(kThreads, (P <= 6 && sizeof(Tp) == 4) ? 2 : 1)
    m2m_kernel(Level child, const Tc* __restrict__ Mc, Level par, Tp* __restrict__ Mp,
               __nv_bfloat16* __restrict__ Mhi, __nv_bfloat16* __restrict__ Mlo, int harm, Tp* __restrict__ Mfold) {
  m2m_body<P, Tc, Tp>(child, Mc, par, Mp, Mhi, Mlo, harm, Mfold, native_vblock());
}

// Many (child level, parent level) pairs in one launch (batched solves).
template <int P, typename Tc, typename Tp>
__global__ void __launch_bounds__(kThreads, (P <= 6 && sizeof(Tp) == 4) ? 2 : 1)
    m2m_multi_kernel(const M2mArgs* __restrict__ a, const MultiGrid* __restrict__ g, int n) {
  const int i = multi_item(g, n);
  const M2mArgs& x = a[i];
  m2m_body<P, Tc, Tp>(x.child, static_cast<const Tc*>(x.Mc), x.par, static_cast<Tp*>(x.Mp),
                      static_cast<__nv_bfloat16*>(x.Mhi), static_cast<__nv_bfloat16*>(x.Mlo), x.harm,
                      static_cast<Tp*>(x.Mfold), multi_vblock(g[i]));
}

}  // namespace

template <typename Tc, typename Tp>
cudaError_t launch_m2m(const TreeTables& t, const Level& child, const Tc* Mc, const Level& par, Tp* Mp, void* Mhi,
                       void* Mlo, int harm, Tp* Mfold, cudaStream_t s) {
  const long long threads = child.npar * 8;
  if (threads == 0) return cudaSuccess;
  const int bs = small_grid_block(threads);
  FMM_ORDER_SWITCH(t.p, (m2m_kernel<PP, Tc, Tp><<<(unsigned)((threads + bs - 1) / bs), bs, 0, s>>>(
                            child, Mc, par, Mp, static_cast<__nv_bfloat16*>(Mhi), static_cast<__nv_bfloat16*>(Mlo),
                            harm, Mfold)));
  return cudaGetLastError();
}

template <typename Tc, typename Tp>
cudaError_t launch_m2m_multi(int p, const M2mArgs* args, const MultiGrid* grids, int n, long long blocks, int bs,
                             cudaStream_t s) {
  if (n == 0 || blocks == 0) return cudaSuccess;
  FMM_ORDER_SWITCH(p, (m2m_multi_kernel<PP, Tc, Tp><<<(unsigned)blocks, bs, 0, s>>>(args, grids, n)));
  return cudaGetLastError();
}
template cudaError_t launch_m2m_multi<float, float>(int, const M2mArgs*, const MultiGrid*, int, long long, int,
                                                    cudaStream_t);
template cudaError_t launch_m2m_multi<double, double>(int, const M2mArgs*, const MultiGrid*, int, long long, int,
                                                      cudaStream_t);

template cudaError_t launch_m2m<float, float>(const TreeTables&, const Level&, const float*, const Level&, float*,
                                              void*, void*, int, float*, cudaStream_t);
template cudaError_t launch_m2m<double, double>(const TreeTables&, const Level&, const double*, const Level&,
                                                double*, void*, void*, int, double*, cudaStream_t);
template cudaError_t launch_m2m<float, double>(const TreeTables&, const Level&, const float*, const Level&, double*,
                                               void*, void*, int, double*, cudaStream_t);

}  // namespace fmmgb
