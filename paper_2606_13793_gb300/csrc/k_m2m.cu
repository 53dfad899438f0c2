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
  m2m_to_parent<P, Tp>(M, p, c, live, par, Mp, Mhi, Mlo, harm, Mfold);
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
