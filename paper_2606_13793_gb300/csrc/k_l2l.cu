// L2L on the CUDA cores (see tree_common.cuh for the layout and conventions).
#include <cuda_bf16.h>

#include "multi.cuh"
#include "tree_common.cuh"

namespace fmmgb {
namespace {
using namespace tree;

// ---------------------------------------------------------------------------
// L2L (Sec. 2.3, eq. L2L, parent centre -> child centre), scaled:
//   Lt_beta(C) = sum_{gamma >= beta} C(gamma,beta) 2^(-1-|gamma|) (+-1/2)^(gamma-beta) Lt_gamma(P)
// Adds to the children's block, which the level's M2L has already written
// (accumulate = 0 overwrites it instead).  harm = 1: the M2L wrote only the
// harmonic components (c <= 1); the others are rebuilt from them first.
// Lp = NULL: no parent locals (the coarsest level: only the rebuild).
template <int P, typename Tp, typename Tc>
__device__ __forceinline__ void l2l_body(const Level& par, const Tp* __restrict__ Lp, const Level& child,
                                         Tc* __restrict__ Lc, int accumulate, int harm, const Tc* __restrict__ Lred,
                                         const VBlock& vb) {
  constexpr int NC = ncoef_c(P);
  const long long t = (long long)vb.x * blockDim.x + threadIdx.x;
  const long long p = t >> 3;  // box of the parent level == parent block of the child level
  const int c = (int)(t & 7);
  if (p >= par.nbox) return;
  Tp L[NC];
  Tc* dst = Lc + p * 8 * NC + c;
  l2l_child<P, Tp, Tc>(L, par, Lp, p, c, accumulate, harm, dst, Lred);
#pragma unroll
  for (int k = 0; k < NC; ++k) dst[k * 8] = Tc(L[k]);
}

template <int P, typename Tp, typename Tc>
__global__ void __launch_bounds__(kThreads) l2l_kernel(Level par, const Tp* __restrict__ Lp, Level child,
                                                       Tc* __restrict__ Lc, int accumulate, int harm,
                                                       const Tc* __restrict__ Lred) {
  l2l_body<P, Tp, Tc>(par, Lp, child, Lc, accumulate, harm, Lred, native_vblock());
}

// Many (parent level, child level) pairs in one launch (batched solves).
template <int P, typename Tp, typename Tc>
__global__ void __launch_bounds__(kThreads) l2l_multi_kernel(const L2lArgs* __restrict__ a,
                                                             const MultiGrid* __restrict__ g, int n) {
  const int i = multi_item(g, n);
  const L2lArgs& x = a[i];
  l2l_body<P, Tp, Tc>(x.par, static_cast<const Tp*>(x.Lp), x.child, static_cast<Tc*>(x.Lc), x.accumulate, x.harm,
                      static_cast<const Tc*>(x.Lred), multi_vblock(g[i]));
}

}  // namespace

template <typename Tp, typename Tc>
cudaError_t launch_l2l(const TreeTables& t, const Level& par, const Tp* Lp, const Level& child, Tc* Lc, int accumulate,
                       int harm, const Tc* Lred, cudaStream_t s) {
  const long long threads = par.nbox * 8;
  if (threads == 0) return cudaSuccess;
  const int bs = small_grid_block(threads);
  FMM_ORDER_SWITCH(t.p, (l2l_kernel<PP, Tp, Tc><<<(unsigned)((threads + bs - 1) / bs), bs, 0, s>>>(par, Lp, child, Lc,
                                                                                          accumulate, harm, Lred)));
  return cudaGetLastError();
}

template <typename Tp, typename Tc>
cudaError_t launch_l2l_multi(int p, const L2lArgs* args, const MultiGrid* grids, int n, long long blocks, int bs,
                             cudaStream_t s) {
  if (n == 0 || blocks == 0) return cudaSuccess;
  FMM_ORDER_SWITCH(p, (l2l_multi_kernel<PP, Tp, Tc><<<(unsigned)blocks, bs, 0, s>>>(args, grids, n)));
  return cudaGetLastError();
}
template cudaError_t launch_l2l_multi<float, float>(int, const L2lArgs*, const MultiGrid*, int, long long, int,
                                                    cudaStream_t);
template cudaError_t launch_l2l_multi<double, double>(int, const L2lArgs*, const MultiGrid*, int, long long, int,
                                                      cudaStream_t);

template cudaError_t launch_l2l<float, float>(const TreeTables&, const Level&, const float*, const Level&, float*, int,
                                              int, const float*, cudaStream_t);
template cudaError_t launch_l2l<double, double>(const TreeTables&, const Level&, const double*, const Level&,
                                                double*, int, int, const double*, cudaStream_t);
template cudaError_t launch_l2l<double, float>(const TreeTables&, const Level&, const double*, const Level&, float*,
                                               int, int, const float*, cudaStream_t);

}  // namespace fmmgb
