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
  const int px = (int)(p % par.n[0]);
  const int py = (int)((p / par.n[0]) % par.n[1]);
  const int pz = (int)(p / ((long long)par.n[0] * par.n[1]));
  const long long gp = ((long long)(pz >> 1) * par.np[1] + (py >> 1)) * par.np[0] + (px >> 1);
  const int cp = (px & 1) | ((py & 1) << 1) | ((pz & 1) << 2);
  Tp L[NC];
  if (Lp) {
    const Tp* src = Lp + gp * 8 * NC + cp;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const int n = (k >= 1) + (k >= 4) + (k >= 10) + (k >= 20) + (k >= 35) + (k >= 56) + (k >= 84) + (k >= 120);
      L[k] = src[k * 8] * Tp(1.0 / (double)(2 << n));  // 2^(-1-|gamma|)
    }
    Tp dp[P + 1];
    powers<P, Tp>(half_offset<Tp>(c, 0), dp);
    shift_down<P, 0, Tp>(L, dp);
    powers<P, Tp>(half_offset<Tp>(c, 1), dp);
    shift_down<P, 1, Tp>(L, dp);
    powers<P, Tp>(half_offset<Tp>(c, 2), dp);
    shift_down<P, 2, Tp>(L, dp);
  } else {
#pragma unroll
    for (int k = 0; k < NC; ++k) L[k] = Tp(0);
  }
  Tc* dst = Lc + p * 8 * NC + c;
  if (accumulate && harm) {
    // The M2L wrote only its c <= 1 locals (in the full rows, tensor cores, or
    // in compact rows [parent][reduced coef][child], CUDA cores).  The
    // parent's shifted locals are harmonic too (an exact re-expansion of a
    // harmonic polynomial), so the sum is: add the c <= 1 values, then rebuild
    // the c >= 2 components of the sum from the Laplace identity, in place.
    constexpr int NR = nred_c(P);
    const Tc* red = Lred ? Lred + p * 8 * NR + c : nullptr;
#pragma unroll
    for (int n = 0; n <= P; ++n)
#pragma unroll
      for (int s = 0; s <= n; ++s)
#pragma unroll
        for (int cc = 0; cc <= 1 && cc <= s; ++cc)
          L[cidx(n - s, s - cc, cc)] +=
              Tp(red ? red[ridx(n - s, s - cc, cc) * 8] : dst[cidx(n - s, s - cc, cc) * 8]);
    harmonic_expand<P, Tp>(L);
#pragma unroll
    for (int k = 0; k < NC; ++k) dst[k * 8] = Tc(L[k]);
  } else {
#pragma unroll
    for (int k = 0; k < NC; ++k) dst[k * 8] = accumulate ? Tc(dst[k * 8] + Tc(L[k])) : Tc(L[k]);
  }
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
