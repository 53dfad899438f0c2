// Shared helpers of the tree kernels (k_p2m.cu, k_m2m.cu, k_l2l.cu, k_leaf.cu):
// P2M, M2M, L2L and the leaf evaluation on the CUDA cores.
//
// One thread owns one box and keeps its expansion in registers: the order p
// is a template parameter, so every coefficient index is a compile-time
// constant.  Threads are numbered (parent box, child) with the child fastest,
// so a warp covers 4 parent blocks and the parent-blocked arrays
// ([coef][child], 8*nc contiguous values per parent) are read and written as
// full 32-byte sectors.  The translations are separable per axis:
//   * P2M / L2P factorise (x - c)^alpha per axis (~b^3 (p+1) * 3 multiply-adds
//     per box instead of b^3 * nc);
//   * M2M / L2L shift one axis at a time, in place, with the half-box offset
//     d = +-1/2 (child units), then siblings are summed by warp shuffles.
// Optional bf16 hi/lo planes (hi = rn(x), lo = rn(x - hi)) are written next to
// the FP32 values for levels whose M2L runs on the tensor cores, and for the
// box-blocked density the tensor-core near field reads.
#include <cuda_bf16.h>

#pragma once
#include "fmm_internal.h"

namespace fmmgb {
namespace tree {

constexpr int kThreads = 256;  // 32 parents x 8 children

__host__ __device__ constexpr int ncoef_c(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

// Index of multi-index (a, b, c) in the canonical order (total order n, then
// a descending, then b descending).
__host__ __device__ constexpr int cidx(int a, int b, int c) {
  return (a + b + c) * (a + b + c + 1) * (a + b + c + 2) / 6 + (b + c) * (b + c + 1) / 2 + c;
}

// Harmonic compression (traceless multipoles): 1/r is harmonic, so its
// derivatives obey D_{g+2z} = -D_{g+2x} - D_{g+2y}, which keeps the total order.
// With the symmetric truncation |alpha| + |beta| <= p this makes the M2L
// contraction depend only on the components with c <= 1 ((p+1)^2 of them
// instead of nc(p)), exactly:
//   * multipoles fold onto c <= 1 (in the scaled variables
//     Mt_(a+2,b,c-2) -= (a+2)(a+1)/(c(c-1)) Mt_(a,b,c), likewise for b, taking c
//     from the top down);
//   * locals (Laplacian of the potential = 0 in the box) are rebuilt from c <= 1:
//     Lt_(a,b,c) = -[(a+2)(a+1) Lt_(a+2,b,c-2) + (b+2)(b+1) Lt_(a,b+2,c-2)] / (c(c-1)).
// Reduced components are ordered like the canonical order restricted to c <= 1.
__host__ __device__ constexpr int nred_c(int p) { return (p + 1) * (p + 1); }
__host__ __device__ constexpr int ridx(int a, int b, int c) {
  return (a + b + c) * (a + b + c) + ((b + c) == 0 ? 0 : 2 * (b + c) - 1 + c);
}

template <int P, typename T>
__host__ __device__ __forceinline__ void harmonic_fold(T (&M)[(P + 1) * (P + 2) * (P + 3) / 6]) {
#pragma unroll
  for (int c = P; c >= 2; --c)
#pragma unroll
    for (int a = 0; a + c <= P; ++a)
#pragma unroll
      for (int b = 0; a + b + c <= P; ++b) {
        const T f = M[cidx(a, b, c)] * T(1.0 / (double)(c * (c - 1)));
        M[cidx(a + 2, b, c - 2)] -= T((a + 2) * (a + 1)) * f;
        M[cidx(a, b + 2, c - 2)] -= T((b + 2) * (b + 1)) * f;
      }
}

template <int P, typename T>
__host__ __device__ __forceinline__ void harmonic_expand(T (&L)[(P + 1) * (P + 2) * (P + 3) / 6]) {
#pragma unroll
  for (int c = 2; c <= P; ++c)
#pragma unroll
    for (int a = 0; a + c <= P; ++a)
#pragma unroll
      for (int b = 0; a + b + c <= P; ++b)
        L[cidx(a, b, c)] = -(T((a + 2) * (a + 1)) * L[cidx(a + 2, b, c - 2)] +
                             T((b + 2) * (b + 1)) * L[cidx(a, b + 2, c - 2)]) *
                           T(1.0 / (double)(c * (c - 1)));
}

__host__ __device__ constexpr int binom_c(int n, int k) {
  int r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

template <typename T>
__device__ __forceinline__ void store_split(__nv_bfloat16* hi, __nv_bfloat16* lo, size_t i, T x) {
  const float f = (float)x;
  const __nv_bfloat16 h = __float2bfloat16_rn(f);
  hi[i] = h;
  lo[i] = __float2bfloat16_rn(f - __bfloat162float(h));
}

// In-place upward (multipole) shift along axis Q by d:
//   M'_{..a..} = sum_{a' <= a} C(a, a') d^(a - a') M_{..a'..}
template <int P, int Q, typename T>
__host__ __device__ __forceinline__ void shift_up(T (&M)[ncoef_c(P)], const T (&dp)[P + 1]) {
#pragma unroll
  for (int u = 0; u <= P; ++u)
#pragma unroll
    for (int v = 0; u + v <= P; ++v)
#pragma unroll
      for (int a = P - u - v; a >= 1; --a) {
        T s = M[Q == 0 ? cidx(a, u, v) : (Q == 1 ? cidx(u, a, v) : cidx(u, v, a))];
#pragma unroll
        for (int k = 0; k < a; ++k) {
          const int id = Q == 0 ? cidx(k, u, v) : (Q == 1 ? cidx(u, k, v) : cidx(u, v, k));
          s = fma(T(binom_c(a, k)) * dp[a - k], M[id], s);
        }
        M[Q == 0 ? cidx(a, u, v) : (Q == 1 ? cidx(u, a, v) : cidx(u, v, a))] = s;
      }
}

// In-place downward (local) shift along axis Q by d:
//   L'_{..a..} = sum_{a' >= a} C(a', a) d^(a' - a) L_{..a'..}
template <int P, int Q, typename T>
__host__ __device__ __forceinline__ void shift_down(T (&L)[ncoef_c(P)], const T (&dp)[P + 1]) {
#pragma unroll
  for (int u = 0; u <= P; ++u)
#pragma unroll
    for (int v = 0; u + v <= P; ++v)
#pragma unroll
      for (int a = 0; a < P - u - v; ++a) {
        T s = L[Q == 0 ? cidx(a, u, v) : (Q == 1 ? cidx(u, a, v) : cidx(u, v, a))];
#pragma unroll
        for (int k = a + 1; k <= P - u - v; ++k) {
          const int id = Q == 0 ? cidx(k, u, v) : (Q == 1 ? cidx(u, k, v) : cidx(u, v, k));
          s = fma(T(binom_c(k, a)) * dp[k - a], L[id], s);
        }
        L[Q == 0 ? cidx(a, u, v) : (Q == 1 ? cidx(u, a, v) : cidx(u, v, a))] = s;
      }
}

template <int P, typename T>
__host__ __device__ __forceinline__ void powers(T x, T (&dp)[P + 1]) {
  dp[0] = T(1);
#pragma unroll
  for (int k = 1; k <= P; ++k) dp[k] = dp[k - 1] * x;
}

// Child c of a parent box sits at +-1/2 child box along each axis.
template <typename T>
__host__ __device__ __forceinline__ T half_offset(int c, int q) {
  return ((c >> q) & 1) ? T(0.5) : T(-0.5);
}

struct Box {
  long long par;  // parent block index
  int c;          // child index
  int x, y, z;    // box coordinates at the child level
  bool real;      // inside the level's extent
};

__device__ __forceinline__ Box box_of(const Level& lv, long long t) {
  Box B;
  B.par = t >> 3;
  B.c = (int)(t & 7);
  const int px = (int)(B.par % lv.np[0]);
  const int py = (int)((B.par / lv.np[0]) % lv.np[1]);
  const int pz = (int)(B.par / ((long long)lv.np[0] * lv.np[1]));
  B.x = 2 * px + (B.c & 1);
  B.y = 2 * py + ((B.c >> 1) & 1);
  B.z = 2 * pz + (B.c >> 2);
  B.real = B.par < lv.npar && B.x < lv.n[0] && B.y < lv.n[1] && B.z < lv.n[2];
  return B;
}

inline unsigned grid_threads(long long threads) { return (unsigned)((threads + kThreads - 1) / kThreads); }

// Block size of the coarse-level shifts (M2M / L2L): a grid that would not
// give every SM a block of kThreads runs warp-sized blocks instead, so its few
// warps spread over the SMs (the FP64 levels are bound by each SM's DFMA rate:
// at 512^3 their launches drop from ~50 to a few microseconds).
inline int small_grid_block(long long threads) { return threads < 152LL * kThreads ? 32 : kThreads; }

#define FMM_ORDER_SWITCH(p, ...)                          \
  switch (p) {                                            \
    case 0: { constexpr int PP = 0; __VA_ARGS__; } break; \
    case 1: { constexpr int PP = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int PP = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int PP = 3; __VA_ARGS__; } break; \
    case 4: { constexpr int PP = 4; __VA_ARGS__; } break; \
    case 5: { constexpr int PP = 5; __VA_ARGS__; } break; \
    case 6: { constexpr int PP = 6; __VA_ARGS__; } break; \
    case 7: { constexpr int PP = 7; __VA_ARGS__; } break; \
    case 8: { constexpr int PP = 8; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;                \
  }

// M2M (Sec. 2.1, eq. M2M_general) of one child's scaled multipoles M (in
// registers, overwritten) onto its parent p, a box of level `par`; lane c =
// the child (lanes 8j .. 8j + 7 of a warp are one parent's 8 children, all 32
// lanes take part in the shuffles), `live` false for padding lanes.  Writes
// the parent's scaled multipoles 2^-|alpha| sum_children ... into Mp (its own
// parent-blocked slot) and, when given, the bf16 hi / lo planes and the
// folded harmonic rows.
template <int P, typename Tp>
__device__ __forceinline__ void m2m_to_parent(Tp (&M)[ncoef_c(P)], long long p, int c, bool live, const Level& par,
                                              Tp* __restrict__ Mp, __nv_bfloat16* __restrict__ Mhi,
                                              __nv_bfloat16* __restrict__ Mlo, int harm, Tp* __restrict__ Mfold) {
  constexpr int NC = ncoef_c(P);
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

// L2L (Sec. 2.3, eq. L2L) of the parent's scaled locals onto child c, plus
// the child's own M2L locals, in registers: the arithmetic of one L2L thread
// (k_l2l.cu).  p: the parent, a box of level `par`; Lp (NULL: no parent
// locals) the parent level's locals; own = the child's row in the child
// level's locals (stride 8: [coef][child]), read where the M2L wrote it
// (accumulate = 1); harm = 1: the M2L wrote only its c <= 1 locals, in own
// or, with Lred, in compact rows; the c >= 2 components are rebuilt.
template <int P, typename Tp, typename Tc>
__device__ __forceinline__ void l2l_child(Tp (&L)[ncoef_c(P)], const Level& par, const Tp* __restrict__ Lp,
                                          long long p, int c, int accumulate, int harm, const Tc* own,
                                          const Tc* __restrict__ Lred) {
  constexpr int NC = ncoef_c(P);
  if (Lp) {
    const int px = (int)(p % par.n[0]);
    const int py = (int)((p / par.n[0]) % par.n[1]);
    const int pz = (int)(p / ((long long)par.n[0] * par.n[1]));
    const long long gp = ((long long)(pz >> 1) * par.np[1] + (py >> 1)) * par.np[0] + (px >> 1);
    const int cp = (px & 1) | ((py & 1) << 1) | ((pz & 1) << 2);
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
  if (accumulate && harm) {
    // The parent's shifted locals are harmonic too (an exact re-expansion of
    // a harmonic polynomial), so the sum is: add the c <= 1 values, then
    // rebuild the c >= 2 components of the sum from the Laplace identity.
    constexpr int NR = nred_c(P);
    const Tc* red = Lred ? Lred + p * 8 * NR + c : nullptr;
#pragma unroll
    for (int n = 0; n <= P; ++n)
#pragma unroll
      for (int s = 0; s <= n; ++s)
#pragma unroll
        for (int cc = 0; cc <= 1 && cc <= s; ++cc)
          L[cidx(n - s, s - cc, cc)] +=
              Tp(red ? red[ridx(n - s, s - cc, cc) * 8] : own[cidx(n - s, s - cc, cc) * 8]);
    harmonic_expand<P, Tp>(L);
  } else if (accumulate) {
#pragma unroll
    for (int k = 0; k < NC; ++k) L[k] = Tp(Tc(own[k * 8]) + Tc(L[k]));
  }
}

}  // namespace tree
}  // namespace fmmgb
