// P2M on the CUDA cores (see tree_common.cuh for the layout and conventions).
#include <cuda_bf16.h>

#include "multi.cuh"
#include "tree_common.cuh"

namespace fmmgb {
namespace {
using namespace tree;

// ---------------------------------------------------------------------------
// P2M (Sec. 2.1, eq. multipole) about each leaf-box centre, scaled:
//   Mt_alpha = sum_cells m ((x - c)/b)^alpha
// plus the box-blocked copy of the density for the near field.
//
// Two threads per box, in adjacent warps: the thread of parity h accumulates
// the coefficients whose z power c has parity h (50 and 34 of the 84 at
// p = 6), so a thread holds about half the expansion in registers and twice
// as many warps fit on an SM to hide the density loads (the second warp's
// reads of the same cells hit L1).  The parity is warp-uniform and selects a
// body instantiated for it, so every register index stays compile-time.
constexpr int kP2mParents = kThreads / 16;  // 2 threads per box, 8 boxes per parent

template <int P>
__host__ __device__ constexpr int ncoef_parity(int h) {
  int n = 0;
  for (int c = h; c <= P; c += 2) n += (P - c + 1) * (P - c + 2) / 2;
  return n;
}

// DIP: dipole sources as well (the transpose of the analytic force's far
// part, the gradient of L2P): dip = [3][cells] weights v_q, each cell adding
// v_q d/de_q (e^alpha) (box units) to the monomial moments of its density.
template <int P, typename T, int h, bool DIP>
__device__ __forceinline__ void p2m_body(const Box& B, const T* __restrict__ rho, int nx, int ny, int b,
                                         const Level& leaf, T* __restrict__ Ms, T* __restrict__ Mr,
                                         T* __restrict__ rho_box, __nv_bfloat16* __restrict__ rhi,
                                         __nv_bfloat16* __restrict__ rlo, int* __restrict__ flag,
                                         const T* __restrict__ dip, long long ncell) {
  constexpr int NC = ncoef_c(P);
  constexpr int NH = ncoef_parity<P>(h);
  T acc[NH > 0 ? NH : 1];  // this thread's coefficients, in canonical order restricted to parity h of c
#pragma unroll
  for (int k = 0; k < NH; ++k) acc[k] = T(0);
  bool bad = false;  // non-finite density (reported through the plan's flag)
  // One z-plane of the box: rows j = 0 .. b-1 of cells m[j][i] -> partial sums
  // t2[(a, bb)] = sum_j yj^bb sum_i m xi^a, then acc += t2 zk^c (this parity).
  // vrow (DIP): the plane's three dipole rows, [3][b * b]
  auto plane = [&](const T* mrow, const T* vrow, int k, const T inv_b) {
    constexpr int N2 = (P + 1) * (P + 2) / 2;
    T t2[N2], t2z[DIP ? N2 : 1];
#pragma unroll
    for (int q = 0; q < N2; ++q) t2[q] = T(0);
    if (DIP) {
#pragma unroll
      for (int q = 0; q < N2; ++q) t2z[q] = T(0);
    }
    for (int j = 0; j < b; ++j) {
      const T yj = (T(j) + T(0.5)) * inv_b - T(0.5);
      // t1: sum_i m xi^a (+ v_x a xi^(a-1)); t1y, t1z: sum_i v_y xi^a, v_z xi^a
      T t1[P + 1], t1y[DIP ? P + 1 : 1], t1z[DIP ? P + 1 : 1];
#pragma unroll
      for (int a = 0; a <= P; ++a) t1[a] = T(0);
      if (DIP) {
#pragma unroll
        for (int a = 0; a <= P; ++a) t1y[a] = T(0), t1z[a] = T(0);
      }
      for (int i = 0; i < b; ++i) {
        const T mi = mrow[j * b + i];
        bad |= !isfinite(mi);
        const T xi = (T(i) + T(0.5)) * inv_b - T(0.5);
        T w = mi;
#pragma unroll
        for (int a = 0; a <= P; ++a) {
          t1[a] += w;
          w *= xi;
        }
        if (DIP) {
          const T vx = vrow[j * b + i], vy = vrow[b * b + j * b + i], vz = vrow[2 * b * b + j * b + i];
          T pw = vx, wy = vy, wz = vz;  // vx xi^(a-1), vy xi^a, vz xi^a
#pragma unroll
          for (int a = 0; a <= P; ++a) {
            if (a >= 1) {
              t1[a] = fma(T(a), pw, t1[a]);
              pw *= xi;
            }
            t1y[a] += wy;
            t1z[a] += wz;
            wy *= xi;
            wz *= xi;
          }
        }
      }
      T ypow[P + 1];
      powers<P, T>(yj, ypow);
#pragma unroll
      for (int a = 0; a <= P; ++a)
#pragma unroll
        for (int bb = 0; a + bb <= P; ++bb) {
          T v = t1[a] * ypow[bb];
          if (DIP) {
            if (bb >= 1) v = fma(t1y[a], T(bb) * ypow[bb - 1], v);
            t2z[(a + bb) * (a + bb + 1) / 2 + bb] = fma(t1z[a], ypow[bb], t2z[(a + bb) * (a + bb + 1) / 2 + bb]);
          }
          t2[(a + bb) * (a + bb + 1) / 2 + bb] += v;
        }
    }
    const T zk = (T(k) + T(0.5)) * inv_b - T(0.5);
    T zpow[P + 1];
    powers<P, T>(zk, zpow);
    int q = 0;
#pragma unroll
    for (int n = 0; n <= P; ++n)
#pragma unroll
      for (int bc = 0; bc <= n; ++bc)  // canonical order: a descending, then b descending
#pragma unroll
        for (int cc = 0; cc <= bc; ++cc) {
          const int a = n - bc, bb = bc - cc;
          if ((cc & 1) != h) continue;
          acc[q] = fma(t2[(a + bb) * (a + bb + 1) / 2 + bb], zpow[cc], acc[q]);
          if (DIP && cc >= 1) acc[q] = fma(t2z[(a + bb) * (a + bb + 1) / 2 + bb], T(cc) * zpow[cc - 1], acc[q]);
          ++q;
        }
  };
  if (B.real) {
    const T inv_b = T(1) / T(b);
    const long long box = ((long long)B.z * leaf.n[1] + B.y) * leaf.n[0] + B.x;
    const int b3 = b * b * b;
    if (sizeof(T) == 4 && b == 4 && !DIP) {
      // two z-planes (8 rows of 16 bytes) in flight per thread before any use
      for (int k0 = 0; k0 < 4; k0 += 2) {
        float4 v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r)
          v[r] = __ldg(reinterpret_cast<const float4*>(
              rho + ((long long)(B.z * 4 + k0 + (r >> 2)) * ny + (B.y * 4 + (r & 3))) * nx + (long long)B.x * 4));
        if (h == 0) {
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const long long e0 = box * 64 + (k0 * 4 + r) * 4;
            if (rho_box) *reinterpret_cast<float4*>(rho_box + e0) = v[r];
            if (rhi) {
              const float m4[4] = {v[r].x, v[r].y, v[r].z, v[r].w};
              __nv_bfloat16 hh[4], ll[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                hh[i] = __float2bfloat16_rn(m4[i]);
                ll[i] = __float2bfloat16_rn(m4[i] - __bfloat162float(hh[i]));
              }
              *reinterpret_cast<uint2*>(rhi + e0) = *reinterpret_cast<const uint2*>(hh);
              *reinterpret_cast<uint2*>(rlo + e0) = *reinterpret_cast<const uint2*>(ll);
            }
          }
        }
        plane(reinterpret_cast<const T*>(&v[0]), nullptr, k0, inv_b);
        plane(reinterpret_cast<const T*>(&v[4]), nullptr, k0 + 1, inv_b);
      }
    } else {
      for (int k = 0; k < b; ++k) {
        T mrow[64];  // b <= 8: one plane of b x b cells
        T vrow[DIP ? 3 * 64 : 1];
        for (int j = 0; j < b; ++j) {
          const long long c0 = ((long long)(B.z * b + k) * ny + (B.y * b + j)) * nx + (long long)B.x * b;
          const T* row = rho + c0;
          const long long e0 = box * b3 + (k * b + j) * b;
          for (int i = 0; i < b; ++i) {
            const T m = row[i];
            mrow[j * b + i] = m;
            if (DIP)
              for (int q = 0; q < 3; ++q) vrow[q * b * b + j * b + i] = dip[q * ncell + c0 + i];
            if (h == 0) {
              if (rho_box) rho_box[e0 + i] = m;
              if (rhi) store_split(rhi, rlo, (size_t)(e0 + i), m);
            }
          }
        }
        plane(mrow, DIP ? vrow : nullptr, k, inv_b);
      }
    }
  }
  if (bad && h == 0) atomicOr(flag, 1);
  // into the block's staged parent rows [parent][coef][child] (rows padded
  // by 8 values so the four parents of a warp fall in different banks)
  T* dst = Ms + (B.par & (kP2mParents - 1)) * (8 * NC + 8) + B.c;
  int q = 0;
#pragma unroll
  for (int n = 0; n <= P; ++n)
#pragma unroll
    for (int bc = 0; bc <= n; ++bc)
#pragma unroll
      for (int cc = 0; cc <= bc; ++cc) {
        const int a = n - bc, bb = bc - cc;
        if ((cc & 1) != h) continue;
        dst[cidx(a, bb, cc) * 8] = acc[q];
        ++q;
      }
  if (Mr) {
    // harmonic planes: this thread's parity class folds onto c = h (the fold
    // keeps the parity of c), staged as [parent][reduced coef][child]
    constexpr int NR = nred_c(P);
    T f[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) f[k] = T(0);
    int r = 0;
#pragma unroll
    for (int n = 0; n <= P; ++n)
#pragma unroll
      for (int bc = 0; bc <= n; ++bc)
#pragma unroll
        for (int cc = 0; cc <= bc; ++cc) {
          if ((cc & 1) != h) continue;
          f[cidx(n - bc, bc - cc, cc)] = acc[r];
          ++r;
        }
    harmonic_fold<P, T>(f);
    T* dr = Mr + (B.par & (kP2mParents - 1)) * (8 * NR + 8) + B.c;
#pragma unroll
    for (int n = h; n <= P; ++n)
#pragma unroll
      for (int s = h; s <= n; ++s) dr[ridx(n - s, s - h, h) * 8] = f[cidx(n - s, s - h, h)];
  }
}

// A block (256 threads, 128 boxes) covers kP2mParents whole parents, so its
// output is one contiguous run of parent rows: staged in shared memory and
// written with 16-byte stores (FP32 rows, and the bf16 hi/lo planes).
template <int P, typename T, bool DIP>
__device__ __forceinline__ void p2m_block(const T* __restrict__ rho, int nx, int ny, int b, const Level& leaf,
                                          T* __restrict__ Mleaf, __nv_bfloat16* __restrict__ Mhi,
                                          __nv_bfloat16* __restrict__ Mlo, T* __restrict__ rho_box,
                                          __nv_bfloat16* __restrict__ rhi, __nv_bfloat16* __restrict__ rlo,
                                          int* __restrict__ flag, int harm, T* __restrict__ Mfold,
                                          const T* __restrict__ dip, long long ncell, const VBlock& vb) {
  constexpr int NC = ncoef_c(P);
  constexpr int ROW = 8 * NC;     // values per parent row
  constexpr int ROWP = ROW + 8;   // staged row pitch
  constexpr int ROWR = 8 * nred_c(P);  // values per parent row of the harmonic planes
  extern __shared__ __align__(16) unsigned char p2m_smem[];
  T* Ms = reinterpret_cast<T*>(p2m_smem);
  T* Mr = (harm && (Mhi || Mfold)) ? Ms + kP2mParents * ROWP : nullptr;
  const long long t = (long long)vb.x * kThreads + threadIdx.x;
  const long long w = t >> 5;
  const Box B = box_of(leaf, (w >> 1) * 32 + (t & 31));
  if (B.par < leaf.npar) {
    if (w & 1)
      p2m_body<P, T, 1, DIP>(B, rho, nx, ny, b, leaf, Ms, Mr, rho_box, rhi, rlo, flag, dip, ncell);
    else
      p2m_body<P, T, 0, DIP>(B, rho, nx, ny, b, leaf, Ms, Mr, rho_box, rhi, rlo, flag, dip, ncell);
  }
  __syncthreads();
  const long long p0 = (long long)vb.x * kP2mParents;
  const long long np = min((long long)kP2mParents, leaf.npar - p0);
  if (np <= 0) return;
  const int count = (int)np * ROW;  // a multiple of 8
  const long long g0 = p0 * ROW;
  if (sizeof(T) == 4) {
    float4* out = reinterpret_cast<float4*>(Mleaf + g0);
    for (int i = threadIdx.x; i < count / 4; i += kThreads) {
      const int pr = i / (ROW / 4), wi = i % (ROW / 4);
      out[i] = *reinterpret_cast<const float4*>(Ms + pr * ROWP + wi * 4);
    }
  } else {
    for (int i = threadIdx.x; i < count; i += kThreads) Mleaf[g0 + i] = Ms[(i / ROW) * ROWP + i % ROW];
  }
  if (Mfold) {  // the folded multipoles in the level's type (CUDA-core harmonic M2L)
    const int pc = (int)np * ROWR;
    for (int i = threadIdx.x; i < pc; i += kThreads) Mfold[p0 * ROWR + i] = Mr[(i / ROWR) * (ROWR + 8) + i % ROWR];
  }
  if (Mhi) {  // 8 values -> 16 bytes of hi and 16 bytes of lo
    const int rl = Mr ? ROWR : ROW, rp = Mr ? ROWR + 8 : ROWP;
    const T* src = Mr ? Mr : Ms;
    const int pc = (int)np * rl;
    const long long h0 = p0 * rl;
    for (int i = threadIdx.x; i < pc / 8; i += kThreads) {
      const T* v = src + (i / (rl / 8)) * rp + (i % (rl / 8)) * 8;
      __nv_bfloat16 hh[8], ll[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float x = (float)v[q];
        hh[q] = __float2bfloat16_rn(x);
        ll[q] = __float2bfloat16_rn(x - __bfloat162float(hh[q]));
      }
      reinterpret_cast<uint4*>(Mhi + h0)[i] = *reinterpret_cast<const uint4*>(hh);
      reinterpret_cast<uint4*>(Mlo + h0)[i] = *reinterpret_cast<const uint4*>(ll);
    }
  }
}

template <int P, typename T, bool DIP>
__global__ void __launch_bounds__(kThreads) p2m_kernel(const T* __restrict__ rho, int nx, int ny, int b, Level leaf,
                                                       T* __restrict__ Mleaf, __nv_bfloat16* __restrict__ Mhi,
                                                       __nv_bfloat16* __restrict__ Mlo, T* __restrict__ rho_box,
                                                       __nv_bfloat16* __restrict__ rhi,
                                                       __nv_bfloat16* __restrict__ rlo, int* __restrict__ flag,
                                                       int harm, T* __restrict__ Mfold, const T* __restrict__ dip,
                                                       long long ncell) {
  p2m_block<P, T, DIP>(rho, nx, ny, b, leaf, Mleaf, Mhi, Mlo, rho_box, rhi, rlo, flag, harm, Mfold, dip, ncell,
                       native_vblock());
}

// The leaf levels of many solves in one launch (batched solves).
template <int P, typename T>
__global__ void __launch_bounds__(kThreads) p2m_multi_kernel(const P2mArgs* __restrict__ a,
                                                             const MultiGrid* __restrict__ g, int n) {
  __shared__ P2mArgs x;  // the item's arguments, read by the body from shared memory
  const int i = multi_item(g, n);
  if (threadIdx.x == 0 && threadIdx.y == 0) x = a[i];
  __syncthreads();
  p2m_block<P, T, false>(static_cast<const T*>(x.rho), x.nx, x.ny, x.b, x.leaf, static_cast<T*>(x.Mleaf),
                         static_cast<__nv_bfloat16*>(x.Mhi), static_cast<__nv_bfloat16*>(x.Mlo),
                         static_cast<T*>(x.rho_box), static_cast<__nv_bfloat16*>(x.rho_hi),
                         static_cast<__nv_bfloat16*>(x.rho_lo), x.flag, x.harm, static_cast<T*>(x.Mfold), nullptr,
                         x.ncell, multi_vblock(g[i]));
}

template <int P, typename T>
cudaError_t p2m_multi_launch(const P2mArgs* args, const MultiGrid* grids, int n, long long blocks, int harm_rows,
                             cudaStream_t s) {
  constexpr size_t full = (size_t)kP2mParents * (8 * ncoef_c(P) + 8) * sizeof(T);
  constexpr size_t red0 = (size_t)kP2mParents * (8 * nred_c(P) + 8) * sizeof(T);
  constexpr size_t red = full + red0 <= 227 * 1024 ? red0 : 0;
  if (harm_rows && red == 0) return cudaErrorInvalidValue;
  const size_t smem = full + (harm_rows ? red : 0);
  static bool attr = false;
  if (!attr && full + red > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(p2m_multi_kernel<P, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(full + red));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  p2m_multi_kernel<P, T><<<(unsigned)blocks, kThreads, smem, s>>>(args, grids, n);
  return cudaGetLastError();
}

template <int P, typename T, bool DIP>
cudaError_t p2m_launch_dip(unsigned blocks, size_t smem, size_t attr_bytes, cudaStream_t s, const T* rho, int nx,
                           int ny, int b, Level leaf, T* Mleaf, __nv_bfloat16* Mhi, __nv_bfloat16* Mlo, T* rho_box,
                           __nv_bfloat16* rhi, __nv_bfloat16* rlo, int* flag, int harm, T* Mfold, const T* dip,
                           long long ncell) {
  static bool attr = false;
  if (!attr && attr_bytes > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(p2m_kernel<P, T, DIP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)attr_bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  p2m_kernel<P, T, DIP><<<blocks, kThreads, smem, s>>>(rho, nx, ny, b, leaf, Mleaf, Mhi, Mlo, rho_box, rhi, rlo, flag,
                                                       harm, Mfold, dip, ncell);
  return cudaGetLastError();
}

template <int P, typename T>
cudaError_t p2m_launch(unsigned blocks, cudaStream_t s, const T* rho, int nx, int ny, int b, Level leaf, T* Mleaf,
                __nv_bfloat16* Mhi, __nv_bfloat16* Mlo, T* rho_box, __nv_bfloat16* rhi, __nv_bfloat16* rlo, int* flag,
                int harm, T* Mfold, const T* dip, long long ncell) {
  constexpr size_t full = (size_t)kP2mParents * (8 * ncoef_c(P) + 8) * sizeof(T);
  // staged harmonic rows, where they fit beside the full ones (the plan folds
  // nothing at FP64 order 8, which would not)
  constexpr size_t red0 = (size_t)kP2mParents * (8 * nred_c(P) + 8) * sizeof(T);
  constexpr size_t red = full + red0 <= 227 * 1024 ? red0 : 0;
  if (harm && (Mhi || Mfold) && red == 0) return cudaErrorInvalidValue;
  const size_t smem = full + ((harm && (Mhi || Mfold)) ? red : 0);
  if (dip)
    return p2m_launch_dip<P, T, true>(blocks, smem, full + red, s, rho, nx, ny, b, leaf, Mleaf, Mhi, Mlo, rho_box, rhi,
                                      rlo, flag, harm, Mfold, dip, ncell);
  return p2m_launch_dip<P, T, false>(blocks, smem, full + red, s, rho, nx, ny, b, leaf, Mleaf, Mhi, Mlo, rho_box, rhi,
                                     rlo, flag, harm, Mfold, nullptr, ncell);
}

}  // namespace

template <typename T>
cudaError_t launch_p2m(const TreeTables& t, const T* rho, const int dims[3], const Level& leaf, T* Mleaf, T* rho_box,
                       void* Mhi, void* Mlo, void* rho_hi, void* rho_lo, int* flag, int harm, T* Mfold,
                       cudaStream_t s, const T* dip) {
  const long long threads = leaf.npar * 16;  // two threads per box
  if (threads == 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  FMM_ORDER_SWITCH(t.p, (e = p2m_launch<PP, T>(grid_threads(threads), s,
                            rho, dims[0], dims[1], t.b, leaf, Mleaf, static_cast<__nv_bfloat16*>(Mhi),
                            static_cast<__nv_bfloat16*>(Mlo), rho_box, static_cast<__nv_bfloat16*>(rho_hi),
                            static_cast<__nv_bfloat16*>(rho_lo), flag, harm, Mfold, dip,
                            (long long)dims[0] * dims[1] * dims[2])));
  return e;
}

template <typename T>
cudaError_t launch_p2m_multi(int p, const P2mArgs* args, const MultiGrid* grids, int n, long long blocks,
                             int harm_rows, cudaStream_t s) {
  if (n == 0 || blocks == 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  FMM_ORDER_SWITCH(p, (e = p2m_multi_launch<PP, T>(args, grids, n, blocks, harm_rows, s)));
  return e;
}
template cudaError_t launch_p2m_multi<float>(int, const P2mArgs*, const MultiGrid*, int, long long, int,
                                             cudaStream_t);
template cudaError_t launch_p2m_multi<double>(int, const P2mArgs*, const MultiGrid*, int, long long, int,
                                              cudaStream_t);

template cudaError_t launch_p2m<float>(const TreeTables&, const float*, const int*, const Level&, float*, float*,
                                       void*, void*, void*, void*, int*, int, float*, cudaStream_t, const float*);
template cudaError_t launch_p2m<double>(const TreeTables&, const double*, const int*, const Level&, double*, double*,
                                        void*, void*, void*, void*, int*, int, double*, cudaStream_t, const double*);

}  // namespace fmmgb
