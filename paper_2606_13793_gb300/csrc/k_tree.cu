// Small utility kernels of the tree: zero fill and the debug export of a level.
#include "fmm_internal.h"

namespace fmmgb {
namespace {

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

template <typename T>
__global__ void scaled_copy_kernel(const T* __restrict__ src, size_t count, T sc, T* __restrict__ dst) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = sc * src[i];
}

}  // namespace

template <typename T>
cudaError_t launch_scaled_copy(const T* src, size_t count, double sc, T* dst, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  size_t blocks = (count + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  scaled_copy_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(src, count, (T)sc, dst);
  return cudaGetLastError();
}
template cudaError_t launch_scaled_copy<float>(const float*, size_t, double, float*, cudaStream_t);
template cudaError_t launch_scaled_copy<double>(const double*, size_t, double, double*, cudaStream_t);

template <typename T>
cudaError_t launch_zero(T* p, size_t count, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  size_t blocks = (count + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  zero_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(p, count);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_export_level(const T* src, const Level& lv, int what, double h, const int8_t* mi, int nc,
                                double* dst, cudaStream_t s) {
  export_level_kernel<T><<<256, 256, 0, s>>>(src, lv, what, h, mi, nc, dst);
  return cudaGetLastError();
}

template cudaError_t launch_zero<float>(float*, size_t, cudaStream_t);
template cudaError_t launch_zero<double>(double*, size_t, cudaStream_t);
template cudaError_t launch_export_level<float>(const float*, const Level&, int, double, const int8_t*, int, double*,
                                                cudaStream_t);
template cudaError_t launch_export_level<double>(const double*, const Level&, int, double, const int8_t*, int,
                                                 double*, cudaStream_t);

}  // namespace fmmgb
