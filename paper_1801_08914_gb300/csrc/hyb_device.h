// Device helpers shared by the element translation units (hyb_element.cu, hyb_mixed.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hyb {
namespace dev {

__device__ __forceinline__ int64_t tri(int i, int j) { return (int64_t)i * (i + 1) / 2 + j; }

// Local dof index of the component-c function with 1-D node indices (i0, i1, i2):
// interior dofs first (x, y, z components, first index fastest), then faces x0 x1 y0 y1 z0 z1.
template <int K>
__device__ __forceinline__ int local_index(int c, int i0, int i1, int i2) {
  constexpr int P = K + 2, p = K + 1, NI = 3 * K * p * p, NFN = p * p;
  const int ic = c == 0 ? i0 : c == 1 ? i1 : i2;
  if (ic > 0 && ic < P - 1) {
    const int r0 = c == 0 ? K : p, r1 = c == 1 ? K : p;
    const int j0 = i0 - (c == 0), j1 = i1 - (c == 1), j2 = i2 - (c == 2);
    return c * K * p * p + j0 + r0 * (j1 + r1 * j2);
  }
  const int side = ic == 0 ? 0 : 1;
  const int t0 = c == 0 ? i1 : i0;
  const int t1 = c == 2 ? i1 : i2;
  return NI + (2 * c + side) * NFN + t0 + p * t1;
}

// slot of the symmetric pair (a, b) in the 6-vector (00, 11, 22, 10, 20, 21)
__device__ __forceinline__ int gslot(int a, int b) {
  if (a == b) return a;
  const int hi = a > b ? a : b, lo = a > b ? b : a;
  return hi == 1 ? 3 : (lo == 0 ? 4 : 5);
}

// Row index i of the packed lower-triangle position t (t = i(i+1)/2 + j, j <= i).
__device__ __forceinline__ int tri_row(int t) {
  int i = (int)((sqrtf((float)(8 * t + 1)) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  while (i * (i + 1) / 2 > t) --i;
  return i;
}

// 1 / sqrt(d) by Newton-Raphson on f(r) = r^-2 - d from a single-precision seed:
// r <- r (3 - d r^2) / 2, two steps (23 -> 46 -> full FP64 bits). Falls back to the
// library square root outside the single-precision range.
__device__ __forceinline__ double rsqrt_newton(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  double r = (double)rsqrtf((float)d);
  r = r * fma(-0.5 * d, r * r, 1.5);
  r = r * fma(-0.5 * d, r * r, 1.5);
  return r;
}
// single precision: the hardware estimate and one Newton step
__device__ __forceinline__ float rsqrt_newton(float d) {
  float r = rsqrtf(d);
  return r * fmaf(-0.5f * d, r * r, 1.5f);
}

__device__ __forceinline__ void set_error(int* status, long long* err_elem, int code, long long e) {
  if (atomicCAS(status, 0, code) == 0) *err_elem = e;
}

}  // namespace dev
}  // namespace hyb
