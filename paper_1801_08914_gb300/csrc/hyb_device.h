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
// 1 / sqrt(d) for a positive normal double, without FP64 conversions or range branches (on
// GPUs whose FP64 unit takes tens of cycles per warp instruction, those dominate a pivot):
// write d = m 4^s with m in [1, 4); build m as a float from its exponent and leading mantissa
// bits with integer operations, take the single-precision hardware estimate of m^{-1/2}, and
// scale it by 2^{-s} back into a double, again with integer operations (about 21 correct
// bits). One third-order step of the binomial series (1 - e)^{-1/2} = 1 + e/2 + 3 e^2/8 + ...
// with e = 1 - d r0^2 then gives the full double: the neglected term 5 e^3 / 16 is below
// 2^-60. u = d r0 is rounded before e = 1 - u r0 is formed; that adds about 2^-53 to e and so
// to the result. The caller checks that d is a positive normal number (a negative, zero or
// non-finite d gives a meaningless value, no trap).
__device__ __forceinline__ double rsqrt_h3(double d) {
  const int hi = __double2hiint(d), lo = __double2loint(d);
  const int ex = ((hi >> 20) & 0x7ff) - 1023;
  const int s = ex >> 1;                                    // floor(ex / 2)
  const unsigned mb = ((unsigned)(127 + ex - 2 * s) << 23) | (((unsigned)hi & 0xfffffu) << 3) |
                      ((unsigned)lo >> 29);
  const unsigned rb = __float_as_uint(rsqrtf(__uint_as_float(mb)));
  const int rexp = (int)((rb >> 23) & 0xffu) - 127;
  const double r0 = __hiloint2double((int)(((unsigned)(rexp + 1023 - s) << 20) | ((rb & 0x7fffffu) >> 3)),
                                     (int)((rb & 7u) << 29));
  const double u = d * r0;
  const double e = fma(-u, r0, 1.0);
  const double ep = e * fma(e, 0.375, 0.5);
  return fma(r0, ep, r0);
}
// Exact float -> double widening with integer operations (sign, re-biased exponent, mantissa
// shifted into place), for kernels where an FP64-pipe conversion per value is the cost; zero,
// denormal, infinite and NaN inputs take the hardware conversion.
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)f;
  const unsigned hi = (u & 0x80000000u) | ((e + (1023u - 127u)) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)((u & 7u) << 29));
}
// d > 0, finite and normal, from its high word (integer compares only)
__device__ __forceinline__ bool positive_normal(double d) {
  const int hi = __double2hiint(d);
  return hi > 0x000fffff && hi < 0x7ff00000;
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
