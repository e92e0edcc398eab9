// Back substitution after the reduced solve, one CTA per element, FP64.
//
// Hybridization (Thm 2.1): x_T = A_T^{-1}(f_T - C_T^T lambda_T). With the stored
// factor L (interior rows L_ii, L_bi) and Y = L_bb^{-1}, and z = L^{-1} f:
//   w = D lambda_T,  x_b = Y^T (z_b - Y w),  x_i = L_ii^{-T}(z_i - L_bi^T x_b).
// Static condensation (Sec. 3.1): u_b from the global face dofs (essential
// values on boundary faces), u_i = A_ii^{-1}(f_i - A_ib u_b) = L_ii^{-T}(z_i - L_bi^T u_b).
// The stored factor is read once, row by row (coalesced): this pass is bound by HBM.
#include <cuda_runtime.h>

#include "hyb_internal.h"

namespace hyb {

namespace {

__device__ __forceinline__ int64_t tri(int i, int j) { return (int64_t)i * (i + 1) / 2 + j; }

template <int K, int MODE>
__device__ __forceinline__ void recover_body(const RecoverArgs& a, const int64_t e) {
  constexpr int p = K + 1, NFN = p * p, NI = 3 * K * p * p, NB = 6 * NFN, N = NI + NB;
  constexpr int NT = K <= 1 ? 64 : K == 2 ? 128 : 256;
  constexpr int64_t TRI = (int64_t)N * (N + 1) / 2;
  __shared__ double x[N];
  __shared__ double w[NB];
  __shared__ double rhs[NI > 0 ? NI : 1];
  const int tid = threadIdx.x;
  const int64_t es = a.slot ? (int64_t)a.slot[e] : e;
  const double* L = a.Lstore + es * TRI;
  const double* z = a.zstore + e * (int64_t)N;
  const int32_t* ef = a.elem_face + 6 * e;

  if (MODE == MODE_HYB) {
    for (int ib = tid; ib < NB; ib += NT) {
      const int fa = ef[ib / NFN], m = ib % NFN;
      w[ib] = fa < 0 ? 0.0 : (((ib / NFN) & 1) ? 1.0 : -1.0) * a.wf[m] * a.lambda[(int64_t)fa * NFN + m];
    }
    __syncthreads();
    // t = z_b - Y w   (row i of Y is contiguous)
    for (int i = tid; i < NB; i += NT) {
      const double* Yi = L + tri(NI + i, NI);
      double acc = 0.0;
      for (int m = 0; m <= i; ++m) acc = fma(Yi[m], w[m], acc);
      x[NI + i] = z[NI + i] - acc;
    }
    __syncthreads();
    // x_b = Y^T t : thread i walks rows m >= i, consecutive threads read consecutive columns
    for (int i = tid; i < NB; i += NT) {
      double acc = 0.0;
      for (int m = i; m < NB; ++m) acc = fma(L[tri(NI + m, NI + i)], x[NI + m], acc);
      w[i] = acc;
    }
    __syncthreads();
    for (int i = tid; i < NB; i += NT) x[NI + i] = w[i];
  } else {
    for (int ib = tid; ib < NB; ib += NT) {
      const int fa = ef[ib / NFN], m = ib % NFN;
      double v;
      // boundary faces: the essential value, kept unchanged in z by the identity rows
      if (fa >= 0) v = a.lambda[(int64_t)fa * NFN + m];
      else v = z[NI + ib];
      x[NI + ib] = v;
    }
  }
  __syncthreads();
  if (NI > 0) {
    // rhs = z_i - L_bi^T x_b
    for (int r = tid; r < NI; r += NT) {
      double acc = z[r];
      for (int m = 0; m < NB; ++m) acc = fma(-L[tri(NI + m, r)], x[NI + m], acc);
      rhs[r] = acc;
    }
    __syncthreads();
    // L_ii^T x_i = rhs, column-oriented from the last row
    for (int r = NI - 1; r >= 0; --r) {
      if (tid == 0) x[r] = rhs[r] / L[tri(r, r)];
      __syncthreads();
      const double xr = x[r];
      const double* Lr = L + tri(r, 0);
      for (int s = tid; s < r; s += NT) rhs[s] = fma(-Lr[s], xr, rhs[s]);
      __syncthreads();
    }
  }
  double* u = a.u + e * (int64_t)N;
  for (int i = tid; i < N; i += NT) u[i] = x[i];
}

template <int K, int MODE>
__global__ void recover_kernel(RecoverArgs a) {
  if ((int64_t)blockIdx.x >= a.n_elem) return;
  recover_body<K, MODE>(a, a.elem_list ? (int64_t)a.elem_list[blockIdx.x] : (int64_t)blockIdx.x);
}

template <int K, int MODE>
__global__ void recover_kernel_batch(const RecoverArgs* probs, const int2* items, int64_t n_items) {
  if ((int64_t)blockIdx.x >= n_items) return;
  const int2 it = items[blockIdx.x];
  const RecoverArgs a = probs[it.x];
  recover_body<K, MODE>(a, it.y);
}

template <int K>
cudaError_t launch_k(const RecoverArgs& a, cudaStream_t s, Prof* prof) {
  constexpr int NT = K <= 1 ? 64 : K == 2 ? 128 : 256;
  if (a.n_elem == 0) return cudaSuccess;
  const int tok = prof_begin(prof, HYB_K_RECOVER, s);
  if (a.mode == MODE_HYB) recover_kernel<K, MODE_HYB><<<(unsigned)a.n_elem, NT, 0, s>>>(a);
  else recover_kernel<K, MODE_SC><<<(unsigned)a.n_elem, NT, 0, s>>>(a);
  prof_end(prof, tok, s);
  return cudaGetLastError();
}

}  // namespace

template <int K>
cudaError_t launch_batch_k(int mode, const RecoverArgs* probs, const int2* items, int64_t n, cudaStream_t s,
                           Prof* prof) {
  constexpr int NT = K <= 1 ? 64 : K == 2 ? 128 : 256;
  if (n == 0) return cudaSuccess;
  const int tok = prof_begin(prof, HYB_K_RECOVER, s);
  if (mode == MODE_HYB) recover_kernel_batch<K, MODE_HYB><<<(unsigned)n, NT, 0, s>>>(probs, items, n);
  else recover_kernel_batch<K, MODE_SC><<<(unsigned)n, NT, 0, s>>>(probs, items, n);
  prof_end(prof, tok, s);
  return cudaGetLastError();
}

cudaError_t launch_recover_batch(int k, int mode, const RecoverArgs* probs, const int2* items, int64_t n,
                                 cudaStream_t s, Prof* prof) {
  switch (k) {
    case 0: return launch_batch_k<0>(mode, probs, items, n, s, prof);
    case 1: return launch_batch_k<1>(mode, probs, items, n, s, prof);
    case 2: return launch_batch_k<2>(mode, probs, items, n, s, prof);
    case 3: return launch_batch_k<3>(mode, probs, items, n, s, prof);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_recover(const RecoverArgs& a, cudaStream_t s, Prof* prof) {
  switch (a.k) {
    case 0: return launch_k<0>(a, s, prof);
    case 1: return launch_k<1>(a, s, prof);
    case 2: return launch_k<2>(a, s, prof);
    case 3: return launch_k<3>(a, s, prof);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hyb
