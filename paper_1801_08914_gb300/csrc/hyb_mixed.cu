// Mixed-precision element elimination for hybridization (arXiv:1801.08914, Sec. 3.2).
//
// A_T = alpha M + beta K is badly conditioned (kappa ~ (beta/alpha) h^-2): an FP32
// Cholesky of it loses every digit of C A^{-1} C^T on fine meshes. The paper's
// hybridized mixed form gives the same H (H = H~) from well-conditioned pieces:
// with K = D G D^T (D the geometry-free divergence coefficients of the RT_k basis in
// the Q_k Lagrange basis on the Gauss-Legendre nodes, G the beta / det J weighted
// Q_k mass),
//    A^{-1} = M^{-1} - M^{-1} D Z^{-1} D^T M^{-1},   Z = G^{-1} + D^T M^{-1} D,
// where M (the alpha mass) and Z stay well conditioned at any contrast. In FP32:
//    L_M = chol(M), Xd = L_M^{-1} D, L_Z = chol(G^{-1} + Xd^T Xd),
//    Y = L_M,bb^{-1}, P = Xd_b^T Y, V = L_Z^{-1} P,
//    (A^{-1})_bb = Y^T Y - V^T V,   S_T = D_c (A^{-1})_bb D_c   (C_T = [0 D_c]),
// accumulated into the FP64 CSR values, and the load term g_T = C_T A^{-1} f_T from one
// FP32 solve (both carry FP32-level error, which the global FP64 refinement removes). The
// recovery x_T = A^{-1}(f_T - C_T^T lambda) is refined in the mixed variables (x, q),
// q = G D^T x, against FP64 residuals of that (well-conditioned) saddle system, with M, D,
// D^T and G applied matrix-free in FP64; refining A x = f directly does not converge at
// high contrast because the two Woodbury terms cancel in FP32.
#include <cuda_runtime.h>

#include <type_traits>

#include "hyb_device.h"
#include "hyb_internal.h"
#include "hyb_tc.cuh"
#include "hyb_tiles.cuh"

namespace hyb {

__constant__ RefTables c_refm[kMaxOrder + 1];

cudaError_t launch_mass_maps(cudaStream_t s);

// The reference tables, then the per-order mass-assembly destination tables the element kernels read.
cudaError_t upload_ref_tables_mixed(const RefTables* tabs, int count, cudaStream_t s) {
  const cudaError_t e = cudaMemcpyToSymbolAsync(c_refm, tabs, sizeof(RefTables) * count, 0, cudaMemcpyHostToDevice, s);
  return e == cudaSuccess ? launch_mass_maps(s) : e;
}

namespace {

using dev::gslot;
using dev::local_index;
using dev::set_error;
using dev::tri;
using dev::tri_row;

// ---------------------------------------------------------------- CTA-wide building blocks

// out[o2][o1][o0] = sum_{i} in[i2][i1][i0] A0(i0,o0) A1(i1,o1) A2(i2,o2), with
// A_d(i,o) = fwd ? T_d[i*Q + o] (interpolation) : T_d[o*Q + i] (testing).
template <typename T, int NT>
__device__ void contract3(const T* in, int n0, int n1, int n2, int m0, int m1, int m2, const T* A0, const T* A1,
                          const T* A2, int Q, bool fwd, T* t1, T* t2, T* out, bool acc_out) {
  const int tid = threadIdx.x;
  for (int t = tid; t < m0 * n1 * n2; t += NT) {
    const int o0 = t % m0, i1 = (t / m0) % n1, i2 = t / (m0 * n1);
    T acc = 0;
    for (int i0 = 0; i0 < n0; ++i0) acc = fma(in[(i2 * n1 + i1) * n0 + i0], fwd ? A0[i0 * Q + o0] : A0[o0 * Q + i0], acc);
    t1[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < m0 * m1 * n2; t += NT) {
    const int o0 = t % m0, o1 = (t / m0) % m1, i2 = t / (m0 * m1);
    T acc = 0;
    for (int i1 = 0; i1 < n1; ++i1) acc = fma(t1[(i2 * n1 + i1) * m0 + o0], fwd ? A1[i1 * Q + o1] : A1[o1 * Q + i1], acc);
    t2[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < m0 * m1 * m2; t += NT) {
    const int o0 = t % m0, o1 = (t / m0) % m1, o2 = t / (m0 * m1);
    T acc = 0;
    for (int i2 = 0; i2 < n2; ++i2) acc = fma(t2[(i2 * m1 + o1) * m0 + o0], fwd ? A2[i2 * Q + o2] : A2[o2 * Q + i2], acc);
    out[t] = acc_out ? out[t] + acc : acc;
  }
  __syncthreads();
}

// FP64 geometry at the Gauss points from the monomial coefficients Mc of the trilinear map:
// g6[s][q] = w (J^T J)_s / det J (6 symmetric entries), gd[q] = w / det J.
template <int K, int NT>
__device__ void geometry64(const double* Mc, const double* qx, const double* qw, double* g6, double* gd,
                           int* status, long long* err_elem, int64_t e) {
  constexpr int Q = K + 2, NQ = Q * Q * Q;
  for (int q = threadIdx.x; q < NQ; q += NT) {
    const int q0 = q % Q, q1 = (q / Q) % Q, q2 = q / (Q * Q);
    const double x0 = qx[q0], x1 = qx[q1], x2 = qx[q2];
    const double x12 = x1 * x2, x02 = x0 * x2, x01 = x0 * x1;
    double J[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      J[r][0] = fma(Mc[21 + r], x12, fma(Mc[15 + r], x2, fma(Mc[12 + r], x1, Mc[3 + r])));
      J[r][1] = fma(Mc[21 + r], x02, fma(Mc[18 + r], x2, fma(Mc[12 + r], x0, Mc[6 + r])));
      J[r][2] = fma(Mc[21 + r], x01, fma(Mc[18 + r], x1, fma(Mc[15 + r], x0, Mc[9 + r])));
    }
    const double det = J[0][0] * fma(J[1][1], J[2][2], -J[1][2] * J[2][1]) -
                       J[0][1] * fma(J[1][0], J[2][2], -J[1][2] * J[2][0]) +
                       J[0][2] * fma(J[1][0], J[2][1], -J[1][1] * J[2][0]);
    if (!(det > 0.0)) set_error(status, err_elem, HYB_ERR_MESH, e);
    const double s = qw[q0] * qw[q1] * qw[q2] / det;
    g6[0 * NQ + q] = s * fma(J[0][0], J[0][0], fma(J[1][0], J[1][0], J[2][0] * J[2][0]));
    g6[1 * NQ + q] = s * fma(J[0][1], J[0][1], fma(J[1][1], J[1][1], J[2][1] * J[2][1]));
    g6[2 * NQ + q] = s * fma(J[0][2], J[0][2], fma(J[1][2], J[1][2], J[2][2] * J[2][2]));
    g6[3 * NQ + q] = s * fma(J[0][1], J[0][0], fma(J[1][1], J[1][0], J[2][1] * J[2][0]));
    g6[4 * NQ + q] = s * fma(J[0][2], J[0][0], fma(J[1][2], J[1][0], J[2][2] * J[2][0]));
    g6[5 * NQ + q] = s * fma(J[0][2], J[0][1], fma(J[1][2], J[1][1], J[2][2] * J[2][1]));
    gd[q] = s;
  }
  __syncthreads();
}

// Monomial coefficients of the trilinear map of element e, and the FP64 tables (one CTA).
template <int K, int NT>
__device__ void load_element64(const ElemArgs& a, int64_t e, double* X8, double* Mc, double* Vc, double* Dc,
                               double* Vo, double* qx, double* qw, double* wf) {
  constexpr int P = K + 2, p = K + 1, Q = K + 2;
  const int tid = threadIdx.x;
  const int ex = (int)(e % a.nx), ey = (int)((e / a.nx) % a.ny), ez = (int)(e / ((int64_t)a.nx * a.ny));
  const RefTables& rt = c_refm[K];
  for (int i = tid; i < P * Q; i += NT) {
    Vc[i] = rt.Vc[i / Q][i % Q];
    Dc[i] = rt.Dc[i / Q][i % Q];
  }
  for (int i = tid; i < p * Q; i += NT) Vo[i] = rt.Vo[i / Q][i % Q];
  for (int i = tid; i < Q; i += NT) { qx[i] = rt.qx[i]; qw[i] = rt.qw[i]; }
  for (int i = tid; i < p * p; i += NT) wf[i] = rt.wf[i];
  if (tid < 24) {
    const int c = tid / 3, d = tid % 3;
    const int64_t v = (ex + (c & 1)) + (int64_t)(a.nx + 1) * ((ey + ((c >> 1) & 1)) + (int64_t)(a.ny + 1) * (ez + (c >> 2)));
    X8[tid] = a.vertices[3 * v + d];
  }
  __syncthreads();
  if (tid < 3) {
    const int d = tid;
    const double x0 = X8[d], x1 = X8[3 + d], x2 = X8[6 + d], x3 = X8[9 + d];
    const double x4 = X8[12 + d], x5 = X8[15 + d], x6 = X8[18 + d], x7 = X8[21 + d];
    Mc[d] = x0;
    Mc[3 + d] = x1 - x0;
    Mc[6 + d] = x2 - x0;
    Mc[9 + d] = x4 - x0;
    Mc[12 + d] = (x3 - x2) - (x1 - x0);
    Mc[15 + d] = (x5 - x4) - (x1 - x0);
    Mc[18 + d] = (x6 - x4) - (x2 - x0);
    Mc[21 + d] = ((x7 - x6) - (x5 - x4)) - ((x3 - x2) - (x1 - x0));
  }
  __syncthreads();
}

// y = A x for the element operator (alpha mass + beta div, no boundary conditions), FP64,
// by sum factorisation; with_div = false gives the unit mass when alpha = 1.
template <int K, int NT>
__device__ void apply_A64(const double* x, double* y, double alpha, double beta, bool with_div, const double* g6,
                          const double* gd, const double* Vc, const double* Dc, const double* Vo, double* U,
                          double* Wv, double* Dv, double* xc, double* t1, double* t2) {
  constexpr int P = K + 2, p = K + 1, Q = K + 2, NQ = Q * Q * Q;
  const int tid = threadIdx.x;
  for (int c = 0; c < 3; ++c) {
    const int n0 = c == 0 ? P : p, n1 = c == 1 ? P : p, n2 = c == 2 ? P : p;
    for (int t = tid; t < n0 * n1 * n2; t += NT) {
      const int i0 = t % n0, i1 = (t / n0) % n1, i2 = t / (n0 * n1);
      xc[t] = x[local_index<K>(c, i0, i1, i2)];
    }
    __syncthreads();
    contract3<double, NT>(xc, n0, n1, n2, Q, Q, Q, c == 0 ? Vc : Vo, c == 1 ? Vc : Vo, c == 2 ? Vc : Vo, Q, true,
                          t1, t2, U + c * NQ, false);
    if (with_div)
      contract3<double, NT>(xc, n0, n1, n2, Q, Q, Q, c == 0 ? Dc : Vo, c == 1 ? Dc : Vo, c == 2 ? Dc : Vo, Q, true,
                            t1, t2, Dv, c > 0);
  }
  for (int t = tid; t < 3 * NQ; t += NT) {
    const int c = t / NQ, q = t % NQ;
    Wv[t] = alpha * (g6[gslot(c, 0) * NQ + q] * U[q] + g6[gslot(c, 1) * NQ + q] * U[NQ + q] +
                     g6[gslot(c, 2) * NQ + q] * U[2 * NQ + q]);
  }
  if (with_div)
    for (int q = tid; q < NQ; q += NT) Dv[q] *= beta * gd[q];
  __syncthreads();
  for (int c = 0; c < 3; ++c) {
    const int n0 = c == 0 ? P : p, n1 = c == 1 ? P : p, n2 = c == 2 ? P : p;
    contract3<double, NT>(Wv + c * NQ, Q, Q, Q, n0, n1, n2, c == 0 ? Vc : Vo, c == 1 ? Vc : Vo, c == 2 ? Vc : Vo, Q,
                          false, t1, t2, xc, false);
    if (with_div)
      contract3<double, NT>(Dv, Q, Q, Q, n0, n1, n2, c == 0 ? Dc : Vo, c == 1 ? Dc : Vo, c == 2 ? Dc : Vo, Q, false,
                            t1, t2, xc, true);
    for (int t = tid; t < n0 * n1 * n2; t += NT) {
      const int i0 = t % n0, i1 = (t / n0) % n1, i2 = t / (n0 * n1);
      y[local_index<K>(c, i0, i1, i2)] = xc[t];
    }
    __syncthreads();
  }
}

// y = alpha M x (the Piola-mapped mass, no boundary conditions), FP64, by sum factorisation
// with the three components in every pass: interpolation to the Gauss points in three
// contractions, the 3 x 3 geometric factor, testing in three contractions; 7 barriers.
// t1, t2: 3 P Q Q doubles each.
template <int K, int NT>
__device__ void apply_mass64(const double* x, double* y, double alpha, const double* g6, const double* Vc,
                             const double* Vo, double* U, double* Wv, double* t1, double* t2) {
  constexpr int P = K + 2, p = K + 1, Q = K + 2, NQ = Q * Q * Q;
  // component c has n0 x n1 x n2 dofs: P along its own axis, p across
  constexpr int S1 = Q * p * p, S1B = Q * P * p;              // stage-1 items of c = 0, of c = 1, 2
  constexpr int S2A = Q * Q * p, S2B = Q * Q * P;             // stage-2 items of c = 0, 1 and of c = 2
  const int tid = threadIdx.x;
  auto nd = [](int c, int d) { return c == d ? P : p; };
  auto tab = [&](int c, int d) { return c == d ? Vc : Vo; };
  // forward stage 1: t1[c][i2][i1][o0] = sum_i0 x[c](i0, i1, i2) T(i0, o0)
  for (int t = tid; t < S1 + 2 * S1B; t += NT) {
    const int c = t < S1 ? 0 : (t < S1 + S1B ? 1 : 2);
    const int l = t - (c == 0 ? 0 : (c == 1 ? S1 : S1 + S1B));
    const int n0 = nd(c, 0), n1 = nd(c, 1);
    const int o0 = l % Q, i1 = (l / Q) % n1, i2 = l / (Q * n1);
    const double* A = tab(c, 0);
    double acc = 0.0;
    for (int i0 = 0; i0 < n0; ++i0) acc = fma(x[local_index<K>(c, i0, i1, i2)], A[i0 * Q + o0], acc);
    t1[t] = acc;
  }
  __syncthreads();
  // forward stage 2: t2[c][i2][o1][o0] = sum_i1 t1[c][i2][i1][o0] T(i1, o1)
  for (int t = tid; t < 2 * S2A + S2B; t += NT) {
    const int c = t < S2A ? 0 : (t < 2 * S2A ? 1 : 2);
    const int l = t - c * S2A;
    const int n1 = nd(c, 1);
    const int o0 = l % Q, o1 = (l / Q) % Q, i2 = l / (Q * Q);
    const double* A = tab(c, 1);
    const double* src = t1 + (c == 0 ? 0 : (c == 1 ? S1 : S1 + S1B));
    double acc = 0.0;
    for (int i1 = 0; i1 < n1; ++i1) acc = fma(src[(i2 * n1 + i1) * Q + o0], A[i1 * Q + o1], acc);
    t2[t] = acc;
  }
  __syncthreads();
  // forward stage 3: U[c][o2][o1][o0] = sum_i2 t2[c][i2][o1][o0] T(i2, o2)
  for (int t = tid; t < 3 * NQ; t += NT) {
    const int c = t / NQ, l = t % NQ;
    const int n2 = nd(c, 2);
    const int o01 = l % (Q * Q), o2 = l / (Q * Q);
    const double* A = tab(c, 2);
    const double* src = t2 + c * S2A;
    double acc = 0.0;
    for (int i2 = 0; i2 < n2; ++i2) acc = fma(src[i2 * Q * Q + o01], A[i2 * Q + o2], acc);
    U[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < 3 * NQ; t += NT) {
    const int c = t / NQ, q = t % NQ;
    Wv[t] = alpha * (g6[gslot(c, 0) * NQ + q] * U[q] + g6[gslot(c, 1) * NQ + q] * U[NQ + q] +
                     g6[gslot(c, 2) * NQ + q] * U[2 * NQ + q]);
  }
  __syncthreads();
  // test stage 1: t1[c][q2][q1][i0] = sum_q0 Wv[c][q2][q1][q0] T(i0, q0)
  constexpr int B1A = p * Q * Q, B1B = P * Q * Q;             // items of c = 0 (P) and c = 1, 2 (p)
  for (int t = tid; t < B1B + 2 * B1A; t += NT) {
    const int c = t < B1B ? 0 : (t < B1B + B1A ? 1 : 2);
    const int l = t - (c == 0 ? 0 : (c == 1 ? B1B : B1B + B1A));
    const int n0 = nd(c, 0);
    const int i0 = l % n0, q1 = (l / n0) % Q, q2 = l / (n0 * Q);
    const double* A = tab(c, 0);
    const double* src = Wv + c * NQ + (q2 * Q + q1) * Q;
    double acc = 0.0;
    for (int q0 = 0; q0 < Q; ++q0) acc = fma(src[q0], A[i0 * Q + q0], acc);
    t1[t] = acc;
  }
  __syncthreads();
  // test stage 2: t2[c][q2][i1][i0] = sum_q1 t1[c][q2][q1][i0] T(i1, q1)
  constexpr int B2A = P * p * Q, B2B = p * p * Q;             // items of c = 0, 1 (n0 n1 = P p) and c = 2 (p p)
  for (int t = tid; t < 2 * B2A + B2B; t += NT) {
    const int c = t < B2A ? 0 : (t < 2 * B2A ? 1 : 2);
    const int l = t - c * B2A;
    const int n0 = nd(c, 0), n1 = nd(c, 1);
    const int i0 = l % n0, i1 = (l / n0) % n1, q2 = l / (n0 * n1);
    const double* A = tab(c, 1);
    const double* src = t1 + (c == 0 ? 0 : (c == 1 ? B1B : B1B + B1A));
    double acc = 0.0;
    for (int q1 = 0; q1 < Q; ++q1) acc = fma(src[(q2 * Q + q1) * n0 + i0], A[i1 * Q + q1], acc);
    t2[t] = acc;
  }
  __syncthreads();
  // test stage 3: y[c](i0, i1, i2) = sum_q2 t2[c][q2][i1][i0] T(i2, q2)
  constexpr int NC = P * p * p;
  for (int t = tid; t < 3 * NC; t += NT) {
    const int c = t / NC, l = t % NC;
    const int n0 = nd(c, 0), n1 = nd(c, 1);
    const int i0 = l % n0, i1 = (l / n0) % n1, i2 = l / (n0 * n1);
    const double* A = tab(c, 2);
    const double* src = t2 + c * B2A;
    double acc = 0.0;
    for (int q2 = 0; q2 < Q; ++q2) acc = fma(src[(q2 * n1 + i1) * n0 + i0], A[i2 * Q + q2], acc);
    y[local_index<K>(c, i0, i1, i2)] = acc;
  }
  __syncthreads();
}

// y = D' q (D' the divergence coefficients with zero rows on essential dofs), FP64.
template <int K, int NT>
__device__ void apply_D64(const double* q, double* y, const int* dofcode, const double* DcO, int bmask) {
  constexpr int p = K + 1, NI = 3 * K * p * p, NFN = p * p, N = NI + 6 * NFN;
  for (int i = threadIdx.x; i < N; i += NT) {
    double acc = 0.0;
    if (!(i >= NI && ((bmask >> ((i - NI) / NFN)) & 1))) {
      const int code = dofcode[i];
      const int c = code & 3, i0 = (code >> 2) & 63, i1 = (code >> 8) & 63, i2 = (code >> 14) & 63;
      const int ic = c == 0 ? i0 : c == 1 ? i1 : i2;
      for (int ac = 0; ac < p; ++ac) {
        const int a0 = c == 0 ? ac : i0, a1 = c == 1 ? ac : i1, a2 = c == 2 ? ac : i2;
        acc = fma(DcO[ic * p + ac], q[a0 + p * (a1 + p * a2)], acc);
      }
    }
    y[i] = acc;
  }
  __syncthreads();
}

// t = D'^T x (Q_k node values), FP64.
template <int K, int NT>
__device__ void apply_Dt64(const double* x, double* t, const double* DcO, int bmask) {
  constexpr int P = K + 2, p = K + 1, NI = 3 * K * p * p, NFN = p * p;
  for (int a = threadIdx.x; a < p * p * p; a += NT) {
    const int a0 = a % p, a1 = (a / p) % p, a2 = a / (p * p);
    double acc = 0.0;
    for (int c = 0; c < 3; ++c) {
      const int ac = c == 0 ? a0 : c == 1 ? a1 : a2;
      for (int ic = 0; ic < P; ++ic) {
        const int i0 = c == 0 ? ic : a0, i1 = c == 1 ? ic : a1, i2 = c == 2 ? ic : a2;
        const int i = local_index<K>(c, i0, i1, i2);
        if (i >= NI && ((bmask >> ((i - NI) / NFN)) & 1)) continue;
        acc = fma(DcO[ic * p + ac], x[i], acc);
      }
    }
    t[a] = acc;
  }
  __syncthreads();
}

// w = G v with G the Q_k mass weighted by beta / det J (sum factorisation), FP64.
template <int K, int NT>
__device__ void apply_G64(const double* v, double* w, double beta, const double* gd, const double* Vo, double* U,
                          double* t1, double* t2) {
  constexpr int p = K + 1, Q = K + 2, NQ = Q * Q * Q;
  contract3<double, NT>(v, p, p, p, Q, Q, Q, Vo, Vo, Vo, Q, true, t1, t2, U, false);
  for (int q = threadIdx.x; q < NQ; q += NT) U[q] *= beta * gd[q];
  __syncthreads();
  contract3<double, NT>(U, Q, Q, Q, p, p, p, Vo, Vo, Vo, Q, false, t1, t2, w, false);
}

#include "hyb_mixed_tiled.cuh"

// Opt in to the kernel's shared memory (with the largest carve-out) before its first launch.
template <typename F>
cudaError_t prepare_smem(F* kernel, size_t bytes) {
  cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
  if (err == cudaSuccess) err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return err;
}

template <int K>
cudaError_t launch_mixed_batch_k(const ElemArgs* probs, const int2* items, int64_t n, int colour, bool recover,
                                 const double* const* lams, double* const* us, int grid, cudaStream_t s, Prof* prof) {
  using S = MT<K>;
  if (n == 0) return cudaSuccess;
  cudaError_t err;
  if (!recover) {
    if ((err = prepare_smem(mixed_load_kernel_batch<K>, LoadShape<K>::SMEM)) != cudaSuccess) return err;
    if ((err = prepare_smem(element_tiled_kernel_batch<K>, S::SMEM_ASM)) != cudaSuccess) return err;
    int tok = prof_begin(prof, HYB_K_ELEMENT, s);
    mixed_load_kernel_batch<K><<<(unsigned)n, LoadShape<K>::NT, LoadShape<K>::SMEM, s>>>(probs, items, n);
    prof_end(prof, tok, s);
    tok = prof_begin(prof, HYB_K_ELEMENT, s);
    const unsigned g = (unsigned)(grid > 0 && grid < n ? grid : n);
    element_tiled_kernel_batch<K><<<g, S::NT, S::SMEM_ASM, s>>>(probs, items, n, colour);
    prof_end(prof, tok, s);
  } else {
    if ((err = prepare_smem(recover_tiled_kernel_batch<K>, S::SMEM)) != cudaSuccess) return err;
    const int tok = prof_begin(prof, HYB_K_RECOVER, s);
    recover_tiled_kernel_batch<K><<<(unsigned)n, S::NT, S::SMEM, s>>>(probs, lams, us, items, n);
    prof_end(prof, tok, s);
  }
  return cudaGetLastError();
}

template <int K>
cudaError_t launch_mixed_k(const ElemArgs& a, cudaStream_t s, Prof* prof, bool recover, const double* lambda,
                           double* u) {
  using S = MT<K>;
  if (a.n_list == 0) return cudaSuccess;
  cudaError_t err;
  if (!recover) {
    if ((err = prepare_smem(mixed_load_kernel<K>, LoadShape<K>::SMEM)) != cudaSuccess) return err;
    if ((err = prepare_smem(element_tiled_kernel<K>, S::SMEM_ASM)) != cudaSuccess) return err;
    int tok = prof_begin(prof, HYB_K_ELEMENT, s);
    mixed_load_kernel<K><<<(unsigned)a.n_list, LoadShape<K>::NT, LoadShape<K>::SMEM, s>>>(a);
    prof_end(prof, tok, s);
    tok = prof_begin(prof, HYB_K_ELEMENT, s);
    element_tiled_kernel<K><<<(unsigned)a.n_list, S::NT, S::SMEM_ASM, s>>>(a);
    prof_end(prof, tok, s);
  } else {
    if ((err = prepare_smem(recover_tiled_kernel<K>, S::SMEM)) != cudaSuccess) return err;
    const int tok = prof_begin(prof, HYB_K_RECOVER, s);
    recover_tiled_kernel<K><<<(unsigned)a.n_list, S::NT, S::SMEM, s>>>(a, lambda, u);
    prof_end(prof, tok, s);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mass_maps(cudaStream_t s) {
  mass_map_kernel<0><<<1, 192, 0, s>>>();
  mass_map_kernel<1><<<1, 192, 0, s>>>();
  mass_map_kernel<2><<<1, 192, 0, s>>>();
  mass_map_kernel<3><<<1, 192, 0, s>>>();
  return cudaGetLastError();
}

// FP32-path store per element: the tiles of L_M | Xd | L_Z | G^{-1} for the recovery.
int64_t mixed_store_floats(int k) {
  switch (k) {
    case 0: return MT<0>::STORE;
    case 1: return MT<1>::STORE;
    case 2: return MT<2>::STORE;
    case 3: return MT<3>::STORE;
  }
  return 0;
}

cudaError_t launch_element_mixed(int k, const ElemArgs& a, cudaStream_t s, Prof* prof) {
  switch (k) {
    case 0: return launch_mixed_k<0>(a, s, prof, false, nullptr, nullptr);
    case 1: return launch_mixed_k<1>(a, s, prof, false, nullptr, nullptr);
    case 2: return launch_mixed_k<2>(a, s, prof, false, nullptr, nullptr);
    case 3: return launch_mixed_k<3>(a, s, prof, false, nullptr, nullptr);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_mixed_batch(int k, const ElemArgs* probs, const int2* items, int64_t n, int colour, bool recover,
                               const double* const* lams, double* const* us, int grid, cudaStream_t s, Prof* prof) {
  switch (k) {
    case 0: return launch_mixed_batch_k<0>(probs, items, n, colour, recover, lams, us, grid, s, prof);
    case 1: return launch_mixed_batch_k<1>(probs, items, n, colour, recover, lams, us, grid, s, prof);
    case 2: return launch_mixed_batch_k<2>(probs, items, n, colour, recover, lams, us, grid, s, prof);
    case 3: return launch_mixed_batch_k<3>(probs, items, n, colour, recover, lams, us, grid, s, prof);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_recover_mixed(int k, const ElemArgs& a, const double* lambda, double* u, cudaStream_t s,
                                 Prof* prof) {
  switch (k) {
    case 0: return launch_mixed_k<0>(a, s, prof, true, lambda, u);
    case 1: return launch_mixed_k<1>(a, s, prof, true, lambda, u);
    case 2: return launch_mixed_k<2>(a, s, prof, true, lambda, u);
    case 3: return launch_mixed_k<3>(a, s, prof, true, lambda, u);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hyb

namespace hyb {
int mixed_batch_ctas_per_sm(int k) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (k) {
    case 0: e = prepare_smem(element_tiled_kernel_batch<0>, MT<0>::SMEM_ASM); if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, element_tiled_kernel_batch<0>, MT<0>::NT, MT<0>::SMEM_ASM); break;
    case 1: e = prepare_smem(element_tiled_kernel_batch<1>, MT<1>::SMEM_ASM); if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, element_tiled_kernel_batch<1>, MT<1>::NT, MT<1>::SMEM_ASM); break;
    case 2: e = prepare_smem(element_tiled_kernel_batch<2>, MT<2>::SMEM_ASM); if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, element_tiled_kernel_batch<2>, MT<2>::NT, MT<2>::SMEM_ASM); break;
    case 3: e = prepare_smem(element_tiled_kernel_batch<3>, MT<3>::SMEM_ASM); if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, element_tiled_kernel_batch<3>, MT<3>::NT, MT<3>::SMEM_ASM); break;
  }
  return e == cudaSuccess ? n : 0;
}
}  // namespace hyb
