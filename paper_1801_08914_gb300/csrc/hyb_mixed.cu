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
// accumulated into the FP64 CSR values. The load term g_T = C_T A^{-1} f_T and the
// recovery x_T = A^{-1}(f_T - C_T^T lambda) are refined in the mixed variables (x, q),
// q = G D^T x, against FP64 residuals of that (well-conditioned) saddle system, with M, D,
// D^T and G applied matrix-free in FP64; refining A x = f directly does not converge at
// high contrast because the two Woodbury terms cancel in FP32.
#include <cuda_runtime.h>

#include "hyb_device.h"
#include "hyb_internal.h"

namespace hyb {

__constant__ RefTables c_refm[kMaxOrder + 1];

cudaError_t upload_ref_tables_mixed(const RefTables* tabs, int count, cudaStream_t s) {
  return cudaMemcpyToSymbolAsync(c_refm, tabs, sizeof(RefTables) * count, 0, cudaMemcpyHostToDevice, s);
}

namespace {

using dev::gslot;
using dev::local_index;
using dev::set_error;
using dev::tri;
using dev::tri_row;

template <int K>
struct MX {
  static constexpr int P = K + 2, p = K + 1, Q = K + 2, NQ = Q * Q * Q;
  static constexpr int NFN = p * p, NI = 3 * K * p * p, NB = 6 * NFN, N = NI + NB, NC = P * p * p;
  static constexpr int NQK = p * p * p;                   // dimension of Q_k
  static constexpr int NT = K == 0 ? 64 : K == 1 ? 128 : 256;
  static constexpr bool BIG_SMEM = K <= 2;                // L_M and Xd in shared memory
  static constexpr int TRI = N * (N + 1) / 2, TRIB = NB * (NB + 1) / 2;
  static constexpr int64_t STORE = (int64_t)TRI + (int64_t)N * NQK + 2 * NQK * NQK;   // L_M | Xd | L_Z | G^{-1}
  // FP64 shared region
  static constexpr int TMP64 = P * Q * Q;
  static constexpr int D64 = 24 + 24 + 2 * P * Q + p * Q + 2 * Q + NFN + 7 * NQ /*g6, gd*/ + 4 * N /*f x r u*/ +
                             3 * NQ /*U*/ + 3 * NQ /*W*/ + NQ /*Dv*/ + NC /*xc*/ + 2 * TMP64 + 8 +
                             NQK /*q*/ + (N > NQ ? N : NQ) /*rq*/ + P * p /*DcO*/;
  // FP32 shared region
  static constexpr int T1SZ = Q * Q * P * P, T2SZ = Q * P * P * p * p;
  static constexpr int ASMF = T1SZ + T2SZ + 7 * NQ;
  static constexpr int VA = NB * NB > 2 * NQK * NQK ? NB * NB : 2 * NQK * NQK;
  static constexpr int VREG = VA > ASMF ? VA : ASMF;
  static constexpr int TABF = 2 * P * Q + p * Q + P * P * Q + P * p * Q + p * p * Q + P * p;
  static constexpr int F32 = TABF + NQK * NQK /*Z*/ + TRIB /*Y*/ + TRIB /*S*/ + VREG + 2 * N /*colbuf invd*/ +
                             2 * N /*vec*/ + 3 * NQK + 8 + (BIG_SMEM ? TRI + N * NQK : 0);
  static constexpr size_t SMEM = sizeof(double) * D64 + sizeof(float) * F32 + sizeof(int) * N;
};

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

// In-place Cholesky of a packed (ld < 0) or full row-major (ld = row stride) lower triangle,
// optionally fused with the forward substitution X <- L^{-1} X of an n x m row-major block.
// Right-looking; every trailing update (triangle and right-hand sides) is spread over all
// threads, two barriers per column. Returns false (in every thread) on a non-positive pivot.
template <int NT>
__device__ bool chol32(float* A, int n, int ld, float* colbuf, float* invd, float* flag, float* X = nullptr,
                       int m = 0) {
  const int tid = threadIdx.x;
  auto at = [&](int i, int j) -> float& { return ld < 0 ? A[tri(i, j)] : A[i * ld + j]; };
  if (tid == 0) flag[0] = n > 0 ? at(0, 0) : 1.0f;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const float d = flag[0];
    if (!(d > 0.0f) || !(d < INFINITY)) return false;
    const float r = dev::rsqrt_newton(d);
    for (int i = j + 1 + tid; i < n; i += NT) {
      const float v = at(i, j) * r;
      at(i, j) = v;
      colbuf[i] = v;
    }
    if (tid == 0) {
      at(j, j) = d * r;
      invd[j] = r;
    }
    for (int a = tid; a < m; a += NT) X[j * m + a] *= r;       // row j of L^{-1} X is final
    __syncthreads();
    // trailing update, one row per warp (lanes along the contiguous packed row, then along
    // the right-hand sides): no per-entry index arithmetic, which would dominate in FP32
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int NW = NT / 32;
    for (int i = j + 1 + warp; i < n; i += NW) {
      const float lij = colbuf[i];
      for (int l = j + 1 + lane; l <= i; l += 32) {
        const float v = fmaf(-lij, colbuf[l], at(i, l));
        at(i, l) = v;
        if (i == j + 1) flag[0] = v;                           // the next pivot (l == j + 1 here)
      }
      for (int a = lane; a < m; a += 32) X[i * m + a] = fmaf(-lij, X[j * m + a], X[i * m + a]);
    }
    __syncthreads();
  }
  return true;
}

// Register-resident Cholesky of the packed lower triangle A (n = N) fused with X <- L^{-1} X
// (N x M, row-major), for matrices whose entries fit in the registers of the CTA: thread t owns
// packed entries t, t + NT, ... and right-hand-side entries t, t + NT, ..., with their (row,
// column) precomputed, so each column step is two predicated passes over registers:
//   B: scale column j by 1/sqrt(pivot) and publish it (and row j of X) to shared memory;
//   C: rank-1 update of the entries right of column j; the owner of (j+1, j+1) publishes the
//      next pivot.
// Results are written back to A and X. Returns false (in every thread) on a bad pivot.
template <int N, int M, int NT>
__device__ bool chol32_reg(float* A, float* X, float* colbuf, float* xrow, float* invd, float* piv) {
  constexpr int TRI = N * (N + 1) / 2, ST = (TRI + NT - 1) / NT, SX = (N * M + NT - 1) / NT;
  const int tid = threadIdx.x;
  float av[ST], xv[SX];
  int ak[ST], xk[SX];                              // (row << 16) | column, packed
#pragma unroll
  for (int s = 0; s < ST; ++s) {
    const int t = tid + s * NT;
    if (t < TRI) {
      const int i = tri_row(t);
      ak[s] = (i << 16) | (t - i * (i + 1) / 2);
      av[s] = A[t];
    } else {
      ak[s] = 0xffff;                                // row 0, column 65535: never active
      av[s] = 0.f;
    }
  }
#pragma unroll
  for (int s = 0; s < SX; ++s) {
    const int u = tid + s * NT;
    if (u < N * M) {
      xk[s] = ((u / M) << 16) | (u % M);
      xv[s] = X[u];
    } else {
      xk[s] = -1;                                    // row -1: never active
      xv[s] = 0.f;
    }
  }
  if (tid == 0) piv[0] = A[0];
  __syncthreads();
  bool ok = true;
  for (int j = 0; j < N; ++j) {
    const float d = piv[0];
    if (!(d > 0.0f) || !(d < INFINITY)) { ok = false; break; }
    const float r = dev::rsqrt_newton(d);
#pragma unroll
    for (int s = 0; s < ST; ++s) {
      const int i = ak[s] >> 16, l = ak[s] & 0xffff;
      if (l == j) {
        if (i == j) {
          av[s] = d * r;
          invd[j] = r;
        } else {
          av[s] *= r;
          colbuf[i] = av[s];
        }
      }
    }
#pragma unroll
    for (int s = 0; s < SX; ++s)
      if ((xk[s] >> 16) == j) {
        xv[s] *= r;
        xrow[xk[s] & 0xffff] = xv[s];
      }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < ST; ++s) {
      const int i = ak[s] >> 16, l = ak[s] & 0xffff;
      if (l > j && l < N) {
        av[s] = fmaf(-colbuf[i], colbuf[l], av[s]);
        if (l == j + 1 && i == j + 1) piv[0] = av[s];
      }
    }
#pragma unroll
    for (int s = 0; s < SX; ++s) {
      const int i = xk[s] >> 16;
      if (i > j) xv[s] = fmaf(-colbuf[i], xrow[xk[s] & 0xffff], xv[s]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int s = 0; s < ST; ++s)
    if (tid + s * NT < TRI) A[tid + s * NT] = av[s];
#pragma unroll
  for (int s = 0; s < SX; ++s)
    if (tid + s * NT < N * M) X[tid + s * NT] = xv[s];
  __syncthreads();
  return ok;
}

// Single-warp triangular solves with a packed lower factor L (invd = 1 / diag):
// forward L y = v in place, and backward L^T x = y in place.
__device__ void warp_fwd(const float* L, const float* invd, float* v, int n) {
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < n; ++j) {
    if (lane == (j & 31)) v[j] *= invd[j];
    __syncwarp();
    const float vj = v[j];
    for (int i = j + 1 + lane; i < n; i += 32) v[i] = fmaf(-L[tri(i, j)], vj, v[i]);
    __syncwarp();
  }
}
__device__ void warp_bwd(const float* L, const float* invd, float* v, int n) {
  const int lane = threadIdx.x & 31;
  for (int j = n - 1; j >= 0; --j) {
    if (lane == (j & 31)) v[j] *= invd[j];
    __syncwarp();
    const float vj = v[j];
    const float* Lj = L + tri(j, 0);
    for (int i = lane; i < j; i += 32) v[i] = fmaf(-Lj[i], vj, v[i]);
    __syncwarp();
  }
}
// same with a full row-major lower factor of leading dimension ld
__device__ void warp_fwd_full(const float* L, int ld, float* v, int n) {
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < n; ++j) {
    if (lane == (j & 31)) v[j] /= L[j * ld + j];
    __syncwarp();
    const float vj = v[j];
    for (int i = j + 1 + lane; i < n; i += 32) v[i] = fmaf(-L[i * ld + j], vj, v[i]);
    __syncwarp();
  }
}
__device__ void warp_bwd_full(const float* L, int ld, float* v, int n) {
  const int lane = threadIdx.x & 31;
  for (int j = n - 1; j >= 0; --j) {
    if (lane == (j & 31)) v[j] /= L[j * ld + j];
    __syncwarp();
    const float vj = v[j];
    for (int i = lane; i < j; i += 32) v[i] = fmaf(-L[j * ld + i], vj, v[i]);
    __syncwarp();
  }
}

// x = A_lo^{-1} v in FP32 with the Woodbury factors (warp 0 only): y = L_M^{-1} v,
// t = Xd^T y, s = Z^{-1} t, y -= Xd s, x = L_M^{-T} y. v is overwritten by x.
template <int K>
__device__ void woodbury_solve_warp(const float* LM, const float* invdM, const float* Xd, const float* LZ, float* v,
                                    float* t) {
  constexpr int p = K + 1, N = 3 * K * p * p + 6 * p * p, NQK = p * p * p;
  const int lane = threadIdx.x & 31;
  warp_fwd(LM, invdM, v, N);
  for (int a = lane; a < NQK; a += 32) {
    float acc = 0.f;
    for (int i = 0; i < N; ++i) acc = fmaf(Xd[i * NQK + a], v[i], acc);
    t[a] = acc;
  }
  __syncwarp();
  warp_fwd_full(LZ, NQK, t, NQK);
  warp_bwd_full(LZ, NQK, t, NQK);
  for (int i = lane; i < N; i += 32) {
    float acc = v[i];
    for (int a = 0; a < NQK; ++a) acc = fmaf(-Xd[i * NQK + a], t[a], acc);
    v[i] = acc;
  }
  __syncwarp();
  warp_bwd(LM, invdM, v, N);
}

// One FP32 solve of the mixed-form saddle system (warp 0): with r1, rho in v (n) and t (n_q),
//   y = L_M^{-1} r1,  dq = Z^{-1} (G^{-1} rho + Xd^T y),  dx = L_M^{-T} (y - Xd dq);
// v receives dx and t receives dq.
template <int K>
__device__ void mixed_solve_warp(const float* LM, const float* invdM, const float* Xd, const float* LZ,
                                 const float* Gi, float* v, float* t, float* tmp) {
  constexpr int p = K + 1, N = 3 * K * p * p + 6 * p * p, NQK = p * p * p;
  const int lane = threadIdx.x & 31;
  warp_fwd(LM, invdM, v, N);
  for (int a = lane; a < NQK; a += 32) {
    float acc = 0.f;
    for (int b = 0; b < NQK; ++b) acc = fmaf(Gi[a * NQK + b], t[b], acc);
    for (int i = 0; i < N; ++i) acc = fmaf(Xd[i * NQK + a], v[i], acc);
    tmp[a] = acc;
  }
  __syncwarp();
  for (int a = lane; a < NQK; a += 32) t[a] = tmp[a];
  __syncwarp();
  warp_fwd_full(LZ, NQK, t, NQK);
  warp_bwd_full(LZ, NQK, t, NQK);
  for (int i = lane; i < N; i += 32) {
    float acc = v[i];
    for (int a = 0; a < NQK; ++a) acc = fmaf(-Xd[i * NQK + a], t[a], acc);
    v[i] = acc;
  }
  __syncwarp();
  warp_bwd(LM, invdM, v, N);
}

// Iterative refinement of the element solve in the mixed variables (x, q = G D^T x):
//   r1 = f - M x - D q (free rows), f_e - x_e (essential rows),  rho = G D^T x - q,
// corrected by the FP32 block solve. This system is well conditioned at any contrast, so the
// FP64 residuals drive x to FP64 accuracy where refining A x = f directly would not converge.
template <int K, int NT>
__device__ void refine_mixed(const double* f, double* x, double* q, int steps, double alpha, double beta, int bmask,
                             const double* g6, const double* gd, const double* Vc, const double* Dc, const double* Vo,
                             const double* DcO64, const int* dofcode, const float* LM, const float* invdM,
                             const float* Xd, const float* LZ, const float* Gi, double* r, double* ut, double* rq,
                             double* U, double* Wv, double* Dv, double* xc, double* t1, double* t2, float* vec,
                             float* tq, float* tmp) {
  constexpr int p = K + 1, NI = 3 * K * p * p, NFN = p * p, N = NI + 6 * NFN, NQK = p * p * p;
  const int tid = threadIdx.x;
  auto is_e = [&](int i) { return i >= NI && ((bmask >> ((i - NI) / NFN)) & 1); };
  for (int i = tid; i < N; i += NT) x[i] = 0.0;
  for (int a = tid; a < NQK; a += NT) q[a] = 0.0;
  __syncthreads();
  for (int it = 0; it <= steps; ++it) {
    // r1 = f - M x~ - D q on free rows, f_e - x_e on essential rows
    for (int i = tid; i < N; i += NT) ut[i] = is_e(i) ? 0.0 : x[i];
    __syncthreads();
    apply_A64<K, NT>(ut, r, alpha, 0.0, false, g6, gd, Vc, Dc, Vo, U, Wv, Dv, xc, t1, t2);
    apply_D64<K, NT>(q, rq, dofcode, DcO64, bmask);
    for (int i = tid; i < N; i += NT) vec[i] = (float)(is_e(i) ? f[i] - x[i] : f[i] - r[i] - rq[i]);
    __syncthreads();
    // rho = G D^T x - q
    apply_Dt64<K, NT>(ut, rq, DcO64, bmask);
    apply_G64<K, NT>(rq, r, beta, gd, Vo, U, t1, t2);
    for (int a = tid; a < NQK; a += NT) tq[a] = (float)(r[a] - q[a]);
    __syncthreads();
    if (tid < 32) mixed_solve_warp<K>(LM, invdM, Xd, LZ, Gi, vec, tq, tmp);
    __syncthreads();
    for (int i = tid; i < N; i += NT) x[i] += (double)vec[i];
    for (int a = tid; a < NQK; a += NT) q[a] += (double)tq[a];
    __syncthreads();
  }
}

// ---------------------------------------------------------------- element kernel (FP32 path)
template <int K>
__device__ __forceinline__ void element_mixed_body(const ElemArgs& args, const int64_t e, double* smem) {
  using S = MX<K>;
  constexpr int P = S::P, p = S::p, Q = S::Q, NQ = S::NQ, NFN = S::NFN, NI = S::NI, NB = S::NB, N = S::N;
  constexpr int NQK = S::NQK, NT = S::NT, NC = S::NC;
  const int tid = threadIdx.x;
  const int64_t slot = args.slot ? args.slot[e] : e;
  float* store = args.Lstore32 + slot * S::STORE;

  // ---- shared memory: FP64 region then FP32 region then ints
  double* d = smem;
  double* X8 = d; d += 24;
  double* Mc = d; d += 24;
  double* Vc = d; d += P * Q;
  double* Dc = d; d += P * Q;
  double* Vo = d; d += p * Q;
  double* qx = d; d += Q;
  double* qw = d; d += Q;
  double* wf = d; d += NFN;
  double* g6 = d; d += 6 * NQ;
  double* gd = d; d += NQ;
  double* f = d; d += N;
  double* x = d; d += N;
  double* r = d; d += N;
  double* ut = d; d += N;
  double* U = d; d += 3 * NQ;
  double* Wv = d; d += 3 * NQ;
  double* Dv = d; d += NQ;
  double* xc = d; d += NC;
  double* t1 = d; d += S::TMP64;
  double* t2 = d; d += S::TMP64;
  d += 8;
  double* qv = d; d += NQK;
  double* rq = d; d += (N > NQ ? N : NQ);
  double* DcO64 = d; d += P * p;
  float* fl = reinterpret_cast<float*>(d);
  float* Vcf = fl; fl += P * Q;
  float* Dcf = fl; fl += P * Q;
  float* Vof = fl; fl += p * Q;
  float* VcVc = fl; fl += P * P * Q;
  float* VcVo = fl; fl += P * p * Q;
  float* VoVo = fl; fl += p * p * Q;
  float* DcO = fl; fl += P * p;
  float* Z = fl; fl += NQK * NQK;
  float* Y = fl; fl += S::TRIB;
  float* Sb = fl; fl += S::TRIB;
  float* V = fl; fl += S::VREG;               // scratch: mass assembly | G, L_G^{-1} | P, V
  float* colbuf = fl; fl += N;
  float* invd = fl; fl += N;
  float* vec = fl; fl += N;
  fl += N;
  float* tq = fl; fl += NQK;
  fl += NQK;
  float* tmpq = fl; fl += NQK;
  float* flag = fl; fl += 8;
  float* LM = S::BIG_SMEM ? fl : store;
  if (S::BIG_SMEM) fl += S::TRI;
  float* Xd = S::BIG_SMEM ? fl : store + S::TRI;
  if (S::BIG_SMEM) fl += N * NQK;
  int* dofcode = reinterpret_cast<int*>(fl);  // per local dof: c | i0 << 2 | i1 << 8 | i2 << 14
  float* LZs = store + S::TRI + (int64_t)N * NQK;
  float* Gis = LZs + NQK * NQK;

  load_element64<K, NT>(args, e, X8, Mc, Vc, Dc, Vo, qx, qw, wf);
  const RefTables& rt = c_refm[K];
  for (int i = tid; i < P * p; i += NT) DcO64[i] = rt.DcO[i / p][i % p];
  for (int i = tid; i < P * Q; i += NT) { Vcf[i] = (float)Vc[i]; Dcf[i] = (float)Dc[i]; }
  for (int i = tid; i < p * Q; i += NT) Vof[i] = (float)Vo[i];
  for (int i = tid; i < P * p; i += NT) DcO[i] = (float)rt.DcO[i / p][i % p];
  for (int t = tid; t < 3 * NC; t += NT) {
    const int c = t / NC, fi = t % NC;
    const int n0 = c == 0 ? P : p, n1 = c == 1 ? P : p;
    const int i0 = fi % n0, i1 = (fi / n0) % n1, i2 = fi / (n0 * n1);
    dofcode[local_index<K>(c, i0, i1, i2)] = c | (i0 << 2) | (i1 << 8) | (i2 << 14);
  }
  __syncthreads();
  for (int i = tid; i < P * P * Q; i += NT) {
    const int q = i % Q, b = (i / Q) % P, a = i / (Q * P);
    VcVc[i] = Vcf[a * Q + q] * Vcf[b * Q + q];
  }
  for (int i = tid; i < P * p * Q; i += NT) {
    const int q = i % Q, b = (i / Q) % p, a = i / (Q * p);
    VcVo[i] = Vcf[a * Q + q] * Vof[b * Q + q];
  }
  for (int i = tid; i < p * p * Q; i += NT) {
    const int q = i % Q, b = (i / Q) % p, a = i / (Q * p);
    VoVo[i] = Vof[a * Q + q] * Vof[b * Q + q];
  }
  geometry64<K, NT>(Mc, qx, qw, g6, gd, args.status, args.err_elem, e);
  const double alpha = args.alpha[e], beta = args.beta[e];

  // ---- FP64 load f = M c and essential values: f_f -= (A u_e)_f, f_e = u_e
  const double* coef = args.load + e * (int64_t)N;
  for (int i = tid; i < N; i += NT) ut[i] = coef[i];
  __syncthreads();
  apply_A64<K, NT>(ut, f, 1.0, 0.0, false, g6, gd, Vc, Dc, Vo, U, Wv, Dv, xc, t1, t2);
  const int32_t* ef = args.elem_face + e * 6;
  int bmask = 0;
#pragma unroll
  for (int a = 0; a < 6; ++a) bmask |= (ef[a] < 0) << a;
  auto is_e = [&](int i) { return i >= NI && ((bmask >> ((i - NI) / NFN)) & 1); };
  if (bmask) {
    const double* ue = args.ess ? args.ess + e * (int64_t)N : nullptr;
    if (ue) {
      for (int i = tid; i < N; i += NT) ut[i] = is_e(i) ? ue[i] : 0.0;
      __syncthreads();
      apply_A64<K, NT>(ut, r, alpha, beta, true, g6, gd, Vc, Dc, Vo, U, Wv, Dv, xc, t1, t2);
      for (int i = tid; i < N; i += NT) f[i] = is_e(i) ? ue[i] : f[i] - r[i];
    } else {
      for (int i = tid; i < N; i += NT)
        if (is_e(i)) f[i] = 0.0;
    }
    __syncthreads();
  }
  double* fs = args.zstore + e * (int64_t)N;   // the modified load, kept for the recovery
  for (int i = tid; i < N; i += NT) fs[i] = f[i];

  // ---- G = Q_k mass weighted by beta / det J (full, into Z), then G^{-1}
  {
    float* Gd32 = V;                          // [NQ]
    float* T1 = V + NQ;                       // [Q][Q][p][p]
    float* T2 = T1 + Q * Q * p * p;           // [Q][p^4]
    for (int q = tid; q < NQ; q += NT) Gd32[q] = (float)(beta * gd[q]);
    __syncthreads();
    for (int t = tid; t < Q * Q * p * p; t += NT) {        // T1[q2][q1][a0][b0]
      const int b0 = t % p, a0 = (t / p) % p, q1 = (t / (p * p)) % Q, q2 = t / (p * p * Q);
      float acc = 0.f;
      for (int q0 = 0; q0 < Q; ++q0) acc = fmaf(Gd32[(q2 * Q + q1) * Q + q0], VoVo[(a0 * p + b0) * Q + q0], acc);
      T1[t] = acc;
    }
    __syncthreads();
    for (int t = tid; t < Q * p * p * p * p; t += NT) {    // T2[q2][a1][b1][a0][b0]
      const int b0 = t % p, a0 = (t / p) % p, b1 = (t / (p * p)) % p, a1 = (t / (p * p * p)) % p, q2 = t / (p * p * p * p);
      float acc = 0.f;
      for (int q1 = 0; q1 < Q; ++q1) acc = fmaf(T1[((q2 * Q + q1) * p + a0) * p + b0], VoVo[(a1 * p + b1) * Q + q1], acc);
      T2[t] = acc;
    }
    __syncthreads();
    for (int t = tid; t < NQK * NQK; t += NT) {            // G[a][b], a = a0 + p (a1 + p a2)
      const int a = t / NQK, b = t % NQK;
      const int a0 = a % p, a1 = (a / p) % p, a2 = a / (p * p);
      const int b0 = b % p, b1 = (b / p) % p, b2 = b / (p * p);
      float acc = 0.f;
      for (int q2 = 0; q2 < Q; ++q2)
        acc = fmaf(T2[(((q2 * p + a1) * p + b1) * p + a0) * p + b0], VoVo[(a2 * p + b2) * Q + q2], acc);
      Z[t] = acc;
    }
    __syncthreads();
  }
  if (!chol32<NT>(Z, NQK, NQK, colbuf, invd, flag)) {
    if (tid == 0) set_error(args.status, args.err_elem, HYB_ERR_NOT_SPD, e);
    return;
  }
  {
    float* Li = V;                            // L_G^{-1}, full lower
    for (int t = tid; t < NQK * NQK; t += NT) Li[t] = 0.f;
    __syncthreads();
    for (int m = 0; m < NQK; ++m) {
      const float im = invd[m];
      for (int jj = tid; jj <= m; jj += NT) Li[m * NQK + jj] = (jj == m) ? im : Li[m * NQK + jj] * im;
      __syncthreads();
      const int w = m + 1, cnt = (NQK - 1 - m) * w;
      for (int t = tid; t < cnt; t += NT) {
        const int i = m + 1 + t / w, jj = t % w;
        Li[i * NQK + jj] = fmaf(-Z[i * NQK + m], Li[m * NQK + jj], Li[i * NQK + jj]);
      }
      __syncthreads();
    }
    for (int t = tid; t < NQK * NQK; t += NT) {            // G^{-1} = L^{-T} L^{-1}, into Z
      const int a = t / NQK, b = t % NQK;
      const int lo = a > b ? a : b;
      float acc = 0.f;
      for (int m = lo; m < NQK; ++m) acc = fmaf(Li[m * NQK + a], Li[m * NQK + b], acc);
      V[NQK * NQK + t] = acc;
    }
    __syncthreads();
    for (int t = tid; t < NQK * NQK; t += NT) {
      Z[t] = V[NQK * NQK + t];
      Gis[t] = V[NQK * NQK + t];
    }
    __syncthreads();
  }

  // ---- FP32 alpha-mass M (packed lower) by sum factorisation, essential rows -> identity
  {
    float* Ga32 = V;                          // [6][NQ]
    float* T1 = V + 6 * NQ;
    float* T2 = T1 + S::T1SZ;
    for (int t = tid; t < 6 * NQ; t += NT) Ga32[t] = (float)(alpha * g6[t]);
    __syncthreads();
    for (int blk = 0; blk < 6; ++blk) {
      const int c = blk < 3 ? blk : (blk == 3 ? 1 : 2);
      const int cp = blk < 3 ? blk : (blk == 5 ? 1 : 0);
      const bool diag = c == cp;
      const int da = c, db = diag ? (c + 1) % 3 : cp, dL = 3 - da - db;
      const int nia = P, nja = diag ? P : p, nib = p, njb = diag ? p : P;
      const int sa = da == 0 ? 1 : da == 1 ? Q : Q * Q;
      const int sb = db == 0 ? 1 : db == 1 ? Q : Q * Q;
      const int sL = dL == 0 ? 1 : dL == 1 ? Q : Q * Q;
      const float* Gm = Ga32 + gslot(c, cp) * NQ;
      const float* Pm = diag ? VcVc : VcVo;
      const int n1 = Q * Q * nia * nja;
      for (int idx = tid; idx < n1; idx += NT) {
        int rr = idx;
        const int ja = rr % nja; rr /= nja;
        const int ia = rr % nia; rr /= nia;
        const int qL = rr % Q, qb = rr / Q;
        float acc = 0.f;
        for (int qa = 0; qa < Q; ++qa) acc = fmaf(Gm[qa * sa + qb * sb + qL * sL], Pm[(ia * nja + ja) * Q + qa], acc);
        T1[idx] = acc;
      }
      __syncthreads();
      const int n2 = Q * nia * nja * nib * njb;
      for (int idx = tid; idx < n2; idx += NT) {
        int rr = idx;
        const int jb = rr % njb; rr /= njb;
        const int ib = rr % nib; rr /= nib;
        const int ja = rr % nja; rr /= nja;
        const int ia = rr % nia, qL = rr / nia;
        float acc = 0.f;
        for (int qb = 0; qb < Q; ++qb) {
          const float tv = T1[((qb * Q + qL) * nia + ia) * nja + ja];
          acc = fmaf(tv, diag ? VoVo[(ib * p + jb) * Q + qb] : VcVo[(jb * p + ib) * Q + qb], acc);
        }
        T2[idx] = acc;
      }
      __syncthreads();
      const int s2 = nia * nja * nib * njb;
      for (int idx = tid; idx < s2 * p * p; idx += NT) {
        int rr = idx;
        const int jL = rr % p; rr /= p;
        const int iL = rr % p; rr /= p;
        const int jb = rr % njb; rr /= njb;
        const int ib = rr % nib; rr /= nib;
        const int ja = rr % nja, ia = rr / nja;
        const int i0 = da == 0 ? ia : db == 0 ? ib : iL, i1 = da == 1 ? ia : db == 1 ? ib : iL;
        const int i2 = da == 2 ? ia : db == 2 ? ib : iL;
        const int j0 = da == 0 ? ja : db == 0 ? jb : jL, j1 = da == 1 ? ja : db == 1 ? jb : jL;
        const int j2 = da == 2 ? ja : db == 2 ? jb : jL;
        const int ra = local_index<K>(c, i0, i1, i2), sa2 = local_index<K>(cp, j0, j1, j2);
        if (diag && ra < sa2) continue;
        const int tt = ((ia * nja + ja) * nib + ib) * njb + jb;
        float acc = 0.f;
        for (int qL = 0; qL < Q; ++qL) acc = fmaf(T2[qL * s2 + tt], VoVo[(iL * p + jL) * Q + qL], acc);
        LM[ra >= sa2 ? tri(ra, sa2) : tri(sa2, ra)] = acc;
      }
      __syncthreads();
    }
    if (bmask) {
      for (int a = 0; a < 6; ++a) {
        if (!((bmask >> a) & 1)) continue;
        for (int t = tid; t < NFN * N; t += NT) {
          const int m = t / N, j = t % N, i = NI + a * NFN + m;
          LM[i >= j ? tri(i, j) : tri(j, i)] = (i == j) ? 1.f : 0.f;
        }
        __syncthreads();
      }
    }
  }

  // ---- D' (divergence coefficients, zero rows on essential dofs) into Xd, then
  // ---- L_M = chol(M) fused with Xd = L_M^{-1} D'
  for (int t = tid; t < N * NQK; t += NT) {
    const int i = t / NQK, a = t % NQK;
    float v = 0.f;
    if (!is_e(i)) {
      const int code = dofcode[i];
      const int c = code & 3, i0 = (code >> 2) & 63, i1 = (code >> 8) & 63, i2 = (code >> 14) & 63;
      const int a0 = a % p, a1 = (a / p) % p, a2 = a / (p * p);
      const bool match = (c == 0 || i0 == a0) && (c == 1 || i1 == a1) && (c == 2 || i2 == a2);
      if (match) v = DcO[(c == 0 ? i0 : c == 1 ? i1 : i2) * p + (c == 0 ? a0 : c == 1 ? a1 : a2)];
    }
    Xd[t] = v;
  }
  __syncthreads();
  bool spd;
  if constexpr (S::BIG_SMEM) spd = chol32_reg<N, NQK, NT>(LM, Xd, colbuf, vec, invd, flag);
  else spd = chol32<NT>(LM, N, -1, colbuf, invd, flag, Xd, NQK);
  if (!spd) {
    if (tid == 0) set_error(args.status, args.err_elem, HYB_ERR_NOT_SPD, e);
    return;
  }
  // ---- Z = G^{-1} + Xd^T Xd, L_Z = chol(Z)
  for (int t = tid; t < NQK * NQK; t += NT) {
    const int a = t / NQK, b = t % NQK;
    if (b > a) continue;
    float acc = Z[t];
    for (int i = 0; i < N; ++i) acc = fmaf(Xd[i * NQK + a], Xd[i * NQK + b], acc);
    Z[t] = acc;
  }
  __syncthreads();
  if (!chol32<NT>(Z, NQK, NQK, colbuf, vec, flag)) {
    if (tid == 0) set_error(args.status, args.err_elem, HYB_ERR_NOT_SPD, e);
    return;
  }
  for (int t = tid; t < NQK * NQK; t += NT) {
    const int a = t / NQK, b = t % NQK;
    LZs[t] = b <= a ? Z[t] : 0.f;
  }
  if (S::BIG_SMEM) {
    for (int t = tid; t < S::TRI; t += NT) store[t] = LM[t];
    for (int t = tid; t < N * NQK; t += NT) store[S::TRI + t] = Xd[t];
  }
  __syncthreads();

  // ---- g_T = D_c (A^{-1} f)_b: FP32 mixed-form solve, three refinement steps on FP64 residuals
  refine_mixed<K, NT>(f, x, qv, 3, alpha, beta, bmask, g6, gd, Vc, Dc, Vo, DcO64, dofcode, LM, invd, Xd, Z, Gis, r,
                      ut, rq, U, Wv, Dv, xc, t1, t2, vec, tq, tmpq);
  const int32_t* bo_face = ef;
  for (int ib = tid; ib < NB; ib += NT) {
    const int a = ib / NFN, m1 = ib % NFN;
    if (bo_face[a] < 0) continue;
    const double v = ((a & 1) ? 1.0 : -1.0) * wf[m1] * x[NI + ib];
    const int64_t gi = (int64_t)bo_face[a] * NFN + m1;
    if (args.colour == 1) args.rhs[gi] += v;
    else args.rhs[gi] = v;
  }

  // ---- Y = L_M,bb^{-1} (packed), P = Xd_b^T Y, V = L_Z^{-1} P, S = Y^T Y - V^T V
  for (int t = tid; t < S::TRIB; t += NT) Y[t] = 0.f;
  __syncthreads();
  for (int m = 0; m < NB; ++m) {
    const float im = invd[NI + m];
    for (int jj = tid; jj <= m; jj += NT) Y[tri(m, jj)] = (jj == m) ? im : Y[tri(m, jj)] * im;
    __syncthreads();
    const int w = m + 1, cnt = (NB - 1 - m) * w;
    for (int t = tid; t < cnt; t += NT) {
      const int i = m + 1 + t / w, jj = t % w;
      Y[tri(i, jj)] = fmaf(-LM[tri(NI + i, NI + m)], Y[tri(m, jj)], Y[tri(i, jj)]);
    }
    __syncthreads();
  }
  for (int t = tid; t < NQK * NB; t += NT) {              // P[a][jb]
    const int a = t / NB, jb = t % NB;
    float acc = 0.f;
    for (int m = jb; m < NB; ++m) acc = fmaf(Xd[(NI + m) * NQK + a], Y[tri(m, jb)], acc);
    V[t] = acc;
  }
  __syncthreads();
  for (int jb = tid; jb < NB; jb += NT) {                 // V = L_Z^{-1} P, column by column
    for (int a = 0; a < NQK; ++a) {
      float acc = V[a * NB + jb];
      for (int b = 0; b < a; ++b) acc = fmaf(-Z[a * NQK + b], V[b * NB + jb], acc);
      V[a * NB + jb] = acc / Z[a * NQK + a];
    }
  }
  __syncthreads();
  for (int t = tid; t < S::TRIB; t += NT) {
    const int i = tri_row(t), jj = t - i * (i + 1) / 2;
    float acc = 0.f;
    for (int m = i; m < NB; ++m) acc = fmaf(Y[tri(m, i)], Y[tri(m, jj)], acc);
    for (int a = 0; a < NQK; ++a) acc = fmaf(-V[a * NB + i], V[a * NB + jj], acc);
    Sb[t] = acc;
  }
  __syncthreads();
  // ---- scatter S_T = D_c S D_c into the FP64 CSR values
  const int64_t* boff = args.blockoff + e * 36;
  for (int t = tid; t < NB * NB; t += NT) {
    const int ib = t / NB, jb = t % NB;
    const int a = ib / NFN, m1 = ib % NFN, b = jb / NFN, m2 = jb % NFN;
    if (bo_face[a] < 0 || bo_face[b] < 0) continue;
    const double dd = (((a ^ b) & 1) ? -1.0 : 1.0) * wf[m1] * wf[m2];
    const double v = dd * (double)Sb[ib >= jb ? tri(ib, jb) : tri(jb, ib)];
    const int64_t r0 = args.row_ptr[(int64_t)bo_face[a] * NFN];
    const int64_t rl = args.row_ptr[(int64_t)bo_face[a] * NFN + 1] - r0;
    const int64_t pos = boff[a * 6 + b] + m1 * rl + m2;
    if (a == b && args.colour == 1) args.val[pos] += v;
    else args.val[pos] = v;
  }
}

template <int K>
__global__ void __launch_bounds__(MX<K>::NT) element_mixed_kernel(ElemArgs args) {
  extern __shared__ double smem[];
  const int64_t li = blockIdx.x;
  if (li >= args.n_list) return;
  element_mixed_body<K>(args, args.elem_list[li], smem);
}

template <int K>
__global__ void __launch_bounds__(MX<K>::NT) element_mixed_kernel_batch(const ElemArgs* probs, const int2* items,
                                                                       int64_t n_items, int colour) {
  extern __shared__ double smem[];
  const int64_t li = blockIdx.x;
  if (li >= n_items) return;
  const int2 it = items[li];
  ElemArgs a = probs[it.x];
  a.colour = colour;
  element_mixed_body<K>(a, it.y, smem);
}

// ---------------------------------------------------------------- recovery (FP32 + FP64 refinement)
template <int K>
__device__ __forceinline__ void recover_mixed_body(const ElemArgs& args, const int64_t e, const double* lambda,
                                                   double* u, double* smem) {
  using S = MX<K>;
  constexpr int P = S::P, p = S::p, Q = S::Q, NQ = S::NQ, NFN = S::NFN, NI = S::NI, N = S::N;
  constexpr int NQK = S::NQK, NT = S::NT, NC = S::NC;
  const int tid = threadIdx.x;
  const int64_t slot = args.slot ? args.slot[e] : e;
  const float* store = args.Lstore32 + slot * S::STORE;
  const float* LM = store;
  const float* Xd = store + S::TRI;
  const float* LZ = store + S::TRI + (int64_t)N * NQK;
  double* d = smem;
  double* X8 = d; d += 24;
  double* Mc = d; d += 24;
  double* Vc = d; d += P * Q;
  double* Dc = d; d += P * Q;
  double* Vo = d; d += p * Q;
  double* qx = d; d += Q;
  double* qw = d; d += Q;
  double* wf = d; d += NFN;
  double* g6 = d; d += 6 * NQ;
  double* gd = d; d += NQ;
  double* f = d; d += N;
  double* x = d; d += N;
  double* r = d; d += N;
  double* ut = d; d += N;
  double* U = d; d += 3 * NQ;
  double* Wv = d; d += 3 * NQ;
  double* Dv = d; d += NQ;
  double* xc = d; d += NC;
  double* t1 = d; d += S::TMP64;
  double* t2 = d; d += S::TMP64;
  d += 8;
  double* qv = d; d += NQK;
  double* rq = d; d += (N > NQ ? N : NQ);
  double* DcO64 = d; d += P * p;
  float* fl = reinterpret_cast<float*>(d);
  float* vec = fl; fl += N;
  float* tq = fl; fl += NQK;
  float* tmpq = fl; fl += NQK;
  float* invd = fl; fl += N;
  int* dofcode = reinterpret_cast<int*>(fl + 8);

  const float* Gi = LZ + NQK * NQK;
  load_element64<K, NT>(args, e, X8, Mc, Vc, Dc, Vo, qx, qw, wf);
  {
    const RefTables& rt = c_refm[K];
    for (int i = tid; i < P * p; i += NT) DcO64[i] = rt.DcO[i / p][i % p];
    for (int t = tid; t < 3 * NC; t += NT) {
      const int c = t / NC, fi = t % NC;
      const int n0 = c == 0 ? P : p, n1 = c == 1 ? P : p;
      const int i0 = fi % n0, i1 = (fi / n0) % n1, i2 = fi / (n0 * n1);
      dofcode[local_index<K>(c, i0, i1, i2)] = c | (i0 << 2) | (i1 << 8) | (i2 << 14);
    }
  }
  geometry64<K, NT>(Mc, qx, qw, g6, gd, args.status, args.err_elem, e);
  const double alpha = args.alpha[e], beta = args.beta[e];
  const int32_t* ef = args.elem_face + e * 6;
  int bmask = 0;
#pragma unroll
  for (int a = 0; a < 6; ++a) bmask |= (ef[a] < 0) << a;
  auto is_e = [&](int i) { return i >= NI && ((bmask >> ((i - NI) / NFN)) & 1); };
  const double* fs = args.zstore + e * (int64_t)N;
  for (int i = tid; i < N; i += NT) {
    double v = fs[i];
    if (i >= NI) {
      const int a = (i - NI) / NFN, m = (i - NI) % NFN;
      if (ef[a] >= 0) v -= ((a & 1) ? 1.0 : -1.0) * wf[m] * lambda[(int64_t)ef[a] * NFN + m];
    }
    f[i] = v;                                  // f_T - C_T^T lambda
    invd[i] = 1.0f / LM[tri(i, i)];
  }
  __syncthreads();
  refine_mixed<K, NT>(f, x, qv, 3, alpha, beta, bmask, g6, gd, Vc, Dc, Vo, DcO64, dofcode, LM, invd, Xd, LZ, Gi, r,
                      ut, rq, U, Wv, Dv, xc, t1, t2, vec, tq, tmpq);
  double* ue = u + e * (int64_t)N;
  for (int i = tid; i < N; i += NT) ue[i] = x[i];
}

template <int K>
__global__ void __launch_bounds__(MX<K>::NT) recover_mixed_kernel(ElemArgs args, const double* lambda, double* u) {
  extern __shared__ double smem[];
  const int64_t li = blockIdx.x;
  if (li >= args.n_list) return;
  recover_mixed_body<K>(args, args.elem_list[li], lambda, u, smem);
}

// batched recovery: per-problem multipliers and outputs in BatchRecover
template <int K>
__global__ void __launch_bounds__(MX<K>::NT) recover_mixed_kernel_batch(const ElemArgs* probs, const double* const* lams,
                                                                       double* const* us, const int2* items,
                                                                       int64_t n_items) {
  extern __shared__ double smem[];
  const int64_t li = blockIdx.x;
  if (li >= n_items) return;
  const int2 it = items[li];
  const ElemArgs a = probs[it.x];
  recover_mixed_body<K>(a, it.y, lams[it.x], us[it.x], smem);
}

#include "hyb_mixed_tiled.cuh"

template <int K>
cudaError_t launch_mixed_batch_k(const ElemArgs* probs, const int2* items, int64_t n, int colour, bool recover,
                                 const double* const* lams, double* const* us, cudaStream_t s, Prof* prof) {
  if (n == 0) return cudaSuccess;
  cudaError_t err;
  if constexpr (K >= 1) {
    using S = MT<K>;
    if (!recover) {
      err = cudaFuncSetAttribute(element_tiled_kernel_batch<K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
      if (err == cudaSuccess) err = cudaFuncSetAttribute(element_tiled_kernel_batch<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)S::SMEM);
      if (err != cudaSuccess) return err;
      const int tok = prof_begin(prof, HYB_K_ELEMENT, s);
      element_tiled_kernel_batch<K><<<(unsigned)n, S::NT, S::SMEM, s>>>(probs, items, n, colour);
      prof_end(prof, tok, s);
    } else {
      err = cudaFuncSetAttribute(recover_tiled_kernel_batch<K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
      if (err == cudaSuccess) err = cudaFuncSetAttribute(recover_tiled_kernel_batch<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)S::SMEM);
      if (err != cudaSuccess) return err;
      const int tok = prof_begin(prof, HYB_K_RECOVER, s);
      recover_tiled_kernel_batch<K><<<(unsigned)n, S::NT, S::SMEM, s>>>(probs, lams, us, items, n);
      prof_end(prof, tok, s);
    }
    return cudaGetLastError();
  } else {
  using S = MX<K>;
  if (!recover) {
    err = cudaFuncSetAttribute(element_mixed_kernel_batch<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    if (err != cudaSuccess) return err;
    const int tok = prof_begin(prof, HYB_K_ELEMENT, s);
    element_mixed_kernel_batch<K><<<(unsigned)n, S::NT, S::SMEM, s>>>(probs, items, n, colour);
    prof_end(prof, tok, s);
  } else {
    err = cudaFuncSetAttribute(recover_mixed_kernel_batch<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    if (err != cudaSuccess) return err;
    const int tok = prof_begin(prof, HYB_K_RECOVER, s);
    recover_mixed_kernel_batch<K><<<(unsigned)n, S::NT, S::SMEM, s>>>(probs, lams, us, items, n);
    prof_end(prof, tok, s);
  }
  return cudaGetLastError();
  }
}

template <int K>
cudaError_t launch_mixed_k(const ElemArgs& a, cudaStream_t s, Prof* prof, bool recover, const double* lambda,
                           double* u) {
  if (a.n_list == 0) return cudaSuccess;
  cudaError_t err;
  if constexpr (K >= 1) {
    using S = MT<K>;
    if (!recover) {
      err = cudaFuncSetAttribute(element_tiled_kernel<K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
      if (err == cudaSuccess) err = cudaFuncSetAttribute(element_tiled_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
      if (err != cudaSuccess) return err;
      const int tok = prof_begin(prof, HYB_K_ELEMENT, s);
      element_tiled_kernel<K><<<(unsigned)a.n_list, S::NT, S::SMEM, s>>>(a);
      prof_end(prof, tok, s);
    } else {
      err = cudaFuncSetAttribute(recover_tiled_kernel<K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
      if (err == cudaSuccess) err = cudaFuncSetAttribute(recover_tiled_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
      if (err != cudaSuccess) return err;
      const int tok = prof_begin(prof, HYB_K_RECOVER, s);
      recover_tiled_kernel<K><<<(unsigned)a.n_list, S::NT, S::SMEM, s>>>(a, lambda, u);
      prof_end(prof, tok, s);
    }
    return cudaGetLastError();
  } else {
  using S = MX<K>;
  if (!recover) {
    err = cudaFuncSetAttribute(element_mixed_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    if (err != cudaSuccess) return err;
    const int tok = prof_begin(prof, HYB_K_ELEMENT, s);
    element_mixed_kernel<K><<<(unsigned)a.n_list, S::NT, S::SMEM, s>>>(a);
    prof_end(prof, tok, s);
  } else {
    err = cudaFuncSetAttribute(recover_mixed_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    if (err != cudaSuccess) return err;
    const int tok = prof_begin(prof, HYB_K_RECOVER, s);
    recover_mixed_kernel<K><<<(unsigned)a.n_list, S::NT, S::SMEM, s>>>(a, lambda, u);
    prof_end(prof, tok, s);
  }
  return cudaGetLastError();
  }
}

}  // namespace

// FP32-path store per element: L_M | Xd | L_Z | G^{-1} for the recovery (packed triangles
// for RT_0, tiles for RT_1 to RT_3).
int64_t mixed_store_floats(int k) {
  switch (k) {
    case 0: return MX<0>::STORE;
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
                               const double* const* lams, double* const* us, cudaStream_t s, Prof* prof) {
  switch (k) {
    case 0: return launch_mixed_batch_k<0>(probs, items, n, colour, recover, lams, us, s, prof);
    case 1: return launch_mixed_batch_k<1>(probs, items, n, colour, recover, lams, us, s, prof);
    case 2: return launch_mixed_batch_k<2>(probs, items, n, colour, recover, lams, us, s, prof);
    case 3: return launch_mixed_batch_k<3>(probs, items, n, colour, recover, lams, us, s, prof);
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
