// Element-by-element elimination for algebraic hybridization and static
// condensation (arXiv:1801.08914, Thm 2.1 / eq. 2.4, Sec. 3.1, Sec. 5), FP64.
//
// One CTA eliminates one hexahedron:
//   1. geometry at the (k+2)^3 Gauss points: w J^T J / det J and w / det J;
//   2. A_T = alpha M_T + beta K_T by sum factorisation over the three
//      directions (the RT_k basis and the rule are tensor products);
//   3. f_T = M_T c_T matrix-free (load given by broken-RT_k coefficients);
//   4. essential dofs: f -= A_{:,e} u_e, rows / columns of A replaced by I;
//   5. right-looking Cholesky of the packed lower triangle (interior dofs
//      first, the 2x2 block form of Sec. 5), fused with z = L^{-1} f;
//      static condensation stops after the interior columns, leaving
//      S_hat = A_bb - A_bi A_ii^{-1} A_ib in the trailing block;
//   6. hybridization: Y = L_bb^{-1}, S_T = D Y^T Y D, g_T = D Y^T z_b where
//      C_T = [0 D] is diagonal (signed face Gauss weights, zero on boundary faces);
//   7. atomic-free scatter into the CSR values of the face-multiplier system:
//      a face block shared by two elements is stored by colour 0 and
//      incremented by colour 1 in a later launch, every other block has one owner.
// The factor (with Y in place of L_bb for hybridization) and z are stored for
// the back substitution.
#include <cuda_runtime.h>

#include "hyb_device.h"
#include "hyb_internal.h"
#include "hyb_tiles.cuh"

namespace hyb {

__constant__ RefTables c_ref[kMaxOrder + 1];

cudaError_t upload_ref_tables(const RefTables* tabs, int count, cudaStream_t s) {
  return cudaMemcpyToSymbolAsync(c_ref, tabs, sizeof(RefTables) * count, 0, cudaMemcpyHostToDevice, s);
}

namespace {

using dev::tri;
using dev::local_index;
using dev::gslot;
using dev::tri_row;
using dev::rsqrt_newton;
using dev::set_error;

template <int K>
struct EK {
  static constexpr int P = K + 2, p = K + 1, Q = K + 2, NQ = Q * Q * Q;
  static constexpr int NFN = p * p, NI = 3 * K * p * p, NB = 6 * NFN, N = NI + NB;
  static constexpr int NC = P * p * p;                 // functions per component
  static constexpr int NT = K == 0 ? 32 : K == 1 ? 64 : K == 2 ? 256 : 512;
  // RT_2 and RT_3: the elimination runs on NFN x NFN tiles (element_tail_tiled; one tile per
  // face, 3k tiles per interior component block): interior block L_ii and interface rows L_bi
  // resident together, then the Schur complement of the face block. A_T is assembled into the
  // element's factor store in HBM there (packed), so that the tiles fit beside it.
  static constexpr bool TILED_PATH = K >= 2;
  static constexpr bool A_SMEM = !TILED_PATH;
  static constexpr int TB = TILED_PATH ? NFN : 16, TI = NI / TB, TBB = NB / TB;
  static constexpr int MR = K == 2 ? 3 : 2, MC = MR;         // register micro-tiles of the updates
  static constexpr int R1 = TI * (TI + 1) / 2 * TB * TB;     // L_ii tiles, later the face-block tiles
  static constexpr int R2 = TBB * TI * TB * TB;              // L_bi tiles, later Y = L_bb^{-1} (NB x NB)
  // the face block needs its own tiles and those of S = Y^T Y (2 x 21 tiles): past R1 where R1
  // is smaller (RT_2: 21 tiles)
  static constexpr int RX = 2 * TBB * (TBB + 1) / 2 * TB * TB > R1 ? 2 * TBB * (TBB + 1) / 2 * TB * TB - R1 : 0;
  static constexpr int TILED = TILED_PATH ? R1 + R2 + RX : 0;
  static constexpr int TRI = N * (N + 1) / 2;
  static constexpr int TRIB = NB * (NB + 1) / 2;
  // 1-D tables: Vc, Dc (P x Q), Vo (p x Q), products VcVc, DcDc (P P Q), VcVo, DcVo (P p Q), VoVo (p p Q)
  static constexpr int TAB = 2 * P * Q + p * Q + 2 * P * P * Q + 2 * P * p * Q + p * p * Q + 2 * Q + NFN;
  // assembly scratch: T1, T2, Gu[6], Ga[6], Gd; load scratch: 2 x 3 x (P P Q) buffers, U[3], W[3]
  static constexpr int T1SZ = 2 * Q * Q * P * P;
  static constexpr int T2SZ = Q * P * P * p * p;
  static constexpr int LBUF = 3 * P * P * Q;
  static constexpr int ASM = T1SZ + T2SZ + 13 * NQ + 2 * LBUF + 6 * NQ;
  static constexpr int POST = 2 * TRIB;                // Y, Y^T Y (row-major packed)
  static constexpr int UNION0 = ASM > POST ? ASM : POST;
  static constexpr int UNION = UNION0 > TILED ? UNION0 : TILED;
  static constexpr int SMEM_DOUBLES = (A_SMEM ? TRI : 0) + 3 * N + 48 + TAB + UNION + 4;
  static constexpr size_t SMEM_BYTES = sizeof(double) * SMEM_DOUBLES;
};

struct Tabs {
  const double *Vc, *Dc, *Vo;                  // [P][Q], [P][Q], [p][Q]
  const double *VcVc, *DcDc, *VcVo, *DcVo, *VoVo;   // [a][b][q] products
};

// Block (c, cp) of alpha M + beta K, c >= cp, written into the packed lower triangle of A.
// Directions are contracted one at a time (sum factorisation); the mass and divergence
// terms share every stage after the directions in which their 1-D factors differ.
template <int K>
__device__ void assemble_block(int c, int cp, const Tabs& tb, const double* Ga, const double* Gd,
                               double* T1, double* T2, double* A) {
  using S = EK<K>;
  constexpr int P = S::P, p = S::p, Q = S::Q, NT = S::NT;
  const int tid = threadIdx.x;
  const bool diag = c == cp;
  const int da = c;
  const int db = diag ? (c + 1) % 3 : cp;
  const int dL = 3 - da - db;
  const int nia = P, nja = diag ? P : p;                   // along da (== c)
  const int nib = p, njb = diag ? p : P;                   // along db
  constexpr int niL = p, njL = p;                          // along dL (neither c nor cp)
  const int sa = da == 0 ? 1 : da == 1 ? Q : Q * Q;
  const int sb = db == 0 ? 1 : db == 1 ? Q : Q * Q;
  const int sL = dL == 0 ? 1 : dL == 1 ? Q : Q * Q;
  const double* Gm = Ga + gslot(c, cp) * S::NQ;
  const double* Pm = diag ? tb.VcVc : tb.VcVo;             // [ia][ja][q]
  const double* Pd = diag ? tb.DcDc : tb.DcVo;

  // stage 1: contract q_a
  const int n1 = Q * Q * nia * nja;
  for (int idx = tid; idx < n1; idx += NT) {
    int r = idx;
    const int ja = r % nja; r /= nja;
    const int ia = r % nia; r /= nia;
    const int qL = r % Q;
    const int qb = r / Q;
    const double* pm = Pm + (ia * nja + ja) * Q;
    const double* pd = Pd + (ia * nja + ja) * Q;
    double accm = 0.0, accd = 0.0;
#pragma unroll
    for (int qa = 0; qa < Q; ++qa) {
      const int q = qa * sa + qb * sb + qL * sL;
      accm = fma(Gm[q], pm[qa], accm);
      accd = fma(Gd[q], pd[qa], accd);
    }
    if (diag) {
      T1[idx] = accm + accd;
    } else {
      T1[idx] = accm;
      T1[n1 + idx] = accd;
    }
  }
  __syncthreads();

  // stage 2: contract q_b
  const int n2 = Q * nia * nja * nib * njb;
  for (int idx = tid; idx < n2; idx += NT) {
    int r = idx;
    const int jb = r % njb; r /= njb;
    const int ib = r % nib; r /= nib;
    const int ja = r % nja; r /= nja;
    const int ia = r % nia;
    const int qL = r / nia;
    double acc = 0.0;
#pragma unroll
    for (int qb = 0; qb < Q; ++qb) {
      const int t1 = ((qb * Q + qL) * nia + ia) * nja + ja;
      if (diag) {
        acc = fma(T1[t1], tb.VoVo[(ib * p + jb) * Q + qb], acc);
      } else {
        // rows: open in db; columns: closed value (mass) / closed derivative (div) in db == cp
        acc = fma(T1[t1], tb.VcVo[(jb * p + ib) * Q + qb], acc);
        acc = fma(T1[n1 + t1], tb.DcVo[(jb * p + ib) * Q + qb], acc);
      }
    }
    T2[idx] = acc;
  }
  __syncthreads();

  // stage 3: contract q_L and write the lower triangle
  const int n3 = nia * nja * nib * njb * niL * njL;
  const int s2 = nia * nja * nib * njb;
  for (int idx = tid; idx < n3; idx += NT) {
    int r = idx;
    const int jL = r % njL; r /= njL;
    const int iL = r % niL; r /= niL;
    const int jb = r % njb; r /= njb;
    const int ib = r % nib; r /= nib;
    const int ja = r % nja;
    const int ia = r / nja;
    const int i0 = da == 0 ? ia : db == 0 ? ib : iL;
    const int i1 = da == 1 ? ia : db == 1 ? ib : iL;
    const int i2 = da == 2 ? ia : db == 2 ? ib : iL;
    const int j0 = da == 0 ? ja : db == 0 ? jb : jL;
    const int j1 = da == 1 ? ja : db == 1 ? jb : jL;
    const int j2 = da == 2 ? ja : db == 2 ? jb : jL;
    const int rr = local_index<K>(c, i0, i1, i2);
    const int ss = local_index<K>(cp, j0, j1, j2);
    if (diag && rr < ss) continue;
    const int t2 = (((ia * nja + ja) * nib + ib) * njb + jb);
    const double* pv = tb.VoVo + (iL * p + jL) * Q;
    double acc = 0.0;
#pragma unroll
    for (int qL = 0; qL < Q; ++qL) acc = fma(T2[qL * s2 + t2], pv[qL], acc);
    A[rr >= ss ? tri(rr, ss) : tri(ss, rr)] = acc;
  }
  __syncthreads();
}

// f = M c with M the unit-coefficient mass, by sum factorisation: interpolate the three
// reference components of the coefficient field at the Gauss points, apply the weights
// w J^T J / det J, test against the basis. B0, B1 hold 3 x (P P Q) doubles each.
template <int K>
__device__ void load_vector(const double* coef, const Tabs& tb, const double* Gu, double* B0, double* B1,
                            double* U, double* W, double* f) {
  using S = EK<K>;
  constexpr int P = S::P, p = S::p, Q = S::Q, NQ = S::NQ, NT = S::NT, LB = P * P * Q;
  const int tid = threadIdx.x;
  auto nn = [](int c, int d) { return c == d ? P : p; };
  auto tab = [&](int c, int d) { return c == d ? tb.Vc : tb.Vo; };
  // Z1[c][i2][i1][q0] = sum_i0 coef * T0[i0][q0]
  for (int t = tid; t < 3 * LB; t += NT) {
    const int c = t / LB, r = t % LB;
    const int n0 = nn(c, 0), n1 = nn(c, 1), n2 = nn(c, 2);
    if (r >= n2 * n1 * Q) continue;
    const int q0 = r % Q, i1 = (r / Q) % n1, i2 = r / (Q * n1);
    const double* T = tab(c, 0);
    double acc = 0.0;
    for (int i0 = 0; i0 < n0; ++i0) acc = fma(coef[local_index<K>(c, i0, i1, i2)], T[i0 * Q + q0], acc);
    B0[t] = acc;
  }
  __syncthreads();
  // Z2[c][i2][q1][q0] = sum_i1 Z1 * T1[i1][q1]
  for (int t = tid; t < 3 * LB; t += NT) {
    const int c = t / LB, r = t % LB;
    const int n1 = nn(c, 1), n2 = nn(c, 2);
    if (r >= n2 * Q * Q) continue;
    const int q0 = r % Q, q1 = (r / Q) % Q, i2 = r / (Q * Q);
    const double* T = tab(c, 1);
    double acc = 0.0;
    for (int i1 = 0; i1 < n1; ++i1) acc = fma(B0[c * LB + (i2 * n1 + i1) * Q + q0], T[i1 * Q + q1], acc);
    B1[t] = acc;
  }
  __syncthreads();
  // U[c][q] = sum_i2 Z2 * T2[i2][q2]
  for (int t = tid; t < 3 * NQ; t += NT) {
    const int c = t / NQ, q = t % NQ;
    const int q0 = q % Q, q1 = (q / Q) % Q, q2 = q / (Q * Q);
    const int n2 = nn(c, 2);
    const double* T = tab(c, 2);
    double acc = 0.0;
    for (int i2 = 0; i2 < n2; ++i2) acc = fma(B1[c * LB + (i2 * Q + q1) * Q + q0], T[i2 * Q + q2], acc);
    U[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < 3 * NQ; t += NT) {
    const int c = t / NQ, q = t % NQ;
    W[t] = Gu[gslot(c, 0) * NQ + q] * U[q] + Gu[gslot(c, 1) * NQ + q] * U[NQ + q] +
           Gu[gslot(c, 2) * NQ + q] * U[2 * NQ + q];
  }
  __syncthreads();
  // Y1[c][q2][q1][i0] = sum_q0 W * T0[i0][q0]
  for (int t = tid; t < 3 * LB; t += NT) {
    const int c = t / LB, r = t % LB;
    const int n0 = nn(c, 0);
    if (r >= Q * Q * n0) continue;
    const int i0 = r % n0, q1 = (r / n0) % Q, q2 = r / (n0 * Q);
    const double* T = tab(c, 0);
    double acc = 0.0;
    for (int q0 = 0; q0 < Q; ++q0) acc = fma(W[c * NQ + (q2 * Q + q1) * Q + q0], T[i0 * Q + q0], acc);
    B0[t] = acc;
  }
  __syncthreads();
  // Y2[c][q2][i1][i0] = sum_q1 Y1 * T1[i1][q1]
  for (int t = tid; t < 3 * LB; t += NT) {
    const int c = t / LB, r = t % LB;
    const int n0 = nn(c, 0), n1 = nn(c, 1);
    if (r >= Q * n1 * n0) continue;
    const int i0 = r % n0, i1 = (r / n0) % n1, q2 = r / (n0 * n1);
    const double* T = tab(c, 1);
    double acc = 0.0;
    for (int q1 = 0; q1 < Q; ++q1) acc = fma(B0[c * LB + (q2 * Q + q1) * n0 + i0], T[i1 * Q + q1], acc);
    B1[t] = acc;
  }
  __syncthreads();
  // f[c][i2][i1][i0] = sum_q2 Y2 * T2[i2][q2]
  for (int t = tid; t < 3 * S::NC; t += NT) {
    const int c = t / S::NC, r = t % S::NC;
    const int n0 = nn(c, 0), n1 = nn(c, 1);
    const int i0 = r % n0, i1 = (r / n0) % n1, i2 = r / (n0 * n1);
    const double* T = tab(c, 2);
    double acc = 0.0;
    for (int q2 = 0; q2 < Q; ++q2) acc = fma(B1[c * LB + (q2 * n1 + i1) * n0 + i0], T[i2 * Q + q2], acc);
    f[local_index<K>(c, i0, i1, i2)] = acc;
  }
  __syncthreads();
}

// ---- RT_3 elimination on tiles, after the assembly has written A_T (packed, row-major
// lower, essential rows already identity) to its factor slot A and the load to f:
//   1. the first TI tile columns (interior dofs) with all rows in shared memory: L_ii and L_bi
//      (blocked right-looking Cholesky restricted to those columns);
//   2. z_i = L_ii^{-1} f_i, f_b -= L_bi z_i; L_ii and L_bi go to the factor slot;
//   3. the face block A_bb - L_bi L_bi^T (its Schur complement, Sec. 3.1);
//   4. static condensation: scatter it and f_b; hybridization: L_bb = chol(.), z_b, Y = L_bb^{-1},
//      S_T = D Y^T Y D and g_T = D Y^T z_b scattered, Y into the slot in place of L_bb.
// The factor slot keeps the packed layout the recovery reads.

// The face block of the hybridization in one look-ahead pass over its 6 x 6 tiles of 16 x 16:
// L_bb = chol(A_bb - L_bi L_bi^T) (packed tiles in Lt, diagonal tiles inverted), Y = L_bb^{-1}
// (row-major in Y, ld 96, formed from the identity) and S = Y^T Y (lower tiles, packed, in Sg).
// Once tile column J is scaled, block row J of Y is final too, so the trailing update of L_bb,
// the update of Y's later block rows and the rank-16 term Y_J^T Y_J of S share one phase; it
// fills the sub-partitions that the one-warp diagonal step (warp 0, look-ahead) leaves idle.
// Two barriers per tile column. Returns false in every thread on a bad pivot.
template <int TB, int NT, int MR, int MC>
__device__ bool face_block_hyb(double* Lt, double* Y, double* Sg, double* flag) {
  constexpr int T = 6, NB = T * TB, TT = TB * TB, PM = (TB / MR) * (TB / MC);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto tp = [&](int I, int J) { return Lt + tiles::tcol(I, J, T) * TT; };
  for (int t = tid; t < NB * NB; t += NT) Y[t] = (t / NB == t % NB) ? 1.0 : 0.0;
  for (int t = tid; t < T * (T + 1) / 2 * TT; t += NT) Sg[t] = 0.0;
  if (tid == 0) flag[0] = 0.0;
  __syncthreads();
  if (warp == 0) tiles::diag_step<double, TB>(tp(0, 0), flag, tiles::NoOut{});
  __syncthreads();
  for (int J = 0; J < T; ++J) {
    if (flag[0] != 0.0) return false;
    const double* Dv = tp(J, J);
    const int nrows = (T - J - 1) * TB, ncy = (J + 1) * TB;   // Y_J: zero beyond column ncy
    double* YJ = Y + J * TB * NB;
    for (int it = tid; it < nrows + ncy; it += NT) {
      if (it < nrows) tiles::panel_row_item<double, TB>(Dv, tp(J + 1 + it / TB, J), it % TB);
      else tiles::scale_rows_item<double, TB>(Dv, YJ, NB, it - nrows);
    }
    __syncthreads();
    const bool next = J + 1 < T;
    const int m = T - J - 1, npairs = m * (m + 1) / 2;
    if (next && warp == 0) {
      double* Dn = tp(J + 1, J + 1);
      const double* P = tp(J + 1, J);
      for (int u = lane; u < PM; u += 32) {
        const int r0 = (u / (TB / MC)) * MR, c0 = (u % (TB / MC)) * MC;
        if (r0 + MR - 1 >= c0) tiles::syrk_micro<double, TB, MR, MC>(P, P, Dn, r0, c0);
      }
      __syncwarp();
      tiles::diag_step<double, TB>(Dn, flag, tiles::NoOut{});
    } else {
      const int q0 = next ? 1 : 0;
      const int na = (npairs - q0) * PM;                  // trailing tile pairs of L_bb
      const int xm = (TB / MR) * (ncy / MC), nb = m * xm;  // Y's later block rows
      const int nsc = (J + 1) * (J + 2) / 2 * PM;          // S tiles (I2 >= J2, both <= J)
      const tiles::LaWorkers wk(NT, (na + nb + nsc) * TB * MR * MC / 32);
      const int t0 = next ? wk.id : tid, nth = next ? wk.n : NT;
      for (int it = t0 >= 0 ? t0 : na + nb + nsc; it < na + nb + nsc; it += nth) {
        if (it < na) {
          const int q = q0 + it / PM, u = it % PM;
          int kp = 0, rem = q;
          while (rem >= m - kp) { rem -= m - kp; ++kp; }
          const int K2 = J + 1 + kp, I = K2 + rem;
          tiles::syrk_micro<double, TB, MR, MC>(tp(I, J), tp(K2, J), tp(I, K2), (u / (TB / MC)) * MR,
                                                (u % (TB / MC)) * MC);
        } else if (it < na + nb) {
          const int it2 = it - na, ti = it2 / xm, u = it2 % xm;
          tiles::gemm_x_micro<double, TB, MR, MC>(tp(J + 1 + ti, J), YJ, Y + (J + 1 + ti) * TB * NB, NB,
                                                  (u / (ncy / MC)) * MR, (u % (ncy / MC)) * MC);
        } else {
          const int it3 = it - na - nb, q = it3 / PM, u = it3 % PM;
          int I2 = 0;
          while ((I2 + 1) * (I2 + 2) / 2 <= q) ++I2;
          const int J2 = q - I2 * (I2 + 1) / 2;
          const int a0 = (u / (TB / MC)) * MR, b0 = (u % (TB / MC)) * MC;
          if (I2 == J2 && a0 + MR - 1 < b0) continue;
          double acc[MR][MC];
#pragma unroll
          for (int i = 0; i < MR; ++i)
#pragma unroll
            for (int j = 0; j < MC; ++j) acc[i][j] = 0.0;
#pragma unroll 4
          for (int k = 0; k < TB; ++k) {
            double x[MR], y[MC];
#pragma unroll
            for (int i = 0; i < MR; ++i) x[i] = YJ[k * NB + I2 * TB + a0 + i];
#pragma unroll
            for (int j = 0; j < MC; ++j) y[j] = YJ[k * NB + J2 * TB + b0 + j];
#pragma unroll
            for (int i = 0; i < MR; ++i)
#pragma unroll
              for (int j = 0; j < MC; ++j) acc[i][j] = fma(x[i], y[j], acc[i][j]);
          }
          double* St = Sg + tiles::tcol(I2, J2, T) * TT;
#pragma unroll
          for (int i = 0; i < MR; ++i)
#pragma unroll
            for (int j = 0; j < MC; ++j) St[(a0 + i) + (b0 + j) * TB] += acc[i][j];
        }
      }
    }
    __syncthreads();
  }
  return true;
}

template <int K, int MODE>
__device__ void element_tail_tiled(const ElemArgs& args, const int64_t e, double* A, double* f, double* R,
                                   double* flag, const double* wf) {
  using S = EK<K>;
  constexpr int NI = S::NI, NB = S::NB, NFN = S::NFN, NT = S::NT, TB = S::TB, TI = S::TI, TBB = S::TBB;
  constexpr int T = TI + TBB, TT = TB * TB, MR = S::MR, MC = S::MC;   // small micro-tiles: more items to spread
  const int tid = threadIdx.x;
  double* R1 = R;                                   // L_ii tiles (packed over TI), then A_bb tiles
  double* R2 = R + S::R1;                           // L_bi tiles [I - TI][J], then Y
  auto tp = [&](int I, int J) -> double* {
    return I < TI ? R1 + tiles::tcol(I, J, TI) * TT : R2 + ((I - TI) * TI + J) * TT;
  };
  // ---- 1. load the interior tile columns, eliminate them. Consecutive threads read
  // consecutive columns of one row (contiguous in packed A); four loads in flight per thread.
  constexpr int NLD = S::R1 + S::R2, LB = 4;
  for (int t0 = tid; t0 < NLD; t0 += LB * NT) {
    double v[LB];
    int dst[LB];
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int t = t0 + u * NT;
      dst[u] = -1;
      v[u] = 0.0;
      if (t < NLD) {
        int I, J;
        const int w = t % TT;
        if (t < S::R1) {
          int rem = t / TT;
          J = 0;
          while (rem >= TI - J) { rem -= TI - J; ++J; }
          I = J + rem;
        } else {
          const int tile = (t - S::R1) / TT;
          I = TI + tile / TI;
          J = tile % TI;
        }
        const int r = w / TB, c = w % TB, i = I * TB + r, j = J * TB + c;
        dst[u] = t - w + r + c * TB;
        if (i >= j) v[u] = A[tri(i, j)];
      }
    }
#pragma unroll
    for (int u = 0; u < LB; ++u)
      if (dst[u] >= 0) R[dst[u]] = v[u];
  }
  __syncthreads();
  if (!tiles::tile_chol_la<double, TB, MR, MC, NT>(tp, T, TI, TI, flag, [](int) { return tiles::NoOut{}; })) {
    if (tid == 0) set_error(args.status, args.err_elem, HYB_ERR_NOT_SPD, e);
    return;
  }
  // ---- 2. forward substitution of the load; the factor tiles to the slot, the diagonal ones
  // as the inverses of their triangles (lower, what the recovery's blocked back substitution
  // applies)
  tiles::tile_fwd_vec<double, TB, NT>(R1, TI, f);
  for (int ib = tid; ib < NB; ib += NT) {
    const int I = ib / TB, r = ib % TB;
    double s = 0.0;
    for (int J = 0; J < TI; ++J) {
      const double* L = R2 + (I * TI + J) * TT;
#pragma unroll
      for (int c = 0; c < TB; ++c) s = fma(L[r + c * TB], f[J * TB + c], s);
    }
    f[NI + ib] -= s;
  }
  for (int t = tid; t < S::R1 + S::R2; t += NT) {
    int I, J;
    const int w = t % TT;
    if (t < S::R1) {
      int rem = t / TT;
      J = 0;
      while (rem >= TI - J) { rem -= TI - J; ++J; }
      I = J + rem;
      if (I == J && w % TB < w / TB) continue;     // strict upper part of an inverted diagonal tile
    } else {
      const int tile = (t - S::R1) / TT;
      I = TI + tile / TI;
      J = tile % TI;
    }
    A[tri(I * TB + w % TB, J * TB + w / TB)] = R[t];
  }
  __syncthreads();
  // ---- 3. the face block and its Schur complement A_bb - L_bi L_bi^T (packed tiles in R1)
  constexpr int NBB = TBB * (TBB + 1) / 2 * TT;
  for (int t0 = tid; t0 < NBB; t0 += LB * NT) {
    double v[LB];
    int dst[LB];
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int t = t0 + u * NT;
      dst[u] = -1;
      v[u] = 0.0;
      if (t < NBB) {
        int rem = t / TT, J = 0;
        while (rem >= TBB - J) { rem -= TBB - J; ++J; }
        const int I = J + rem, w = t % TT;
        const int r = w / TB, c = w % TB, i = NI + I * TB + r, j = NI + J * TB + c;
        dst[u] = t - w + r + c * TB;
        if (i >= j) v[u] = A[tri(i, j)];
      }
    }
#pragma unroll
    for (int u = 0; u < LB; ++u)
      if (dst[u] >= 0) R1[dst[u]] = v[u];
  }
  __syncthreads();
  {
    constexpr int PM = (TB / MR) * (TB / MC);
    for (int it = tid; it < TBB * (TBB + 1) / 2 * PM; it += NT) {
      const int tile = it / PM, u = it % PM;
      int rem = tile, J2 = 0;
      while (rem >= TBB - J2) { rem -= TBB - J2; ++J2; }
      const int I2 = J2 + rem;
      const int r0 = (u / (TB / MC)) * MR, c0 = (u % (TB / MC)) * MC;
      double acc[MR][MC];
#pragma unroll
      for (int a = 0; a < MR; ++a)
#pragma unroll
        for (int b = 0; b < MC; ++b) acc[a][b] = 0.0;
      for (int J = 0; J < TI; ++J) {
        const double* LA = R2 + (I2 * TI + J) * TT;
        const double* LB = R2 + (J2 * TI + J) * TT;
#pragma unroll 4
        for (int k = 0; k < TB; ++k) {
          double x[MR], y[MC];
#pragma unroll
          for (int a = 0; a < MR; ++a) x[a] = LA[r0 + a + k * TB];
#pragma unroll
          for (int b = 0; b < MC; ++b) y[b] = LB[c0 + b + k * TB];
#pragma unroll
          for (int a = 0; a < MR; ++a)
#pragma unroll
            for (int b = 0; b < MC; ++b) acc[a][b] = fma(x[a], y[b], acc[a][b]);
        }
      }
      double* C = R1 + tile * TT;
#pragma unroll
      for (int a = 0; a < MR; ++a)
#pragma unroll
        for (int b = 0; b < MC; ++b) C[(r0 + a) + (c0 + b) * TB] -= acc[a][b];
    }
  }
  __syncthreads();
  const int32_t* ef = args.elem_face + e * 6;
  const int64_t* boff = args.blockoff + e * 36;
  __shared__ int64_t s_row0[6];
  __shared__ int s_rlen[6];
  if (tid < 6) {
    const int64_t r0 = ef[tid] >= 0 ? args.row_ptr[(int64_t)ef[tid] * NFN] : 0;
    s_row0[tid] = r0;
    s_rlen[tid] = ef[tid] >= 0 ? (int)(args.row_ptr[(int64_t)ef[tid] * NFN + 1] - r0) : 0;
  }
  __shared__ double s_ww[2 * NFN * NFN];             // +-w_m1 w_m2 (sign of the face pair)
  for (int t = tid; t < 2 * NFN * NFN; t += NT) {
    const int m1 = (t / NFN) % NFN, m2 = t % NFN;
    s_ww[t] = (t < NFN * NFN ? 1.0 : -1.0) * wf[m1] * wf[m2];
  }
  __syncthreads();
  auto put = [&](int ib, int jb, double v, bool weighted) {
    const int a = ib / NFN, m1 = ib % NFN, b = jb / NFN, m2 = jb % NFN;
    if (ef[a] < 0 || ef[b] < 0) return;
    if (weighted) v *= s_ww[((a ^ b) & 1) * NFN * NFN + m1 * NFN + m2];
    const int64_t pos = boff[a * 6 + b] + m1 * (int64_t)s_rlen[a] + m2;
    if (a == b && args.colour == 1) args.val[pos] += v;
    else args.val[pos] = v;
  };
  if (MODE == MODE_SC) {
    // ---- 4a. static condensation: the Schur complement and rhs_b = f_b - L_bi z_i
    double* zs = args.zstore + e * (int64_t)S::N;
    for (int i = tid; i < S::N; i += NT) zs[i] = f[i];
    for (int t = tid; t < NB * NB; t += NT) {
      const int ib = t / NB, jb = t % NB;
      const int gi = ib >= jb ? ib : jb, gj = ib >= jb ? jb : ib;
      put(ib, jb, R1[tiles::tcol(gi / TB, gj / TB, TBB) * TT + (gi % TB) + (gj % TB) * TB], false);
    }
    for (int ib = tid; ib < NB; ib += NT) {
      const int a = ib / NFN, m1 = ib % NFN;
      if (ef[a] < 0) continue;
      const int64_t gi = (int64_t)ef[a] * NFN + m1;
      if (args.colour == 1) args.rhs[gi] += f[NI + ib];
      else args.rhs[gi] = f[NI + ib];
    }
    return;
  }
  // ---- 4b. hybridization: L_bb, Y = L_bb^{-1} (in R2) and S = Y^T Y (tiles after the
  // face block's in R1, or past R2 where R1 holds only the face block) in one pass; x0_b,
  // g_T, S_T scattered, P = S into the store
  double* Y = R2;                                    // [NB][NB], row-major
  double* Sg = S::RX > 0 ? R + S::R1 + S::R2 : R1 + TBB * (TBB + 1) / 2 * TT;
  static_assert(2 * TBB * (TBB + 1) / 2 * TT <= S::R1 + S::RX && NB * NB <= S::R2, "face block buffers");
  if (!face_block_hyb<TB, NT, MR, MC>(R1, Y, Sg, flag)) {
    if (tid == 0) set_error(args.status, args.err_elem, HYB_ERR_NOT_SPD, e);
    return;
  }
  tiles::tile_fwd_vec<double, TB, NT>(R1, TBB, f + NI);
  double* zs = args.zstore + e * (int64_t)S::N;
  for (int i = tid; i < NI; i += NT) zs[i] = f[i];
  for (int ib = tid; ib < NB; ib += NT) {           // x0_b = Y^T z_b (stored), g_T = D x0_b
    const int a = ib / NFN, m1 = ib % NFN;
    double acc = 0.0;
    for (int m = ib; m < NB; ++m) acc = fma(Y[m * NB + ib], f[NI + m], acc);
    zs[NI + ib] = acc;
    if (ef[a] < 0) continue;
    const double v = ((a & 1) ? 1.0 : -1.0) * wf[m1] * acc;
    const int64_t gi = (int64_t)ef[a] * NFN + m1;
    if (args.colour == 1) args.rhs[gi] += v;
    else args.rhs[gi] = v;
  }
  for (int t = tid; t < NB * NB; t += NT) {          // S_T = D S D, both triangles from the lower tiles
    const int ib = t / NB, jb = t % NB;
    const int gi = ib >= jb ? ib : jb, gj = ib >= jb ? jb : ib;
    put(ib, jb, Sg[tiles::tcol(gi / TB, gj / TB, TBB) * TT + (gi % TB) + (gj % TB) * TB], true);
  }
  double* Pst = A + S::TRI;                          // P = Y^T Y for the recovery, full square
  for (int t = tid; t < NB * NB; t += NT) {
    const int ib = t / NB, jb = t % NB;
    const int gi = ib >= jb ? ib : jb, gj = ib >= jb ? jb : ib;
    __stcs(Pst + t, Sg[tiles::tcol(gi / TB, gj / TB, TBB) * TT + (gi % TB) + (gj % TB) * TB]);
  }
}

template <int K, int MODE>
__device__ __forceinline__ void element_body(const ElemArgs& args, const int64_t e, double* smem) {
  using S = EK<K>;
  constexpr int P = S::P, p = S::p, Q = S::Q, NQ = S::NQ, NFN = S::NFN, NI = S::NI, NB = S::NB, N = S::N;
  constexpr int NT = S::NT;
  const int tid = threadIdx.x;
  const int64_t es = args.slot ? args.slot[e] : e;       // index into the FP64 factor store
  const int ex = (int)(e % args.nx), ey = (int)((e / args.nx) % args.ny), ez = (int)(e / ((int64_t)args.nx * args.ny));

  // ---- shared memory carve-up
  double* sp = smem;
  double* A = S::A_SMEM ? sp : args.Lstore + es * fp64_store_doubles(K);
  if (S::A_SMEM) sp += S::TRI;
  double* f = sp; sp += N;
  double* colbuf = sp; sp += N;
  double* invd = sp; sp += N;
  double* X8 = sp; sp += 24;
  double* Mc = sp; sp += 24;                // monomial coefficients of the trilinear map
  double* Vc = sp; sp += P * Q;
  double* Dc = sp; sp += P * Q;
  double* Vo = sp; sp += p * Q;
  double* VcVc = sp; sp += P * P * Q;
  double* DcDc = sp; sp += P * P * Q;
  double* VcVo = sp; sp += P * p * Q;
  double* DcVo = sp; sp += P * p * Q;
  double* VoVo = sp; sp += p * p * Q;
  double* qx = sp; sp += Q;
  double* qw = sp; sp += Q;
  double* wf = sp; sp += NFN;
  double* flag = sp; sp += 4;
  double* U = sp;                           // union region
  double* T1 = U;
  double* T2 = T1 + S::T1SZ;
  double* Gu = T2 + S::T2SZ;                // [6][NQ] unit-coefficient mass weights
  double* Ga = Gu + 6 * NQ;                 // [6][NQ] alpha-scaled
  double* Gd = Ga + 6 * NQ;                 // [NQ]    beta-scaled divergence weights
  double* LB0 = Gd + NQ;                    // load scratch
  double* LB1 = LB0 + S::LBUF;
  double* Uq = LB1 + S::LBUF;               // [3][NQ]
  double* Wq = Uq + 3 * NQ;                 // [3][NQ]
  double* Y = U;                            // after the factorisation: L_bb^{-1}, row-major packed
  double* YtY = U + S::TRIB;

  const RefTables& rt = c_ref[K];
  for (int i = tid; i < P * Q; i += NT) {
    Vc[i] = rt.Vc[i / Q][i % Q];
    Dc[i] = rt.Dc[i / Q][i % Q];
  }
  for (int i = tid; i < p * Q; i += NT) Vo[i] = rt.Vo[i / Q][i % Q];
  for (int i = tid; i < Q; i += NT) { qx[i] = rt.qx[i]; qw[i] = rt.qw[i]; }
  for (int i = tid; i < NFN; i += NT) wf[i] = rt.wf[i];
  if (tid < 24) {
    const int c = tid / 3, d = tid % 3;
    const int64_t v = (ex + (c & 1)) + (int64_t)(args.nx + 1) * ((ey + ((c >> 1) & 1)) + (int64_t)(args.ny + 1) * (ez + (c >> 2)));
    X8[tid] = args.vertices[3 * v + d];
  }
  __syncthreads();
  for (int i = tid; i < P * P * Q; i += NT) {
    const int q = i % Q, b = (i / Q) % P, a = i / (Q * P);
    VcVc[i] = Vc[a * Q + q] * Vc[b * Q + q];
    DcDc[i] = Dc[a * Q + q] * Dc[b * Q + q];
  }
  for (int i = tid; i < P * p * Q; i += NT) {
    const int q = i % Q, b = (i / Q) % p, a = i / (Q * p);
    VcVo[i] = Vc[a * Q + q] * Vo[b * Q + q];
    DcVo[i] = Dc[a * Q + q] * Vo[b * Q + q];
  }
  for (int i = tid; i < p * p * Q; i += NT) {
    const int q = i % Q, b = (i / Q) % p, a = i / (Q * p);
    VoVo[i] = Vo[a * Q + q] * Vo[b * Q + q];
  }
  // trilinear map x = m0 + m1 x0 + m2 x1 + m3 x2 + m4 x0 x1 + m5 x0 x2 + m6 x1 x2 + m7 x0 x1 x2
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

  // ---- 1. geometry: J columns from the monomial form, w J^T J / det J and w / det J
  const double alpha = args.alpha[e], beta = args.beta[e];
  for (int q = tid; q < NQ; q += NT) {
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
    if (!(det > 0.0)) set_error(args.status, args.err_elem, HYB_ERR_MESH, e);
    const double s = qw[q0] * qw[q1] * qw[q2] / det;
    double g[6];
    g[0] = fma(J[0][0], J[0][0], fma(J[1][0], J[1][0], J[2][0] * J[2][0]));
    g[1] = fma(J[0][1], J[0][1], fma(J[1][1], J[1][1], J[2][1] * J[2][1]));
    g[2] = fma(J[0][2], J[0][2], fma(J[1][2], J[1][2], J[2][2] * J[2][2]));
    g[3] = fma(J[0][1], J[0][0], fma(J[1][1], J[1][0], J[2][1] * J[2][0]));
    g[4] = fma(J[0][2], J[0][0], fma(J[1][2], J[1][0], J[2][2] * J[2][0]));
    g[5] = fma(J[0][2], J[0][1], fma(J[1][2], J[1][1], J[2][2] * J[2][1]));
    const double as = alpha * s;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      Gu[t * NQ + q] = s * g[t];
      Ga[t * NQ + q] = as * g[t];
    }
    Gd[q] = beta * s;
  }
  __syncthreads();

  // ---- 2. A_T by sum factorisation (6 blocks, c >= cp)
  const Tabs tb{Vc, Dc, Vo, VcVc, DcDc, VcVo, DcVo, VoVo};
  assemble_block<K>(0, 0, tb, Ga, Gd, T1, T2, A);
  assemble_block<K>(1, 1, tb, Ga, Gd, T1, T2, A);
  assemble_block<K>(2, 2, tb, Ga, Gd, T1, T2, A);
  assemble_block<K>(1, 0, tb, Ga, Gd, T1, T2, A);
  assemble_block<K>(2, 0, tb, Ga, Gd, T1, T2, A);
  assemble_block<K>(2, 1, tb, Ga, Gd, T1, T2, A);

  // ---- 3. load f = M c
  load_vector<K>(args.load + e * (int64_t)N, tb, Gu, LB0, LB1, Uq, Wq, f);

  // ---- 4. essential dofs on boundary faces: f -= A_{:,e} u_e, then rows / columns -> identity
  const int32_t* ef = args.elem_face + e * 6;
  int bmask = 0;
#pragma unroll
  for (int a = 0; a < 6; ++a) bmask |= (ef[a] < 0 && !args.natural) << a;
  if (bmask) {
    const double* ue = args.ess ? args.ess + e * (int64_t)N : nullptr;
    if (ue) {
      for (int i = tid; i < N; i += NT) {
        const bool ie = i >= NI && ((bmask >> ((i - NI) / NFN)) & 1);
        if (ie) continue;
        double acc = f[i];
        for (int a = 0; a < 6; ++a) {
          if (!((bmask >> a) & 1)) continue;
          for (int m = 0; m < NFN; ++m) {
            const int j = NI + a * NFN + m;
            acc = fma(-A[i >= j ? tri(i, j) : tri(j, i)], ue[j], acc);
          }
        }
        colbuf[i] = acc;
      }
      __syncthreads();
      for (int i = tid; i < N; i += NT) {
        const bool ie = i >= NI && ((bmask >> ((i - NI) / NFN)) & 1);
        f[i] = ie ? ue[i] : colbuf[i];
      }
    } else {
      for (int i = tid; i < NB; i += NT)
        if ((bmask >> (i / NFN)) & 1) f[NI + i] = 0.0;
    }
    __syncthreads();
    for (int a = 0; a < 6; ++a) {
      if (!((bmask >> a) & 1)) continue;
      for (int t = tid; t < NFN * N; t += NT) {
        const int m = t / N, j = t % N;
        const int i = NI + a * NFN + m;
        A[i >= j ? tri(i, j) : tri(j, i)] = (i == j) ? 1.0 : 0.0;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  if constexpr (S::TILED_PATH) {
    element_tail_tiled<K, MODE>(args, e, A, f, U, flag, wf);
    return;
  }

  // ---- 5. Cholesky (right-looking, packed lower) fused with z = L^{-1} f. Every trailing
  // update is spread over all threads (entry (i, l) of the trailing triangle, then f), and the
  // thread that updates the next diagonal entry prepares the next pivot.
  const int jend = MODE == MODE_SC ? NI : N;
  if (tid == 0) {
    const double d = jend > 0 ? A[0] : 1.0;
    const double r = rsqrt_newton(d);
    flag[0] = d;
    flag[1] = d * r;
    flag[2] = r;
  }
  __syncthreads();
  for (int j = 0; j < jend; ++j) {
    const double d = flag[0];
    if (!(d > 0.0) || !(d < INFINITY)) {
      if (tid == 0) set_error(args.status, args.err_elem, HYB_ERR_NOT_SPD, e);
      return;                               // uniform: every thread read the same pivot
    }
    const double inv = flag[2];
    for (int i = j + 1 + tid; i < N; i += NT) {
      const double v = A[tri(i, j)] * inv;
      A[tri(i, j)] = v;
      colbuf[i] = v;
    }
    if (tid == 0) {
      A[tri(j, j)] = flag[1];
      invd[j] = inv;
      f[j] = f[j] * inv;                    // z_j
    }
    __syncthreads();
    const double zj = f[j];
    const int m = N - 1 - j;
    const int T = m * (m + 1) / 2;
    for (int t = tid; t < T + m; t += NT) {
      if (t < T) {
        const int ii = tri_row(t), ll = t - ii * (ii + 1) / 2;
        const int i = j + 1 + ii, l = j + 1 + ll;
        const double v = fma(-colbuf[i], colbuf[l], A[tri(i, l)]);
        A[tri(i, l)] = v;
        if (t == 0 && j + 1 < jend) {        // next pivot, from its final value
          const double r = rsqrt_newton(v);
          flag[0] = v;
          flag[1] = v * r;
          flag[2] = r;
        }
      } else {
        const int i = j + 1 + (t - T);
        f[i] = fma(-colbuf[i], zj, f[i]);
      }
    }
    __syncthreads();
  }

  // ---- store z (hybridization: z_i here, the face part x0_b = Y^T z_b below)
  double* zs = args.zstore + e * (int64_t)N;
  for (int i = tid; i < (MODE == MODE_HYB ? NI : N); i += NT) zs[i] = f[i];

  // C_T = [0 D]: D_i = sign(face) * face weight on interior faces, 0 on boundary faces
  const int32_t* bo_face = ef;
  const int64_t* boff = args.blockoff + e * 36;

  if (MODE == MODE_HYB) {
    // ---- 6a. Y = L_bb^{-1} by right-looking forward elimination (row-major packed)
    for (int t = tid; t < S::TRIB; t += NT) Y[t] = 0.0;
    __syncthreads();
    for (int m = 0; m < NB; ++m) {
      const double im = invd[NI + m];
      for (int jj = tid; jj <= m; jj += NT) Y[tri(m, jj)] = (jj == m) ? im : Y[tri(m, jj)] * im;
      __syncthreads();
      const int w = m + 1, cnt = (NB - 1 - m) * w;
      for (int t = tid; t < cnt; t += NT) {
        const int i = m + 1 + t / w, jj = t % w;
        Y[tri(i, jj)] = fma(-A[tri(NI + i, NI + m)], Y[tri(m, jj)], Y[tri(i, jj)]);
      }
      __syncthreads();
    }
    // ---- 6b. Y^T Y (lower): (Y^T Y)_{i jj} = sum_{m >= i} Y_{m i} Y_{m jj}
    for (int t = tid; t < S::TRIB; t += NT) {
      const int i = tri_row(t), jj = t - i * (i + 1) / 2;
      double acc = 0.0;
      for (int m = i; m < NB; ++m) acc = fma(Y[tri(m, i)], Y[tri(m, jj)], acc);
      YtY[t] = acc;
    }
    __syncthreads();
    // ---- 7. scatter S_T = D Y^T Y D and g_T = D Y^T z_b
    for (int t = tid; t < NB * NB; t += NT) {
      const int ib = t / NB, jb = t % NB;
      const int a = ib / NFN, m1 = ib % NFN, b = jb / NFN, m2 = jb % NFN;
      if (bo_face[a] < 0 || bo_face[b] < 0) continue;
      const double dd = (((a ^ b) & 1) ? -1.0 : 1.0) * wf[m1] * wf[m2];
      const double v = dd * YtY[ib >= jb ? tri(ib, jb) : tri(jb, ib)];
      const int64_t r0 = args.row_ptr[(int64_t)bo_face[a] * NFN];
      const int64_t rl = args.row_ptr[(int64_t)bo_face[a] * NFN + 1] - r0;
      const int64_t pos = boff[a * 6 + b] + m1 * rl + m2;
      if (a == b && args.colour == 1) args.val[pos] += v;
      else args.val[pos] = v;
    }
    for (int ib = tid; ib < NB; ib += NT) {
      const int a = ib / NFN, m1 = ib % NFN;
      double acc = 0.0;
      for (int m = ib; m < NB; ++m) acc = fma(Y[tri(m, ib)], f[NI + m], acc);
      zs[NI + ib] = acc;
      if (bo_face[a] < 0) continue;
      const double v = ((a & 1) ? 1.0 : -1.0) * wf[m1] * acc;
      const int64_t gi = (int64_t)bo_face[a] * NFN + m1;
      if (args.colour == 1) args.rhs[gi] += v;
      else args.rhs[gi] = v;
    }
    __syncthreads();
    // ---- store the factor (the recovery reads its interior rows) and P = Y^T Y, full square
    double* Ls = args.Lstore + es * fp64_store_doubles(K);
    if (S::A_SMEM)
      for (int t = tid; t < S::TRI; t += NT) __stcs(Ls + t, A[t]);
    for (int t = tid; t < NB * NB; t += NT) {
      const int i = t / NB, jj = t % NB;
      __stcs(Ls + S::TRI + t, YtY[i >= jj ? tri(i, jj) : tri(jj, i)]);
    }
  } else {
    // ---- static condensation: scatter S_hat (trailing block) and rhs_b = f_b - L_bi z_i
    for (int t = tid; t < NB * NB; t += NT) {
      const int ib = t / NB, jb = t % NB;
      const int a = ib / NFN, m1 = ib % NFN, b = jb / NFN, m2 = jb % NFN;
      if (bo_face[a] < 0 || bo_face[b] < 0) continue;
      const double v = A[ib >= jb ? tri(NI + ib, NI + jb) : tri(NI + jb, NI + ib)];
      const int64_t r0 = args.row_ptr[(int64_t)bo_face[a] * NFN];
      const int64_t rl = args.row_ptr[(int64_t)bo_face[a] * NFN + 1] - r0;
      const int64_t pos = boff[a * 6 + b] + m1 * rl + m2;
      if (a == b && args.colour == 1) args.val[pos] += v;
      else args.val[pos] = v;
    }
    for (int ib = tid; ib < NB; ib += NT) {
      const int a = ib / NFN, m1 = ib % NFN;
      if (bo_face[a] < 0) continue;
      const int64_t gi = (int64_t)bo_face[a] * NFN + m1;
      if (args.colour == 1) args.rhs[gi] += f[NI + ib];
      else args.rhs[gi] = f[NI + ib];
    }
    if (S::A_SMEM) {
      double* Ls = args.Lstore + es * fp64_store_doubles(K);
      for (int t = tid; t < S::TRI; t += NT) Ls[t] = A[t];
    }
  }
}

template <int K, int MODE>
__global__ void __launch_bounds__(EK<K>::NT) element_kernel(ElemArgs args) {
  extern __shared__ double smem[];
  const int64_t li = blockIdx.x;
  if (li >= args.n_list) return;
  element_body<K, MODE>(args, args.elem_list[li], smem);
}

// Many problems in one launch: work item (problem, element) with per-problem arguments. A CTA
// takes items blockIdx.x, blockIdx.x + gridDim.x, ...: one per CTA when the grid covers them,
// several (persistent CTAs) when the batch's autotuner chose a smaller grid.
template <int K, int MODE>
__global__ void __launch_bounds__(EK<K>::NT) element_kernel_batch(const ElemArgs* probs, const int2* items,
                                                                  int64_t n_items, int colour) {
  extern __shared__ double smem[];
  for (int64_t li = blockIdx.x; li < n_items; li += gridDim.x) {
    const int2 it = items[li];
    ElemArgs a = probs[it.x];
    a.colour = colour;
    element_body<K, MODE>(a, it.y, smem);
    __syncthreads();                         // the next item overwrites this one's shared memory
  }
}

// det J > 0 at the 8 corners and every Gauss point of every element.
template <int K>
__global__ void check_geometry_kernel(ElemArgs args) {
  constexpr int Q = K + 2, NQ = Q * Q * Q;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= args.n_elem) return;
  const int ex = (int)(e % args.nx), ey = (int)((e / args.nx) % args.ny), ez = (int)(e / ((int64_t)args.nx * args.ny));
  double X[24];
  for (int c = 0; c < 8; ++c) {
    const int64_t v = (ex + (c & 1)) + (int64_t)(args.nx + 1) * ((ey + ((c >> 1) & 1)) + (int64_t)(args.ny + 1) * (ez + (c >> 2)));
    for (int d = 0; d < 3; ++d) X[3 * c + d] = args.vertices[3 * v + d];
  }
  const RefTables& rt = c_ref[K];
  bool ok = true;
  for (int q = 0; q < NQ + 8; ++q) {
    double x0, x1, x2;
    if (q < NQ) {
      x0 = rt.qx[q % Q]; x1 = rt.qx[(q / Q) % Q]; x2 = rt.qx[q / (Q * Q)];
    } else {
      const int c = q - NQ;
      x0 = c & 1; x1 = (c >> 1) & 1; x2 = c >> 2;
    }
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int c = 0; c < 8; ++c) {
      const int s0 = c & 1, s1 = (c >> 1) & 1, s2 = c >> 2;
      const double f0 = s0 ? x0 : 1.0 - x0, f1 = s1 ? x1 : 1.0 - x1, f2 = s2 ? x2 : 1.0 - x2;
      const double d0 = (s0 ? 1.0 : -1.0) * f1 * f2, d1 = f0 * (s1 ? 1.0 : -1.0) * f2, d2 = f0 * f1 * (s2 ? 1.0 : -1.0);
      for (int r = 0; r < 3; ++r) {
        J[r][0] += X[3 * c + r] * d0;
        J[r][1] += X[3 * c + r] * d1;
        J[r][2] += X[3 * c + r] * d2;
      }
    }
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    ok = ok && (det > 0.0);
  }
  if (!ok) set_error(args.status, args.err_elem, HYB_ERR_MESH, e);
}

template <int K>
cudaError_t launch_element_k(int mode, const ElemArgs& a, cudaStream_t s, Prof* prof) {
  using S = EK<K>;
  if (a.n_list == 0) return cudaSuccess;
  const size_t smem = S::SMEM_BYTES;
  cudaError_t err;
  if (mode == MODE_HYB) {
    err = cudaFuncSetAttribute(element_kernel<K, MODE_HYB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int tok = prof_begin(prof, HYB_K_ELEMENT, s);
    element_kernel<K, MODE_HYB><<<(unsigned)a.n_list, S::NT, smem, s>>>(a);
    prof_end(prof, tok, s);
  } else {
    err = cudaFuncSetAttribute(element_kernel<K, MODE_SC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int tok = prof_begin(prof, HYB_K_ELEMENT, s);
    element_kernel<K, MODE_SC><<<(unsigned)a.n_list, S::NT, smem, s>>>(a);
    prof_end(prof, tok, s);
  }
  return cudaGetLastError();
}

}  // namespace

template <int K>
cudaError_t launch_element_batch_k(int mode, const ElemArgs* probs, const int2* items, int64_t n, int colour,
                                   int grid, cudaStream_t s, Prof* prof) {
  using S = EK<K>;
  if (n == 0) return cudaSuccess;
  const unsigned g = (unsigned)(grid > 0 && grid < n ? grid : n);
  const size_t smem = S::SMEM_BYTES;
  cudaError_t err;
  const int tok = prof_begin(prof, HYB_K_ELEMENT, s);
  if (mode == MODE_HYB) {
    err = cudaFuncSetAttribute(element_kernel_batch<K, MODE_HYB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    element_kernel_batch<K, MODE_HYB><<<g, S::NT, smem, s>>>(probs, items, n, colour);
  } else {
    err = cudaFuncSetAttribute(element_kernel_batch<K, MODE_SC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    element_kernel_batch<K, MODE_SC><<<g, S::NT, smem, s>>>(probs, items, n, colour);
  }
  prof_end(prof, tok, s);
  return cudaGetLastError();
}

cudaError_t launch_element_batch(int k, int mode, const ElemArgs* probs, const int2* items, int64_t n, int colour,
                                 int grid, cudaStream_t s, Prof* prof) {
  switch (k) {
    case 0: return launch_element_batch_k<0>(mode, probs, items, n, colour, grid, s, prof);
    case 1: return launch_element_batch_k<1>(mode, probs, items, n, colour, grid, s, prof);
    case 2: return launch_element_batch_k<2>(mode, probs, items, n, colour, grid, s, prof);
    case 3: return launch_element_batch_k<3>(mode, probs, items, n, colour, grid, s, prof);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_element(int k, int mode, const ElemArgs& a, cudaStream_t s, Prof* prof) {
  switch (k) {
    case 0: return launch_element_k<0>(mode, a, s, prof);
    case 1: return launch_element_k<1>(mode, a, s, prof);
    case 2: return launch_element_k<2>(mode, a, s, prof);
    case 3: return launch_element_k<3>(mode, a, s, prof);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_check_geometry(int k, const ElemArgs& a, cudaStream_t s, Prof* prof) {
  const int nt = 128;
  const unsigned nb = (unsigned)((a.n_elem + nt - 1) / nt);
  if (nb == 0) return cudaSuccess;
  const int tok = prof_begin(prof, HYB_K_SETUP, s);
  switch (k) {
    case 0: check_geometry_kernel<0><<<nb, nt, 0, s>>>(a); break;
    case 1: check_geometry_kernel<1><<<nb, nt, 0, s>>>(a); break;
    case 2: check_geometry_kernel<2><<<nb, nt, 0, s>>>(a); break;
    case 3: check_geometry_kernel<3><<<nb, nt, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  prof_end(prof, tok, s);
  return cudaGetLastError();
}

}  // namespace hyb

namespace hyb {
// CTAs of the batched element kernel of order k that fit on one SM at once (the autotuner's unit).
int element_batch_ctas_per_sm(int k) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (k) {
    case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, element_kernel_batch<0, MODE_HYB>, EK<0>::NT, EK<0>::SMEM_BYTES); break;
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, element_kernel_batch<1, MODE_HYB>, EK<1>::NT, EK<1>::SMEM_BYTES); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, element_kernel_batch<2, MODE_HYB>, EK<2>::NT, EK<2>::SMEM_BYTES); break;
    case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, element_kernel_batch<3, MODE_HYB>, EK<3>::NT, EK<3>::SMEM_BYTES); break;
  }
  return e == cudaSuccess ? n : 0;
}
}  // namespace hyb
