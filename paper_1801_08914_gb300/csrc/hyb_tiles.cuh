// Blocked dense kernels on TB x TB tiles in shared memory, generic in the scalar type (float
// for the mixed-precision elimination, double for the FP64 one). Used inside element kernels:
// every function is called by all threads of the CTA unless it says one warp.
//
// Tile layout: a lower-triangular matrix of T x T tiles is stored as "packed tiles", column
// of tiles after column of tiles (tile (I, J), I >= J, at J T - J (J - 1) / 2 + I - J), each
// tile column-major inside. After a factorisation a diagonal tile holds the inverse of its
// triangle (what the panel step, the triangular solves and inverses use). tile_chol_la takes a
// tile-address functor instead, so that a factorisation can run over tiles split between
// several regions (the FP64 elimination keeps the interior and the interface rows apart).
#pragma once

#include <cuda_runtime.h>

#include "hyb_device.h"

namespace hyb {
namespace tiles {

__device__ __forceinline__ int tcol(int I, int J, int T) { return J * T - J * (J - 1) / 2 + (I - J); }

// tile address of packed tiles
template <typename F, int TB>
struct Packed {
  F* base;
  int T;
  __device__ __forceinline__ F* operator()(int I, int J) const { return base + tcol(I, J, T) * (TB * TB); }
};

// no write-out of the diagonal factor
struct NoOut {
  template <typename F>
  __device__ __forceinline__ void operator()(int, int, F) const {}
};

// ---- one warp: Cholesky of the lower triangle of a TB x TB column-major tile in place,
// then replace it by the inverse of the factor (strict upper part zero). Lane i holds row i
// of the factor and column i of its inverse in registers; the columns of the factor travel
// by shuffles, so there is no shared-memory round trip or index arithmetic inside the
// elimination. The inverse is formed right-looking in the same pass: once column k of L is
// known, x_k = x_k / L_kk is final in every lane's column and x_l -= L_lk x_k for l > k, with
// the L_lk the factor update has just fetched (the lane's own x_k needs no shuffle). No
// data-dependent exit: a bad pivot only sets a flag, so the loops unroll and every array stays
// in registers. out(i, l, L_il) receives the factor itself (l <= i); flag[0] = 1 on a bad
// pivot (non-positive or non-finite), in which case nothing is written.
template <typename F, int TB, typename Out>
__device__ __forceinline__ void diag_factor_invert(F* D, F* flag, const Out& out) {
  const int lane = threadIdx.x & 31;
  constexpr unsigned FULL = 0xffffffffu;
  F row[TB], x[TB];
#pragma unroll
  for (int l = 0; l < TB; ++l) {
    row[l] = (lane < TB && l <= lane) ? D[lane + l * TB] : F(0);
    x[l] = l == lane ? F(1) : F(0);
  }
  bool ok = true;
#pragma unroll
  for (int k = 0; k < TB; ++k) {
    const F d = __shfl_sync(FULL, row[k], k);             // pivot, after the previous updates
    ok = ok && d > F(0) && d < F(INFINITY);
    const F r = dev::rsqrt_newton(d);
    row[k] = lane == k ? d * r : row[k] * r;               // column k of L (rows > k, and the pivot)
    x[k] *= r;                                             // x_k of this lane's column, final
#pragma unroll
    for (int l = k + 1; l < TB; ++l) {
      const F lk = __shfl_sync(FULL, row[k], l);          // L_lk
      if (lane >= l) row[l] = fma(-row[k], lk, row[l]);    // row_i[l] -= L_ik L_lk, k < l <= i
      x[l] = fma(-lk, x[k], x[l]);
    }
  }
  if (!ok) {
    if (lane == 0) flag[0] = F(1);
    __syncwarp();
    return;
  }
  if (lane < TB) {
#pragma unroll
    for (int l = 0; l < TB; ++l)
      if (l <= lane) out(lane, l, row[l]);
#pragma unroll
    for (int i = 0; i < TB; ++i) D[i + lane * TB] = x[i];
  }
  __syncwarp();
}

// ---- one warp, TB at most 16: the same factorisation and inversion with two columns per
// instruction (an odd TB leaves the last column pair half empty). On this part an FP64 warp instruction holds its sub-partition's
// FP64 unit as long as its dependent successor waits, whatever the number of active lanes, so
// what counts is the number of instructions the warp issues; in FP32 the halved per-lane
// arrays keep the factor in registers inside large kernels. Lane (i, h) = (lane & 15,
// lane >> 4) keeps the columns l = 2 j + h of row i in c[j] and the rows 2 j + h of column i of
// L^{-1} in x[j] (lanes with i >= TB carry zeros). The inverse is formed right-looking in the
// same pass, with the L_lk the factor update has just fetched. FP64 pivots take their inverse
// square root from rsqrt_h3 (no FP64 conversions or branches) and are checked on their
// integer bits. About half the instructions of the one-row-per-lane form.
template <typename F, int TB, typename Out>
__device__ __forceinline__ void diag_factor_invert2(F* D, F* flag, const Out& out) {
  static_assert(TB <= 16, "two half-warps of at most 8 columns");
  constexpr int H = (TB + 1) / 2;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, i = lane & 15, h = lane >> 4;
  F c[H], x[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    const int l = 2 * j + h;
    c[j] = (i < TB && l <= i) ? D[i + l * TB] : F(0);
    x[j] = l == i ? F(1) : F(0);
  }
  bool ok = true;
#pragma unroll
  for (int k = 0; k < TB; ++k) {
    const int jk = k >> 1, hk = k & 1;
    const F d = __shfl_sync(FULL, c[jk], k + 16 * hk);             // pivot, after the updates
    F r;
    if constexpr (sizeof(F) == 8) {
      ok = ok && dev::positive_normal(d);
      r = dev::rsqrt_h3(d);
    } else {
      ok = ok && d > F(0) && d < F(INFINITY);
      r = dev::rsqrt_newton(d);
    }
    const F lik = __shfl_sync(FULL, c[jk], (i & 15) + 16 * hk) * r; // L_ik (L_kk in row k)
    if (h == hk) {
      c[jk] = lik;
      x[jk] *= r;                                                  // x_k of column i, final
    }
    const F xk = __shfl_sync(FULL, x[jk], (i & 15) + 16 * hk);
#pragma unroll
    for (int j = (k + 1) >> 1; j < H; ++j) {
      const int l = 2 * j + h;
      const F llk = __shfl_sync(FULL, lik, l);                     // L_lk, from row l
      if (l > k && l <= i) c[j] = fma(-lik, llk, c[j]);
      if (l > k) x[j] = fma(-llk, xk, x[j]);
    }
  }
  __syncwarp();
  if (!ok) {
    if (lane == 0) flag[0] = F(1);
    __syncwarp();
    return;
  }
  if (i < TB) {
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const int l = 2 * j + h;
      if (l <= i) out(i, l, c[j]);
      if (l < TB) D[l + i * TB] = x[j];
    }
  }
  __syncwarp();
}

template <typename F, int TB, typename Out>
__device__ __forceinline__ void diag_step(F* D, F* flag, const Out& out) {
  if constexpr (TB <= 16) diag_factor_invert2<F, TB>(D, flag, out);
  else diag_factor_invert<F, TB>(D, flag, out);
}

// Workers of a look-ahead update phase, while warp 0 factors the next diagonal tile. Warps w
// run on sub-partition w % 4. A small update leaves sub-partition 0 to warp 0 alone (its
// dependent chain would otherwise wait behind the other warps' FP64 instructions there); a
// large one uses every other warp. `work` = FP64 warp instructions of the update.
struct LaWorkers {
  int id, n;   // worker index (-1: not a worker) and worker count
  __device__ LaWorkers(int nthreads, int work) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (work > 3000) {
      id = warp == 0 ? -1 : (int)threadIdx.x - 32;
      n = nthreads - 32;
    } else {
      id = (warp & 3) == 0 ? -1 : (warp - (warp >> 2) - 1) * 32 + lane;
      n = (nthreads >> 5) / 4 * 3 * 32;
    }
  }
};


// ---- one thread: column cx of X_J <- Dinv_J X_J (X_J: TB rows, row-major with ld MX)
template <typename F, int TB>
__device__ __forceinline__ void scale_rows_item(const F* Dv, F* XJ, int MX, int cx) {
  F x[TB];
#pragma unroll
  for (int k = 0; k < TB; ++k) x[k] = XJ[k * MX + cx];
#pragma unroll
  for (int r = 0; r < TB; ++r) {
    F s = F(0);
#pragma unroll
    for (int k = 0; k <= r; ++k) s = fma(Dv[r + k * TB], x[k], s);
    XJ[r * MX + cx] = s;
  }
}

// ---- one thread: row r of a panel tile A_IJ <- A_IJ Dinv_J^T (Dinv lower triangular)
template <typename F, int TB>
__device__ __forceinline__ void panel_row_item(const F* Dv, F* A, int r) {
  F a[TB];
#pragma unroll
  for (int k = 0; k < TB; ++k) a[k] = A[r + k * TB];
#pragma unroll
  for (int c = 0; c < TB; ++c) {
    F s = F(0);
#pragma unroll
    for (int k = 0; k <= c; ++k) s = fma(a[k], Dv[c + k * TB], s);
    A[r + c * TB] = s;
  }
}

// ---- one thread: C (MR x MC block at r0, c0) -= A(rows r0..) * B(rows c0..)^T, K dim TB,
// A and B column-major TB x TB tiles; C column-major with leading dimension TB.
template <typename F, int TB, int MR, int MC>
__device__ __forceinline__ void syrk_micro(const F* A, const F* B, F* C, int r0, int c0) {
  F acc[MR][MC];
#pragma unroll
  for (int i = 0; i < MR; ++i)
#pragma unroll
    for (int j = 0; j < MC; ++j) acc[i][j] = F(0);
#pragma unroll 2
  for (int k = 0; k < TB; ++k) {
    F a[MR], b[MC];
#pragma unroll
    for (int i = 0; i < MR; ++i) a[i] = A[r0 + i + k * TB];
#pragma unroll
    for (int j = 0; j < MC; ++j) b[j] = B[c0 + j + k * TB];
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
      for (int j = 0; j < MC; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
#pragma unroll
  for (int i = 0; i < MR; ++i)
#pragma unroll
    for (int j = 0; j < MC; ++j) C[(r0 + i) + (c0 + j) * TB] -= acc[i][j];
}

// ---- one thread: XI (MR x MC block at r0, c0; row-major, ld MX) -= A(rows r0..) * XJ, K dim TB
template <typename F, int TB, int MR, int MC>
__device__ __forceinline__ void gemm_x_micro(const F* A, const F* XJ, F* XI, int MX, int r0, int c0) {
  F acc[MR][MC];
#pragma unroll
  for (int i = 0; i < MR; ++i)
#pragma unroll
    for (int j = 0; j < MC; ++j) acc[i][j] = F(0);
#pragma unroll 2
  for (int k = 0; k < TB; ++k) {
    F a[MR], b[MC];
#pragma unroll
    for (int i = 0; i < MR; ++i) a[i] = A[r0 + i + k * TB];
#pragma unroll
    for (int j = 0; j < MC; ++j) b[j] = XJ[k * MX + c0 + j];
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
      for (int j = 0; j < MC; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
#pragma unroll
  for (int i = 0; i < MR; ++i)
#pragma unroll
    for (int j = 0; j < MC; ++j) XI[(r0 + i) * MX + c0 + j] -= acc[i][j];
}

// ---- blocked right-looking Cholesky of the tile columns J < Jend of a T x T tile triangle
// (tiles addressed by tp), fused with X <- L^{-1} X (T TB rows, ld MX; X may be null). The
// rank-TB updates reach the tiles (I, K2) with K2 < Kend only: with Jend = Kend = T this is
// the whole factorisation; with Jend = Kend = TI < T it eliminates the first TI tile columns
// and leaves the trailing block untouched (its Schur update is the caller's). out(J) gives the
// write-out functor of diagonal tile J. Per tile column: the CTA scales the panel (one thread
// per row) and the rows of X (one thread per column); then, with a look-ahead of one tile
// column, warp 0 applies that column's update to the next diagonal tile and factors and
// inverts it while the other warps apply the rest of the update (and of X) with MR x MC
// register micro-tiles, so that the one-warp diagonal step overlaps the CTA-wide update
// instead of running alone between two barriers: two barriers per tile column. Returns false
// in every thread on a bad pivot.
template <typename F, int TB, int MR, int MC, int NT, typename TP, typename OutJ>
__device__ bool tile_chol_la(const TP& tp, int T, int Jend, int Kend, F* flag, const OutJ& out, F* X = nullptr,
                             int MX = 0) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int PM = (TB / MR) * (TB / MC);
  if (tid == 0) flag[0] = F(0);
  __syncthreads();
  if (warp == 0 && Jend > 0) diag_step<F, TB>(tp(0, 0), flag, out(0));
  __syncthreads();
  const int ncx = X ? MX : 0, xm = X ? (TB / MR) * (MX / MC) : 0;
  for (int J = 0; J < Jend; ++J) {
    if (flag[0] != F(0)) return false;
    const F* Dv = tp(J, J);
    const int nrows = (T - J - 1) * TB;
    for (int it = tid; it < nrows + ncx; it += NT) {   // A_IJ <- A_IJ Dinv^T; X_J <- Dinv X_J
      if (it < nrows) panel_row_item<F, TB>(Dv, tp(J + 1 + it / TB, J), it % TB);
      else scale_rows_item<F, TB>(Dv, X + J * TB * MX, MX, it - nrows);
    }
    __syncthreads();
    const int m = T - J - 1, mk = (Kend < T ? Kend : T) - J - 1;
    const bool next = J + 1 < Jend && mk > 0;
    const int npairs = mk * m - mk * (mk - 1) / 2;
    if (next && warp == 0) {
      // pair 0 of the column-by-column enumeration is the next diagonal tile (J+1, J+1): its
      // lower micro-tiles, then its factorisation
      F* Dn = tp(J + 1, J + 1);
      const F* P = tp(J + 1, J);
      for (int u = lane; u < PM; u += 32) {
        const int r0 = (u / (TB / MC)) * MR, c0 = (u % (TB / MC)) * MC;
        if (r0 + MR - 1 >= c0) syrk_micro<F, TB, MR, MC>(P, P, Dn, r0, c0);
      }
      __syncwarp();
      diag_step<F, TB>(Dn, flag, out(J + 1));
    } else {
      const int q0 = next ? 1 : 0;
      const int na = (npairs - q0) * PM, nx = m * xm, ntot = na + nx;
      // FP32: every warp but 0 (the sub-partition contention is an FP64 matter)
      const LaWorkers wk(NT, sizeof(F) == 8 ? ntot * TB * MR * MC / 32 : 1 << 30);
      const int t0 = next ? wk.id : tid, nth = next ? wk.n : NT;
      for (int it = t0 >= 0 ? t0 : ntot; it < ntot; it += nth) {
        if (it < na) {
          const int q = q0 + it / PM, u = it % PM;
          int kp = 0, rem = q;                     // column kp of the trailing part has m - kp tiles
          while (rem >= m - kp) { rem -= m - kp; ++kp; }
          const int K2 = J + 1 + kp, I = K2 + rem;
          syrk_micro<F, TB, MR, MC>(tp(I, J), tp(K2, J), tp(I, K2), (u / (TB / MC)) * MR, (u % (TB / MC)) * MC);
        } else {                                   // X_I -= L_IJ X_J, I > J
          const int it2 = it - na, I = J + 1 + it2 / xm, u = it2 % xm;
          gemm_x_micro<F, TB, MR, MC>(tp(I, J), X + J * TB * MX, X + I * TB * MX, MX, (u / (MX / MC)) * MR,
                                      (u % (MX / MC)) * MC);
        }
      }
    }
    __syncthreads();
  }
  return true;
}

// ---- X <- L^{-1} X for the tiles J0..T-1 of a factored packed tile triangle; X holds the
// rows of those tiles ((J - J0) TB + r), ld MX. LOWER: X is block lower triangular on entry
// (the identity, for L^{-1} itself), so that tile row J - J0 has no nonzero beyond column
// (J - J0 + 1) TB, at every step; the work on those zero columns is skipped.
template <typename F, int TB, int MR, int MC, int NT, bool LOWER = false>
__device__ void tile_fwd_mat(const F* Lt, int T, int J0, F* X, int MX) {
  constexpr int TT = TB * TB;
  const int tid = threadIdx.x;
  for (int J = J0; J < T; ++J) {
    const F* Dv = Lt + tcol(J, J, T) * TT;
    F* XJ = X + (J - J0) * TB * MX;
    const int ncol = LOWER ? (J - J0 + 1) * TB : MX;
    for (int cx = tid; cx < ncol; cx += NT) scale_rows_item<F, TB>(Dv, XJ, MX, cx);
    __syncthreads();
    const int m = T - J - 1, xm = (TB / MR) * (ncol / MC);
    for (int it = tid; it < m * xm; it += NT) {
      const int ti = it / xm, u = it % xm;
      const int I = J + 1 + ti;
      gemm_x_micro<F, TB, MR, MC>(Lt + tcol(I, J, T) * TT, XJ, X + (I - J0) * TB * MX, MX, (u / (ncol / MC)) * MR,
                                  (u % (ncol / MC)) * MC);
    }
    __syncthreads();
  }
}

// ---- X <- L^{-T} X (all T tiles), X row-major with ld MX (small systems).
template <typename F, int TB, int NT>
__device__ void tile_bwd_mat(const F* Lt, int T, F* X, int MX) {
  constexpr int TT = TB * TB;
  const int tid = threadIdx.x;
  for (int J = T - 1; J >= 0; --J) {
    const F* Dv = Lt + tcol(J, J, T) * TT;
    F* XJ = X + J * TB * MX;
    for (int cx = tid; cx < MX; cx += NT) {          // X_J <- Dinv^T X_J
      F x[TB];
#pragma unroll
      for (int k = 0; k < TB; ++k) x[k] = XJ[k * MX + cx];
#pragma unroll
      for (int c = 0; c < TB; ++c) {
        F s = F(0);
#pragma unroll
        for (int r = c; r < TB; ++r) s = fma(Dv[r + c * TB], x[r], s);
        XJ[c * MX + cx] = s;
      }
    }
    __syncthreads();
    for (int it = tid; it < J * TB * MX; it += NT) {   // X_K2 -= L_J,K2^T X_J
      const int row = it / MX, cx = it % MX;
      const int K2 = row / TB, c = row % TB;
      const F* L = Lt + tcol(J, K2, T) * TT;
      F s = F(0);
#pragma unroll
      for (int r = 0; r < TB; ++r) s = fma(L[r + c * TB], XJ[r * MX + cx], s);
      X[row * MX + cx] -= s;
    }
    __syncthreads();
  }
}

// ---- v <- L^{-1} v (one right-hand side, T TB entries)
template <typename F, int TB, int NT>
__device__ void tile_fwd_vec(const F* Lt, int T, F* v) {
  constexpr int TT = TB * TB;
  const int tid = threadIdx.x;
  for (int J = 0; J < T; ++J) {
    const F* Dv = Lt + tcol(J, J, T) * TT;
    F* vJ = v + J * TB;
    if (tid < 32) {
      F y = F(0);
      if (tid < TB) {
#pragma unroll
        for (int k = 0; k < TB; ++k)
          if (k <= tid) y = fma(Dv[tid + k * TB], vJ[k], y);
      }
      __syncwarp();
      if (tid < TB) vJ[tid] = y;
    }
    __syncthreads();
    for (int i = tid; i < (T - J - 1) * TB; i += NT) {
      const int I = J + 1 + i / TB, r = i % TB;
      const F* L = Lt + tcol(I, J, T) * TT;
      F s = F(0);
#pragma unroll
      for (int k = 0; k < TB; ++k) s = fma(L[r + k * TB], vJ[k], s);
      v[I * TB + r] -= s;
    }
    __syncthreads();
  }
}

// ---- v <- L^{-T} v
template <typename F, int TB, int NT>
__device__ void tile_bwd_vec(const F* Lt, int T, F* v) {
  constexpr int TT = TB * TB;
  const int tid = threadIdx.x;
  for (int J = T - 1; J >= 0; --J) {
    const F* Dv = Lt + tcol(J, J, T) * TT;
    F* vJ = v + J * TB;
    if (tid < 32) {
      F x = F(0);
      if (tid < TB) {
#pragma unroll
        for (int r = 0; r < TB; ++r)
          if (r >= tid) x = fma(Dv[r + tid * TB], vJ[r], x);
      }
      __syncwarp();
      if (tid < TB) vJ[tid] = x;
    }
    __syncthreads();
    for (int i = tid; i < J * TB; i += NT) {          // v_K2 -= L_J,K2^T x_J
      const int K2 = i / TB, c = i % TB;
      const F* L = Lt + tcol(J, K2, T) * TT;
      F s = F(0);
#pragma unroll
      for (int t = 0; t < TB; ++t) {
        const int r = (c + t) % TB;                  // rotated start: no bank conflicts across c
        s = fma(L[r + c * TB], vJ[r], s);
      }
      v[i] -= s;
    }
    __syncthreads();
  }
}

}  // namespace tiles
}  // namespace hyb
