// Back substitution after the reduced solve, one CTA per element, FP64.
//
// Hybridization (Thm 2.1): x_T = A_T^{-1}(f_T - C_T^T lambda_T), C_T = [0 D]. With the stored
// factor (interior rows L_ii, L_bi of the Cholesky factor L of A_T), z_i = L_ii^{-1} f_i, the
// face part of the load solve x0_b = (A_T^{-1} f_T)_b and P = (A_T^{-1})_bb = Y^T Y
// (Y = L_bb^{-1}; D P D is the element's S_T), all written by the element kernel:
//   w = D lambda_T,  x_b = x0_b - P w,  x_i = L_ii^{-T}(z_i - L_bi^T x_b).
// Static condensation (Sec. 3.1): u_b from the global face dofs (essential values on boundary
// faces), u_i = A_ii^{-1}(f_i - A_ib u_b) = L_ii^{-T}(z_i - L_bi^T u_b).
//
// Data movement: L_ii (the leading tri(NI) doubles of the element's packed factor) is copied
// into shared memory by one 1-D bulk copy (cp.async.bulk, completion on an mbarrier) issued
// when the CTA starts, so it lands while the CTA streams P and L_bi from HBM with coalesced
// loads (consecutive threads read consecutive entries of one stored row; P is stored as a full
// square so that x_b = x0_b - P w reads it once, column by column). The back substitution runs
// on BS-row blocks from shared memory. The tiled element kernels (RT_2, RT_3) store each
// diagonal block of L_ii as the inverse of its triangle (BS = the tile size), so a block's
// unknowns are one short triangular product (8 lanes per unknown, shuffle sums); RT_0/RT_1
// store the factor itself and one warp solves the diagonal triangle (shuffle broadcasts,
// reciprocal pivots formed in parallel beforehand). Then every thread applies the block's
// rows to the rows above it: two barriers per block instead of two per row. Every
// stored double feeds one FMA, so on this part (2 FP64 FMAs per clock per SM) the kernel is
// bound by FP64 issue, slightly above the HBM time of its bytes.
#include <cuda_runtime.h>

#include "hyb_device.h"
#include "hyb_internal.h"

namespace hyb {

namespace {

__device__ __forceinline__ int64_t tri(int i, int j) { return (int64_t)i * (i + 1) / 2 + j; }

template <int K>
struct RK {
  static constexpr int p = K + 1, NFN = p * p, NI = 3 * K * p * p, NB = 6 * NFN, N = NI + NB;
  static constexpr int TRI = N * (N + 1) / 2, TRII = NI * (NI + 1) / 2;
  static constexpr int NT = K <= 1 ? 32 : K == 2 ? 128 : 512;
  static constexpr bool INV = K >= 2;                          // diagonal blocks stored inverted
  static constexpr int BS = INV ? NFN : K == 1 ? 12 : 1;       // divides NI, <= 32
  static constexpr int NBLK = NI / BS;
  static_assert(NBLK * BS == NI, "whole blocks");
  static constexpr int CP = NT / NB > 0 ? NT / NB : 1;         // column chunks of x_b = x0_b - P w
  static constexpr int CI = NT / (NI > 0 ? NI : 1) > 0 ? NT / (NI > 0 ? NI : 1) : 1;   // of L_bi^T x_b
  static constexpr int LII_BYTES = (TRII * 8 + 15) / 16 * 16;  // bulk copy: a multiple of 16 bytes
  static constexpr int LII = LII_BYTES / 8;
  // shared memory (doubles): L_ii | x (N) | w (NB) | rhs (NI) | 1/L_rr (NI) | chunk partials
  static constexpr int PART = (CP * NB > CI * NI ? CP * NB : CI * NI);
  static constexpr int SMEM_DOUBLES = LII + N + NB + NI + NI + PART;
  static constexpr size_t SMEM = sizeof(double) * SMEM_DOUBLES;
  static_assert(K == 0 || NI % BS == 0, "blocks split the interior rows");
  static_assert(BS <= 32 && (!INV || 8 * BS <= NT), "one warp per diagonal block; 8 lanes per unknown");
  static_assert(fp64_store_doubles(K) >= TRI + NB * NB, "store holds the packed factor and P");
  static_assert((fp64_store_doubles(K) * 8) % 16 == 0 && (LII == 0 || TRI >= LII), "bulk copy alignment");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void csync() { __syncthreads(); }

template <int K, int MODE>
__device__ __forceinline__ void recover_body(const RecoverArgs& a, const int64_t e, double* sm) {
  using R = RK<K>;
  constexpr int NI = R::NI, NB = R::NB, N = R::N, NFN = R::NFN, NT = R::NT, BS = R::BS;
  constexpr int CP = R::CP, CI = R::CI;
  __shared__ uint64_t mbar;
  double* lii = sm;                       // L_ii, packed rows (bulk copy target, 16-byte aligned)
  double* x = lii + R::LII;               // x_i (solved in place of rhs), x_b
  double* w = x + N;                      // D lambda_T
  double* rhs = w + NB;
  double* invd = rhs + NI;
  double* part = invd + NI;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t es = a.slot ? (int64_t)a.slot[e] : e;
  const double* L = a.Lstore + es * fp64_store_doubles(K);
  const double* z = a.zstore + e * (int64_t)N;
  const int32_t* ef = a.elem_face + 6 * e;

  // ---- L_ii into shared memory (lands during the x_b and L_bi^T x_b passes)
  if constexpr (NI > 0) {
    if (tid == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&mbar)),
                   "r"((uint32_t)R::LII_BYTES)
                   : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32(lii)),
          "l"(L), "r"((uint32_t)R::LII_BYTES), "r"(smem_u32(&mbar))
          : "memory");
    }
  }

  // ---- x_b
  if (MODE == MODE_HYB) {
    for (int ib = tid; ib < NB; ib += NT) {
      const int fa = ef[ib / NFN], m = ib % NFN;
      w[ib] = fa < 0 ? 0.0 : (((ib / NFN) & 1) ? 1.0 : -1.0) * a.wf[m] * a.lambda[(int64_t)fa * NFN + m];
    }
    csync();
    // x_b = x0_b - P w: thread (j, c) sums column j of P over the rows of chunk c
    const double* P = L + R::TRI;
    if (tid < CP * NB) {
      const int j = tid % NB, c = tid / NB;
      constexpr int M0 = (NB + CP - 1) / CP;
      const int m0 = c * M0, m1 = m0 + M0 < NB ? m0 + M0 : NB;
      double acc = 0.0;
#pragma unroll 8
      for (int m = m0; m < m1; ++m) acc = fma(__ldcs(P + (int64_t)m * NB + j), w[m], acc);
      part[c * NB + j] = acc;
    }
    csync();
    for (int j = tid; j < NB; j += NT) {
      double s = part[j];
      for (int c = 1; c < CP; ++c) s += part[c * NB + j];
      x[NI + j] = z[NI + j] - s;
    }
  } else {
    for (int ib = tid; ib < NB; ib += NT) {
      const int fa = ef[ib / NFN], m = ib % NFN;
      // boundary faces: the essential value, kept unchanged in z by the identity rows
      x[NI + ib] = fa >= 0 ? a.lambda[(int64_t)fa * NFN + m] : z[NI + ib];
    }
  }
  csync();

  if constexpr (NI > 0) {
    // ---- rhs = z_i - L_bi^T x_b: thread (i, c) walks the stored rows NI + m of chunk c
    if (tid < CI * NI) {
      const int i = tid % NI, c = tid / NI;
      constexpr int M0 = (NB + CI - 1) / CI;
      const int m0 = c * M0, m1 = m0 + M0 < NB ? m0 + M0 : NB;
      double acc = 0.0;
#pragma unroll 8
      for (int m = m0; m < m1; ++m) acc = fma(__ldcs(L + tri(NI + m, i)), x[NI + m], acc);
      part[c * NI + i] = acc;
    }
    {
      // L_ii has landed (bounded waits: a copy that never completes is reported, not waited on)
      uint32_t done = 0;
      auto poll = [&](long long limit) {
        for (long long it = 0; it < limit && !done; ++it)
          asm volatile(
              "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\nselp.u32 %0, 1, 0, p;\n}"
              : "=r"(done)
              : "r"(smem_u32(&mbar))
              : "memory");
      };
      poll(1ll << 24);
      if (!__syncthreads_and(done != 0)) {
        poll(1ll << 28);       // the copy in flight may still write: let it finish before the CTA exits
        if (tid == 0 && a.status) dev::set_error(a.status, a.err_elem, HYB_ERR_TIMEOUT, e);
        return;                // uniform: every thread saw the same barrier result
      }
    }
    for (int i = tid; i < NI; i += NT) {
      double s = part[i];
      for (int c = 1; c < CI; ++c) s += part[c * NI + i];
      rhs[i] = z[i] - s;
      if constexpr (!R::INV) invd[i] = 1.0 / lii[tri(i, i)];
    }
    csync();
    // ---- L_ii^T x_i = rhs by blocks of BS rows, last block first
    for (int blk = R::NBLK - 1; blk >= 0; --blk) {
      const int r0 = blk * BS;
      if constexpr (R::INV) {
        // x_J = Dinv^T rhs_J, Dinv = L_JJ^{-1} (lower): unknown c sums over the rows r >= c,
        // the 8 lanes of its group taking every 8th row
        const int c = tid >> 3, q = tid & 7;
        double acc = 0.0;
        if (c < BS)
#pragma unroll
          for (int r = q; r < BS; r += 8)
            if (r >= c) acc = fma(lii[tri(r0 + r, r0 + c)], rhs[r0 + r], acc);
        if (warp < (8 * BS + 31) / 32) {   // whole warps (lanes past the last unknown add zeros)
          acc += __shfl_xor_sync(0xffffffffu, acc, 4);
          acc += __shfl_xor_sync(0xffffffffu, acc, 2);
          acc += __shfl_xor_sync(0xffffffffu, acc, 1);
          if (q == 0 && c < BS) x[r0 + c] = acc;
        }
      } else if (warp == 0) {
        double v = lane < BS ? rhs[r0 + lane] : 0.0;
#pragma unroll
        for (int r = BS - 1; r >= 0; --r) {
          const double xr = __shfl_sync(0xffffffffu, v * invd[r0 + (lane < BS ? lane : 0)], r);
          if (lane < r) v = fma(-lii[tri(r0 + r, r0 + lane)], xr, v);
          if (lane == r) x[r0 + r] = xr;
        }
      }
      csync();
      // rows above the block: rhs_s -= sum_r L(r0 + r, s) x_{r0 + r} (two partial sums)
      for (int s = tid; s < r0; s += NT) {
        double a0 = rhs[s], a1 = 0.0;
#pragma unroll
        for (int r = 0; r + 1 < BS; r += 2) {
          a0 = fma(-lii[tri(r0 + r, s)], x[r0 + r], a0);
          a1 = fma(-lii[tri(r0 + r + 1, s)], x[r0 + r + 1], a1);
        }
        if (BS & 1) a0 = fma(-lii[tri(r0 + BS - 1, s)], x[r0 + BS - 1], a0);
        rhs[s] = a0 + a1;
      }
      csync();
    }
  }
  double* u = a.u + e * (int64_t)N;
  for (int i = tid; i < N; i += NT) __stcs(u + i, x[i]);
}

template <int K, int MODE>
__global__ void __launch_bounds__(RK<K>::NT) recover_kernel(RecoverArgs a) {
  extern __shared__ __align__(16) double rsm[];
  if ((int64_t)blockIdx.x >= a.n_elem) return;
  recover_body<K, MODE>(a, a.elem_list ? (int64_t)a.elem_list[blockIdx.x] : (int64_t)blockIdx.x, rsm);
}

template <int K, int MODE>
__global__ void __launch_bounds__(RK<K>::NT) recover_kernel_batch(const RecoverArgs* probs, const int2* items,
                                                                   int64_t n_items) {
  extern __shared__ __align__(16) double rsm[];
  if ((int64_t)blockIdx.x >= n_items) return;
  const int2 it = items[blockIdx.x];
  recover_body<K, MODE>(probs[it.x], it.y, rsm);
}

template <class F>
cudaError_t set_smem(F* kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int K>
cudaError_t launch_k(const RecoverArgs& a, cudaStream_t s, Prof* prof) {
  using R = RK<K>;
  if (a.n_elem == 0) return cudaSuccess;
  cudaError_t err = a.mode == MODE_HYB ? set_smem(recover_kernel<K, MODE_HYB>, R::SMEM)
                                       : set_smem(recover_kernel<K, MODE_SC>, R::SMEM);
  if (err != cudaSuccess) return err;
  const int tok = prof_begin(prof, HYB_K_RECOVER, s);
  if (a.mode == MODE_HYB) recover_kernel<K, MODE_HYB><<<(unsigned)a.n_elem, R::NT, R::SMEM, s>>>(a);
  else recover_kernel<K, MODE_SC><<<(unsigned)a.n_elem, R::NT, R::SMEM, s>>>(a);
  prof_end(prof, tok, s);
  return cudaGetLastError();
}

}  // namespace

template <int K>
cudaError_t launch_batch_k(int mode, const RecoverArgs* probs, const int2* items, int64_t n, cudaStream_t s,
                           Prof* prof) {
  using R = RK<K>;
  if (n == 0) return cudaSuccess;
  cudaError_t err = mode == MODE_HYB ? set_smem(recover_kernel_batch<K, MODE_HYB>, R::SMEM)
                                     : set_smem(recover_kernel_batch<K, MODE_SC>, R::SMEM);
  if (err != cudaSuccess) return err;
  const int tok = prof_begin(prof, HYB_K_RECOVER, s);
  if (mode == MODE_HYB) recover_kernel_batch<K, MODE_HYB><<<(unsigned)n, R::NT, R::SMEM, s>>>(probs, items, n);
  else recover_kernel_batch<K, MODE_SC><<<(unsigned)n, R::NT, R::SMEM, s>>>(probs, items, n);
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
