// Tiled FP32 element elimination of the hybridized mixed form (RT_0 to RT_3)
// (arXiv:1801.08914, Sec. 3.2; the factorisation of Sec. 3.1 applied to the alpha mass M).
// Included by hyb_mixed.cu inside namespace hyb { namespace { ... } }; it uses that
// translation unit's FP64 helpers (geometry64, load_element64, apply_mass64/A64/D64/Dt64/G64) and
// its constant tables.
//
// The algebra (hyb_mixed.cu's header derives it):
//    L_M = chol(M), Xd = L_M^{-1} D, L_Z = chol(G^{-1} + Xd^T Xd),
//    Y = L_M,bb^{-1}, P = Xd_b^T Y, V = L_Z^{-1} P,  (A^{-1})_bb = Y^T Y - V^T V,
// with the matrices held as TB x TB tiles in shared memory so that every step is a short
// sequence of CTA-wide passes:
//  * L_M and L_Z: packed lower tiles, column of tiles after column of tiles (tile (I, J),
//    I >= J, at J T - J (J - 1) / 2 + I - J), column-major inside a tile. After the
//    factorisation a diagonal tile holds the inverse of its triangle, which is what the
//    panel step, the triangular solves and the inverse Y use.
//  * Cholesky: right-looking by tile columns; per column the CTA scales the panel (and the
//    matching rows of the fused right-hand sides), then warp 0 factors and inverts the next
//    diagonal tile (look-ahead) while the other warps apply the rank-TB update to the
//    trailing tiles with MR x MC register micro-tiles: two barriers per tile column.
//  * Triangular solves with one right-hand side (the refinement): two barriers per tile.
// TB divides both the interior and the face block of the local ordering (interior dofs
// first), so the face block is a trailing square of whole tiles. The assembly stores the
// tiles of L_M and L_Z, Xd and G^{-1} per element (211 KB at RT_3, 50 KB at RT_2); the
// recovery copies them back into shared memory and runs only the refined solve.

template <int K>
struct TileShape;
template <>
struct TileShape<0> {
  static constexpr int TB = 6, MR = 3, MC = 3, NT = 64, MINB = 8, MINB_ASM = 8;
};
template <>
struct TileShape<1> {
  // 6 x 6 tiles (6 tile columns): 17% faster element phase than 12 x 12 at 64^3
  static constexpr int TB = 6, MR = 3, MC = 3, NT = 128, MINB = 4, MINB_ASM = 4;
};
template <>
struct TileShape<2> {
  // one 9 x 9 tile per face (6 interior + 6 face tile columns): the diagonal tiles take the
  // two-column factor, and the kernel needs no stack; 18 x 18 tiles (one-row-per-lane factor,
  // 200-byte stack frame) ran the 64^3 element phase at half this rate. The recovery: 3 CTAs
  // per SM; the assembly, without the FP64 residual scratch: 4 CTAs per SM (64 registers)
  static constexpr int TB = 9, MR = 3, MC = 3, NT = 256, MINB = 3, MINB_ASM = 4;
};
template <>
struct TileShape<3> {
  static constexpr int TB = 16, MR = 4, MC = 4, NT = 512, MINB = 1, MINB_ASM = 1;   // 227 KB of shared memory
};

// S = Y^T Y - V^T V on the tensor cores (s_tensor) where the dead shared memory after Y | P
// holds the split operands: RT_3 (one CTA per SM, 227 KB)
template <int K>
constexpr bool kTensorS = K == 3;

template <int K>
struct MT {
  using TS = TileShape<K>;
  static constexpr int TB = TS::TB, MR = TS::MR, MC = TS::MC, NT = TS::NT, MINB = TS::MINB, MINB_ASM = TS::MINB_ASM;
  static constexpr int P = K + 2, p = K + 1, Q = K + 2, NQ = Q * Q * Q;
  static constexpr int NFN = p * p, NI = 3 * K * p * p, NB = 6 * NFN, N = NI + NB, NC = P * p * p;
  static constexpr int NQK = p * p * p;
  static constexpr int T = N / TB, TI = NI / TB, TQ = (NQK + TB - 1) / TB, NQP = TQ * TB;
  static constexpr int TT = TB * TB;
  static constexpr int LT = T * (T + 1) / 2 * TT;          // L_M tiles
  static constexpr int ZTS = TQ * (TQ + 1) / 2 * TT;       // L_Z tiles
  static constexpr int ZTSA = (ZTS + 3) / 4 * 4;           // their region, 16-byte aligned
  // Xd, row-major with XS columns: L_M^{-1} D' in columns < NQK (zero up to NQP); where it fits
  // (RT_0..RT_2), column NQP carries the load f_T through the factorisation (y = L_M^{-1} f_T for
  // the assembly's g_T) and the rest of the last MC-group is zero
  static constexpr bool FUSED_F = K <= 2;
  static constexpr int XS = NQP + (FUSED_F ? MC : 0);
  static constexpr int XD = N * XS;
  static constexpr int LT_INTERIOR = (TI * T - TI * (TI - 1) / 2) * TT;   // tile columns J < TI
  static constexpr int YPS = NB * NB + NQP * NB;           // Y | P (= V) after the refinement
  static constexpr bool YPS_IN_LT = YPS <= LT_INTERIOR;
  static constexpr int TMP64 = 3 * P * Q * Q;             // apply_mass64 scratch (all three components)
  static constexpr int D64 = 24 + 24 + 2 * P * Q + p * Q + 2 * Q + NFN + 7 * NQ /*g6 gd*/ + 4 * N /*f x r ut*/ +
                             3 * NQ /*U*/ + 3 * NQ /*Wv*/ + NQ /*Dv*/ + NC /*xc*/ + 2 * TMP64 + 8 + NQK /*qv*/ +
                             (N > NQ ? N : NQ) /*rq*/ + P * p /*DcO64*/;
  static constexpr int TABF = (2 * P * Q + p * Q + P * P * Q + P * p * Q + p * p * Q + P * p + 3) / 4 * 4;
  // scratch before the factorisation (in the L_M region): G, its tiles, the G^{-1} solve,
  // the sum-factorisation temporaries; mass-assembly temporaries (in the Xd region)
  static constexpr int GSCR = NQK * NQK + ZTS + NQP * NQP + Q * Q * p * p + Q * p * p * p * p + NQ;
  static constexpr int MSCR = 6 * NQ + Q * Q * P * P + Q * P * P * p * p;
  static constexpr int LTA = ((LT > GSCR ? LT : GSCR) + 3) / 4 * 4;   // L_M region (only RT_0 needs the padding)
  static constexpr int XDA = ((XD > MSCR ? XD : MSCR) + 3) / 4 * 4;   // Xd region
  static constexpr int64_t STORE = ((int64_t)LTA + XDA + ZTSA + NQK * NQK + 3) / 4 * 4;   // L_M | Xd | L_Z | G^{-1}
  static constexpr int F32 = TABF + LTA + XDA + ZTSA + N /*vec*/ + 2 * NQP /*tq tmpq*/ + 32 /*ybuf*/ + 8 /*flag*/ +
                             (YPS_IN_LT ? 0 : YPS);
  static constexpr size_t SMEM = sizeof(double) * D64 + sizeof(float) * F32 + sizeof(int) * N;
  // the assembly keeps only the geometry, the load and the solution in FP64 (the load is formed by
  // mixed_load_kernel, and the assembly's element solve is not refined)
  static constexpr int D64_ASM = (24 + 24 + 2 * P * Q + p * Q + 2 * Q + NFN + 7 * NQ + 2 * N + 8 + NQK + P * p + 1) / 2 * 2;
  static constexpr size_t SMEM_ASM = sizeof(double) * D64_ASM + sizeof(float) * F32 + sizeof(int) * N;
  static_assert(N % TB == 0 && NI % TB == 0, "tiles must split the interior and face blocks");
  static_assert(TB % MR == 0 && TB % MC == 0 && NQP % MC == 0 && NB % MC == 0, "micro-tile shape");
  static_assert(TB <= 32, "one warp per diagonal tile");
  static_assert(ZTSA % 4 == 0 && (D64 * 2) % 4 == 0, "16-byte aligned tile blocks");
};

// Refinement steps of the recovery's element solve: every step multiplies the error by about
// kappa(M, Z) u_32 <= 5e-5, so one step takes the FP32 solve (1e-7) to ~5e-12, below what the
// global FP64 refinement needs: its residual, the jump C u of the recovered flux, is only as
// accurate as u_T. The assembly's load term g_T = C_T A^{-1} f_T is left at the FP32 solve's
// accuracy (no refinement step): its error enters the reduced right-hand side as the FP32 S_T's
// error enters H, and the global refinement, whose residual does not depend on g, removes both.
constexpr int kRefineSteps = 1;

using tiles::tcol;

// S = Y^T Y - V^T V on the tensor cores (tcgen05 kind::tf32), split-TF32: X = [Y; V]^T (NB rows,
// K = NB + NQP, padded to multiples of 8) is split into TF32 parts X = X_hi + X_lo (each rounded
// to nearest), and S = X_hi^T X_hi + T + T^T with T = X_hi^T X_lo (the sign of the V rows via
// the MMA's negated A), which keeps FP32-level accuracy (Ootomo and Yokota's error-compensated
// TF32 products; the dropped X_lo^T X_lo term is below FP32 rounding). Both products are one
// M = 128 x N x 8 MMA per K step, accumulated in TMEM (S in columns 0.., T in columns 128..).
// X_hi and X_lo take dead shared memory (xhi: 128 rows' worth may be read, the padding rows
// landing in xlo). put(i, j, s) receives S(i, j) once per unordered pair and its mirror.
// Returns false (after freeing the TMEM) if the MMAs did not complete within the poll limit.
template <int K>
struct TensorS {
  using S = MT<K>;
  static constexpr int NB = S::NB, NQP = S::NQP;
  static constexpr int KY = (NB + 7) / 8 * 8, KV = (NQP + 7) / 8 * 8, KK = KY + KV;
  static constexpr int NPAD = (NB + 15) / 16 * 16;     // MMA N: a multiple of 16 for M = 128
  static constexpr int XFLOATS = NPAD * KK;            // one operand, rows >= NB zero
  static constexpr uint32_t SBO = (KK / 4) * 128;
};

template <int K, class Put>
__device__ bool s_tensor(const float* Y, const float* Pv, float* xhi, float* xlo, Put put) {
  using TS = TensorS<K>;
  constexpr int NB = TS::NB, NQP = TS::NQP, KY = TS::KY, KK = TS::KK, NPAD = TS::NPAD, NT = MT<K>::NT;
  static_assert(NT % 128 == 0, "whole lane quarters of warps");
  __shared__ uint64_t mbar;
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int t = tid; t < NPAD * KK; t += NT) {
    const int r = t % NPAD, k = t / NPAD;
    float x = 0.0f;
    if (r < NB) {
      if (k < NB) x = Y[k * NB + r];
      else if (k >= KY && k - KY < NQP) x = Pv[(k - KY) * NB + r];
    }
    const float hi = tc::to_tf32(x);
    const int o = tc::kmajor_offset(r, k, KK) >> 2;
    xhi[o] = hi;
    xlo[o] = tc::to_tf32(x - hi);
  }
  if (warp == 0) tc::tmem_alloc(&tbase, 256);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = tbase;
  if (tid == 0) {
    const uint32_t ahi = tc::smem_addr(xhi), alo = tc::smem_addr(xlo);
#pragma unroll 1
    for (int ks = 0; ks < KK / 8; ++ks) {
      const uint32_t id = tc::idesc_tf32(128, NPAD, ks * 8 >= KY);
      const uint64_t dhi = tc::smem_desc(ahi + ks * 256, 128, TS::SBO);
      const uint64_t dlo = tc::smem_desc(alo + ks * 256, 128, TS::SBO);
      tc::mma_tf32(tm, dhi, dhi, id, ks > 0);
      tc::mma_tf32(tm + 128, dhi, dlo, id, ks > 0);
    }
    tc::commit(&mbar);
  }
  bool ok = tc::mbar_wait(&mbar, 0, 1ll << 22);
  if (!ok) tc::mbar_wait(&mbar, 0, 1ll << 26);   // let MMAs in flight finish before the TMEM is freed
  tc::fence_after_sync();
  // T into shared memory (over X_lo, read by the completed MMAs), then S = S_hh + T + T^T
  constexpr int TLD = NB + 1;
  float* Ts = xlo;
  const int q = warp & 3, g = warp >> 2;                 // lane quarter, column group
  constexpr int NG = NT / 128, CW = (NPAD / NG + 7) / 8 * 8;
  const int i = q * 32 + lane;
  if (ok && q * 32 < NB)
    for (int c = g * CW; c < (g + 1) * CW && c < NPAD; c += 8) {
      float v[8];
      tc::tmem_ld8(tm + 128, q, c, v);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (i < NB && c + j < NB) Ts[i * TLD + c + j] = v[j];
    }
  __syncthreads();
  if (ok && q * 32 < NB)
    for (int c = g * CW; c < (g + 1) * CW && c < NPAD; c += 8) {
      float v[8];
      tc::tmem_ld8(tm, q, c, v);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int jj = c + j;
        if (i < NB && jj <= i) {
          const float sv = v[j] + Ts[i * TLD + jj] + Ts[jj * TLD + i];
          put(i, jj, sv);
          if (jj != i) put(jj, i, sv);
        }
      }
    }
  tc::fence_before_sync();
  __syncthreads();                                       // every thread is past the wait and the loads
  if (warp == 0) tc::tmem_dealloc(tm, 256);
  if (tid == 0) tc::mbar_inval(&mbar);
  return ok;
}

// FP32 tile factorisations of this kernel: whole triangles, no write-out of the factor,
// look-ahead form (warp 0 factors the next diagonal tile during the trailing update)
template <int TB, int MR, int MC, int NT>
__device__ __forceinline__ bool chol_tiles32(float* Lt, int T, float* X, int MX, float* flag) {
  return tiles::tile_chol_la<float, TB, MR, MC, NT>(tiles::Packed<float, TB>{Lt, T}, T, T, T, flag,
                                                    [](int) { return tiles::NoOut{}; }, X, MX);
}

// ---- CTA: one FP32 solve of the mixed-form saddle system with the tiled factors.
// In: v = r1 (N), t = rho (NQK, padded to NQP with zeros). Out: v = dx, t = dq, where
//   y = L_M^{-1} r1,  dq = Z^{-1} (G^{-1} rho + Xd^T y),  dx = L_M^{-T} (y - Xd dq).
template <int K>
__device__ void mixed_solve_tiled(const float* Lt, const float* Xd, const float* Zt, const float* Gi, float* v,
                                  float* t, float* tmp) {
  using S = MT<K>;
  constexpr int N = S::N, NQK = S::NQK, NQP = S::NQP, NT = S::NT;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  tiles::tile_fwd_vec<float, S::TB, NT>(Lt, S::T, v);
  for (int a = warp; a < NQP; a += NT / 32) {
    float acc = 0.0f;
    if (a < NQK) {
      for (int b = lane; b < NQK; b += 32) acc = fmaf(Gi[a * NQK + b], t[b], acc);
      for (int i = lane; i < N; i += 32) acc = fmaf(Xd[i * S::XS + a], v[i], acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) tmp[a] = acc;
  }
  __syncthreads();
  for (int a = tid; a < NQP; a += NT) t[a] = tmp[a];
  __syncthreads();
  tiles::tile_fwd_vec<float, S::TB, NT>(Zt, S::TQ, t);
  tiles::tile_bwd_vec<float, S::TB, NT>(Zt, S::TQ, t);
  for (int i = tid; i < N; i += NT) {
    float acc = v[i];
    for (int a = 0; a < NQK; ++a) acc = fmaf(-Xd[i * S::XS + a], t[a], acc);
    v[i] = acc;
  }
  __syncthreads();
  tiles::tile_bwd_vec<float, S::TB, NT>(Lt, S::T, v);
}

// ---- refinement of the element solve in the mixed variables (x, q = G D^T x) against FP64
// residuals of that saddle system (well conditioned at any contrast; refining A x = f
// directly would not converge, the two Woodbury terms cancelling in FP32):
//   r1 = f - M x - D q on free rows, f_e - x_e on essential rows;  rho = G D^T x - q;
// each correction is one tiled FP32 solve.
template <int K>
__device__ void refine_tiled(const double* f, double* x, double* q, int steps, double alpha, double beta, int bmask,
                             const double* g6, const double* gd, const double* Vc, const double* Dc, const double* Vo,
                             const double* DcO64, const int* dofcode, const float* Lt, const float* Xd,
                             const float* Zt, const float* Gi, double* r, double* ut, double* rq, double* U,
                             double* Wv, double* Dv, double* xc, double* t1, double* t2, float* vec, float* tq,
                             float* tmp) {
  using S = MT<K>;
  constexpr int NI = S::NI, NFN = S::NFN, N = S::N, NQK = S::NQK, NQP = S::NQP, NT = S::NT;
  const int tid = threadIdx.x;
  auto is_e = [&](int i) { return i >= NI && ((bmask >> ((i - NI) / NFN)) & 1); };
  for (int i = tid; i < N; i += NT) x[i] = 0.0;
  for (int a = tid; a < NQK; a += NT) q[a] = 0.0;
  __syncthreads();
  for (int it = 0; it <= steps; ++it) {
    if (it == 0) {                                  // x = 0, q = 0: the residuals are (f, 0)
      for (int i = tid; i < N; i += NT) vec[i] = (float)f[i];
      for (int a = tid; a < NQP; a += NT) tq[a] = 0.0f;
      __syncthreads();
    } else {
      for (int i = tid; i < N; i += NT) ut[i] = is_e(i) ? 0.0 : x[i];
      __syncthreads();
      apply_mass64<K, NT>(ut, r, alpha, g6, Vc, Vo, U, Wv, t1, t2);
      apply_D64<K, NT>(q, rq, dofcode, DcO64, bmask);
      for (int i = tid; i < N; i += NT) vec[i] = (float)(is_e(i) ? f[i] - x[i] : f[i] - r[i] - rq[i]);
      __syncthreads();
      apply_Dt64<K, NT>(ut, rq, DcO64, bmask);
      apply_G64<K, NT>(rq, r, beta, gd, Vo, U, t1, t2);
      for (int a = tid; a < NQP; a += NT) tq[a] = a < NQK ? (float)(r[a] - q[a]) : 0.0f;
      __syncthreads();
    }
    mixed_solve_tiled<K>(Lt, Xd, Zt, Gi, vec, tq, tmp);
    for (int i = tid; i < N; i += NT) x[i] += (double)vec[i];
    for (int a = tid; a < NQK; a += NT) q[a] += (double)tq[a];
    __syncthreads();
  }
}

// ---- The alpha mass M = (alpha u, v) of RT_K by sum factorisation, one (c, c') component block
// at a time: blk 0..2 the diagonal blocks (c, c), 3..5 the blocks (1, 0), (2, 0), (2, 1). Along
// da (= c) the rows take the closed 1-D basis and the columns the closed (diagonal) or open one,
// along db the rows take the open basis and the columns the open (diagonal) or closed one (db =
// c' off the diagonal), and along the remaining direction dL both take the open basis. The last
// contraction (over the dL quadrature points) writes output idx = ((((ia nja + ja) nib + ib) njb
// + jb) p + iL) p + jL, i.e. M(local_index(c, i), local_index(c', j)) with i, j the 1-D indices
// gathered per direction.
template <int K, int blk>
struct MassBlk {
  static constexpr int P = K + 2, p = K + 1;
  static constexpr int c = blk < 3 ? blk : (blk == 3 ? 1 : 2);
  static constexpr int cp = blk < 3 ? blk : (blk == 5 ? 1 : 0);
  static constexpr bool diag = c == cp;
  static constexpr int da = c, db = diag ? (c + 1) % 3 : cp, dL = 3 - da - db;
  static constexpr int nia = P, nja = diag ? P : p, nib = p, njb = diag ? p : P;
  static constexpr int s2 = nia * nja * nib * njb;     // outputs of the second contraction
  static constexpr int OUT = s2 * p * p;               // outputs of the last one
};

// Entries of one block before the symmetry cut, and each order's offset into the table below.
__host__ __device__ constexpr int mass_map_per(int k) { return (k + 2) * (k + 2) * (k + 1) * (k + 1) * (k + 1) * (k + 1); }
__host__ __device__ constexpr int mass_map_off(int k) { return k == 0 ? 0 : mass_map_off(k - 1) + 6 * mass_map_per(k - 1); }

// Per order and block, the outputs of the last contraction that land in the stored lower
// triangle of M, in increasing idx, each packed as (idx << 16) | (its offset in the L_M tile
// layout); g_mass_cnt holds their number. Filled by mass_map_kernel (every context setup writes
// the same values) so that the element kernel spends no integer work on local indices and tile
// positions in that pass.
__device__ uint32_t g_mass_map[mass_map_off(kMaxOrder + 1)];
__device__ int g_mass_cnt[(kMaxOrder + 1) * 6];

// Offset in the L_M tile layout of output idx of block blk, or -1 above the diagonal of M.
template <int K, int blk>
__device__ int mass_dst(int idx) {
  using B = MassBlk<K, blk>;
  using S = MT<K>;
  constexpr int p = B::p, da = B::da, db = B::db, nja = B::nja, nib = B::nib, njb = B::njb;
  constexpr int TB = S::TB, T = S::T, TT = S::TT;
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
  const int ra = local_index<K>(B::c, i0, i1, i2), sa = local_index<K>(B::cp, j0, j1, j2);
  if (B::diag && ra < sa) return -1;
  const int gi = ra >= sa ? ra : sa, gj = ra >= sa ? sa : ra;
  return tcol(gi / TB, gj / TB, T) * TT + (gi % TB) + (gj % TB) * TB;
}

// One warp per block: the kept outputs compacted in order by ballots.
template <int K>
__global__ void __launch_bounds__(192) mass_map_kernel() {
  static_assert(MT<K>::LT <= 65536 && mass_map_per(K) <= 65536, "16-bit fields");
  const int blk = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* map = g_mass_map + mass_map_off(K) + blk * mass_map_per(K);
  int n = 0;
  for (int base = 0; base < mass_map_per(K); base += 32) {
    const int idx = base + lane;
    int d = -1;
    if (idx < mass_map_per(K)) {
      switch (blk) {
        case 0: d = mass_dst<K, 0>(idx); break;
        case 1: d = mass_dst<K, 1>(idx); break;
        case 2: d = mass_dst<K, 2>(idx); break;
        case 3: d = mass_dst<K, 3>(idx); break;
        case 4: d = mass_dst<K, 4>(idx); break;
        default: d = mass_dst<K, 5>(idx); break;
      }
    }
    const unsigned keep = __ballot_sync(0xffffffffu, d >= 0);
    if (d >= 0) map[n + __popc(keep & ((1u << lane) - 1u))] = ((uint32_t)idx << 16) | (uint32_t)d;
    n += __popc(keep);
  }
  if (lane == 0) g_mass_cnt[K * 6 + blk] = n;
}

// ---- the element: factorisation (both modes), then either S_T / g_T (assembly) or the
// recovery u_T = A^{-1}(f_T - C_T^T lambda).
template <int K, bool RECOVER>
__device__ void element_tiled_body(const ElemArgs& args, const int64_t e, double* smem, const double* lambda,
                                   double* u_out) {
  using S = MT<K>;
  constexpr int P = S::P, p = S::p, Q = S::Q, NQ = S::NQ, NFN = S::NFN, NI = S::NI, NB = S::NB, N = S::N;
  constexpr int NQK = S::NQK, NQP = S::NQP, NT = S::NT, NC = S::NC, TB = S::TB, MR = S::MR, MC = S::MC;
  constexpr int T = S::T, TQ = S::TQ, TT = S::TT;
  const int tid = threadIdx.x;
  const int64_t slot = args.slot ? args.slot[e] : e;
  float* store = args.Lstore32 + slot * S::STORE;                // this element's factors (global)
  float* Gi = store + S::LTA + S::XDA + S::ZTSA;                  // G^{-1}

  // ---- shared memory
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
  double *r = nullptr, *ut = nullptr, *U = nullptr, *Wv = nullptr, *Dv = nullptr, *xc = nullptr, *t1 = nullptr,
         *t2 = nullptr, *rq = nullptr;
  if constexpr (RECOVER) {                        // the refinement's FP64 residual scratch
    r = d; d += N;
    ut = d; d += N;
    U = d; d += 3 * NQ;
    Wv = d; d += 3 * NQ;
    Dv = d; d += NQ;
    xc = d; d += NC;
    t1 = d; d += S::TMP64;
    t2 = d; d += S::TMP64;
  }
  d += 8;
  double* qv = d; d += NQK;
  if constexpr (RECOVER) {
    rq = d; d += (N > NQ ? N : NQ);
  }
  double* DcO64 = d; d += P * p;
  d = smem + (RECOVER ? S::D64 : S::D64_ASM);      // the float region starts where the launch sized it
  float* fl = reinterpret_cast<float*>(d);
  float* Vcf = fl; fl += P * Q;
  float* Dcf = fl; fl += P * Q;
  float* Vof = fl; fl += p * Q;
  float* VcVc = fl; fl += P * P * Q;
  float* VcVo = fl; fl += P * p * Q;
  float* VoVo = fl; fl += p * p * Q;
  float* DcO = fl; fl += S::TABF - (2 * P * Q + p * Q + P * P * Q + P * p * Q + p * p * Q);
  float* Lt = fl; fl += S::LTA;
  float* Xd = fl; fl += S::XDA;
  float* Zt = fl; fl += S::ZTSA;
  float* vec = fl; fl += N;
  float* tq = fl; fl += NQP;
  float* tmpq = fl; fl += NQP;
  fl += 32;                                       // spare
  float* flag = fl; fl += 8;
  float* yps = S::YPS_IN_LT ? Lt : fl;
  if (!S::YPS_IN_LT) fl += S::YPS;
  int* dofcode = reinterpret_cast<int*>(fl);

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
  const int32_t* ef = args.elem_face + e * 6;
  int bmask = 0;
#pragma unroll
  for (int a = 0; a < 6; ++a) bmask |= (ef[a] < 0 && !args.natural) << a;
  auto is_e = [&](int i) { return i >= NI && ((bmask >> ((i - NI) / NFN)) & 1); };

  // ---- FP64 right-hand side f_T = M_T c_T (essential values folded in), formed by
  // mixed_load_kernel before the assembly; the recovery subtracts C^T lambda
  double* fs = args.zstore + e * (int64_t)N;
  for (int i = tid; i < N; i += NT) {
    double v = fs[i];
    if (RECOVER && i >= NI) {
      const int a = (i - NI) / NFN, m = (i - NI) % NFN;
      if (ef[a] >= 0) v -= ((a & 1) ? 1.0 : -1.0) * wf[m] * lambda[(int64_t)ef[a] * NFN + m];
    }
    f[i] = v;                                    // f_T, or f_T - C_T^T lambda
  }
  __syncthreads();

  if (RECOVER) {
    // ---- the stored factors back into shared memory
    const float4* src = reinterpret_cast<const float4*>(store);
    float4* dst = reinterpret_cast<float4*>(Lt);
    constexpr int NV = (S::LTA + S::XDA + S::ZTSA) / 4;         // Lt | Xd | Zt are contiguous
    for (int t = tid; t < NV; t += NT) dst[t] = __ldcs(src + t);
    __syncthreads();
  } else {
  // G^{-1} (the Q_k mass weighted by beta / det J, inverted in FP32) is in the element's store:
  // mixed_load_kernel formed it before this launch
  // ---- FP32 alpha-mass M into the L_M tiles (lower triangle), essential rows -> identity.
  // Temporaries in the Xd region, which is free until D' is written.
  for (int t = tid; t < S::LT; t += NT) Lt[t] = 0.0f;
  __syncthreads();
  {
    float* Ga32 = Xd;                             // [6][NQ]
    float* T1 = Xd + 6 * NQ;
    float* T2 = T1 + Q * Q * P * P;
    for (int t = tid; t < 6 * NQ; t += NT) Ga32[t] = (float)(alpha * g6[t]);
    __syncthreads();
    // one (c, cp) block of the mass per call, block index a compile-time constant so that the
    // index decompositions divide by constants
    auto mass_block = [&](auto blk_c) {
      constexpr int blk = decltype(blk_c)::value;
      using B = MassBlk<K, blk>;
      constexpr int c = B::c, cp = B::cp;
      constexpr bool diag = B::diag;
      constexpr int da = B::da, db = B::db, dL = B::dL;
      constexpr int nia = B::nia, nja = B::nja, nib = B::nib, njb = B::njb;
      constexpr int sa = da == 0 ? 1 : da == 1 ? Q : Q * Q;
      constexpr int sb = db == 0 ? 1 : db == 1 ? Q : Q * Q;
      constexpr int sL = dL == 0 ? 1 : dL == 1 ? Q : Q * Q;
      const float* Gm = Ga32 + gslot(c, cp) * NQ;
      const float* Pm = diag ? VcVc : VcVo;
      constexpr int n1 = Q * Q * nia * nja;
      for (int idx = tid; idx < n1; idx += NT) {
        int rr = idx;
        const int ja = rr % nja; rr /= nja;
        const int ia = rr % nia; rr /= nia;
        const int qL = rr % Q, qb = rr / Q;
        float acc = 0.f;
#pragma unroll
        for (int qa = 0; qa < Q; ++qa) acc = fmaf(Gm[qa * sa + qb * sb + qL * sL], Pm[(ia * nja + ja) * Q + qa], acc);
        T1[idx] = acc;
      }
      __syncthreads();
      constexpr int n2 = Q * nia * nja * nib * njb;
      for (int idx = tid; idx < n2; idx += NT) {
        int rr = idx;
        const int jb = rr % njb; rr /= njb;
        const int ib = rr % nib; rr /= nib;
        const int ja = rr % nja; rr /= nja;
        const int ia = rr % nia, qL = rr / nia;
        float acc = 0.f;
#pragma unroll
        for (int qb = 0; qb < Q; ++qb) {
          const float tv = T1[((qb * Q + qL) * nia + ia) * nja + ja];
          acc = fmaf(tv, diag ? VoVo[(ib * p + jb) * Q + qb] : VcVo[(jb * p + ib) * Q + qb], acc);
        }
        T2[idx] = acc;
      }
      __syncthreads();
      constexpr int s2 = B::s2;
      // outputs in the lower triangle of M, with their tile offsets, from the per-order table
      const uint32_t* map = g_mass_map + mass_map_off(K) + blk * mass_map_per(K);
      const int cnt = g_mass_cnt[K * 6 + blk];
      for (int t = tid; t < cnt; t += NT) {
        const uint32_t m = __ldg(map + t);
        const int idx = (int)(m >> 16);
        const int tt = idx / (p * p), ij = idx - tt * (p * p);   // ij = iL p + jL
        float acc = 0.f;
#pragma unroll
        for (int qL = 0; qL < Q; ++qL) acc = fmaf(T2[qL * s2 + tt], VoVo[ij * Q + qL], acc);
        Lt[m & 0xffffu] = acc;
      }
      // the next block's first pass touches only T1 (last read before the barrier above) and
      // its second pass, which overwrites T2, follows a barrier
      if constexpr (blk == 5) __syncthreads();
    };
    mass_block(std::integral_constant<int, 0>{});
    mass_block(std::integral_constant<int, 1>{});
    mass_block(std::integral_constant<int, 2>{});
    mass_block(std::integral_constant<int, 3>{});
    mass_block(std::integral_constant<int, 4>{});
    mass_block(std::integral_constant<int, 5>{});
    if (bmask) {
      for (int t = tid; t < NB * N; t += NT) {   // essential rows and columns -> identity
        const int i = NI + t / N, j = t % N;
        if (!is_e(i)) continue;
        const int gi = i >= j ? i : j, gj = i >= j ? j : i;
        Lt[tcol(gi / TB, gj / TB, T) * TT + (gi % TB) + (gj % TB) * TB] = (i == j) ? 1.f : 0.f;
      }
      __syncthreads();
    }
  }

  // ---- D' (zero rows on essential dofs, zero columns beyond NQK) into Xd, then the tiled
  // Cholesky of M fused with Xd <- L_M^{-1} D'. The component-c function with 1-D nodes
  // (i0, i1, i2) meets only the p functions of Q_k whose other two indices equal its own:
  // D'(i, a) = DcO[i_c][a_c] there, zero elsewhere; so Xd is cleared and those p entries per free
  // row written.
  {
    static_assert((N * S::XS + 3) / 4 * 4 <= S::XDA, "Xd cleared in whole float4");
    float4* x4 = reinterpret_cast<float4*>(Xd);
    for (int t = tid; t < (N * S::XS + 3) / 4; t += NT) x4[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  for (int t = tid; t < N * p; t += NT) {
    const int i = t / p, j = t - (t / p) * p;
    if (is_e(i)) continue;
    const int code = dofcode[i];
    const int c = code & 3, i0 = (code >> 2) & 63, i1 = (code >> 8) & 63, i2 = (code >> 14) & 63;
    const int a0 = c == 0 ? j : i0, a1 = c == 1 ? j : i1, a2 = c == 2 ? j : i2;
    Xd[i * S::XS + a0 + p * (a1 + p * a2)] = DcO[(c == 0 ? i0 : c == 1 ? i1 : i2) * p + j];
  }
  if constexpr (S::FUSED_F)                        // the load, carried through the factorisation
    for (int i = tid; i < N; i += NT) Xd[i * S::XS + NQP] = (float)f[i];
  __syncthreads();
  if (!chol_tiles32<TB, MR, MC, NT>(Lt, T, Xd, S::XS, flag)) {
    if (tid == 0) set_error(args.status, args.err_elem, HYB_ERR_NOT_SPD, e);
    return;
  }
  // ---- Z = G^{-1} + Xd^T Xd (padded with the identity) into the L_Z tiles, then its Cholesky
  {
    constexpr int PM = (TB / MR) * (TB / MC);
    constexpr int NP = TQ * (TQ + 1) / 2;
    for (int it = tid; it < NP * PM; it += NT) {
      const int tile = it / PM, u = it % PM;
      int J = 0, rem = tile;
      while (rem >= TQ - J) { rem -= TQ - J; ++J; }
      const int I = J + rem;
      const int r0 = (u / (TB / MC)) * MR, c0 = (u % (TB / MC)) * MC;
      float acc[MR][MC];
#pragma unroll
      for (int i = 0; i < MR; ++i)
#pragma unroll
        for (int j = 0; j < MC; ++j) acc[i][j] = 0.0f;
      for (int k = 0; k < N; ++k) {
        float a[MR], b[MC];
#pragma unroll
        for (int i = 0; i < MR; ++i) a[i] = Xd[k * S::XS + I * TB + r0 + i];
#pragma unroll
        for (int j = 0; j < MC; ++j) b[j] = Xd[k * S::XS + J * TB + c0 + j];
#pragma unroll
        for (int i = 0; i < MR; ++i)
#pragma unroll
          for (int j = 0; j < MC; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
      float* Zq = Zt + tile * TT;
#pragma unroll
      for (int i = 0; i < MR; ++i)
#pragma unroll
        for (int j = 0; j < MC; ++j) {
          const int gi = I * TB + r0 + i, gj = J * TB + c0 + j;
          const float g = (gi < NQK && gj < NQK) ? Gi[gi * NQK + gj] : (gi == gj ? 1.0f : 0.0f);
          Zq[(r0 + i) + (c0 + j) * TB] = acc[i][j] + g;
        }
    }
    __syncthreads();
    if (!chol_tiles32<TB, MR, MC, NT>(Zt, TQ, nullptr, 0, flag)) {
      if (tid == 0) set_error(args.status, args.err_elem, HYB_ERR_NOT_SPD, e);
      return;
    }
  }
  {
    // ---- keep the factors for the recovery
    const float4* src = reinterpret_cast<const float4*>(Lt);
    float4* dst = reinterpret_cast<float4*>(store);
    constexpr int NV = (S::LTA + S::XDA + S::ZTSA) / 4;
    for (int t = tid; t < NV; t += NT) __stcs(dst + t, src[t]);
  }
  }

  // ---- the refined element solve: u_T (recovery)
  if constexpr (RECOVER)
    refine_tiled<K>(f, x, qv, kRefineSteps, alpha, beta, bmask, g6, gd, Vc, Dc, Vo, DcO64, dofcode, Lt, Xd, Zt, Gi, r,
                    ut, rq, U, Wv, Dv, xc, t1, t2, vec, tq, tmpq);
  auto scatter_rhs = [&](auto xb) {              // g_T = D_c x_b on the interior faces
    for (int ib = tid; ib < NB; ib += NT) {
      const int a = ib / NFN, m1 = ib % NFN;
      if (ef[a] < 0) continue;
      const double v = ((a & 1) ? 1.0 : -1.0) * wf[m1] * (double)xb(ib);
      const int64_t gi = (int64_t)ef[a] * NFN + m1;
      if (args.colour == 1) args.rhs[gi] += v;
      else args.rhs[gi] = v;
    }
  };
  if constexpr (RECOVER) {
    double* ue = u_out + e * (int64_t)N;
    for (int i = tid; i < N; i += NT) ue[i] = x[i];
  } else {
    {
      // (A^{-1} f)_b of the mixed form from y = L_M^{-1} f: t = Z^{-1} Xd^T y, v = y - Xd t, and
      // (A^{-1} f)_b = L_bb^{-T} v_b = Y^T v_b once Y is formed below (the backward solve's face
      // rows need only v_b). y is column NQP of Xd where the load rode through the
      // factorisation (RT_0..RT_2), else one forward solve. The FP32 solve of the recovery's first
      // step, without its backward solve (and, where fused, without its forward one).
      const int lane = tid & 31, warp = tid >> 5;
      if constexpr (!S::FUSED_F) {
        for (int i = tid; i < N; i += NT) vec[i] = (float)f[i];
        __syncthreads();
        tiles::tile_fwd_vec<float, TB, NT>(Lt, T, vec);
      }
      auto y = [&](int i) { return S::FUSED_F ? Xd[i * S::XS + NQP] : vec[i]; };
      for (int a = warp; a < NQP; a += NT / 32) {
        float acc = 0.0f;
        if (a < NQK)
          for (int i = lane; i < N; i += 32) acc = fmaf(Xd[i * S::XS + a], y(i), acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) tq[a] = acc;
      }
      __syncthreads();
      tiles::tile_fwd_vec<float, TB, NT>(Zt, TQ, tq);
      tiles::tile_bwd_vec<float, TB, NT>(Zt, TQ, tq);
      for (int j = tid; j < NB; j += NT) {
        const float* xr = Xd + (NI + j) * S::XS;
        float acc = y(NI + j);
        for (int a = 0; a < NQK; ++a) acc = fmaf(-xr[a], tq[a], acc);
        vec[NI + j] = acc;
      }
    }

    // ---- Y = L_M,bb^{-1}, P = Xd_b^T Y, V = L_Z^{-1} P, S = Y^T Y - V^T V. The buffers take the
    // interior tile columns of L_M (no longer needed) where they fit.
    float* Y = yps;                                 // [NB][NB]
    float* Pv = Y + NB * NB;                        // [NQP][NB]
    __syncthreads();
    for (int t = tid; t < NB * NB; t += NT) Y[t] = (t / NB == t % NB) ? 1.0f : 0.0f;
    __syncthreads();
    tiles::tile_fwd_mat<float, TB, MR, MC, NT>(Lt, T, S::TI, Y, NB);
    {
      __syncthreads();
      // x_b = Y^T v_b (Y lower triangular, row-major), scattered as g_T = D_c x_b
      scatter_rhs([&](int j) {
        float acc = 0.0f;
        for (int k = j; k < NB; ++k) acc = fmaf(Y[k * NB + j], vec[NI + k], acc);
        return acc;
      });
    }
    {
      constexpr int RM = NQP / MR, CM = NB / MC;
      for (int it = tid; it < RM * CM; it += NT) {  // P[a][j] = sum_i Xd[NI + i][a] Y[i][j]
        const int a0 = (it / CM) * MR, j0 = (it % CM) * MC;
        float acc[MR][MC];
  #pragma unroll
        for (int i = 0; i < MR; ++i)
  #pragma unroll
          for (int j = 0; j < MC; ++j) acc[i][j] = 0.0f;
        for (int k = 0; k < NB; ++k) {
          float a[MR], b[MC];
  #pragma unroll
          for (int i = 0; i < MR; ++i) a[i] = Xd[(NI + k) * S::XS + a0 + i];
  #pragma unroll
          for (int j = 0; j < MC; ++j) b[j] = Y[k * NB + j0 + j];
  #pragma unroll
          for (int i = 0; i < MR; ++i)
  #pragma unroll
            for (int j = 0; j < MC; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
  #pragma unroll
        for (int i = 0; i < MR; ++i)
  #pragma unroll
          for (int j = 0; j < MC; ++j) Pv[(a0 + i) * NB + j0 + j] = acc[i][j];
      }
    }
    __syncthreads();
    tiles::tile_fwd_mat<float, TB, MR, MC, NT>(Zt, TQ, 0, Pv, NB);
    // ---- S[i][j] = sum_m Y[m][i] Y[m][j] - sum_a V[a][i] V[a][j] for i >= j, in register
    // micro-tiles, scattered as S_T = D_c S D_c straight into the FP64 CSR values: entry (i, j)
    // and its mirror (j, i) get the same value, so both face blocks of a pair are bitwise
    // transposed.
    __shared__ int64_t s_row0[6];
    __shared__ int s_rlen[6];
    __shared__ float s_wf[NFN];
    if (tid < 6) {
      const int64_t r0 = ef[tid] >= 0 ? args.row_ptr[(int64_t)ef[tid] * NFN] : 0;
      s_row0[tid] = r0;
      s_rlen[tid] = ef[tid] >= 0 ? (int)(args.row_ptr[(int64_t)ef[tid] * NFN + 1] - r0) : 0;
    }
    for (int m = tid; m < NFN; m += NT) s_wf[m] = (float)wf[m];
    __syncthreads();
    const int64_t* boff = args.blockoff + e * 36;
    // S_T = D_c S D_c in FP32 (S itself carries ~1e-7), widened exactly to FP64 with integer
    // operations: no FP64 instruction per entry
    auto put = [&](int ib, int jb, float sv) {
      const int a = ib / NFN, m1 = ib % NFN, b = jb / NFN, m2 = jb % NFN;
      if (ef[a] < 0 || ef[b] < 0) return;
      const float w = sv * (s_wf[m1] * s_wf[m2]);      // w_m1 w_m2 = w_m2 w_m1: the mirror gets the same value
      const double v = dev::widen_f32(((a ^ b) & 1) ? -w : w);
      const int64_t pos = boff[a * 6 + b] + m1 * (int64_t)s_rlen[a] + m2;
      if (a == b && args.colour == 1) args.val[pos] += v;
      else args.val[pos] = v;
    };
    if constexpr (kTensorS<K>) {
      static_assert(S::YPS_IN_LT && S::YPS + TensorS<K>::XFLOATS <= S::LTA && TensorS<K>::XFLOATS <= S::XDA &&
                        (128 - TensorS<K>::NPAD) * TensorS<K>::KK <= S::XDA,
                    "X_hi after Y | P in the L_M region, X_lo over Xd, the padding rows of X_hi inside X_lo");
      if (!s_tensor<K>(Y, Pv, Lt + S::YPS, Xd, put) && tid == 0)
        set_error(args.status, args.err_elem, HYB_ERR_TIMEOUT, e);
    } else {
      constexpr int RM = NB / MR, CM = NB / MC;
      constexpr bool kMicroInFace = NFN % MR == 0 && NFN % MC == 0;
      for (int it = tid; it < RM * CM; it += NT) {
        const int i0 = (it / CM) * MR, j0 = (it % CM) * MC;
        if (i0 + MR - 1 < j0) continue;             // strictly above the diagonal
        // where the micro-tiles split the face blocks, a micro-tile lies in one face pair: skip
        // it whole when either face is on the boundary (put drops those entries)
        if constexpr (kMicroInFace) {
          if (ef[i0 / NFN] < 0 || ef[j0 / NFN] < 0) continue;
        }
        float acc[MR][MC];
  #pragma unroll
        for (int i = 0; i < MR; ++i)
  #pragma unroll
          for (int j = 0; j < MC; ++j) acc[i][j] = 0.0f;
        for (int k = 0; k < NB; ++k) {
          float a[MR], b[MC];
  #pragma unroll
          for (int i = 0; i < MR; ++i) a[i] = Y[k * NB + i0 + i];
  #pragma unroll
          for (int j = 0; j < MC; ++j) b[j] = Y[k * NB + j0 + j];
  #pragma unroll
          for (int i = 0; i < MR; ++i)
  #pragma unroll
            for (int j = 0; j < MC; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        for (int k = 0; k < NQK; ++k) {
          float a[MR], b[MC];
  #pragma unroll
          for (int i = 0; i < MR; ++i) a[i] = Pv[k * NB + i0 + i];
  #pragma unroll
          for (int j = 0; j < MC; ++j) b[j] = Pv[k * NB + j0 + j];
  #pragma unroll
          for (int i = 0; i < MR; ++i)
  #pragma unroll
            for (int j = 0; j < MC; ++j) acc[i][j] = fmaf(-a[i], b[j], acc[i][j]);
        }
        if constexpr (kMicroInFace) {
          // put with the face pair (a, b) decoded once per micro-tile; the same values and
          // positions entry by entry
          const int a = i0 / NFN, b = j0 / NFN, m10 = i0 - a * NFN, m20 = j0 - b * NFN;
          const int64_t pab = boff[a * 6 + b], pba = boff[b * 6 + a];
          const int64_t la = s_rlen[a], lb = s_rlen[b];
          const bool neg = (a ^ b) & 1, add = a == b && args.colour == 1;
  #pragma unroll
          for (int i = 0; i < MR; ++i)
  #pragma unroll
            for (int j = 0; j < MC; ++j) {
              const int ib = i0 + i, jb = j0 + j;
              if (ib < jb) continue;
              const int m1 = m10 + i, m2 = m20 + j;
              const float w = acc[i][j] * (s_wf[m1] * s_wf[m2]);
              const double v = dev::widen_f32(neg ? -w : w);
              const int64_t pos = pab + m1 * la + m2;
              if (add) args.val[pos] += v;
              else args.val[pos] = v;
              if (ib != jb) {
                const int64_t pos2 = pba + m2 * lb + m1;
                if (add) args.val[pos2] += v;
                else args.val[pos2] = v;
              }
            }
        } else {
  #pragma unroll
          for (int i = 0; i < MR; ++i)
  #pragma unroll
            for (int j = 0; j < MC; ++j) {
              const int ib = i0 + i, jb = j0 + j;
              if (ib < jb) continue;
              put(ib, jb, acc[i][j]);
              if (ib != jb) put(jb, ib, acc[i][j]);
            }
        }
      }
    }
  }
}

// ---- FP64 element load of the mixed path, before the FP32 elimination: f_T = M_T c_T by sum
// factorisation; on boundary faces with essential data f_T -= A_{:,e} u_e (free rows) and
// f_T = u_e (essential rows), zero essential data clearing the essential rows. Stored in the
// element's slot of zstore, where the assembly (g_T) and the recovery read it. The same kernel
// then forms the element's G^{-1} (g_inverse), which needs only the geometry and beta.
// Layout (floats, every piece 16-byte aligned) of g_inverse's shared-memory scratch.
template <int K>
struct GScratch {
  using S = MT<K>;
  static constexpr int p = S::p, Q = S::Q;
  static constexpr int r4(int n) { return (n + 3) / 4 * 4; }
  static constexpr int VOVO = 0, GD = VOVO + r4(p * p * Q), GF = GD + r4(S::NQ), GT = GF + r4(S::NQK * S::NQK);
  static constexpr int XG = GT + r4(S::ZTS), T1 = XG + r4(S::NQP * S::NQP), T2 = T1 + r4(Q * Q * p * p);
  static constexpr int FLAG = T2 + r4(Q * p * p * p * p), TOTAL = FLAG + 8;
};

template <int K>
struct LoadShape {
  static constexpr int P = K + 2, p = K + 1, Q = K + 2, NQ = Q * Q * Q, NFN = p * p, N = 3 * K * p * p + 6 * NFN;
  static constexpr int NC = P * p * p, TMP64 = 3 * P * Q * Q, NT = 128;
  static constexpr int D64 = 24 + 24 + 2 * P * Q + p * Q + 2 * Q + NFN + 7 * NQ + 3 * N + 6 * NQ + NQ + NC + 2 * TMP64;
  // the G^{-1} scratch (floats) starts where the FP64 load scratch (after f_T) started
  static constexpr int PREFIX = (24 + 24 + 2 * P * Q + p * Q + 2 * Q + NFN + 7 * NQ + N + 1) / 2 * 2;
  using S = MT<K>;
  static constexpr int GF = GScratch<K>::TOTAL;
  static constexpr int DTOT = D64 > PREFIX + (GF + 1) / 2 ? D64 : PREFIX + (GF + 1) / 2;
  static constexpr size_t SMEM = sizeof(double) * DTOT;
};

// ---- G^{-1} of one element into its FP32 store (CTA of NT threads): the Q_k mass weighted by
// beta / det J (gd: det J times the quadrature weights) by sum factorisation in FP32, its tiled
// Cholesky with the identity carried along (X = L^{-1}), then X = L^{-T} L^{-1}. fl: GF floats.
// Returns false (every thread) if G is not positive definite.
template <int K, int NT>
__device__ bool g_inverse(double beta, const double* gd, const double* Vo, float* fl, float* Gi) {
  using S = MT<K>;
  constexpr int p = S::p, Q = S::Q, NQ = S::NQ, NQK = S::NQK, NQP = S::NQP, TB = S::TB, TT = S::TT, TQ = S::TQ;
  const int tid = threadIdx.x;
  using GS = GScratch<K>;
  float* VoVo = fl + GS::VOVO;                  // [p][p][Q]
  float* Gd32 = fl + GS::GD;                    // [NQ]
  float* Gf = fl + GS::GF;                      // [NQK][NQK]
  float* Gt = fl + GS::GT;                      // tiles of the padded G
  float* Xg = fl + GS::XG;                      // [NQP][NQP]: identity -> L^{-1} -> G^{-1}
  float* T1 = fl + GS::T1;                      // [Q][Q][p][p]
  float* T2 = fl + GS::T2;                      // [Q][p^4]
  float* flag = fl + GS::FLAG;
  for (int i = tid; i < p * p * Q; i += NT) {
    const int q = i % Q, b = (i / Q) % p, a = i / (Q * p);
    VoVo[i] = (float)Vo[a * Q + q] * (float)Vo[b * Q + q];
  }
  for (int q = tid; q < NQ; q += NT) Gd32[q] = (float)(beta * gd[q]);
  __syncthreads();
  for (int t = tid; t < Q * Q * p * p; t += NT) {
    const int b0 = t % p, a0 = (t / p) % p, q1 = (t / (p * p)) % Q, q2 = t / (p * p * Q);
    float acc = 0.f;
    for (int q0 = 0; q0 < Q; ++q0) acc = fmaf(Gd32[(q2 * Q + q1) * Q + q0], VoVo[(a0 * p + b0) * Q + q0], acc);
    T1[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < Q * p * p * p * p; t += NT) {
    const int b0 = t % p, a0 = (t / p) % p, b1 = (t / (p * p)) % p, a1 = (t / (p * p * p)) % p, q2 = t / (p * p * p * p);
    float acc = 0.f;
    for (int q1 = 0; q1 < Q; ++q1) acc = fmaf(T1[((q2 * Q + q1) * p + a0) * p + b0], VoVo[(a1 * p + b1) * Q + q1], acc);
    T2[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < NQK * NQK; t += NT) {
    const int a = t / NQK, b = t % NQK;
    const int a0 = a % p, a1 = (a / p) % p, a2 = a / (p * p);
    const int b0 = b % p, b1 = (b / p) % p, b2 = b / (p * p);
    float acc = 0.f;
    for (int q2 = 0; q2 < Q; ++q2)
      acc = fmaf(T2[(((q2 * p + a1) * p + b1) * p + a0) * p + b0], VoVo[(a2 * p + b2) * Q + q2], acc);
    Gf[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < S::ZTS; t += NT) {      // pack the lower tiles of [[G, 0], [0, I]]
    const int tile = t / TT, w = t % TT, rr = w % TB, cc = w / TB;
    int J = 0, rem = tile;
    while (rem >= TQ - J) { rem -= TQ - J; ++J; }
    const int I = J + rem, i = I * TB + rr, j = J * TB + cc;
    Gt[t] = (i < NQK && j < NQK) ? Gf[i * NQK + j] : (i == j ? 1.0f : 0.0f);
  }
  for (int t = tid; t < NQP * NQP; t += NT) Xg[t] = (t / NQP == t % NQP) ? 1.0f : 0.0f;
  __syncthreads();
  if (!chol_tiles32<TB, S::MR, S::MC, NT>(Gt, TQ, Xg, NQP, flag)) return false;
  tiles::tile_bwd_mat<float, TB, NT>(Gt, TQ, Xg, NQP);
  for (int t = tid; t < NQK * NQK; t += NT) Gi[t] = Xg[(t / NQK) * NQP + t % NQK];
  return true;
}

template <int K>
__device__ void mixed_load_body(const ElemArgs& args, const int64_t e, double* smem) {
  using L = LoadShape<K>;
  constexpr int P = L::P, p = L::p, Q = L::Q, NQ = L::NQ, NFN = L::NFN, N = L::N, NT = L::NT;
  constexpr int NI = 3 * K * p * p;
  const int tid = threadIdx.x;
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
  double* ut = d; d += N;
  double* r = d; d += N;
  double* U = d; d += 3 * NQ;
  double* Wv = d; d += 3 * NQ;
  double* Dv = d; d += NQ;
  double* xc = d; d += L::NC;
  double* t1 = d; d += L::TMP64;
  double* t2 = d; d += L::TMP64;
  load_element64<K, NT>(args, e, X8, Mc, Vc, Dc, Vo, qx, qw, wf);
  geometry64<K, NT>(Mc, qx, qw, g6, gd, args.status, args.err_elem, e);
  const double alpha = args.alpha[e], beta = args.beta[e];
  const int32_t* ef = args.elem_face + e * 6;
  int bmask = 0;
#pragma unroll
  for (int a = 0; a < 6; ++a) bmask |= (ef[a] < 0 && !args.natural) << a;
  auto is_e = [&](int i) { return i >= NI && ((bmask >> ((i - NI) / NFN)) & 1); };
  const double* coef = args.load + e * (int64_t)N;
  for (int i = tid; i < N; i += NT) ut[i] = coef[i];
  __syncthreads();
  apply_mass64<K, NT>(ut, f, 1.0, g6, Vc, Vo, U, Wv, t1, t2);
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
  double* fs = args.zstore + e * (int64_t)N;
  for (int i = tid; i < N; i += NT) fs[i] = f[i];
  __syncthreads();                               // the FP64 scratch after f_T is free
  const int64_t slot = args.slot ? args.slot[e] : e;
  float* Gi = args.Lstore32 + slot * MT<K>::STORE + MT<K>::LTA + MT<K>::XDA + MT<K>::ZTSA;
  if (!g_inverse<K, NT>(beta, gd, Vo, reinterpret_cast<float*>(smem + L::PREFIX), Gi) && tid == 0)
    set_error(args.status, args.err_elem, HYB_ERR_NOT_SPD, e);
}

template <int K>
__global__ void __launch_bounds__(LoadShape<K>::NT, 8) mixed_load_kernel(ElemArgs args) {
  extern __shared__ double smem[];
  const int64_t li = blockIdx.x;
  if (li >= args.n_list) return;
  mixed_load_body<K>(args, args.elem_list[li], smem);
}

template <int K>
__global__ void __launch_bounds__(LoadShape<K>::NT, 8) mixed_load_kernel_batch(const ElemArgs* probs, const int2* items,
                                                                           int64_t n_items) {
  extern __shared__ double smem[];
  const int64_t li = blockIdx.x;
  if (li >= n_items) return;
  const int2 it = items[li];
  mixed_load_body<K>(probs[it.x], it.y, smem);
}

template <int K>
__global__ void __launch_bounds__(MT<K>::NT, MT<K>::MINB_ASM) element_tiled_kernel(ElemArgs args) {
  extern __shared__ double smem[];
  const int64_t li = blockIdx.x;
  if (li >= args.n_list) return;
  element_tiled_body<K, false>(args, args.elem_list[li], smem, nullptr, nullptr);
}

template <int K>
__global__ void __launch_bounds__(MT<K>::NT, MT<K>::MINB_ASM) element_tiled_kernel_batch(const ElemArgs* probs, const int2* items,
                                                                        int64_t n_items, int colour) {
  extern __shared__ double smem[];
  for (int64_t li = blockIdx.x; li < n_items; li += gridDim.x) {   // persistent when the grid is smaller
    const int2 it = items[li];
    ElemArgs a = probs[it.x];
    a.colour = colour;
    element_tiled_body<K, false>(a, it.y, smem, nullptr, nullptr);
    __syncthreads();
  }
}

template <int K>
__global__ void __launch_bounds__(MT<K>::NT, MT<K>::MINB) recover_tiled_kernel(ElemArgs args, const double* lambda, double* u) {
  extern __shared__ double smem[];
  const int64_t li = blockIdx.x;
  if (li >= args.n_list) return;
  element_tiled_body<K, true>(args, args.elem_list[li], smem, lambda, u);
}

template <int K>
__global__ void __launch_bounds__(MT<K>::NT, MT<K>::MINB) recover_tiled_kernel_batch(const ElemArgs* probs,
                                                                        const double* const* lams, double* const* us,
                                                                        const int2* items, int64_t n_items) {
  extern __shared__ double smem[];
  const int64_t li = blockIdx.x;
  if (li >= n_items) return;
  const int2 it = items[li];
  const ElemArgs a = probs[it.x];
  element_tiled_body<K, true>(a, it.y, smem, lams[it.x], us[it.x]);
}
