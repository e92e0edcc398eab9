// Aggregation multigrid preconditioner for the reduced system, and CG preconditioned by it.
//
// Sec. 4: H = C A^{-1} C^T is spectrally equivalent to a mesh-dependent H^1-type norm of the
// face functions, so an H^1-type algebraic multigrid preconditions it with iteration counts
// that do not grow with the mesh (Sec. 6.1 uses BoomerAMG). The paper does not define the
// multigrid; this one is built for the structured hexahedral mesh:
//  * level 0 is H itself (the face-block CSR of the context); every interior face belongs to
//    the 2 x 2 x 2 block of cells (i / 2, j / 2, l / 2) of its grid position, and all nodes of
//    the faces of a block share one coarse unknown (piecewise-constant tentative prolongation:
//    the constant is the near-null vector of an H^1-type operator);
//  * levels 1.. are structured grids with 27-point operators stored as 27 coefficient arrays
//    ([27][n], offset (dx, dy, dz) at (dx+1) + 3 (dy+1) + 9 (dz+1)), each aggregated 2 x 2 x 2
//    into the next; Galerkin coarse operators A_{l+1} = P^T A_l P are sums of fine entries, formed
//    by gathers in a fixed order (bitwise reproducible); a block without faces gets x = 0;
//  * the smoother is the Chebyshev iteration of a fixed degree for D^{-1} A on
//    [lmax / 30, lmax], lmax = 1.1 x a 12-step power estimate in the D inner product (start
//    s_i = ((7919 i) mod 101) / 101 - 1/2), the same before and after the coarse correction,
//    so the V-cycle is symmetric positive definite; each Chebyshev step is one kernel that
//    multiplies and updates the residual, the direction and the iterate together;
//  * the coarsest level (at most `coarsest` unknowns) is solved with its dense inverse, formed
//    on the device by Gauss-Jordan elimination in one CTA.
// Everything after set-up is a fixed sequence of kernels with device-resident scalars (the
// Chebyshev coefficients are computed on the device from the power estimates), so one PCG
// iteration, V-cycle included, is captured once as a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hyb_internal.h"

namespace hyb {

namespace {

constexpr int kT = 256;            // threads per block
constexpr int kMaxDeg = 4;
constexpr int kVecBlocks = 152 * 8;
constexpr int kPowerSteps = 12;
constexpr double kRatio = 30.0;

// Chebyshev coefficients of one level (device): d_1 = D^-1 r / theta; step k = 1..deg-1:
// d_{k+1} = c1[k] d_k + c2[k] D^-1 r_k
struct Coef {
  double inv_theta;
  double c1[kMaxDeg], c2[kMaxDeg];
  double lam;                      // power estimate of lmax(D^-1 A) (without the margin)
};

struct FaceOp {                    // level 0: the face-block CSR of H
  const int64_t* row_ptr;
  const int32_t* col;
  const double* val;
  int64_t nfaces;
};

// level 0 from the FP32 copy of a mixed context: H_ij / (d_i d_j) rounded to FP32 (d = sqrt of
// the diagonal), every face's column list padded to a multiple of 8 (value 0, column 0), so
// (H v)_i = d_i sum_j Ht_ij (d_j v_j) with the products and row sums in FP32 over an FP32 copy
// of d v that the kernel producing v writes beside it
struct Face32Op {
  const int64_t* fptr;
  const int32_t* col;
  const float* val;
  const double* dsq;
  int64_t nfaces;
};

struct GridOp {                    // levels >= 1: 27-point operator on a bx x by x bz grid
  const double* A;                 // [27][n]
  int bx, by, bz;
  int64_t n;
};

int cuda_status_of(cudaError_t e) {
  if (e == cudaSuccess) return HYB_OK;
  return e == cudaErrorMemoryAllocation ? HYB_ERR_OOM : HYB_ERR_CUDA;
}

__device__ __forceinline__ bool stopped(const int* flags) { return flags && (flags[F_CONV] | flags[F_BRK]); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block sum to thread 0 (fixed order)
__device__ __forceinline__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
#pragma unroll
    for (int k = 0; k < kT / 32; ++k) t += sh[threadIdx.x + 32 * k];
    t = warp_sum(t);
  }
  __syncthreads();
  return t;
}

__device__ __forceinline__ bool last_block(int* ticket) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  return last;
}

// sum of gridDim.x partials part[b * stride + off] by the last block, fixed order
__device__ __forceinline__ double sum_partials(const double* part, int stride, int off, double* sh) {
  double v = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kT) v += __ldcg(part + (int64_t)b * stride + off);
  return block_sum(v, sh);
}

// ---- operator applications: w = (A v)_i for the rows a thread (group) owns, then an epilogue

// Epilogue kinds of the fused Chebyshev kernels (r, x, d: the level's vectors; din the
// direction multiplied, dout the next one):
//   RES:   r = b - A x;           dout = D^-1 r / theta      (start from a nonzero x; x += dout later)
//   STEP:  r -= A din;            dout = c1 din + c2 D^-1 r;  x += (defer ? din : 0) + dout
//   FINAL: r -= A din;            x += (defer ? din : 0)      (residual after pre-smoothing)
//   MATV:  dout = A din           (power iteration, PCG product q = H p with p.q partials)
enum Kind { K_RES = 0, K_STEP = 1, K_FINAL = 2, K_MATV = 3 };

struct Vecs {
  const double* b;
  double* x;
  double* r;
  const double* din;
  double* dout;
  const double* dinv;
  const Coef* coef;
  int k;                   // STEP: step index (1..deg-1)
  int defer;               // x += din still pending
  int* flags;              // skip when the PCG has stopped (null: never)
  const float* x32;        // FP32 level 0: the scaled FP32 copies of x (RES) and din (the others)
  const float* din32;
  float* out32;            // FP32 level 0: where the scaled copy of dout goes (null: none)
  const double* dsq;
  double* partial;         // MATV: per-block partial sums of din . dout (null: none)
  int* ticket;
  double* scal;            // MATV with partials: PCG scalars (alpha = rz / pq)
};

template <int KIND>
__device__ __forceinline__ double epilogue(const Vecs& v, int64_t i, double w) {
  if constexpr (KIND == K_RES) {
    const double r = v.b[i] - w;
    v.r[i] = r;
    const double dn = v.dinv[i] * r * v.coef->inv_theta;
    v.dout[i] = dn;
    if (v.out32) v.out32[i] = (float)(v.dsq[i] * dn);
    return 0.0;
  } else if constexpr (KIND == K_STEP) {
    const double r = v.r[i] - w;
    v.r[i] = r;
    const double dn = fma(v.coef->c1[v.k], v.din[i], v.coef->c2[v.k] * v.dinv[i] * r);
    v.dout[i] = dn;
    if (v.out32) v.out32[i] = (float)(v.dsq[i] * dn);
    v.x[i] += v.defer ? v.din[i] + dn : dn;
    return 0.0;
  } else if constexpr (KIND == K_FINAL) {
    v.r[i] -= w;
    if (v.defer) v.x[i] += v.din[i];
    return 0.0;
  } else {
    v.dout[i] = w;
    return v.din[i] * w;
  }
}

template <int KIND>
__device__ __forceinline__ void finish_matv(const Vecs& v, double dot, double* sh) {
  if (KIND != K_MATV || !v.partial) return;
  dot = block_sum(dot, sh);
  if (threadIdx.x == 0) v.partial[blockIdx.x] = dot;
  if (last_block(v.ticket)) {
    const double s = sum_partials(v.partial, 1, 0, sh);
    if (threadIdx.x == 0) {
      v.scal[S_PQ] = s;
      if (!(s > 0.0) || !(s < INFINITY)) {
        v.scal[S_ALPHA] = 0.0;
        v.flags[F_BRK] = 1;
      } else {
        v.scal[S_ALPHA] = v.scal[S_RZ] / s;
      }
      *v.ticket = 0;
    }
  }
}

// level 0: four lanes per face, NFN row sums per lane, shuffle-combined; lane g finishes the
// rows m = g, g + 4, ...
template <int NFN, int KIND>
__global__ void __launch_bounds__(kT) face_kernel(FaceOp op, Vecs v) {
  __shared__ double sh[kT];
  if (stopped(v.flags)) return;
  const int lane = threadIdx.x & 31, gl = lane & 3;
  const int64_t f = ((int64_t)blockIdx.x * kT + threadIdx.x) >> 2;
  const double* src = KIND == K_RES ? v.x : v.din;
  double acc[NFN];
#pragma unroll
  for (int m = 0; m < NFN; ++m) acc[m] = 0.0;
  if (f < op.nfaces) {
    const int64_t lo = op.row_ptr[f * NFN];
    const int len = (int)(op.row_ptr[f * NFN + 1] - lo);
    for (int t = gl; t < len; t += 4) {
      const double s = __ldg(src + op.col[lo + t]);
#pragma unroll
      for (int m = 0; m < NFN; ++m) acc[m] = fma(__ldcs(op.val + lo + (int64_t)m * len + t), s, acc[m]);
    }
  }
#pragma unroll
  for (int m = 0; m < NFN; ++m) {
    acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], 1);
    acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], 2);
  }
  double dot = 0.0;
  if (f < op.nfaces) {
#pragma unroll
    for (int m = 0; m < NFN; ++m)
      if ((m & 3) == gl) dot += epilogue<KIND>(v, f * NFN + m, acc[m]);
  }
  finish_matv<KIND>(v, dot, sh);
}

// level 0 from the FP32 copy: eight lanes per face over the padded column list (one aligned
// 32-byte sector of values per row and step), FP32 row sums combined across the lanes, widened
// and scaled by d_i; lane g finishes the rows m = g, g + 8, ...
template <int NFN, int KIND>
__global__ void __launch_bounds__(kT) face32_kernel(Face32Op op, Vecs v) {
  __shared__ double sh[kT];
  if (stopped(v.flags)) return;
  const int lane = threadIdx.x & 31, gl = lane & 7;
  const int64_t f = ((int64_t)blockIdx.x * kT + threadIdx.x) >> 3;
  const float* src = KIND == K_RES ? v.x32 : v.din32;
  float acc[NFN];
#pragma unroll
  for (int m = 0; m < NFN; ++m) acc[m] = 0.0f;
  if (f < op.nfaces) {
    const int64_t c0 = op.fptr[f];
    const int len = (int)(op.fptr[f + 1] - c0);
    const float* vb = op.val + (int64_t)NFN * c0;
#pragma unroll 2
    for (int t = gl; t < len; t += 8) {
      const float s = __ldg(src + __ldcs(op.col + c0 + t));
#pragma unroll
      for (int m = 0; m < NFN; ++m) acc[m] = fmaf(__ldcs(vb + (int64_t)m * len + t), s, acc[m]);
    }
  }
#pragma unroll
  for (int m = 0; m < NFN; ++m) {
    acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], 1);
    acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], 2);
    acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], 4);
  }
  double dot = 0.0;
  if (f < op.nfaces) {
#pragma unroll
    for (int m = 0; m < NFN; ++m)
      if ((m & 7) == gl) {
        const int64_t i = f * NFN + m;
        dot += epilogue<KIND>(v, i, (double)acc[m] * op.dsq[i]);
      }
  }
  finish_matv<KIND>(v, dot, sh);
}

__device__ __forceinline__ void grid_xyz(int64_t i, int bx, int by, int& x, int& y, int& z) {
  x = (int)(i % bx);
  y = (int)((i / bx) % by);
  z = (int)(i / ((int64_t)bx * by));
}

template <int KIND>
__global__ void __launch_bounds__(kT) grid_kernel(GridOp op, Vecs v) {
  __shared__ double sh[kT];
  if (stopped(v.flags)) return;
  const double* src = KIND == K_RES ? v.x : v.din;
  double dot = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < op.n; i += (int64_t)gridDim.x * kT) {
    int x, y, z;
    grid_xyz(i, op.bx, op.by, x, y, z);
    double w = 0.0;
#pragma unroll
    for (int o = 0; o < 27; ++o) {
      const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
      const int xx = x + dx, yy = y + dy, zz = z + dz;
      if (xx < 0 || yy < 0 || zz < 0 || xx >= op.bx || yy >= op.by || zz >= op.bz) continue;
      w = fma(op.A[(int64_t)o * op.n + i], src[i + dx + (int64_t)op.bx * (dy + (int64_t)op.by * dz)], w);
    }
    dot += epilogue<KIND>(v, i, w);
  }
  finish_matv<KIND>(v, dot, sh);
}

// pre-smoothing from x = 0: r = b, d_1 = D^-1 b / theta, x = d_1
__global__ void __launch_bounds__(kT) start_zero_kernel(int64_t n, Vecs v) {
  if (stopped(v.flags)) return;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    const double b = v.b[i];
    const double d = v.dinv[i] * b * v.coef->inv_theta;
    v.r[i] = b;
    v.dout[i] = d;
    v.x[i] = d;
    if (v.out32) v.out32[i] = (float)(v.dsq[i] * d);
  }
}

// x += d (a deferred update with nothing left to fuse it into: degree 1)
__global__ void __launch_bounds__(kT) add_kernel(int64_t n, double* x, const double* d, const int* flags) {
  if (stopped(flags)) return;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) x[i] += d[i];
}

// restriction from the faces: bc[J] = sum over the faces of block J of their nodes' r
__global__ void __launch_bounds__(kT) restrict_faces_kernel(int64_t nblk, int nfn, const int32_t* blk_ptr,
                                                            const int32_t* blk_faces, const double* r, double* bc,
                                                            const int* flags) {
  if (stopped(flags)) return;
  for (int64_t J = (int64_t)blockIdx.x * kT + threadIdx.x; J < nblk; J += (int64_t)gridDim.x * kT) {
    double s = 0.0;
    for (int t = blk_ptr[J]; t < blk_ptr[J + 1]; ++t) {
      const int64_t f = blk_faces[t];
      for (int m = 0; m < nfn; ++m) s += r[f * nfn + m];
    }
    bc[J] = s;
  }
}

// restriction between grids: bc[J] = sum of r over the (up to 8) children of J
__global__ void __launch_bounds__(kT) restrict_grid_kernel(int fx, int fy, int fz, int cx, int cy, int cz,
                                                           const double* r, double* bc, const int* flags) {
  if (stopped(flags)) return;
  const int64_t nc = (int64_t)cx * cy * cz;
  for (int64_t J = (int64_t)blockIdx.x * kT + threadIdx.x; J < nc; J += (int64_t)gridDim.x * kT) {
    int x, y, z;
    grid_xyz(J, cx, cy, x, y, z);
    double s = 0.0;
    for (int c = 0; c < 8; ++c) {
      const int xx = 2 * x + (c & 1), yy = 2 * y + ((c >> 1) & 1), zz = 2 * z + (c >> 2);
      if (xx < fx && yy < fy && zz < fz) s += r[xx + (int64_t)fx * (yy + (int64_t)fy * zz)];
    }
    bc[J] = s;
  }
}

__global__ void __launch_bounds__(kT) prolong_faces_kernel(int64_t n, int nfn, const int32_t* face_blk,
                                                           const double* xc, double* x, const int* flags,
                                                           float* x32, const double* dsq) {
  if (stopped(flags)) return;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    const double xi = x[i] + xc[face_blk[i / nfn]];
    x[i] = xi;
    if (x32) x32[i] = (float)(dsq[i] * xi);     // the post-smoothing's first product reads it
  }
}

__global__ void __launch_bounds__(kT) prolong_grid_kernel(int fx, int fy, int fz, int cx, int cy, const double* xc,
                                                          double* x, const int* flags) {
  if (stopped(flags)) return;
  const int64_t n = (int64_t)fx * fy * fz;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    int xx, yy, zz;
    grid_xyz(i, fx, fy, xx, yy, zz);
    x[i] += xc[(xx / 2) + (int64_t)cx * ((yy / 2) + (int64_t)cy * (zz / 2))];
  }
}

// coarsest level: x = Ainv b (Ainv symmetric, read by columns: coalesced)
__global__ void __launch_bounds__(kT) dense_apply_kernel(int n, const double* Ainv, const double* b, double* x,
                                                         const int* flags) {
  if (stopped(flags)) return;
  for (int i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s = fma(Ainv[(int64_t)j * n + i], b[j], s);
    x[i] = s;
  }
}

// ---- set-up kernels

// level 1 from H: one warp per block J sums every entry of the face rows of J into the offset
// of its column face's block (per-lane accumulators, then a fixed-order lane sum)
template <int NFN>
__global__ void __launch_bounds__(128) face_coarse_kernel(FaceOp op, int bx, int by, int bz, const int32_t* blk_ptr,
                                                          const int32_t* blk_faces, const int32_t* face_blk,
                                                          double* A1) {
  __shared__ double acc[4][27][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n = (int64_t)bx * by * bz;
  const int64_t J = (int64_t)blockIdx.x * 4 + w;
  if (J >= n) return;                     // whole warps: no block-wide barrier below
  for (int o = 0; o < 27; ++o) acc[w][o][lane] = 0.0;
  int jx, jy, jz;
  grid_xyz(J, bx, by, jx, jy, jz);
  for (int t = blk_ptr[J]; t < blk_ptr[J + 1]; ++t) {
    const int64_t f = blk_faces[t];
    const int64_t lo = op.row_ptr[f * NFN];
    const int len = (int)(op.row_ptr[f * NFN + 1] - lo);
    for (int e = lane; e < NFN * len; e += 32) {
      const int64_t g = op.col[lo + e % len] / NFN;
      int gx, gy, gz;
      grid_xyz(face_blk[g], bx, by, gx, gy, gz);
      const int dx = gx - jx, dy = gy - jy, dz = gz - jz;
      if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) continue;   // not a neighbour block
      acc[w][(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)][lane] += op.val[lo + e];
    }
  }
  __syncwarp();
  if (lane < 27) {
    double s = 0.0;
    for (int l = 0; l < 32; ++l) s += acc[w][lane][l];
    if (lane == 13 && blk_ptr[J] == blk_ptr[J + 1]) s = 1.0;   // no faces: x = 0
    A1[(int64_t)lane * n + J] = s;
  }
}

// level l + 1 from level l: entry (J, oc) sums A_l[o][I] over the children I of J and the
// offsets o whose neighbour I + d(o) lies in block J + d(oc)
__global__ void __launch_bounds__(kT) grid_coarse_kernel(GridOp fine, int cx, int cy, int cz, double* Ac) {
  const int64_t nc = (int64_t)cx * cy * cz;
  for (int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x; t < 27 * nc; t += (int64_t)gridDim.x * kT) {
    const int oc = (int)(t / nc);
    const int64_t J = t % nc;
    int x, y, z;
    grid_xyz(J, cx, cy, x, y, z);
    const int tx = x + oc % 3 - 1, ty = y + (oc / 3) % 3 - 1, tz = z + oc / 9 - 1;
    double s = 0.0;
    for (int c = 0; c < 8; ++c) {
      const int ix = 2 * x + (c & 1), iy = 2 * y + ((c >> 1) & 1), iz = 2 * z + (c >> 2);
      if (ix >= fine.bx || iy >= fine.by || iz >= fine.bz) continue;
      const int64_t I = ix + (int64_t)fine.bx * (iy + (int64_t)fine.by * iz);
      for (int o = 0; o < 27; ++o) {
        const int nx = ix + o % 3 - 1, ny = iy + (o / 3) % 3 - 1, nz = iz + o / 9 - 1;
        if (nx < 0 || ny < 0 || nz < 0 || nx >= fine.bx || ny >= fine.by || nz >= fine.bz) continue;
        if ((nx >> 1) == tx && (ny >> 1) == ty && (nz >> 1) == tz) s += fine.A[(int64_t)o * fine.n + I];
      }
    }
    Ac[t] = s;
  }
}

__global__ void __launch_bounds__(kT) face_dinv_kernel(int64_t n, const int64_t* row_ptr, const int32_t* col,
                                                       const double* val, double* dinv) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    double d = 0.0;
    for (int64_t t = row_ptr[i]; t < row_ptr[i + 1]; ++t)
      if (col[t] == i) d = val[t];
    dinv[i] = 1.0 / d;
  }
}

__global__ void __launch_bounds__(kT) grid_dinv_kernel(int64_t n, const double* A, double* dinv) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    dinv[i] = 1.0 / A[13 * n + i];
}

__global__ void __launch_bounds__(kT) start_vector_kernel(int64_t n, double* v, float* v32, const double* dsq) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    const double s = (double)((7919 * i) % 101) / 101.0 - 0.5;
    v[i] = s;
    if (v32) v32[i] = (float)(dsq[i] * s);
  }
}

// power step after w = A v: lam = v.w / v.Dv, u = D^-1 w, |u|^2 (partials, then the last block)
__global__ void __launch_bounds__(kT) power_reduce_kernel(int64_t n, const double* v, const double* w,
                                                          const double* dinv, double* u, double* partial,
                                                          int* ticket, double* out /* lam, 1/|u| */) {
  __shared__ double sh[kT];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    const double vi = v[i], wi = w[i], di = dinv[i];
    const double ui = wi * di;
    u[i] = ui;
    a = fma(vi, wi, a);
    b = fma(vi, vi / di, b);
    c = fma(ui, ui, c);
  }
  a = block_sum(a, sh);
  b = block_sum(b, sh);
  c = block_sum(c, sh);
  if (threadIdx.x == 0) {
    partial[3 * blockIdx.x] = a;
    partial[3 * blockIdx.x + 1] = b;
    partial[3 * blockIdx.x + 2] = c;
  }
  if (last_block(ticket)) {
    const double sa = sum_partials(partial, 3, 0, sh);
    const double sb = sum_partials(partial, 3, 1, sh);
    const double sc = sum_partials(partial, 3, 2, sh);
    if (threadIdx.x == 0) {
      out[0] = sa / sb;
      out[1] = 1.0 / sqrt(sc);
      *ticket = 0;
    }
  }
}

__global__ void __launch_bounds__(kT) scale_kernel(int64_t n, const double* u, const double* s, double* v, float* v32,
                                                   const double* dsq) {
  const double f = s[1];
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    const double vi = u[i] * f;
    v[i] = vi;
    if (v32) v32[i] = (float)(dsq[i] * vi);
  }
}

// Chebyshev coefficients on [lmax / ratio, lmax], lmax = 1.1 lam
__global__ void coef_kernel(const double* lam, int degree, Coef* c) {
  const double lmax = 1.1 * lam[0];
  const double a = lmax / kRatio, b = lmax;
  const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
  double rho = 1.0 / sigma;
  c->inv_theta = 1.0 / theta;
  c->lam = lam[0];
  for (int k = 0; k < kMaxDeg; ++k) c->c1[k] = c->c2[k] = 0.0;
  for (int k = 1; k < degree; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    c->c1[k] = rn * rho;
    c->c2[k] = 2.0 * rn / delta;
    rho = rn;
  }
}

// dense matrix of the coarsest level (row-major n x n)
__global__ void __launch_bounds__(kT) dense_from_grid_kernel(GridOp op, double* M) {
  const int64_t n = op.n;
  for (int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x; t < n * n; t += (int64_t)gridDim.x * kT) M[t] = 0.0;
}
__global__ void __launch_bounds__(kT) dense_fill_grid_kernel(GridOp op, double* M) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < op.n; i += (int64_t)gridDim.x * kT) {
    int x, y, z;
    grid_xyz(i, op.bx, op.by, x, y, z);
    for (int o = 0; o < 27; ++o) {
      const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
      const int xx = x + dx, yy = y + dy, zz = z + dz;
      if (xx < 0 || yy < 0 || zz < 0 || xx >= op.bx || yy >= op.by || zz >= op.bz) continue;
      M[i * op.n + xx + (int64_t)op.bx * (yy + (int64_t)op.by * zz)] = op.A[(int64_t)o * op.n + i];
    }
  }
}
__global__ void __launch_bounds__(kT) dense_fill_csr_kernel(int64_t n, const int64_t* row_ptr, const int32_t* col,
                                                            const double* val, double* M) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    for (int64_t t = row_ptr[i]; t < row_ptr[i + 1]; ++t) M[i * n + col[t]] = val[t];
}

// in-place Gauss-Jordan inverse of an SPD matrix (no pivoting), one CTA of 1024 threads;
// cr: 2n scratch for the pivot column and row
__global__ void __launch_bounds__(1024) gauss_jordan_kernel(int n, double* M, double* cr, int* status) {
  for (int k = 0; k < n; ++k) {
    const double piv = M[(int64_t)k * n + k];
    if (!(piv > 0.0) || !(piv < INFINITY)) {
      if (threadIdx.x == 0) *status = HYB_ERR_NOT_SPD;
      return;                                   // uniform: every thread read the same pivot
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      cr[i] = M[(int64_t)i * n + k];
      cr[n + i] = M[(int64_t)k * n + i];
    }
    __syncthreads();
    const double ip = 1.0 / piv;
    for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) {
      const int i = (int)(t / n), j = (int)(t % n);
      double v;
      if (i == k && j == k) v = ip;
      else if (i == k) v = cr[n + j] * ip;
      else if (j == k) v = -cr[i] * ip;
      else v = fma(-cr[i] * ip, cr[n + j], M[t]);
      M[t] = v;
    }
    __syncthreads();
  }
}

// ---- PCG kernels (device scalars; the layout solve_impl reads)

// x = 0, r = b, rr0 = r.r
__global__ void __launch_bounds__(kT) pcg0_init_kernel(int64_t n, const double* b, double* x, double* r,
                                                       double* partial, int* flags, double* scal) {
  __shared__ double sh[kT];
  double rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    const double bi = b[i];
    x[i] = 0.0;
    r[i] = bi;
    rr = fma(bi, bi, rr);
  }
  rr = block_sum(rr, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = rr;
  if (last_block(&flags[F_TICKET])) {
    const double s = sum_partials(partial, 1, 0, sh);
    if (threadIdx.x == 0) {
      scal[S_RR0] = s;
      scal[S_RR] = s;
      scal[S_BETA] = 0.0;
      flags[F_IT] = 0;
      flags[F_CONV] = (s == 0.0);
      flags[F_BRK] = 0;
      flags[F_TICKET] = 0;
    }
  }
}

// rz = r.z; first: p = z, else beta = rz / rz_old, p = z + beta p (two passes: the dot first)
__global__ void __launch_bounds__(kT) pcg_rz_kernel(int64_t n, const double* r, const double* z, double* partial,
                                                    int* flags, double* scal, int first) {
  __shared__ double sh[kT];
  if (stopped(flags)) return;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) s = fma(r[i], z[i], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  if (last_block(&flags[F_TICKET])) {
    const double t = sum_partials(partial, 1, 0, sh);
    if (threadIdx.x == 0) {
      scal[S_BETA] = first ? 0.0 : t / scal[S_RZ];
      scal[S_RZ] = t;
      if (!(t > 0.0) || !(t < INFINITY)) flags[F_BRK] = 1;
      flags[F_TICKET] = 0;
    }
  }
}

__global__ void __launch_bounds__(kT) pcg_dir_kernel(int64_t n, const double* z, double* p, const int* flags,
                                                     const double* scal, float* p32, const double* dsq) {
  if (stopped(flags)) return;
  const double beta = scal[S_BETA];
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    const double pi = fma(beta, p[i], z[i]);
    p[i] = pi;
    if (p32) p32[i] = (float)(dsq[i] * pi);
  }
}

// x += alpha p, r -= alpha q, rr = r.r; iteration count and convergence
__global__ void __launch_bounds__(kT) pcg_upd_kernel(int64_t n, double* x, double* r, const double* p,
                                                     const double* q, double* partial, int* flags, double* scal,
                                                     double rtol2) {
  __shared__ double sh[kT];
  if (stopped(flags)) return;
  const double alpha = scal[S_ALPHA];
  double rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    rr = fma(ri, ri, rr);
  }
  rr = block_sum(rr, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = rr;
  if (last_block(&flags[F_TICKET])) {
    const double s = sum_partials(partial, 1, 0, sh);
    if (threadIdx.x == 0) {
      scal[S_RR] = s;
      flags[F_IT] += 1;
      if (s <= rtol2 * scal[S_RR0]) flags[F_CONV] = 1;
      if (!(s < INFINITY)) flags[F_BRK] = 1;
      flags[F_TICKET] = 0;
    }
  }
}

unsigned grid_for(int64_t n) {
  const int64_t b = (n + kT - 1) / kT;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, kVecBlocks));
}

}  // namespace

struct Amg {
  int nfn = 0, degree = 2, coarsest = 512;
  int64_t nfaces = 0, n0 = 0;
  FaceOp H{};
  // level-0 products from the FP32 copy (mixed contexts): the operator, scaled FP32 copies of
  // the vectors the products gather (x of the V-cycle, the two directions, the PCG direction,
  // the power iterate), and the operator the current numeric set-up was made for
  bool use32 = false, numeric32 = false;
  Face32Op H32{};
  float *x32 = nullptr, *d32a = nullptr, *d32b = nullptr, *p32 = nullptr, *pv32 = nullptr;
  // aggregation of the faces (level 0 -> 1)
  int32_t* face_blk = nullptr;     // [nfaces]
  int32_t* blk_ptr = nullptr;      // [n1 + 1]
  int32_t* blk_faces = nullptr;    // [nfaces]
  struct Level {
    int bx = 0, by = 0, bz = 0;
    int64_t n = 0;
    double* A = nullptr;           // levels >= 1
    double *dinv = nullptr, *b = nullptr, *x = nullptr, *r = nullptr, *d0 = nullptr, *d1 = nullptr;
    Coef* coef = nullptr;
  };
  std::vector<Level> lev;          // lev[0]: faces; lev.back(): coarsest (dense inverse)
  double* Ainv = nullptr;
  double* gj_scratch = nullptr;
  // set-up and PCG scratch
  double* partial = nullptr;       // >= 3 * (max grid) doubles
  int* ticket = nullptr;
  double* pscal = nullptr;         // power iteration outputs per level: lam, 1/|u|
  double *pv = nullptr, *pw = nullptr, *pu = nullptr;
  // PCG vectors
  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  int* status = nullptr;
  std::vector<void*> allocs;
  cudaGraphExec_t iter_exec = nullptr;
  cudaGraph_t iter_graph = nullptr;
  const double* iter_b = nullptr;
  double* iter_x = nullptr;
  double iter_rtol = -1.0;
  int* iter_flags = nullptr;
  double* iter_scal = nullptr;
};

namespace {

template <class T>
int amg_alloc(Amg* a, T** p, size_t n) {
  if (n == 0) n = 1;
  if (cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T)) != cudaSuccess) return HYB_ERR_OOM;
  a->allocs.push_back(*p);
  return HYB_OK;
}

int64_t max_face_blocks(const Amg* a) { return (a->nfaces * 4 + kT - 1) / kT; }

// y-style launches of the fused level kernels
template <int KIND>
cudaError_t level_op(const Amg* a, int l, const Vecs& v, cudaStream_t s) {
  const Amg::Level& L = a->lev[l];
  if (l == 0 && a->use32) {
    const unsigned g = (unsigned)((a->nfaces * 8 + kT - 1) / kT);
    switch (a->nfn) {
      case 1: face32_kernel<1, KIND><<<g, kT, 0, s>>>(a->H32, v); break;
      case 4: face32_kernel<4, KIND><<<g, kT, 0, s>>>(a->H32, v); break;
      case 9: face32_kernel<9, KIND><<<g, kT, 0, s>>>(a->H32, v); break;
      case 16: face32_kernel<16, KIND><<<g, kT, 0, s>>>(a->H32, v); break;
      default: return cudaErrorInvalidValue;
    }
  } else if (l == 0) {
    const unsigned g = (unsigned)max_face_blocks(a);
    switch (a->nfn) {
      case 1: face_kernel<1, KIND><<<g, kT, 0, s>>>(a->H, v); break;
      case 4: face_kernel<4, KIND><<<g, kT, 0, s>>>(a->H, v); break;
      case 9: face_kernel<9, KIND><<<g, kT, 0, s>>>(a->H, v); break;
      case 16: face_kernel<16, KIND><<<g, kT, 0, s>>>(a->H, v); break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    GridOp op{L.A, L.bx, L.by, L.bz, L.n};
    grid_kernel<KIND><<<grid_for(L.n), kT, 0, s>>>(op, v);
  }
  return cudaGetLastError();
}

// Chebyshev smoothing on level l of A x = b (b, x: the level's vectors or the caller's at
// level 0). zero: x starts at 0 (pre-smoothing; ends with the residual in L.r); otherwise x
// is updated in place (post-smoothing).
cudaError_t smooth(const Amg* a, int l, const double* b, double* x, bool zero, int* flags, cudaStream_t s) {
  const Amg::Level& L = a->lev[l];
  Vecs v{};
  v.b = b;
  v.x = x;
  v.r = L.r;
  v.dinv = L.dinv;
  v.coef = L.coef;
  v.flags = flags;
  double* d[2] = {L.d0, L.d1};
  float* d32[2] = {nullptr, nullptr};
  if (l == 0 && a->use32) {
    d32[0] = a->d32a;
    d32[1] = a->d32b;
    v.x32 = a->x32;
    v.dsq = a->H32.dsq;
  }
  int cur = 0;
  cudaError_t e;
  bool defer;
  if (zero) {
    v.dout = d[cur];
    v.out32 = d32[cur];
    start_zero_kernel<<<grid_for(L.n), kT, 0, s>>>(L.n, v);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    defer = false;
  } else {
    v.dout = d[cur];
    v.out32 = d32[cur];
    if ((e = level_op<K_RES>(a, l, v, s)) != cudaSuccess) return e;
    defer = true;
  }
  for (int k = 1; k < a->degree; ++k) {
    v.din = d[cur];
    v.din32 = d32[cur];
    v.dout = d[cur ^ 1];
    v.out32 = d32[cur ^ 1];
    v.k = k;
    v.defer = defer;
    if ((e = level_op<K_STEP>(a, l, v, s)) != cudaSuccess) return e;
    defer = false;
    cur ^= 1;
  }
  if (zero) {
    v.din = d[cur];
    v.din32 = d32[cur];
    v.out32 = nullptr;
    v.defer = defer;
    return level_op<K_FINAL>(a, l, v, s);
  }
  if (defer) {
    add_kernel<<<grid_for(L.n), kT, 0, s>>>(L.n, x, d[cur], flags);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

cudaError_t vcycle(const Amg* a, int l, const double* b, double* x, int* flags, cudaStream_t s) {
  const int last = (int)a->lev.size() - 1;
  const Amg::Level& L = a->lev[l];
  cudaError_t e;
  if (l == last) {
    dense_apply_kernel<<<grid_for(L.n), kT, 0, s>>>((int)L.n, a->Ainv, b, x, flags);
    return cudaGetLastError();
  }
  if ((e = smooth(a, l, b, x, true, flags, s)) != cudaSuccess) return e;
  const Amg::Level& C = a->lev[l + 1];
  if (l == 0)
    restrict_faces_kernel<<<grid_for(C.n), kT, 0, s>>>(C.n, a->nfn, a->blk_ptr, a->blk_faces, L.r, C.b, flags);
  else
    restrict_grid_kernel<<<grid_for(C.n), kT, 0, s>>>(L.bx, L.by, L.bz, C.bx, C.by, C.bz, L.r, C.b, flags);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = vcycle(a, l + 1, C.b, C.x, flags, s)) != cudaSuccess) return e;
  if (l == 0)
    prolong_faces_kernel<<<grid_for(L.n), kT, 0, s>>>(L.n, a->nfn, a->face_blk, C.x, x, flags,
                                                      a->use32 ? a->x32 : nullptr, a->H32.dsq);
  else
    prolong_grid_kernel<<<grid_for(L.n), kT, 0, s>>>(L.bx, L.by, L.bz, C.bx, C.by, C.x, x, flags);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return smooth(a, l, b, x, false, flags, s);
}

}  // namespace

void amg_free(Amg* a) {
  if (!a) return;
  if (a->iter_exec) cudaGraphExecDestroy(a->iter_exec);
  if (a->iter_graph) cudaGraphDestroy(a->iter_graph);
  for (void* p : a->allocs) cudaFree(p);
  delete a;
}

// Structure: aggregates, level grids and buffers (once per context).
int amg_create(int nx, int ny, int nz, int nfn, int degree, int coarsest, const int64_t* row_ptr,
               const int32_t* col, const double* val, const int64_t n_iface_axis[3], Amg** out) {
  *out = nullptr;
  if (degree < 1 || degree > kMaxDeg || coarsest < 1 || coarsest > 4096) return HYB_ERR_INVALID_ARG;
  if (nfn != 1 && nfn != 4 && nfn != 9 && nfn != 16) return HYB_ERR_INVALID_ARG;
  Amg* a = new Amg();
  a->nfn = nfn;
  a->degree = degree;
  a->coarsest = coarsest;
  a->nfaces = n_iface_axis[0] + n_iface_axis[1] + n_iface_axis[2];
  a->n0 = a->nfaces * nfn;
  a->H = FaceOp{row_ptr, col, val, a->nfaces};
  int st;
  auto fail = [&](int s) { amg_free(a); return s; };
  Amg::Level L0;
  L0.n = a->n0;
  a->lev.push_back(L0);
  if (a->n0 > coarsest) {
    // aggregates of the faces: the cell block of each face's grid position
    const int dims[3] = {nx, ny, nz};
    const int B[3] = {(nx + 1) / 2, (ny + 1) / 2, (nz + 1) / 2};
    const int64_t n1 = (int64_t)B[0] * B[1] * B[2];
    std::vector<int32_t> fb(a->nfaces), cnt(n1 + 1, 0);
    int64_t f = 0;
    for (int d = 0; d < 3; ++d) {
      const int da = d == 0 ? ny : nx, db = d == 2 ? ny : nz;
      for (int b = 0; b < db; ++b)
        for (int aa = 0; aa < da; ++aa)
          for (int pl = 1; pl < dims[d]; ++pl, ++f) {
            int pos[3];
            pos[d] = pl;
            pos[d == 0 ? 1 : 0] = aa;
            pos[d == 2 ? 1 : 2] = b;
            fb[f] = (pos[0] / 2) + B[0] * ((pos[1] / 2) + B[1] * (pos[2] / 2));
            ++cnt[fb[f] + 1];
          }
    }
    if (f != a->nfaces) return fail(HYB_ERR_INVALID_ARG);
    for (int64_t J = 0; J < n1; ++J) cnt[J + 1] += cnt[J];
    std::vector<int32_t> bf(a->nfaces), pos(cnt.begin(), cnt.end() - 1);
    for (int64_t g = 0; g < a->nfaces; ++g) bf[pos[fb[g]]++] = (int32_t)g;
    if ((st = amg_alloc(a, &a->face_blk, a->nfaces)) || (st = amg_alloc(a, &a->blk_ptr, n1 + 1)) ||
        (st = amg_alloc(a, &a->blk_faces, a->nfaces)))
      return fail(st);
    if (cudaMemcpy(a->face_blk, fb.data(), fb.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(a->blk_ptr, cnt.data(), cnt.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(a->blk_faces, bf.data(), bf.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(HYB_ERR_CUDA);
    int g[3] = {B[0], B[1], B[2]};
    for (;;) {
      Amg::Level L;
      L.bx = g[0];
      L.by = g[1];
      L.bz = g[2];
      L.n = (int64_t)g[0] * g[1] * g[2];
      a->lev.push_back(L);
      if (L.n <= coarsest || (g[0] == 1 && g[1] == 1 && g[2] == 1)) break;
      for (int t = 0; t < 3; ++t) g[t] = (g[t] + 1) / 2;
    }
  }
  const int nl = (int)a->lev.size();
  for (int l = 0; l < nl; ++l) {
    Amg::Level& L = a->lev[l];
    if (l > 0 && (st = amg_alloc(a, &L.A, 27 * L.n))) return fail(st);
    if ((st = amg_alloc(a, &L.dinv, L.n)) || (st = amg_alloc(a, &L.r, L.n)) || (st = amg_alloc(a, &L.d0, L.n)) ||
        (st = amg_alloc(a, &L.d1, L.n)) || (st = amg_alloc(a, &L.coef, 1)))
      return fail(st);
    if (l > 0 && ((st = amg_alloc(a, &L.b, L.n)) || (st = amg_alloc(a, &L.x, L.n)))) return fail(st);
  }
  const int64_t nL = a->lev.back().n;
  const int64_t maxg = std::max<int64_t>(max_face_blocks(a), kVecBlocks);
  if ((st = amg_alloc(a, &a->Ainv, nL * nL)) || (st = amg_alloc(a, &a->gj_scratch, 2 * nL)) ||
      (st = amg_alloc(a, &a->partial, 3 * maxg)) || (st = amg_alloc(a, &a->ticket, 1)) ||
      (st = amg_alloc(a, &a->pscal, 2 * nl)) || (st = amg_alloc(a, &a->pv, a->n0)) ||
      (st = amg_alloc(a, &a->pw, a->n0)) || (st = amg_alloc(a, &a->pu, a->n0)) || (st = amg_alloc(a, &a->z, a->n0)) ||
      (st = amg_alloc(a, &a->status, 1)))
    return fail(st);
  if (cudaMemset(a->ticket, 0, sizeof(int)) != cudaSuccess) return fail(HYB_ERR_CUDA);
  *out = a;
  return HYB_OK;
}

// Level-0 products from a mixed context's FP32 copy (on) or from the FP64 values (off).
// Returns 1 when the choice changed (the numeric set-up must run again: the power estimate of
// level 0 depends on the operator), 0 when not, or a negative status.
int amg_set_fp32(Amg* a, bool on, const float* val32, const int32_t* col32, const int64_t* fptr32, const double* dsq) {
  if (on) {
    if (!val32 || !col32 || !fptr32 || !dsq) return HYB_ERR_INVALID_ARG;
    int st;
    if (!a->x32 && ((st = amg_alloc(a, &a->x32, a->n0)) || (st = amg_alloc(a, &a->d32a, a->n0)) ||
                    (st = amg_alloc(a, &a->d32b, a->n0)) || (st = amg_alloc(a, &a->p32, a->n0)) ||
                    (st = amg_alloc(a, &a->pv32, a->n0))))
      return st;
    a->H32 = Face32Op{fptr32, col32, val32, dsq, a->nfaces};
  }
  const bool changed = a->use32 != on;
  a->use32 = on;
  return changed ? 1 : 0;
}

// Numeric set-up after an assembly: coarse operators, diagonals, power estimates and
// Chebyshev coefficients, the coarsest inverse. No host synchronisation but the final status.
int amg_numeric(Amg* a, cudaStream_t s) {
  cudaError_t e;
  const int nl = (int)a->lev.size();
  face_dinv_kernel<<<grid_for(a->n0), kT, 0, s>>>(a->n0, a->H.row_ptr, a->H.col, a->H.val, a->lev[0].dinv);
  if (nl > 1) {
    Amg::Level& L1 = a->lev[1];
    const unsigned g = (unsigned)((L1.n + 3) / 4);
    switch (a->nfn) {
      case 1: face_coarse_kernel<1><<<g, 128, 0, s>>>(a->H, L1.bx, L1.by, L1.bz, a->blk_ptr, a->blk_faces, a->face_blk, L1.A); break;
      case 4: face_coarse_kernel<4><<<g, 128, 0, s>>>(a->H, L1.bx, L1.by, L1.bz, a->blk_ptr, a->blk_faces, a->face_blk, L1.A); break;
      case 9: face_coarse_kernel<9><<<g, 128, 0, s>>>(a->H, L1.bx, L1.by, L1.bz, a->blk_ptr, a->blk_faces, a->face_blk, L1.A); break;
      case 16: face_coarse_kernel<16><<<g, 128, 0, s>>>(a->H, L1.bx, L1.by, L1.bz, a->blk_ptr, a->blk_faces, a->face_blk, L1.A); break;
    }
    for (int l = 1; l + 1 < nl; ++l) {
      const Amg::Level &F = a->lev[l], &C = a->lev[l + 1];
      grid_coarse_kernel<<<grid_for(27 * C.n), kT, 0, s>>>(GridOp{F.A, F.bx, F.by, F.bz, F.n}, C.bx, C.by, C.bz, C.A);
    }
    for (int l = 1; l < nl; ++l)
      grid_dinv_kernel<<<grid_for(a->lev[l].n), kT, 0, s>>>(a->lev[l].n, a->lev[l].A, a->lev[l].dinv);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status_of(e);
  // power estimates of every smoothed level
  for (int l = 0; l + 1 < nl; ++l) {
    const Amg::Level& L = a->lev[l];
    float* pv32 = l == 0 && a->use32 ? a->pv32 : nullptr;
    start_vector_kernel<<<grid_for(L.n), kT, 0, s>>>(L.n, a->pv, pv32, a->H32.dsq);
    for (int it = 0; it < kPowerSteps; ++it) {
      Vecs v{};
      v.din = a->pv;
      v.din32 = pv32;
      v.dout = a->pw;
      if ((e = level_op<K_MATV>(a, l, v, s)) != cudaSuccess) return cuda_status_of(e);
      power_reduce_kernel<<<grid_for(L.n), kT, 0, s>>>(L.n, a->pv, a->pw, L.dinv, a->pu, a->partial, a->ticket,
                                                       a->pscal + 2 * l);
      scale_kernel<<<grid_for(L.n), kT, 0, s>>>(L.n, a->pu, a->pscal + 2 * l, a->pv, pv32, a->H32.dsq);
    }
    coef_kernel<<<1, 1, 0, s>>>(a->pscal + 2 * l, a->degree, L.coef);
  }
  // coarsest: dense inverse
  const Amg::Level& C = a->lev.back();
  const int nL = (int)C.n;
  if (cudaMemsetAsync(a->status, 0, sizeof(int), s) != cudaSuccess) return HYB_ERR_CUDA;
  if (nl > 1) {
    GridOp op{C.A, C.bx, C.by, C.bz, C.n};
    dense_from_grid_kernel<<<grid_for((int64_t)nL * nL), kT, 0, s>>>(op, a->Ainv);
    dense_fill_grid_kernel<<<grid_for(nL), kT, 0, s>>>(op, a->Ainv);
  } else {
    if (cudaMemsetAsync(a->Ainv, 0, sizeof(double) * nL * nL, s) != cudaSuccess) return HYB_ERR_CUDA;
    dense_fill_csr_kernel<<<grid_for(nL), kT, 0, s>>>(nL, a->H.row_ptr, a->H.col, a->H.val, a->Ainv);
  }
  gauss_jordan_kernel<<<1, 1024, 0, s>>>(nL, a->Ainv, a->gj_scratch, a->status);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status_of(e);
  int hst = 0;
  if (cudaMemcpyAsync(&hst, a->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return HYB_ERR_CUDA;
  // a new operator: the captured iteration is stale
  if (a->iter_exec) {
    cudaGraphExecDestroy(a->iter_exec);
    a->iter_exec = nullptr;
  }
  if (a->iter_graph) {
    cudaGraphDestroy(a->iter_graph);
    a->iter_graph = nullptr;
  }
  return hst;
}

// z = M^{-1} r (one V-cycle; r, z: n0 doubles on the device)
int amg_apply(Amg* a, const double* r, double* z, cudaStream_t s) {
  cudaError_t e = vcycle(a, 0, r, z, nullptr, s);
  return e == cudaSuccess ? HYB_OK : cuda_status_of(e);
}

double amg_lmax(const Amg* a, int level) {
  if (level < 0 || level + 1 >= (int)a->lev.size()) return 0.0;
  Coef c{};
  if (cudaMemcpy(&c, a->lev[level].coef, sizeof(Coef), cudaMemcpyDeviceToHost) != cudaSuccess) return -1.0;
  return c.lam;
}

int amg_levels(const Amg* a, int64_t* sizes, int cap) {
  const int nl = (int)a->lev.size();
  for (int l = 0; l < nl && l < cap; ++l) sizes[l] = a->lev[l].n;
  return nl;
}

// CG preconditioned by one V-cycle per iteration, x = 0 at the start, stop at ||r|| <= rtol
// ||b|| (as the diagonal PCG). pvec: r, p, q work vectors (n0 each); flags / scal: the
// context's PCG scalars. One iteration is captured as a CUDA graph on first use and replayed
// in chunks; the host reads the flags between chunks.
int amg_pcg(Amg* a, const double* b, double rtol, int maxit, double* x, double* r, double* p, double* q,
            int* flags, double* scal, double* partial_unused, cudaStream_t s, int* iters, double* rel_res) {
  (void)partial_unused;
  const int64_t n = a->n0;
  cudaError_t e = cudaMemsetAsync(flags, 0, 4 * sizeof(int), s);
  if (e != cudaSuccess) return cuda_status_of(e);
  pcg0_init_kernel<<<grid_for(n), kT, 0, s>>>(n, b, x, r, a->partial, flags, scal);
  if ((e = vcycle(a, 0, r, a->z, flags, s)) != cudaSuccess) return cuda_status_of(e);
  pcg_rz_kernel<<<grid_for(n), kT, 0, s>>>(n, r, a->z, a->partial, flags, scal, 1);
  float* p32 = a->use32 ? a->p32 : nullptr;
  pcg_dir_kernel<<<grid_for(n), kT, 0, s>>>(n, a->z, p, flags, scal, p32, a->H32.dsq);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status_of(e);
  const double rtol2 = rtol * rtol;
  if (a->iter_exec && (a->iter_b != b || a->iter_x != x || a->iter_rtol != rtol2 || a->iter_flags != flags ||
                       a->iter_scal != scal)) {
    cudaGraphExecDestroy(a->iter_exec);
    cudaGraphDestroy(a->iter_graph);
    a->iter_exec = nullptr;
    a->iter_graph = nullptr;
  }
  if (!a->iter_exec) {
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return HYB_ERR_CUDA;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      Vecs v{};
      v.din = p;
      v.din32 = p32;
      v.dout = q;
      v.flags = flags;
      v.partial = a->partial;
      v.ticket = &flags[F_TICKET];
      v.scal = scal;
      cudaError_t ek = level_op<K_MATV>(a, 0, v, cs);                     // q = H p, alpha
      if (ek == cudaSuccess) {
        pcg_upd_kernel<<<grid_for(n), kT, 0, cs>>>(n, x, r, p, q, a->partial, flags, scal, rtol2);
        ek = vcycle(a, 0, r, a->z, flags, cs);
      }
      if (ek == cudaSuccess) {
        pcg_rz_kernel<<<grid_for(n), kT, 0, cs>>>(n, r, a->z, a->partial, flags, scal, 0);
        pcg_dir_kernel<<<grid_for(n), kT, 0, cs>>>(n, a->z, p, flags, scal, p32, a->H32.dsq);
        ek = cudaGetLastError();
      }
      e = cudaStreamEndCapture(cs, &a->iter_graph);
      if (e == cudaSuccess) e = ek;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&a->iter_exec, a->iter_graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_status_of(e);
    a->iter_b = b;
    a->iter_x = x;
    a->iter_rtol = rtol2;
    a->iter_flags = flags;
    a->iter_scal = scal;
  }
  int hf[4] = {0, 0, 0, 0};
  int done = 0;
  const int chunk = 8;
  for (;;) {
    e = cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status_of(e);
    done = hf[F_IT];
    if (hf[F_CONV] || hf[F_BRK] || done >= maxit) break;
    const int m = std::min(chunk, maxit - done);
    for (int t = 0; t < m && e == cudaSuccess; ++t) e = cudaGraphLaunch(a->iter_exec, s);
    if (e != cudaSuccess) return cuda_status_of(e);
  }
  double hs[4] = {0};
  e = cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status_of(e);
  if (iters) *iters = done;
  if (rel_res) *rel_res = hs[S_RR0] > 0.0 ? std::sqrt(hs[S_RR] / hs[S_RR0]) : 0.0;
  if (hf[F_BRK]) return HYB_ERR_BREAKDOWN;
  if (!hf[F_CONV]) return HYB_ERR_NOT_CONVERGED;
  return HYB_OK;
}

}  // namespace hyb
