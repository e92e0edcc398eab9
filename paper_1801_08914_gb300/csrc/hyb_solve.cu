// Reduced solve: diagonal-preconditioned conjugate gradients on the CSR face
// system (H of eq. 2.4, or the static-condensation matrix S of eq. 3.2),
// stopping when ||r||_2 <= rtol ||r_0||_2 (the paper's criterion, Sec. 6.1).
//
// Every scalar of the iteration lives in device memory: the SpMV kernel
// forms p^T H p, the vector kernel forms r^T z and r^T r, and the last block
// of each grid (ticket counter) finishes the reduction in a fixed block
// order, so results are bitwise reproducible. A converged / breakdown flag
// makes every later kernel of the chunk a no-op, so the host launches
// iterations in chunks and reads the flags once per chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "hyb_internal.h"

namespace hyb {
namespace {

// scal[] slots
enum { S_RZ = 0, S_RR0 = 1, S_RR = 2, S_ALPHA = 3, S_BETA = 4, S_PQ = 5 };
// flags[] slots
enum { F_IT = 0, F_CONV = 1, F_BRK = 2, F_TICKET = 3 };

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum to thread 0 (256 threads).
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (kThreads / 32) ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  return t;
}

// Ticket: returns true in exactly one (the last) block. Thread 0 wrote this block's partial;
// it alone fences before taking a ticket, so the last block sees every partial in L2.
__device__ __forceinline__ bool last_block(int* ticket, int nblocks) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const int t = atomicAdd(ticket, 1);
    last = (t == nblocks - 1);
  }
  __syncthreads();
  return last;
}

// Sum of `count` partials (stride `stride`, offset `off`) by the whole block, fixed order:
// thread t adds entries t, t + 256, ... then the block tree. Result valid in thread 0.
__device__ __forceinline__ double sum_partials(const double* part, int count, int stride, int off, double* sh) {
  double v = 0.0;
  for (int b = threadIdx.x; b < count; b += kThreads) v += __ldcg(part + (int64_t)b * stride + off);
  return block_sum(v, sh);
}

__global__ void diag_inv_kernel(PcgArgs a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int64_t t = a.row_ptr[i]; t < a.row_ptr[i + 1]; ++t)
      if (a.col[t] == i) d = a.val[t];
    a.dinv[i] = 1.0 / d;
  }
}

// x = 0, r = b, p = z = D^{-1} r; rz = r^T z, rr0 = r^T r
__global__ void pcg_init_kernel(PcgArgs a) {
  __shared__ double sh[32];
  double rz = 0.0, rr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double r = a.b[i];
    const double z = a.dinv[i] * r;
    a.x[i] = 0.0;
    a.r[i] = r;
    a.p[i] = z;
    rz = fma(r, z, rz);
    rr = fma(r, r, rr);
  }
  rz = block_sum(rz, sh);
  rr = block_sum(rr, sh);
  if (threadIdx.x == 0) {
    a.partial[2 * blockIdx.x] = rz;
    a.partial[2 * blockIdx.x + 1] = rr;
  }
  if (last_block(&a.flags[F_TICKET], gridDim.x)) {
    const double s0 = sum_partials(a.partial, gridDim.x, 2, 0, sh);
    const double s1 = sum_partials(a.partial, gridDim.x, 2, 1, sh);
    if (threadIdx.x == 0) {
      a.scal[S_RZ] = s0;
      a.scal[S_RR0] = s1;
      a.scal[S_RR] = s1;
      a.flags[F_IT] = 0;
      a.flags[F_CONV] = (s1 == 0.0);
      a.flags[F_BRK] = 0;
      a.flags[F_TICKET] = 0;
    }
  }
}

// q = H p, fused with the partial p^T q; last block: alpha = rz / p^T q.
// The CSR pattern built at set-up gives every row of a face the same column list and
// stores the (k+1)^2 rows of a face back to back. W lanes take one face: each lane
// loads a column index and the gathered p_j once and uses them for all NFN rows,
// so the index stream costs 4 / NFN bytes per nonzero instead of 4.
template <int NFN, int W>
__device__ __forceinline__ void spmv_face_body(const PcgArgs& a, int vb, int nvb, double* sh) {
  if (a.flags[F_CONV] | a.flags[F_BRK]) return;
  constexpr int FPW = 32 / W;                              // faces per warp per step
  const int64_t warp = (vb * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)nvb * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int sub = lane / W, gl = lane % W;
  const int64_t nfaces = a.n / NFN;
  double pq = 0.0;
  for (int64_t base = warp * FPW; base < nfaces; base += nwarps * FPW) {
    const int64_t f = base + sub;
    double acc[NFN];
#pragma unroll
    for (int m = 0; m < NFN; ++m) acc[m] = 0.0;
    if (f < nfaces) {
      const int64_t r0 = f * NFN;
      const int64_t lo = a.row_ptr[r0];
      const int len = (int)(a.row_ptr[r0 + 1] - lo);
#pragma unroll 4
      for (int t = gl; t < len; t += W) {
        const double pj = a.p[a.col[lo + t]];
#pragma unroll
        for (int m = 0; m < NFN; ++m) acc[m] = fma(a.val[lo + (int64_t)m * len + t], pj, acc[m]);
      }
    }
#pragma unroll
    for (int m = 0; m < NFN; ++m) {
#pragma unroll
      for (int o = W / 2; o > 0; o >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o, W);
    }
    if (f < nfaces) {
#pragma unroll
      for (int m = 0; m < NFN; ++m) {
        if (gl == m % W) {
          const int64_t i = f * NFN + m;
          a.q[i] = acc[m];
          pq = fma(a.p[i], acc[m], pq);
        }
      }
    }
  }
  pq = block_sum(pq, sh);
  if (threadIdx.x == 0) a.partial[vb] = pq;
  if (last_block(&a.flags[F_TICKET], nvb)) {
    const double s = sum_partials(a.partial, nvb, 1, 0, sh);
    if (threadIdx.x == 0) {
      a.scal[S_PQ] = s;
      if (!(s > 0.0) || !(s < INFINITY)) a.flags[F_BRK] = 1;
      else a.scal[S_ALPHA] = a.scal[S_RZ] / s;
      a.flags[F_TICKET] = 0;
    }
  }
}

template <int NFN, int W>
__global__ void __launch_bounds__(kThreads) spmv_face_kernel(PcgArgs a) {
  __shared__ double sh[32];
  spmv_face_body<NFN, W>(a, blockIdx.x, gridDim.x, sh);
}

// x += alpha p, r -= alpha q, z = D^{-1} r (into q); rz, rr; last block: beta, convergence.
// Four elements per thread per step with all loads issued first: the kernel is bound by
// memory latency, so independent loads in flight matter more than occupancy.
constexpr int kUnroll = 4;
__device__ __forceinline__ void pcg_update_body(const PcgArgs& a, double rtol2, int vb, int nvb, double* sh) {
  if (a.flags[F_CONV] | a.flags[F_BRK]) return;
  const double alpha = a.scal[S_ALPHA];
  double rz = 0.0, rr = 0.0;
  const int64_t stride = (int64_t)nvb * blockDim.x;
  for (int64_t base = vb * (int64_t)blockDim.x + threadIdx.x; base < a.n; base += kUnroll * stride) {
    double xv[kUnroll], pv[kUnroll], rv[kUnroll], qv[kUnroll], dv[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t i = base + u * stride;
      if (i < a.n) { xv[u] = a.x[i]; pv[u] = a.p[i]; rv[u] = a.r[i]; qv[u] = a.q[i]; dv[u] = a.dinv[i]; }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t i = base + u * stride;
      if (i < a.n) {
        a.x[i] = fma(alpha, pv[u], xv[u]);
        const double r = fma(-alpha, qv[u], rv[u]);
        a.r[i] = r;
        const double z = dv[u] * r;
        a.q[i] = z;
        rz = fma(r, z, rz);
        rr = fma(r, r, rr);
      }
    }
  }
  rz = block_sum(rz, sh);
  rr = block_sum(rr, sh);
  if (threadIdx.x == 0) {
    a.partial[2 * vb] = rz;
    a.partial[2 * vb + 1] = rr;
  }
  if (last_block(&a.flags[F_TICKET], nvb)) {
    const double s0 = sum_partials(a.partial, nvb, 2, 0, sh);
    const double s1 = sum_partials(a.partial, nvb, 2, 1, sh);
    if (threadIdx.x == 0) {
      a.scal[S_BETA] = s0 / a.scal[S_RZ];
      a.scal[S_RZ] = s0;
      a.scal[S_RR] = s1;
      a.flags[F_IT] += 1;
      if (s1 <= rtol2 * a.scal[S_RR0]) a.flags[F_CONV] = 1;
      if (!(s1 < INFINITY)) a.flags[F_BRK] = 1;
      a.flags[F_TICKET] = 0;
    }
  }
}

__global__ void __launch_bounds__(kThreads) pcg_update_kernel(PcgArgs a, double rtol2) {
  __shared__ double sh[32];
  pcg_update_body(a, rtol2, blockIdx.x, gridDim.x, sh);
}

// p = z + beta p
__device__ __forceinline__ void pcg_direction_body(const PcgArgs& a, int vb, int nvb) {
  if (a.flags[F_CONV] | a.flags[F_BRK]) return;
  const double beta = a.scal[S_BETA];
  const int64_t stride = (int64_t)nvb * blockDim.x;
  for (int64_t base = vb * (int64_t)blockDim.x + threadIdx.x; base < a.n; base += kUnroll * stride) {
    double pv[kUnroll], zv[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t i = base + u * stride;
      if (i < a.n) { pv[u] = a.p[i]; zv[u] = a.q[i]; }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t i = base + u * stride;
      if (i < a.n) a.p[i] = fma(beta, pv[u], zv[u]);
    }
  }
}

__global__ void __launch_bounds__(kThreads) pcg_direction_kernel(PcgArgs a) {
  pcg_direction_body(a, blockIdx.x, gridDim.x);
}

// ---- batched forms: block b works for problem blk_prob[b] as its block b - blk_first[that problem]
// of blk_count[that problem]; every problem keeps its own scalars, tickets and flags.
__global__ void __launch_bounds__(kThreads) spmv_batch_kernel(const PcgArgs* probs, const int32_t* blk_prob,
                                                              const int32_t* blk_first, const int32_t* blk_count) {
  __shared__ double sh[32];
  const int pb = blk_prob[blockIdx.x];
  const PcgArgs a = probs[pb];
  const int vb = blockIdx.x - blk_first[pb], nvb = blk_count[pb];
  switch (a.nfn) {
    case 1: spmv_face_body<1, 4>(a, vb, nvb, sh); break;
    case 4: spmv_face_body<4, 2>(a, vb, nvb, sh); break;
    case 9: spmv_face_body<9, 2>(a, vb, nvb, sh); break;
    default: spmv_face_body<16, 2>(a, vb, nvb, sh); break;
  }
}
__global__ void __launch_bounds__(kThreads) update_batch_kernel(const PcgArgs* probs, const int32_t* blk_prob,
                                                                const int32_t* blk_first, const int32_t* blk_count,
                                                                double rtol2) {
  __shared__ double sh[32];
  const int pb = blk_prob[blockIdx.x];
  const PcgArgs a = probs[pb];
  pcg_update_body(a, rtol2, blockIdx.x - blk_first[pb], blk_count[pb], sh);
}
__global__ void __launch_bounds__(kThreads) direction_batch_kernel(const PcgArgs* probs, const int32_t* blk_prob,
                                                                   const int32_t* blk_first, const int32_t* blk_count) {
  const int pb = blk_prob[blockIdx.x];
  const PcgArgs a = probs[pb];
  pcg_direction_body(a, blockIdx.x - blk_first[pb], blk_count[pb]);
}

__global__ void expand_cols_kernel(const int64_t* row_ptr, const int32_t* adj, const int32_t* adj_count,
                                   int64_t n_faces, int nfn, int32_t* col) {
  for (int64_t f = blockIdx.x; f < n_faces; f += gridDim.x) {
    const int cnt = adj_count[f];
    const int len = cnt * nfn;
    for (int m = 0; m < nfn; ++m) {
      const int64_t base = row_ptr[f * nfn + m];
      for (int t = threadIdx.x; t < len; t += blockDim.x)
        col[base + t] = adj[f * 11 + t / nfn] * nfn + t % nfn;
    }
  }
}

}  // namespace

cudaError_t launch_expand_cols(const int64_t* row_ptr, const int32_t* adj, const int32_t* adj_count,
                               int64_t n_faces, int nfn, int32_t* col, cudaStream_t s, Prof* prof) {
  if (n_faces == 0) return cudaSuccess;
  const unsigned nb = (unsigned)(n_faces < 65536 ? n_faces : 65536);
  const int tok = prof_begin(prof, HYB_K_SETUP, s);
  expand_cols_kernel<<<nb, 128, 0, s>>>(row_ptr, adj, adj_count, n_faces, nfn, col);
  prof_end(prof, tok, s);
  return cudaGetLastError();
}

cudaError_t pcg_init(const PcgArgs& a, cudaStream_t s, Prof* prof) {
  cudaError_t err = cudaMemsetAsync(a.flags, 0, 4 * sizeof(int), s);
  if (err != cudaSuccess) return err;
  int tok = prof_begin(prof, HYB_K_PCG_VECTOR, s);
  diag_inv_kernel<<<a.nblocks, kThreads, 0, s>>>(a);
  prof_end(prof, tok, s);
  tok = prof_begin(prof, HYB_K_PCG_VECTOR, s);
  pcg_init_kernel<<<a.nblocks / 4, kThreads, 0, s>>>(a);
  prof_end(prof, tok, s);
  return cudaGetLastError();
}

cudaError_t pcg_iterations(const PcgArgs& a, int count, double rtol, cudaStream_t s, Prof* prof) {
  for (int it = 0; it < count; ++it) {
    int tok = prof_begin(prof, HYB_K_SPMV, s);
    // FP64 is the scarce unit on this part (about 1.2 TFLOP/s): 2 lanes per face keep the
    // cross-lane FP64 reduction to one step per row while the 16 consecutive bytes a face
    // gets per load instruction complete their 32-byte sector on the next iteration.
    const int nbs = a.nblocks * 5 / 8, nbv = a.nblocks / 4;
    switch (a.nfn) {
      case 1: spmv_face_kernel<1, 4><<<nbs, kThreads, 0, s>>>(a); break;
      case 4: spmv_face_kernel<4, 2><<<nbs, kThreads, 0, s>>>(a); break;
      case 9: spmv_face_kernel<9, 2><<<nbs, kThreads, 0, s>>>(a); break;
      case 16: spmv_face_kernel<16, 2><<<nbs, kThreads, 0, s>>>(a); break;
      default: return cudaErrorInvalidValue;
    }
    prof_end(prof, tok, s);
    tok = prof_begin(prof, HYB_K_PCG_VECTOR, s);
    pcg_update_kernel<<<nbv, kThreads, 0, s>>>(a, rtol * rtol);
    prof_end(prof, tok, s);
    tok = prof_begin(prof, HYB_K_PCG_VECTOR, s);
    pcg_direction_kernel<<<nbv, kThreads, 0, s>>>(a);
    prof_end(prof, tok, s);
  }
  return cudaGetLastError();
}

cudaError_t pcg_iterations_batch(const PcgBatch& b, int count, double rtol, cudaStream_t s, Prof* prof) {
  for (int it = 0; it < count; ++it) {
    int tok = prof_begin(prof, HYB_K_SPMV, s);
    spmv_batch_kernel<<<b.n_spmv, kThreads, 0, s>>>(b.probs, b.spmv_prob, b.spmv_first, b.spmv_count);
    prof_end(prof, tok, s);
    tok = prof_begin(prof, HYB_K_PCG_VECTOR, s);
    update_batch_kernel<<<b.n_vec, kThreads, 0, s>>>(b.probs, b.vec_prob, b.vec_first, b.vec_count, rtol * rtol);
    prof_end(prof, tok, s);
    tok = prof_begin(prof, HYB_K_PCG_VECTOR, s);
    direction_batch_kernel<<<b.n_vec, kThreads, 0, s>>>(b.probs, b.vec_prob, b.vec_first, b.vec_count);
    prof_end(prof, tok, s);
  }
  return cudaGetLastError();
}

}  // namespace hyb

// ---------------------------------------------------------------------------
// Allocation-free PCG (hyb_pcg_solve_noalloc). The paper has no counterpart:
// this serves callers that cannot allocate device memory. All solver
// scratch (r, p, q, D^{-1}, block partials, scalars, flags) lives in one
// file-scope device array sized for kNoAllocMaxRows rows; each GPU that loads
// the library holds it until the process exits.
namespace hyb {
namespace {

constexpr int64_t kNoAllocMaxRows = int64_t(1) << 19;     // 524,288 rows
constexpr int kNoAllocBlocks = 152 * 8;
constexpr int64_t kNoAllocDoubles = 4 * kNoAllocMaxRows + 2 * kNoAllocBlocks + 8 + 2;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = static_cast<double*>(ptr);
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace hyb

extern "C" int hyb_pcg_solve_noalloc(const int64_t* row_ptr, const int32_t* col, const double* val,
                                     const double* b, double* x, int64_t n, int rows_per_face, double rtol,
                                     int maxit, void* cuda_stream, int* iters, double* rel_res) {
  using namespace hyb;
  if (!row_ptr || !col || !val || !b || !x) return HYB_ERR_INVALID_ARG;
  if (n < 0 || n > kNoAllocMaxRows || maxit < 0 || !(rtol >= 0.0)) return HYB_ERR_INVALID_ARG;
  if (rows_per_face != 1 && rows_per_face != 4 && rows_per_face != 9 && rows_per_face != 16) return HYB_ERR_INVALID_ARG;
  if (n % rows_per_face != 0) return HYB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  double* base = nullptr;
  cudaError_t e = noalloc_scratch(&base);
  if (e != cudaSuccess) return HYB_ERR_CUDA;
  PcgArgs a{};
  a.n = n;
  a.row_ptr = row_ptr;
  a.col = col;
  a.val = val;
  a.b = b;
  a.x = x;
  a.r = base;
  a.p = base + kNoAllocMaxRows;
  a.q = base + 2 * kNoAllocMaxRows;
  a.dinv = base + 3 * kNoAllocMaxRows;
  a.partial = base + 4 * kNoAllocMaxRows;
  a.scal = a.partial + 2 * kNoAllocBlocks;
  a.flags = reinterpret_cast<int*>(a.scal + 8);
  a.nblocks = kNoAllocBlocks;
  a.nfn = rows_per_face;
  e = pcg_init(a, s, nullptr);                 // clears the flags word, writes every vector it reads
  if (e != cudaSuccess) return HYB_ERR_CUDA;
  int hf[4] = {0, 0, 0, 0};
  double hs[3] = {0, 0, 0};
  int done = 0;
  for (;;) {
    e = cudaMemcpyAsync(hf, a.flags, sizeof(hf), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return HYB_ERR_CUDA;
    done = hf[0];
    if (hf[1] || hf[2] || done >= maxit) break;
    e = pcg_iterations(a, std::min(32, maxit - done), rtol, s, nullptr);
    if (e != cudaSuccess) return HYB_ERR_CUDA;
  }
  e = cudaMemcpyAsync(hs, a.scal, sizeof(hs), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return HYB_ERR_CUDA;
  if (iters) *iters = done;
  if (rel_res) *rel_res = hs[1] > 0.0 ? std::sqrt(hs[2] / hs[1]) : 0.0;
  if (hf[2]) return HYB_ERR_BREAKDOWN;
  if (!hf[1]) return HYB_ERR_NOT_CONVERGED;
  return HYB_OK;
}
