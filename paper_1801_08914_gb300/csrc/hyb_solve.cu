// Reduced solve: diagonal-preconditioned conjugate gradients on the CSR face
// system (H of eq. 2.4, or the static-condensation matrix S of eq. 3.2),
// stopping when ||r||_2 <= rtol ||r_0||_2 (the paper's criterion, Sec. 6.1).
//
// Two forms of the same iteration. The fused form (default) runs 64 iterations in one
// cooperative launch with two grid barriers per iteration (pcg_fused_kernel; a team of
// blocks per problem in the batch form). The three-launch form runs an SpMV kernel that forms
// p^T H p and two vector kernels that form r^T z and r^T r; the last block of each grid
// (ticket counter) finishes the reduction. Every scalar lives in device memory and every
// reduction sums per-block partials in a fixed block order, so results are bitwise
// reproducible. A converged / breakdown flag makes later work of a chunk a no-op, so the
// host launches iterations in chunks and reads the flags once per chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>

#include "hyb_internal.h"

namespace hyb {
namespace {

constexpr int kThreads = 256;

// A problem takes no further iterations once converged, broken down or (maxit > 0) at maxit.
__device__ __forceinline__ bool pcg_stopped(const PcgArgs& a) {
  return (a.flags[F_CONV] | a.flags[F_BRK]) || (a.maxit > 0 && a.flags[F_IT] >= a.maxit);
}

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

// Block-wide sum to thread 0 through shared memory (sh: kThreads doubles): the values are
// stored, then warp 0 adds 8 of them per lane and finishes with one shuffle tree. Far fewer
// FP64 instructions than a shuffle tree in every warp, which matters where the FP64 pipe is
// the bound and every warp instruction occupies it whatever its active lanes.
__device__ __forceinline__ double block_sum_smem(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
#pragma unroll
    for (int k = 0; k < kThreads / 32; ++k) t += sh[threadIdx.x + 32 * k];
    t = warp_sum(t);
  }
  __syncthreads();
  return t;
}

// Row sums of a face shared by W lanes (each lane holds partial sums of the NFN rows).
// Where W divides NFN they reduce-scatter: at each of the log2(W) levels a lane keeps half of
// its current values, sends the other half to its partner and adds what it receives, so lane
// gl ends with the full sums of NFN / W rows, acc[j] being row scatter_row(j, gl), after
// NFN (1 - 1/W) adds instead of NFN log2(W); otherwise every lane reduces every row.
// Row sums per lane padded up to a multiple of W, so that the reduce-scatter applies to any
// number of rows per face (9 rows on 4 lanes: 12 sums, the last 3 always zero).
template <int NFN, int W>
__host__ __device__ constexpr int padded_rows() { return (NFN + W - 1) / W * W; }

template <int NFN, int W>
__device__ __forceinline__ int scatter_row(int j, int gl) {
  int row = j, S = NFN;
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) {
    if (gl & o) row += S / 2;
    S >>= 1;
  }
  return row;
}

template <int NFN, int W, typename T = double>
__device__ __forceinline__ void face_reduce(T (&acc)[NFN], int gl) {
  if constexpr (NFN % W == 0) {
#pragma unroll
    for (int o = W / 2, S = NFN; o > 0; o >>= 1, S >>= 1) {
      const bool hi = gl & o;
#pragma unroll
      for (int j = 0; j < S / 2; ++j) {
        const T keep = hi ? acc[j + S / 2] : acc[j];
        const T send = hi ? acc[j] : acc[j + S / 2];
        acc[j] = keep + __shfl_xor_sync(0xffffffffu, send, o, W);
      }
    }
  } else {
#pragma unroll
    for (int m = 0; m < NFN; ++m) {
#pragma unroll
      for (int o = W / 2; o > 0; o >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o, W);
    }
  }
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


__device__ __forceinline__ void diag_inv_body(const PcgArgs& a, int vb, int nvb) {
  for (int64_t i = vb * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)nvb * blockDim.x) {
    double d = 0.0;
    for (int64_t t = a.row_ptr[i]; t < a.row_ptr[i + 1]; ++t)
      if (a.col[t] == i) d = a.val[t];
    a.dinv[i] = 1.0 / d;
  }
}

// x = 0, r = b, p = z = D^{-1} r; rz = r^T z, rr0 = r^T r (blocks vb of nvb)
__device__ __forceinline__ void pcg_init_body(const PcgArgs& a, int vb, int nvb, double* sh) {
  double rz = 0.0, rr = 0.0;
  for (int64_t i = vb * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)nvb * blockDim.x) {
    const double r = a.b[i];
    const double z = a.dinv[i] * r;
    a.x[i] = 0.0;
    a.r[i] = r;
    a.p[i] = z;
    if (a.z) a.z[i] = z;
    if (a.z32) a.z32[i] = (float)(z * a.dsq[i]);
    rz = fma(r, z, rz);
    rr = fma(r, r, rr);
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
      a.scal[S_RZ] = s0;
      a.scal[S_RR0] = s1;
      a.scal[S_RR] = s1;
      a.scal[S_BETA] = 0.0;
      a.flags[F_IT] = 0;
      a.flags[F_CONV] = (s1 == 0.0);
      a.flags[F_BRK] = 0;
      a.flags[F_TICKET] = 0;
    }
  }
}

__global__ void diag_inv_kernel(PcgArgs a) { diag_inv_body(a, blockIdx.x, gridDim.x); }

__global__ void pcg_init_kernel(PcgArgs a) {
  __shared__ double sh[32];
  pcg_init_body(a, blockIdx.x, gridDim.x, sh);
}

__global__ void diag_inv_batch_kernel(const PcgArgs* probs, const int32_t* blk_prob, const int32_t* blk_first,
                                      const int32_t* blk_count) {
  const int pb = blk_prob[blockIdx.x];
  diag_inv_body(probs[pb], blockIdx.x - blk_first[pb], blk_count[pb]);
}

__global__ void pcg_init_batch_kernel(const PcgArgs* probs, const int32_t* blk_prob, const int32_t* blk_first,
                                      const int32_t* blk_count) {
  __shared__ double sh[32];
  const int pb = blk_prob[blockIdx.x];
  const PcgArgs a = probs[pb];
  pcg_init_body(a, blockIdx.x - blk_first[pb], blk_count[pb], sh);
}

// The WHILE condition of the batched step's PCG loop: 1 while any problem still iterates.
__global__ void pcg_continue_kernel(const PcgArgs* probs, int nprob, cudaGraphConditionalHandle handle) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  int mine = 0;
  for (int p = threadIdx.x; p < nprob; p += blockDim.x) {
    const PcgArgs& a = probs[p];
    const int* f = a.flags;
    if (!(f[F_CONV] | f[F_BRK]) && !(a.maxit > 0 && f[F_IT] >= a.maxit)) mine = 1;
  }
  if (mine) any = 1;                          // benign race: every writer stores 1
  __syncthreads();
  if (threadIdx.x == 0) cudaGraphSetConditional(handle, any ? 1u : 0u);
}

// q = H p, fused with the partial p^T q; last block: alpha = rz / p^T q.
// The CSR pattern built at set-up gives every row of a face the same column list and
// stores the (k+1)^2 rows of a face back to back. W lanes take one face: each lane
// loads a column index and the gathered p_j once and uses them for all NFN rows,
// so the index stream costs 4 / NFN bytes per nonzero instead of 4.
template <int NFN, int W>
__device__ __forceinline__ void spmv_face_body(const PcgArgs& a, int vb, int nvb, double* sh) {
  if (pcg_stopped(a)) return;
  constexpr int FPW = 32 / W;                              // faces per warp per step
  const int64_t warp = (vb * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)nvb * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int sub = lane / W, gl = lane % W;
  const int64_t nfaces = a.n / NFN;
  double pq = 0.0;
  constexpr int NP = padded_rows<NFN, W>();
  for (int64_t base = warp * FPW; base < nfaces; base += nwarps * FPW) {
    const int64_t f = base + sub;
    double acc[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) acc[m] = 0.0;
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
    face_reduce<NP, W>(acc, gl);
    if (f < nfaces) {
      if constexpr (NP % W == 0) {
#pragma unroll
        for (int j = 0; j < NP / W; ++j) {
          const int row = scatter_row<NP, W>(j, gl);
          if (row >= NFN) continue;
          const int64_t i = f * NFN + row;
          a.q[i] = acc[j];
          pq = fma(a.p[i], acc[j], pq);
        }
      } else {
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
  }
  pq = block_sum_smem(pq, sh);
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
  __shared__ double sh[kThreads];
  spmv_face_body<NFN, W>(a, blockIdx.x, gridDim.x, sh);
}

// x += alpha p, r -= alpha q, z = D^{-1} r (into q); rz, rr; last block: beta, convergence.
// Four elements per thread per step with all loads issued first: the kernel is bound by
// memory latency, so independent loads in flight matter more than occupancy.
constexpr int kUnroll = 4;

__device__ __forceinline__ void pcg_update_body(const PcgArgs& a, double rtol2, int vb, int nvb, double* sh) {
  if (pcg_stopped(a)) return;
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
  if (pcg_stopped(a)) return;
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

// ---- fused iterations: one cooperative launch runs up to `count` iterations.
//
// Grid-wide synchronisation is a monotonic arrival counter (64-bit, zeroed before every
// launch, so a team may change size between launches): barrier number B of the launch
// completes when the counter reaches (B + 1) * (blocks in the team). Before
// arriving, thread 0 of each block stores the block's partial sums in one of two buffers
// (alternating with B); after the barrier every block sums all partials itself in block order,
// so every block obtains bitwise the same totals without a serial reduction step. A buffer is
// rewritten two barriers later, after every block has passed the barrier in between and so
// has finished reading it. Waits are bounded: a block that waits longer than a second sets
// flags[F_BRK] = 2, and every block leaves at its next barrier.
constexpr unsigned long long kBarrierNs = 1000000000ull;  // a barrier gives up after 1 s
constexpr long long kBarrierSpins = 1ll << 26;            // and after this many polls in any case

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Every thread of every block calls this; thread 0 has already stored the block's partials.
// Returns false in all threads of the block if the wait ran out (here or in another block).
// The arrival is a release add and the poll an acquire load (gpu scope): after
// __syncthreads the block's earlier stores are ordered before thread 0's release, and the
// acquire that observes the final count orders every other block's stores before this
// block's later loads (the second __syncthreads extends that to all its threads).
__device__ __forceinline__ bool grid_barrier(unsigned long long* count, unsigned long long target, int* flags) {
  __shared__ int brk;
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(count), "l"(1ull) : "memory");
    long long spins = 0;
    const unsigned long long t0 = global_ns();
    while ((long long)(ld_acquire(count) - target) < 0) {
      if (++spins > kBarrierSpins || global_ns() - t0 > kBarrierNs) {
        atomicExch(&flags[F_BRK], 2);
        break;
      }
      if ((spins & 1023) == 0 && ld_relaxed(&flags[F_BRK]) == 2) break;   // another block gave up
      __nanosleep(20);
    }
    brk = ld_relaxed(&flags[F_BRK]) == 2;
  }
  __syncthreads();
  return !brk;
}

// Totals of the 2 * nblk partials in `part` (pairs), fixed order; valid in thread 0.
__device__ __forceinline__ void sum_pairs(const double* part, int nblk, double* sh, double& s0, double& s1) {
  double a0 = 0.0, a1 = 0.0;
  for (int b = threadIdx.x; b < nblk; b += kThreads) {
    a0 += __ldcg(part + 2 * b);
    a1 += __ldcg(part + 2 * b + 1);
  }
  s0 = block_sum_smem(a0, sh);
  s1 = block_sum_smem(a1, sh);
}

struct GridBar {
  unsigned long long count;
  unsigned long long pad;
};

// Fused iteration in two phases separated by the two reductions of CG:
//   S: w = H z;  p = z + beta p;  q = w + beta q  (= H p by linearity);  p^T q
//   U: x += alpha p;  r -= alpha q;  z = D^{-1} r;  r^T z, r^T r
// The SpMV reads z, which the previous U phase finished before its barrier, so the direction
// update rides along with the SpMV instead of needing a third barrier and pass. In exact
// arithmetic the iterates are those of the three-launch form; q is carried by the recursion.
// On the first iteration after initialisation (flags[F_IT] == 0) beta = 0 and q is not read.
// W lanes share a face (face_reduce); each lane then updates the rows it holds.
// The iteration loop of one problem run by nvb cooperating blocks (vb = this block's index
// among them); `bar` is their arrival counter. The single-problem kernel runs it with the
// whole grid, the batch kernel with a team of blocks per problem.
// F32: the operator is the FP32 copy of the values (mixed contexts): each of the W lanes of a
// face forms its share of the face's rows in FP32 (products of FP32 values and the FP32 copy of
// z, ~len / W terms), the lanes' partial sums are reduced in FP32 and the row sums widened to
// FP64; every vector, scalar and reduction of the iteration stays FP64.
template <int NFN, int W, bool F32>
__device__ __forceinline__ void pcg_fused_body(const PcgArgs& a, int count, double rtol2, GridBar* bar, int vb,
                                               int nvb, double* sh, double* bc) {
  constexpr int NP = padded_rows<NFN, W>();
  constexpr bool kScatter = NP % W == 0;
  if (a.flags[F_CONV] | a.flags[F_BRK]) return;
  const int it0 = a.flags[F_IT];                          // no block changes it before all have read it
  const double rr0 = a.scal[S_RR0];
  double rz = a.scal[S_RZ];
  double beta = a.scal[S_BETA];
  bool first = it0 == 0;
  constexpr int FPW = 32 / W;
  const int64_t warp = (vb * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)nvb * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31, sub = lane / W, gl = lane % W;
  const int64_t nfaces = a.n / NFN;
  double* part0 = a.partial;                              // barrier 2i   (p^T q)
  double* part1 = a.partial + 2 * nvb;                    // barrier 2i+1 (r^T z, r^T r)
  for (int it = 0; it < count; ++it) {
    const unsigned long long B = 2ull * (unsigned long long)it;   // the counter is zeroed before every launch
    // ---- S phase
    double pq = 0.0;
    for (int64_t base = warp * FPW; base < nfaces; base += nwarps * FPW) {
      const int64_t f = base + sub;
      using AccT = typename std::conditional<F32, float, double>::type;
      AccT acc[NP];
#pragma unroll
      for (int m = 0; m < NP; ++m) acc[m] = AccT(0);
      if (f < nfaces) {
        if constexpr (F32) {
          const int64_t c0 = __ldcs(a.fptr32 + f);
          const int len = (int)(__ldcs(a.fptr32 + f + 1) - c0);
          const float* vb = a.val32 + NFN * c0;
#pragma unroll 4
          for (int t = gl; t < len; t += W) {
            const float zj = __ldcg(a.z32 + __ldcs(a.col32 + c0 + t));
#pragma unroll
            for (int m = 0; m < NFN; ++m) acc[m] = fmaf(__ldcs(vb + (int64_t)m * len + t), zj, acc[m]);
          }
        } else {
          const int64_t r0 = f * NFN;
          const int64_t lo = __ldcs(a.row_ptr + r0);
          const int len = (int)(__ldcs(a.row_ptr + r0 + 1) - lo);
#pragma unroll 4
          for (int t = gl; t < len; t += W) {
            const double zj = __ldcg(a.z + __ldcs(a.col + lo + t));
#pragma unroll
            for (int m = 0; m < NFN; ++m) acc[m] = fma(__ldcs(a.val + lo + (int64_t)m * len + t), zj, acc[m]);
          }
        }
      }
      face_reduce<NP, W, AccT>(acc, gl);
      if constexpr (kScatter) {
        if (f < nfaces) {
#pragma unroll
          for (int j = 0; j < NP / W; ++j) {
            const int row = scatter_row<NP, W>(j, gl);
            if (row >= NFN) continue;
            const int64_t i = f * NFN + row;
            const double zi = __ldcg(a.z + i);
            const double hz = F32 ? (double)acc[j] * __ldcg(a.dsq + i) : (double)acc[j];
            const double pi = first ? zi : fma(beta, a.p[i], zi);
            const double qi = first ? hz : fma(beta, a.q[i], hz);
            a.p[i] = pi;
            a.q[i] = qi;
            pq = fma(pi, qi, pq);
          }
        }
      } else {
        if (f < nfaces) {
#pragma unroll
          for (int m = 0; m < NFN; ++m)
            if (gl == m % W) {
              const int64_t i = f * NFN + m;
              const double zi = __ldcg(a.z + i);
              const double hz = F32 ? (double)acc[m] * __ldcg(a.dsq + i) : (double)acc[m];
              const double pi = first ? zi : fma(beta, a.p[i], zi);
              const double qi = first ? hz : fma(beta, a.q[i], hz);
              a.p[i] = pi;
              a.q[i] = qi;
              pq = fma(pi, qi, pq);
            }
        }
      }
    }
    first = false;
    pq = block_sum_smem(pq, sh);
    if (threadIdx.x == 0) {
      part0[2 * vb] = pq;
      part0[2 * vb + 1] = 0.0;
    }
    if (!grid_barrier(&bar->count, (B + 1) * nvb, a.flags)) return;
    {
      double tpq, unused;
      sum_pairs(part0, nvb, sh, tpq, unused);
      if (threadIdx.x == 0) {
        bc[0] = tpq;
        bc[1] = rz / tpq;
      }
      __syncthreads();
    }
    const double tpq = bc[0], alpha = bc[1];
    if (!(tpq > 0.0) || !(tpq < INFINITY)) {
      if (vb == 0 && threadIdx.x == 0) { a.flags[F_BRK] = 1; a.scal[S_PQ] = tpq; }
      return;
    }
    // ---- U phase
    double rzl = 0.0, rrl = 0.0;
    {
      const int64_t stride = (int64_t)nvb * blockDim.x;
      for (int64_t i = vb * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += stride) {
        a.x[i] = fma(alpha, a.p[i], a.x[i]);
        const double r = fma(-alpha, a.q[i], a.r[i]);
        a.r[i] = r;
        const double z = a.dinv[i] * r;
        a.z[i] = z;
        if constexpr (F32) a.z32[i] = (float)(z * a.dsq[i]);
        rzl = fma(r, z, rzl);
        rrl = fma(r, r, rrl);
      }
    }
    rzl = block_sum_smem(rzl, sh);
    rrl = block_sum_smem(rrl, sh);
    if (threadIdx.x == 0) {
      part1[2 * vb] = rzl;
      part1[2 * vb + 1] = rrl;
    }
    if (!grid_barrier(&bar->count, (B + 2) * nvb, a.flags)) return;
    {
      double rzn, rrn;
      sum_pairs(part1, nvb, sh, rzn, rrn);
      if (threadIdx.x == 0) {
        bc[0] = rzn;
        bc[1] = rrn;
        bc[2] = rzn / rz;
      }
      __syncthreads();
    }
    const double rzn = bc[0], rrn = bc[1];
    beta = bc[2];
    rz = rzn;
    const bool conv = rrn <= rtol2 * rr0;
    if (vb == 0 && threadIdx.x == 0) {
      a.scal[S_ALPHA] = alpha;
      a.scal[S_BETA] = beta;
      a.scal[S_RZ] = rzn;
      a.scal[S_RR] = rrn;
      a.flags[F_IT] += 1;
      if (conv) a.flags[F_CONV] = 1;
      if (!(rrn < INFINITY)) a.flags[F_BRK] = 1;
    }
    if (conv || !(rrn < INFINITY)) return;
  }
}

// Resident CTAs per SM: two (one for the FP64 form at 16 rows per face). The FP64 form is bound
// by the FP64 pipe (more warps did not help); the FP32-operator form by memory latency, but a
// third CTA per SM (80 registers) cost it more loads in flight per thread than it gained in
// warps (5.9 against 3.9 ms per iteration at 96^3 RT_2), while at 16 rows per face a second CTA
// (128 registers, no spills) helped (2.6 against 2.9 ms at 64^3 RT_3).
template <int NFN, int W, bool F32>
__global__ void __launch_bounds__(kThreads, F32 ? 2 : (NFN <= 9 ? 2 : 1))
    pcg_fused_kernel(PcgArgs a, int count, double rtol2, GridBar* bar) {
  __shared__ double sh[kThreads];
  __shared__ double bc[3];
  pcg_fused_body<NFN, W, F32>(a, count, rtol2, bar, blockIdx.x, gridDim.x, sh, bc);
}

// The FP32 operator of a mixed context: first d_i = sqrt(H_ii), then the scaled values rounded
// to nearest, one warp per row.
__global__ void diag_sqrt_kernel(int64_t n_rows, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                 const double* __restrict__ v, double* __restrict__ dsq) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_rows; i += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int64_t t = row_ptr[i]; t < row_ptr[i + 1]; ++t)
      if (col[t] == i) d = v[t];
    dsq[i] = sqrt(d);
  }
}

// One warp per face: its padded column list and its NFN scaled rows in the FP32 layout.
__global__ void round_values_kernel(int64_t n_faces, int nfn, const int64_t* __restrict__ row_ptr,
                                    const int32_t* __restrict__ col, const double* __restrict__ v,
                                    const int64_t* __restrict__ fptr32, const double* __restrict__ dsq,
                                    float* __restrict__ o, int32_t* __restrict__ col32) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t f = w0; f < n_faces; f += nw) {
    const int64_t r0 = f * nfn, lo = row_ptr[r0];
    const int len = (int)(row_ptr[r0 + 1] - lo);
    const int64_t c0 = fptr32[f];
    const int len32 = (int)(fptr32[f + 1] - c0);
    for (int t = lane; t < len32; t += 32) col32[c0 + t] = t < len ? col[lo + t] : 0;
    for (int m = 0; m < nfn; ++m) {
      const double si = 1.0 / dsq[r0 + m];
      float* orow = o + nfn * c0 + (int64_t)m * len32;
      const double* vrow = v + lo + (int64_t)m * len;
      for (int t = lane; t < len32; t += 32)
        __stcs(orow + t, t < len ? (float)(__ldcs(vrow + t) * si / dsq[col[lo + t]]) : 0.0f);
    }
  }
}

// Batch: block b works for problem team[b].x as block team[b].y of team[b].z, with that
// problem's order (rows per face) and its own barrier counter (PcgArgs::bar): the teams of all
// orders share one launch at two blocks per SM.
__global__ void __launch_bounds__(kThreads, 2)
    pcg_team_kernel(const PcgArgs* __restrict__ probs, const int4* __restrict__ team, int count, double rtol2) {
  __shared__ double sh[kThreads];
  __shared__ double bc[3];
  const int4 t = team[blockIdx.x];
  const PcgArgs& a = probs[t.x];
  GridBar* bar = reinterpret_cast<GridBar*>(a.bar);
  switch (a.nfn) {
    case 1: pcg_fused_body<1, 4, false>(a, count, rtol2, bar, t.y, t.z, sh, bc); break;
    case 4: pcg_fused_body<4, 4, false>(a, count, rtol2, bar, t.y, t.z, sh, bc); break;
    case 9: pcg_fused_body<9, 4, false>(a, count, rtol2, bar, t.y, t.z, sh, bc); break;
    default: pcg_fused_body<16, 4, false>(a, count, rtol2, bar, t.y, t.z, sh, bc); break;
  }
}

// Barrier self-test: `rounds` barriers over a cooperative grid, each checking the fixed-order
// totals of per-block partials; `absent` arrivals are counted as missing (the counter starts
// at -absent), so absent > 0 makes every wait run out.
__global__ void __launch_bounds__(kThreads) barrier_selftest_kernel(int rounds, GridBar* bar, double* part,
                                                                    int* flags) {
  __shared__ double sh[kThreads];
  const int nvb = gridDim.x;
  for (int r = 0; r < rounds; ++r) {
    double* pb = part + (r & 1) * 2 * nvb;
    if (threadIdx.x == 0) {
      pb[2 * blockIdx.x] = 1.0;
      pb[2 * blockIdx.x + 1] = (double)blockIdx.x;
    }
    if (!grid_barrier(&bar->count, (unsigned long long)(r + 1) * nvb, flags)) return;
    double s0, s1;
    sum_pairs(pb, nvb, sh, s0, s1);
    if (threadIdx.x == 0 && (s0 != (double)nvb || s1 != 0.5 * nvb * (nvb - 1.0))) flags[F_BRK] = 1;
  }
}

// ---- refinement helpers
__global__ void __launch_bounds__(kThreads) face_jump_kernel(JumpArgs a) {
  __shared__ double sh[32];
  const int64_t n = a.n_faces * a.nfn;
  double ss = 0.0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = r / a.nfn;
    const int m = (int)(r - f * a.nfn);
    const int lo = a.face_dof[2 * f], hi = a.face_dof[2 * f + 1];
    const double ul = a.u[(int64_t)(lo / 6) * a.n_loc + a.ni + (lo % 6) * a.nfn + m];
    const double uh = a.u[(int64_t)(hi / 6) * a.n_loc + a.ni + (hi % 6) * a.nfn + m];
    const double v = a.wf[m] * (ul - uh);
    a.rho[r] = v;
    ss = fma(v, v, ss);
  }
  ss = block_sum(ss, sh);
  if (threadIdx.x == 0) a.partial[blockIdx.x] = ss;
  if (last_block(a.ticket, gridDim.x)) {
    const double t = sum_partials(a.partial, gridDim.x, 1, 0, sh);
    if (threadIdx.x == 0) {
      *a.norm2 = t;
      *a.ticket = 0;
    }
  }
}

__global__ void __launch_bounds__(kThreads) norm2_kernel(int64_t n, const double* v, double* partial, double* out,
                                                          int* ticket) {
  __shared__ double sh[32];
  double ss = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    ss = fma(v[i], v[i], ss);
  ss = block_sum(ss, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = ss;
  if (last_block(ticket, gridDim.x)) {
    const double t = sum_partials(partial, gridDim.x, 1, 0, sh);
    if (threadIdx.x == 0) {
      *out = t;
      *ticket = 0;
    }
  }
}

__global__ void axpy_kernel(int64_t n, const double* x, double* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}

// ---- batched forms: block b works for problem blk_prob[b] as its block b - blk_first[that problem]
// of blk_count[that problem]; every problem keeps its own scalars, tickets and flags.
__global__ void __launch_bounds__(kThreads) spmv_batch_kernel(const PcgArgs* probs, const int32_t* blk_prob,
                                                              const int32_t* blk_first, const int32_t* blk_count) {
  __shared__ double sh[kThreads];
  const int pb = blk_prob[blockIdx.x];
  const PcgArgs a = probs[pb];
  const int vb = blockIdx.x - blk_first[pb], nvb = blk_count[pb];
  switch (a.nfn) {
    case 1: spmv_face_body<1, 4>(a, vb, nvb, sh); break;
    case 4: spmv_face_body<4, 4>(a, vb, nvb, sh); break;
    case 9: spmv_face_body<9, 4>(a, vb, nvb, sh); break;
    default: spmv_face_body<16, 4>(a, vb, nvb, sh); break;
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

cudaError_t pcg_init_batch(const PcgBatch& b, cudaStream_t s, Prof* prof) {
  int tok = prof_begin(prof, HYB_K_PCG_VECTOR, s);
  diag_inv_batch_kernel<<<b.n_vec, kThreads, 0, s>>>(b.probs, b.vec_prob, b.vec_first, b.vec_count);
  prof_end(prof, tok, s);
  tok = prof_begin(prof, HYB_K_PCG_VECTOR, s);
  pcg_init_batch_kernel<<<b.n_vec, kThreads, 0, s>>>(b.probs, b.vec_prob, b.vec_first, b.vec_count);
  prof_end(prof, tok, s);
  return cudaGetLastError();
}

cudaError_t launch_pcg_continue(const PcgArgs* probs, int nprob, unsigned long long handle, cudaStream_t s) {
  pcg_continue_kernel<<<1, kThreads, 0, s>>>(probs, nprob, (cudaGraphConditionalHandle)handle);
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
      case 4: spmv_face_kernel<4, 4><<<nbs, kThreads, 0, s>>>(a); break;
      case 9: spmv_face_kernel<9, 4><<<nbs, kThreads, 0, s>>>(a); break;
      case 16: spmv_face_kernel<16, 4><<<nbs, kThreads, 0, s>>>(a); break;
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

template <int NFN, int W, bool F32>
cudaError_t launch_fused(const PcgArgs& a, int count, double rtol, void* bar, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_fused_kernel<NFN, W, F32>, kThreads, 0);
  if (e != cudaSuccess) return e;
  int grid = sms * per_sm;
  if (grid > a.nblocks / 2) grid = a.nblocks / 2;         // two buffers of pairs: 4 * grid <= 2 * nblocks
  if (grid < 1) return cudaErrorInvalidConfiguration;
  PcgArgs aa = a;
  double rtol2 = rtol * rtol;
  GridBar* gb = static_cast<GridBar*>(bar);
  void* params[] = {&aa, &count, &rtol2, &gb};
  return cudaLaunchCooperativeKernel((const void*)pcg_fused_kernel<NFN, W, F32>, grid, kThreads, params, 0, s);
}

__global__ void zero_bars_kernel(const PcgArgs* probs, int n) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    probs[p].bar[0] = 0ull;
    probs[p].bar[1] = 0ull;
  }
}

cudaError_t pcg_zero_bars(const PcgArgs* probs, int n, cudaStream_t s) {
  zero_bars_kernel<<<(n + 255) / 256, 256, 0, s>>>(probs, n);
  return cudaGetLastError();
}

cudaError_t pcg_team_capacity(int* blocks) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_team_kernel, kThreads, 0);
  *blocks = sms * per_sm;
  return e;
}

cudaError_t pcg_iterations_team(const PcgArgs* probs, const int4* team, int nblocks, int count, double rtol,
                                cudaStream_t s, Prof* prof) {
  const int tok = prof_begin(prof, HYB_K_PCG_FUSED, s);
  double rtol2 = rtol * rtol;
  void* params[] = {&probs, &team, &count, &rtol2};
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)pcg_team_kernel, nblocks, kThreads, params, 0, s);
  prof_end(prof, tok, s);
  return e;
}

cudaError_t pcg_iterations_fused(const PcgArgs& a, int count, double rtol, void* bar, cudaStream_t s, Prof* prof) {
  const int tok = prof_begin(prof, HYB_K_PCG_FUSED, s);
  cudaError_t e;
  if (a.val32 && (!a.z32 || !a.dsq || !a.fptr32 || !a.col32)) return cudaErrorInvalidValue;
  if (a.val32) {
    // FP32 values: 8 lanes per face load 32 contiguous bytes of a row per step (a full sector),
    // and the lanes' partial sums are reduced in FP32
    switch (a.nfn) {
      case 1: e = launch_fused<1, 8, true>(a, count, rtol, bar, s); break;
      case 4: e = launch_fused<4, 8, true>(a, count, rtol, bar, s); break;
      case 9: e = launch_fused<9, 8, true>(a, count, rtol, bar, s); break;
      case 16: e = launch_fused<16, 8, true>(a, count, rtol, bar, s); break;
      default: e = cudaErrorInvalidValue;
    }
  } else {
    switch (a.nfn) {
      case 1: e = launch_fused<1, 4, false>(a, count, rtol, bar, s); break;
      case 4: e = launch_fused<4, 4, false>(a, count, rtol, bar, s); break;
      case 9: e = launch_fused<9, 4, false>(a, count, rtol, bar, s); break;
      case 16: e = launch_fused<16, 4, false>(a, count, rtol, bar, s); break;
      default: e = cudaErrorInvalidValue;
    }
  }
  prof_end(prof, tok, s);
  return e;
}

cudaError_t launch_round_values(int64_t n_rows, int nfn, const int64_t* row_ptr, const int32_t* col, const double* v,
                                const int64_t* fptr32, double* dsq, float* o, int32_t* col32, cudaStream_t s,
                                Prof* prof) {
  if (n_rows == 0) return cudaSuccess;
  int tok = prof_begin(prof, HYB_K_PCG_VECTOR, s);
  diag_sqrt_kernel<<<152 * 4, kThreads, 0, s>>>(n_rows, row_ptr, col, v, dsq);
  prof_end(prof, tok, s);
  tok = prof_begin(prof, HYB_K_PCG_VECTOR, s);
  round_values_kernel<<<152 * 8, kThreads, 0, s>>>(n_rows / nfn, nfn, row_ptr, col, v, fptr32, dsq, o, col32);
  prof_end(prof, tok, s);
  return cudaGetLastError();
}

cudaError_t launch_face_jump(const JumpArgs& a, cudaStream_t s, Prof* prof) {
  const int tok = prof_begin(prof, HYB_K_PCG_VECTOR, s);
  face_jump_kernel<<<a.nblocks, kThreads, 0, s>>>(a);
  prof_end(prof, tok, s);
  return cudaGetLastError();
}

cudaError_t launch_norm2(int64_t n, const double* v, double* partial, int nblocks, double* out, int* ticket,
                         cudaStream_t s, Prof* prof) {
  const int tok = prof_begin(prof, HYB_K_PCG_VECTOR, s);
  norm2_kernel<<<nblocks, kThreads, 0, s>>>(n, v, partial, out, ticket);
  prof_end(prof, tok, s);
  return cudaGetLastError();
}

cudaError_t launch_axpy(int64_t n, const double* x, double* y, cudaStream_t s, Prof* prof) {
  const int tok = prof_begin(prof, HYB_K_PCG_VECTOR, s);
  axpy_kernel<<<152 * 4, kThreads, 0, s>>>(n, x, y);
  prof_end(prof, tok, s);
  return cudaGetLastError();
}

cudaError_t barrier_selftest(int absent, int rounds, cudaStream_t s, int* result) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, barrier_selftest_kernel, kThreads, 0);
  if (e != cudaSuccess) return e;
  int grid = sms * per_sm;
  if (grid < 1) return cudaErrorInvalidConfiguration;
  // layout: bar (16 bytes) | flags (4 ints) | partials (two buffers of pairs)
  char* buf = nullptr;
  const size_t bytes = 16 + 16 + 4 * sizeof(double) * (size_t)grid;
  e = cudaMalloc(&buf, bytes);
  if (e != cudaSuccess) return e;
  GridBar* bar = reinterpret_cast<GridBar*>(buf);
  int* flags = reinterpret_cast<int*>(buf + 16);
  double* part = reinterpret_cast<double*>(buf + 32);
  const GridBar init{static_cast<unsigned long long>(-(long long)absent), 0ull};
  int hf[4] = {0, 0, 0, 0};
  e = cudaMemsetAsync(buf, 0, bytes, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bar, &init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    void* params[] = {&rounds, &bar, &part, &flags};
    e = cudaLaunchCooperativeKernel((const void*)barrier_selftest_kernel, grid, kThreads, params, 0, s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaError_t ef = cudaFree(buf);
  if (e == cudaSuccess) e = ef;
  *result = hf[F_BRK];
  return e;
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

extern "C" int hyb_barrier_selftest(int absent, int rounds, void* cuda_stream) {
  using namespace hyb;
  if (absent < 0 || absent > 1024 || rounds < 0) return HYB_ERR_INVALID_ARG;
  int result = 0;
  cudaError_t e = barrier_selftest(absent, rounds, static_cast<cudaStream_t>(cuda_stream), &result);
  if (e != cudaSuccess) return HYB_ERR_CUDA;
  if (result == 2) return HYB_ERR_TIMEOUT;
  if (result != 0) return HYB_ERR_BREAKDOWN;
  return HYB_OK;
}
