// Internal declarations shared by the translation units of libhyb.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hyb.h"

namespace hyb {

// Largest supported order and the table sizes it implies.
constexpr int kMaxOrder = 3;
constexpr int kMaxQ = kMaxOrder + 2;      // quadrature points per direction ((k+2)-point Gauss-Legendre)
constexpr int kMaxClosed = kMaxOrder + 2; // Gauss-Lobatto nodes along a component
constexpr int kMaxOpen = kMaxOrder + 1;   // Gauss-Legendre nodes across a component

// 1-D reference tables of one order k, computed on the host (hyb_tables.cpp).
struct RefTables {
  double qx[kMaxQ], qw[kMaxQ];              // quadrature nodes / weights on [0,1]
  double Vc[kMaxClosed][kMaxQ];             // closed Lagrange values at the quadrature nodes
  double Dc[kMaxClosed][kMaxQ];             // their derivatives
  double Vo[kMaxOpen][kMaxQ];               // open Lagrange values
  double wf[kMaxOpen * kMaxOpen];           // face Gauss-Legendre weights (lower axis fastest)
  double DcO[kMaxClosed][kMaxOpen];         // closed Lagrange derivatives at the open nodes (div into Q_k)
};

// Element sizes for order k.
struct Sizes {
  int k, P, p, Q, NQ, nfn, ni, nb, n;
  static Sizes of(int k) {
    Sizes s;
    s.k = k; s.P = k + 2; s.p = k + 1; s.Q = k + 2; s.NQ = s.Q * s.Q * s.Q;
    s.nfn = s.p * s.p; s.ni = 3 * k * s.p * s.p; s.nb = 6 * s.nfn; s.n = s.ni + s.nb;
    return s;
  }
};

enum Mode { MODE_NONE = 0, MODE_HYB = 1, MODE_SC = 2 };

// Device-side view of one problem, passed by value to kernels.
struct ElemArgs {
  int nx, ny, nz;
  int64_t n_elem;
  const double* vertices;
  const double* alpha;
  const double* beta;
  const double* load;
  const double* ess;          // may be null
  const int32_t* elem_list;   // elements of the colour being processed
  int64_t n_list;
  int colour;                 // 0: store shared face blocks, 1: add to them
  const int32_t* elem_face;   // E x 6 interior-face index, -1 on boundary faces
  const int64_t* blockoff;    // E x 36 value offset of face block (a, b) for row node 0, -1 if absent
  const int64_t* row_ptr;
  double* val;                // CSR values of H or S
  double* rhs;                // right-hand side
  double* Lstore;             // packed lower factor, n(n+1)/2 per FP64 element
  double* zstore;             // E x n forward-substituted load (FP64 path) / modified load (FP32 path)
  const int32_t* slot;        // per element: index into its precision's factor store, or null (= e)
  float* Lstore32;            // FP32 path: per element the tiles of L_M | Xd | L_Z | G^{-1}
  int* status;
  long long* err_elem;
  int natural;                // 1: boundary faces carry no essential data (their dofs stay unknowns)
};

// Launch profile: CUDA events around each launch, accumulated per kernel class
// after the owning call has synchronised (hyb_api.cpp).
struct Prof;
int prof_begin(Prof* p, int cls, cudaStream_t s);   // returns a token, -1 when off
void prof_end(Prof* p, int token, cudaStream_t s);

// status helpers
__host__ __device__ inline int64_t tri_size(int n) { return (int64_t)n * (n + 1) / 2; }
// FP64 factor store per element of order k: the packed lower factor of A_T (N (N + 1) / 2
// doubles; the recovery reads its interior rows L_ii and L_bi) followed by P = (A_T^{-1})_bb as
// a full NB x NB square (row-major), rounded up to an even count so that every element's store
// starts on a 16-byte boundary (the recovery bulk-copies L_ii from there).
__host__ __device__ constexpr int64_t fp64_store_doubles(int k) {
  return ((int64_t)(3 * k * (k + 1) * (k + 1) + 6 * (k + 1) * (k + 1)) *
              (3 * k * (k + 1) * (k + 1) + 6 * (k + 1) * (k + 1) + 1) / 2 +
          (int64_t)(6 * (k + 1) * (k + 1)) * (6 * (k + 1) * (k + 1)) + 1) / 2 * 2;
}

// Host-side table construction (hyb_tables.cpp).
void build_ref_tables(int k, RefTables* t);
void build_interface_w(int k, double* W);   // 4 (k+1)^2 x (k+1)^2, row-major

// Kernel launchers (hyb_element.cu, hyb_solve.cu, hyb_recover.cu). Return a cudaError_t.
cudaError_t upload_ref_tables(const RefTables* tabs, int count, cudaStream_t s);
cudaError_t upload_ref_tables_mixed(const RefTables* tabs, int count, cudaStream_t s);
int64_t mixed_store_floats(int k);
cudaError_t launch_element_mixed(int k, const ElemArgs& a, cudaStream_t s, Prof* prof);
cudaError_t launch_recover_mixed(int k, const ElemArgs& a, const double* lambda, double* u, cudaStream_t s,
                                 Prof* prof);
cudaError_t launch_check_geometry(int k, const ElemArgs& a, cudaStream_t s, Prof* prof);
cudaError_t launch_element(int k, int mode, const ElemArgs& a, cudaStream_t s, Prof* prof);
cudaError_t launch_expand_cols(const int64_t* row_ptr, const int32_t* adj, const int32_t* adj_count,
                               int64_t n_faces, int nfn, int32_t* col, cudaStream_t s, Prof* prof);

// Device scalars of a PCG solve: scal[] and flags[] slots (every PCG form, the host reads them)
enum PcgScalar { S_RZ = 0, S_RR0 = 1, S_RR = 2, S_ALPHA = 3, S_BETA = 4, S_PQ = 5 };
enum PcgFlag { F_IT = 0, F_CONV = 1, F_BRK = 2, F_TICKET = 3 };

// Aggregation multigrid preconditioner of the reduced system (hyb_amg.cu).
struct Amg;
int amg_create(int nx, int ny, int nz, int nfn, int degree, int coarsest, const int64_t* row_ptr,
               const int32_t* col, const double* val, const int64_t n_iface_axis[3], Amg** out);
int amg_numeric(Amg* a, cudaStream_t s);   // after every assembly (values of H changed)
int amg_set_fp32(Amg* a, bool on, const float* val32, const int32_t* col32, const int64_t* fptr32, const double* dsq);
int amg_apply(Amg* a, const double* r, double* z, cudaStream_t s);
int amg_pcg(Amg* a, const double* b, double rtol, int maxit, double* x, double* r, double* p, double* q,
            int* flags, double* scal, double* partial_unused, cudaStream_t s, int* iters, double* rel_res);
int amg_levels(const Amg* a, int64_t* sizes, int cap);
double amg_lmax(const Amg* a, int level);
void amg_free(Amg* a);

struct PcgArgs {
  int64_t n;
  const int64_t* row_ptr;
  const int32_t* col;
  const double* val;
  const double* b;
  double* x;
  double* r;
  double* p;
  double* q;
  double* dinv;
  double* z;                 // preconditioned residual (fused form only; NULL otherwise)
  const float* val32;        // mixed contexts, fused form: H_ij / (d_i d_j) rounded to FP32, d_i =
                             // sqrt(H_ii), applied with FP32 products (NULL: the FP64 values)
  const double* dsq;         // with val32: d_i = sqrt(H_ii)
  float* z32;                // with val32: (d z) rounded to FP32 for the SpMV's gathers
  const int64_t* fptr32;     // with val32: its own layout, every face's column list padded to a multiple
                             // of 8 (one 32-byte sector per 8 lanes): face f's list is col32[fptr32[f] ..
                             // fptr32[f+1]) and its NFN rows start at val32[NFN fptr32[f] + m (fptr32[f+1]
                             // - fptr32[f])]; padding entries have value 0 and column 0
  const int32_t* col32;
  int maxit;                 // > 0: the iteration kernels stop this problem after maxit iterations
                             // (the batched step's graph, whose loop runs on the device); <= 0: no limit
  unsigned long long* bar;   // fused form in a batch: this problem's barrier counter (16 bytes, zeroed per launch)
  double* partial;           // per-block partial sums
  double* scal;              // device scalars
  int* flags;                // iteration count / converged / breakdown / ticket
  int nblocks;               // grid size of every PCG kernel (partial holds 2*nblocks)
  int nfn;                   // rows per face ((k+1)^2): rows of a face share their column list
};
// Many independent PCG solves per launch: each problem owns a contiguous range of blocks.
struct PcgBatch {
  const PcgArgs* probs;                     // device, one per problem
  const int32_t *spmv_prob, *spmv_first, *spmv_count;   // device, per SpMV block / per problem
  const int32_t *vec_prob, *vec_first, *vec_count;      // device, per vector block / per problem
  int n_spmv, n_vec;                        // grid sizes
};
cudaError_t pcg_iterations_batch(const PcgBatch& b, int count, double rtol, cudaStream_t s, Prof* prof);
// pcg_init for every problem of a batch in two launches (flags must be zeroed first)
cudaError_t pcg_init_batch(const PcgBatch& b, cudaStream_t s, Prof* prof);
// one block: sets the graph conditional `handle` to 1 while any problem of the batch is neither
// converged nor broken down and below its maxit, else 0 (the WHILE node of the batched step)
cudaError_t launch_pcg_continue(const PcgArgs* probs, int nprob, unsigned long long handle, cudaStream_t s);
cudaError_t pcg_init(const PcgArgs& a, cudaStream_t s, Prof* prof);
// Up to `count` iterations in one cooperative launch (grid barriers between the phases).
// bar: 16 bytes, zeroed before every launch; a.z must be set (pcg_init fills it).
// Stops at convergence or breakdown; a barrier that waits too long sets flags[3rd] = 2
// (reported as HYB_ERR_TIMEOUT).
cudaError_t pcg_iterations_fused(const PcgArgs& a, int count, double rtol, void* bar, cudaStream_t s, Prof* prof);
// Batch form: one cooperative launch runs up to `count` fused iterations for several problems
// (any orders), each on its own team of blocks: block b works for problem team[b].x as block
// team[b].y of team[b].z (device table). nblocks <= pcg_team_capacity.
cudaError_t pcg_iterations_team(const PcgArgs* probs, const int4* team, int nblocks, int count, double rtol,
                                cudaStream_t s, Prof* prof);
cudaError_t pcg_team_capacity(int* blocks);
// zero every problem's barrier counter (before each team launch)
cudaError_t pcg_zero_bars(const PcgArgs* probs, int n, cudaStream_t s);
cudaError_t pcg_iterations(const PcgArgs& a, int count, double rtol, cudaStream_t s, Prof* prof);

// Normal jump of a broken flux: rho = C u (eq. 2.3's constraint), row (f, m) =
// w_m (u of the low-side element - u of the high-side element) at face node m. For the
// locally exact u(lambda) = A^-1 (f - C^T lambda) this is g - H lambda (eq. 2.4).
struct JumpArgs {
  int64_t n_faces;
  int nfn, n_loc, ni;
  const int32_t* face_dof;   // per interior face: 6 e + a of the low side, then of the high side
  const double* u;           // E x n_loc
  double* rho;               // n_faces * nfn
  double* partial;           // >= nblocks doubles
  double* norm2;             // out: rho^T rho
  int* ticket;               // zero on entry, zero on exit
  int nblocks;
  double wf[16];
};
cudaError_t launch_face_jump(const JumpArgs& a, cudaStream_t s, Prof* prof);
// out = v^T v (fixed-order block sums; ticket zero on entry and exit, partial >= nblocks)
cudaError_t launch_norm2(int64_t n, const double* v, double* partial, int nblocks, double* out, int* ticket,
                         cudaStream_t s, Prof* prof);
// y += x
cudaError_t launch_axpy(int64_t n, const double* x, double* y, cudaStream_t s, Prof* prof);
// The FP32 operator of a mixed context's PCG: dsq[i] = sqrt(H_ii), o[t] = (float)(H_ij / (dsq[i]
// dsq[j])) (the diagonally scaled matrix: unit diagonal, |entries| <= 1 for SPD H, so rounding
// it keeps it SPD where rounding H itself would not, e.g. across mass coefficients 10^-8..1);
// the first solve after an assembly runs it (profiled with the PCG's vector kernels)
cudaError_t launch_round_values(int64_t n_rows, int nfn, const int64_t* row_ptr, const int32_t* col, const double* v,
                                const int64_t* fptr32, double* dsq, float* o, int32_t* col32, cudaStream_t s,
                                Prof* prof);

struct RecoverArgs {
  int k;
  int64_t n_elem;             // number of elements to recover (length of elem_list, or all)
  const int32_t* elem_list;   // elements to recover, or null for 0..n_elem-1
  const int32_t* slot;        // factor-store index per element, or null (= e)
  int mode;
  const int32_t* elem_face;
  const double* lambda;       // multipliers (HB) or global face dofs (SC)
  const double* Lstore;       // fp64_store_doubles(k) per element (slot)
  const double* zstore;
  double* u;
  int* status;                // HYB_ERR_TIMEOUT if a bulk copy did not complete in time
  long long* err_elem;
  double wf[kMaxOpen * kMaxOpen];   // face Gauss weights of order k (C_T = [0 D])
};
cudaError_t launch_recover(const RecoverArgs& a, cudaStream_t s, Prof* prof);

// Batched forms: one launch over (problem, element) work items of one order, with the
// per-problem arguments in device arrays.
// grid: CTAs of the element launch; 0 (or >= n) one CTA per item, fewer: every CTA loops over
// the items grid apart (persistent), so each takes about n / grid elements.
cudaError_t launch_element_batch(int k, int mode, const ElemArgs* probs, const int2* items, int64_t n, int colour,
                                 int grid, cudaStream_t s, Prof* prof);
cudaError_t launch_mixed_batch(int k, const ElemArgs* probs, const int2* items, int64_t n, int colour, bool recover,
                               const double* const* lams, double* const* us, int grid, cudaStream_t s, Prof* prof);
// CTAs of the batched element kernels (FP64 / FP32 mixed form) of order k resident on one SM
int element_batch_ctas_per_sm(int k);
int mixed_batch_ctas_per_sm(int k);
cudaError_t launch_recover_batch(int k, int mode, const RecoverArgs* probs, const int2* items, int64_t n,
                                 cudaStream_t s, Prof* prof);

}  // namespace hyb
