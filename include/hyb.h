/*
 * hyb.h -- C ABI of the GB300 library for algebraic hybridization and static
 * condensation of the H(div) form a(u,v) = (alpha u, v) + (beta div u, div v)
 * on structured hexahedral meshes with broken Raviart-Thomas RT_k spaces,
 * k = 0..3 (Dobrev, Kolev, Lee, Tomov, Vassilevski, arXiv:1801.08914).
 *
 * Conventions shared by every entry point
 *  - Every call returns an int status: HYB_OK (0) or a negative HYB_ERR_* code.
 *    No C++ exception crosses this boundary. hyb_status_string() names a code.
 *  - Array arguments are DEVICE pointers (CUDA global memory) to contiguous
 *    float64 / int arrays unless a comment says "host". The caller owns them;
 *    the library never frees or retains a caller pointer beyond the calls
 *    documented to keep it (hyb_setup keeps vertices, alpha and beta).
 *  - The context owns every internal device buffer (reduced CSR system, stored
 *    element factors, solver vectors); hyb_destroy releases them.
 *  - All work is enqueued on the CUDA stream given to hyb_setup. A call returns
 *    after its status word has been copied back, so on return its device work
 *    is complete and its outputs are valid.
 *  - A context is not thread-safe: do not call into one context from two
 *    host threads at once.
 *
 * Numbering (identical on every entry point)
 *  - Element (i,j,l) of an nx*ny*nz mesh has index e = i + nx*(j + ny*l).
 *  - Vertex (i,j,l) has index i + (nx+1)*(j + (ny+1)*l); a vertex is 3 doubles.
 *  - Element-local dofs (n_loc = 3(k+1)^2(k+2)): interior dofs first
 *    (x-component nodes a=1..k, then y, then z; first index fastest), then the
 *    (k+1)^2 dofs of each face in the order x=0, x=1, y=0, y=1, z=0, z=1,
 *    lower tangential axis fastest. A dof is the value of the reference
 *    component along that axis at its node (closed Gauss-Lobatto nodes along
 *    the component, open Gauss-Legendre nodes across it).
 *  - Multipliers (one per Gauss-Legendre node of each interior face): faces by
 *    normal axis x, y, z; within an axis by plane index along the normal
 *    (fastest), then the lower and then the higher tangential cell index;
 *    within a face by node, lower tangential axis fastest. Static
 *    condensation numbers its global face dofs the same way.
 */
#ifndef HYB_H
#define HYB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  HYB_OK = 0,
  HYB_ERR_INVALID_ARG = -1,       /* null pointer, bad size, bad enum, wrong phase order */
  HYB_ERR_UNSUPPORTED_ORDER = -2, /* order outside 0..3 */
  HYB_ERR_MESH = -3,              /* det J <= 0 at a corner or quadrature point */
  HYB_ERR_NOT_SPD = -4,           /* an element matrix failed Cholesky (see hyb_last_error_element) */
  HYB_ERR_NOT_CONVERGED = -5,     /* PCG hit maxit; outputs are still written */
  HYB_ERR_BREAKDOWN = -6,         /* PCG p^T H p <= 0 or non-finite */
  HYB_ERR_CUDA = -7,              /* a CUDA runtime call failed */
  HYB_ERR_OOM = -8,               /* device allocation failed */
  HYB_ERR_TIMEOUT = -9            /* a bounded device-side wait gave up */
};

enum { HYB_FP64 = 0, HYB_MIXED = 1 };

/* Structured hexahedral mesh: (nx+1)(ny+1)(nz+1) vertices, device pointer. */
typedef struct {
  int nx, ny, nz;
  const double* vertices;
} hyb_mesh;

typedef struct hyb_ctx hyb_ctx;

/*
 * hyb_setup -- build the reduced-system pattern and the element metadata.
 *  Paper: the multiplier space and constraint matrix C of Example 2.2 (Sec. 2.4),
 *  the element 2x2 (interior/interface) ordering of Sec. 5.
 *  m          : mesh (nx, ny, nz >= 1); vertices must stay valid until hyb_destroy.
 *  order      : k in 0..3.
 *  alpha,beta : device, nx*ny*nz doubles each, per-element mass and divergence
 *               coefficients (> 0); kept until hyb_destroy.
 *  precision  : HYB_FP64, or HYB_MIXED: elements whose contrast beta/alpha is at most
 *               contrast_threshold are eliminated in FP32 through the hybridized mixed
 *               form (Sec. 3.2: A^-1 = M^-1 - M^-1 D Z^-1 D^T M^-1, every factor well
 *               conditioned): S_T and the load term g_T carry FP32-level error (hyb_refine
 *               removes it), the recovery's element solve is refined against an FP64
 *               residual; the others use the FP64 path. The reduced system is accumulated
 *               in FP64; the PCG keeps its iterate, residual and reductions in FP64 and
 *               applies H from an FP32 copy of its values (hyb_set_mixed_operator); the
 *               recovered u is FP64. Static condensation needs an HYB_FP64 context.
 *  contrast_threshold : HYB_MIXED only (ignored for HYB_FP64); > 0 as given, 0 = autotuned.
 *               The FP32 elimination's relative error in S_T grows like u_32 beta/alpha
 *               (the 1/alpha part of A^-1 on the faces cancels in it); up to 1e6 the FP64
 *               refinement corrects it, at 1e8 it does not. The first HYB_MIXED set-up of
 *               each order on a device times both element kernels on a 16^3 (RT_3: 12^3)
 *               unit-cube mesh: FP32 faster -> threshold 1e6 (elements above it stay
 *               FP64), else 0 (all FP64); the choice is cached for the process.
 *               hyb_get_precision_split reports it. Negative values: HYB_ERR_INVALID_ARG.
 *  cuda_stream: cudaStream_t to enqueue on (NULL = legacy default stream).
 *  out        : host, receives the new context.
 *  Builds the CSR pattern of H (int64 row pointers, int32 columns), per-element
 *  face / scatter tables and checks det J > 0 at every corner and quadrature
 *  point (HYB_ERR_MESH otherwise; hyb_last_error_element gives the element).
 */
int hyb_setup(const hyb_mesh* m, int order, const double* alpha, const double* beta,
              int precision, double contrast_threshold, void* cuda_stream, hyb_ctx** out);

/*
 * hyb_assemble_reduced -- element-by-element elimination and assembly of
 *  H lambda = C A^-1 C^T lambda = C A^-1 f  (Thm 2.1, eq. 2.4; Sec. 5).
 *  Per element: A_T by Gauss quadrature through the Piola map, essential dofs
 *  eliminated, Cholesky A_T = L L^T (interior dofs first), S_T = C_T A_T^-1 C_T^T
 *  and g_T = C_T A_T^-1 f_T, added into the CSR values / right-hand side without
 *  atomics (two element colours).
 *  load : device, E*n_loc doubles: coefficients of f in the broken RT_k basis;
 *         the element load is f_T = M_T c_T with M_T the unit-coefficient mass.
 *  ess  : device, E*n_loc doubles of essential normal-trace dof values, read only
 *         at dofs on boundary faces; NULL means zero.
 *  Keeps the element factors for hyb_recover. HYB_ERR_NOT_SPD names an element.
 */
int hyb_assemble_reduced(hyb_ctx* ctx, const double* load, const double* ess);

/*
 * hyb_solve_reduced -- diagonal-preconditioned CG on the assembled reduced
 *  system (H after hyb_assemble_reduced, S after staticcond_assemble), x0 = 0,
 *  stopping when ||r||_2 <= rtol ||r_0||_2 (the paper's criterion, Sec. 6.1).
 *  lambda : device, N_lambda doubles, receives the solution.
 *  iters, rel_res : host, may be NULL.
 *  By default the iterations run 64 at a time in one cooperative launch (grid-wide
 *  barriers between SpMV, update and direction; the reductions are summed in a fixed
 *  block order, so the result is reproducible); hyb_set_pcg_fused(ctx, 0) selects
 *  three launches per iteration instead. Both give the same iterates up to rounding
 *  of the reductions.
 *  Returns HYB_ERR_NOT_CONVERGED after maxit iterations (lambda still written),
 *  HYB_ERR_BREAKDOWN when p^T H p <= 0 or a residual is not finite, and
 *  HYB_ERR_TIMEOUT when a grid barrier waited longer than about a second (the
 *  kernel then returns; the context stays usable).
 */
int hyb_solve_reduced(hyb_ctx* ctx, double rtol, int maxit, double* lambda,
                      int* iters, double* rel_res);

/*
 * hyb_recover -- back substitution x_T = A_T^-1 (f_T - C_T^T lambda_T) (Thm 2.1)
 *  with essential dofs re-inserted.
 *  lambda : device, N_lambda doubles.   u : device, E*n_loc doubles (broken RT_k dofs).
 *  Requires a preceding hyb_assemble_reduced on this context.
 */
int hyb_recover(hyb_ctx* ctx, const double* lambda, double* u);

/*
 * staticcond_assemble -- static condensation S_hat = A_bb - A_bi A_ii^-1 A_ib per
 *  element and S = [I;W]^T S_hat [I;W] (Sec. 3.1, eq. 3.1-3.2), assembled on the
 *  same CSR pattern as H with right-hand side f_b - A_bi A_ii^-1 f_i.
 *  load, ess : as for hyb_assemble_reduced. Returns HYB_ERR_INVALID_ARG on an HYB_MIXED context.
 */
int staticcond_assemble(hyb_ctx* ctx, const double* load, const double* ess);

/*
 * staticcond_recover -- u_i = A_ii^-1 (f_i - A_ib u_b) per element (Sec. 3.1).
 *  u_face : device, N_lambda doubles, the solved global face dofs.
 *  u      : device, E*n_loc doubles, the broken RT_k dofs (face dofs copied).
 *  Requires a preceding staticcond_assemble on this context.
 */
int staticcond_recover(hyb_ctx* ctx, const double* u_face, double* u);

/*
 * hyb_get_reduced -- borrow the context's reduced system (device pointers owned
 *  by the context, valid until the next assemble or hyb_destroy). Any output
 *  pointer may be NULL. n = N_lambda, nnz = number of stored entries.
 */
int hyb_get_reduced(hyb_ctx* ctx, const int64_t** row_ptr, const int32_t** col,
                    const double** val, const double** rhs, int64_t* n, int64_t* nnz);

/*
 * hyb_export_reduced -- copy the reduced system into caller-owned device arrays
 *  (row_ptr: N_lambda+1 int64, col: nnz int32, val: nnz doubles, rhs: N_lambda
 *  doubles); any pointer may be NULL. Enqueued on the context stream and
 *  complete on return.
 */
int hyb_export_reduced(hyb_ctx* ctx, int64_t* row_ptr, int32_t* col, double* val, double* rhs);

/*
 * hyb_refine -- FP64 iterative refinement of a solved hybridized system. It matters for
 *  mixed-precision contexts, where H was assembled from FP32 element eliminations
 *  (Sec. 3.2's mixed form): the correction equation is eq. 2.4 with the residual as its
 *  right-hand side. Each step
 *    rho = C u                       normal jump of the current flux, FP64 (eq. 2.3's constraint)
 *    H dlambda = rho                 diagonal PCG on the assembled H to inner_rtol
 *    lambda += dlambda, u = hyb_recover(lambda)
 *  For u = A^-1 (f - C^T lambda), which hyb_recover forms with FP64 residual refinement,
 *  the jump C u equals g - H lambda with the exact H, so each step contracts the error of
 *  lambda by about ||I - H_assembled^-1 H|| and u follows.
 *  lambda, u : device, on entry the output of hyb_solve_reduced and hyb_recover; updated.
 *  jump      : host, steps + 1 doubles or NULL; receives ||C u|| / ||g|| before each
 *              step and after the last.
 *  Only after hyb_assemble_reduced (HYB_ERR_INVALID_ARG after static condensation).
 *  Allocates two N_lambda vectors on first use (kept by the context).
 *  An inner solve that stops at maxit is not an error (the next step corrects it).
 */
int hyb_refine(hyb_ctx* ctx, int steps, double inner_rtol, int maxit, double* lambda, double* u,
               double* jump);

/*
 * hyb_set_natural_bc -- boundary reading of the next assembly.
 *  0 (default): every boundary face carries essential normal-trace data (the values
 *  passed as `ess`, zero when NULL); its dofs are eliminated (Sec. 5).
 *  1: natural: the weak form is posed over all of H(div) (eq. 5.1, as in the soft-hard
 *  test of Sec. 6.1); boundary-face dofs stay unknowns of their element, carry no
 *  multiplier, and `ess` is ignored. Hybridization (both precisions), hyb_recover and
 *  hyb_refine follow it; staticcond_assemble returns HYB_ERR_INVALID_ARG (its global
 *  unknowns are the interior faces' dofs).
 *  Resets the context's assembled state. HYB_ERR_INVALID_ARG for other values.
 */
int hyb_set_natural_bc(hyb_ctx* ctx, int natural);

/*
 * hyb_set_pcg_fused -- choose the PCG launch form used by hyb_solve_reduced:
 *  1 (default) one cooperative launch per 64 iterations, 0 three launches per
 *  iteration. Implementation choice with no counterpart in the paper.
 *  HYB_ERR_INVALID_ARG for other values or when the device cannot launch
 *  cooperative kernels.
 */
int hyb_set_pcg_fused(hyb_ctx* ctx, int on);

/*
 * hyb_set_mixed_operator -- HYB_MIXED contexts: the operator that the PCG of hyb_solve_reduced
 *  and hyb_refine applies.
 *  1 (default): when any element is eliminated in FP32, an FP32 copy of the diagonally scaled
 *  H_ij / sqrt(H_ii H_jj) (unit diagonal, so rounding keeps it positive definite even across
 *  coefficients of very different size), rounded once the assembly's FP64 accumulation is
 *  complete. Only when EVERY element took the FP32 path (contrast <= threshold everywhere): an
 *  element above the threshold brings a near-null mode of H whose small eigenvalue FP32 rounding
 *  cannot hold (mass coefficients 10^-8..1 made the PCG break down), so such contexts keep the
 *  FP64 values, as do contexts whose elements all took the FP64 path. Row sums
 *  are formed in FP32 from products of those values and of an FP32 copy of sqrt(H_jj) z_j, then
 *  widened to FP64 and multiplied by sqrt(H_ii); the iterate, residual, direction and every
 *  reduction stay FP64. H of a mixed context carries the FP32
 *  elimination's error (~1e-7 relative) already; the rounding adds error of the same kind and
 *  size. hyb_refine measures its residual as the FP64 jump of the recovered flux, which does not
 *  depend on this operator, so the refined solution does not either.
 *  0: the FP64 values.
 *  The fused form only (hyb_set_pcg_fused(ctx, 1), the default); the three-launch form applies the
 *  FP64 values. Implementation choice with no counterpart in the paper.
 *  HYB_ERR_INVALID_ARG on an HYB_FP64 context or for other values.
 */
int hyb_set_mixed_operator(hyb_ctx* ctx, int fp32);

/* Preconditioners of the reduced-system PCG. */
enum {
  HYB_PC_JACOBI = 0,   /* the diagonal of H (default) */
  HYB_PC_AMG = 1       /* one V-cycle of the aggregation multigrid below */
};

/*
 * hyb_set_preconditioner -- the preconditioner of hyb_solve_reduced and of hyb_refine's inner
 *  solves (arXiv:1801.08914, Sec. 4: H is spectrally equivalent to a mesh-dependent H^1-type
 *  norm of the face functions, so an H^1-type algebraic multigrid gives mesh-independent
 *  iteration counts; Sec. 6.1 uses BoomerAMG). HYB_PC_AMG is this library's own aggregation
 *  multigrid for the structured hexahedral mesh:
 *   - every interior face belongs to the 2x2x2 block of cells (i/2, j/2, l/2) of its grid
 *     position (plane index along its normal, cell indices across); all nodes of a block's
 *     faces share one coarse unknown (piecewise-constant prolongation); coarser levels
 *     aggregate the block grid 2x2x2 again until at most `coarsest` unknowns remain or one
 *     point is left (a block without faces gets the equation x = 0);
 *   - Galerkin coarse operators P^T A P (27-point operators on the block grids);
 *   - Chebyshev smoothing of degree `chebyshev_degree` (1..4) for D^{-1} A on [lmax/30, lmax],
 *     lmax = 1.1 x a 12-step power estimate, the same before and after the coarse correction
 *     (a symmetric positive definite V-cycle);
 *   - the coarsest level solved with its dense inverse (coarsest: 1..4096 unknowns; formed by
 *     Gauss-Jordan elimination in one CTA, so keep it small: 64 is a good default).
 *  Built on the first solve after hyb_setup (buffers: about 5 vectors of n_lambda doubles
 *  plus the coarse levels), its numeric part on the first solve after every assembly. The
 *  PCG starts from lambda = 0 and stops at ||r||_2 <= rtol ||b||_2, as with HYB_PC_JACOBI. Its
 *  products with H (the PCG's and the smoother's on level 0) use the FP64 values, except on
 *  HYB_MIXED contexts that apply the FP32 copy (hyb_set_mixed_operator: every element FP32),
 *  where they run from that copy like the diagonal PCG's; the coarse levels are formed from
 *  the FP64 values in both cases. Static condensation's S is
 *  H(div)-like, not H^1-like: the multigrid is built for H.
 *  HYB_ERR_INVALID_ARG for another kind or parameters out of range.
 */
int hyb_set_preconditioner(hyb_ctx* ctx, int kind, int chebyshev_degree, int coarsest);

/*
 * hyb_amg_apply -- z = M^{-1} r, one V-cycle of the multigrid of hyb_set_preconditioner
 *  (HYB_PC_AMG) for the current assembly. r, z: device, n_lambda doubles each, not
 *  overlapping. Synchronises the context's stream. HYB_ERR_INVALID_ARG before an assembly or
 *  when the preconditioner is not HYB_PC_AMG.
 */
int hyb_amg_apply(hyb_ctx* ctx, const double* r, double* z);

/*
 * hyb_amg_info -- levels of the multigrid (*levels), the unknowns of the first `cap` levels
 *  (sizes, may be null) and the power estimates of lmax(D^{-1} A) of the smoothed levels
 *  (lmax, may be null; 0 for the coarsest). Builds the multigrid if needed (as hyb_amg_apply).
 */
int hyb_amg_info(hyb_ctx* ctx, int* levels, int64_t* sizes, double* lmax, int cap);

/*
 * hyb_barrier_selftest -- exercise the grid barrier of the fused PCG kernel.
 *  Runs `rounds` barrier-and-reduce steps over a cooperative grid (one block per
 *  free slot of every SM) and checks the reduced sums. `absent` arrivals are
 *  counted as missing, so absent > 0 makes the first wait run out: every block
 *  then gives up after about a second and the kernel returns. Implementation
 *  check with no counterpart in the paper. Allocates and frees ~20 KB; synchronises
 *  `cuda_stream`.
 *  Returns HYB_OK, HYB_ERR_TIMEOUT (a wait ran out), HYB_ERR_BREAKDOWN (a wrong
 *  sum) or HYB_ERR_INVALID_ARG (absent outside 0..1024, rounds < 0).
 */
int hyb_barrier_selftest(int absent, int rounds, void* cuda_stream);

/* Kernel classes for the launch profile. */
enum {
  HYB_K_ELEMENT = 0,     /* element elimination (assemble / static condensation) */
  HYB_K_SPMV = 1,        /* CSR SpMV fused with p^T H p (one per PCG iteration) */
  HYB_K_PCG_VECTOR = 2,  /* PCG vector updates, reductions, initialisation */
  HYB_K_RECOVER = 3,     /* back substitution */
  HYB_K_SETUP = 4,       /* set-up kernels (column expansion, geometry check) */
  HYB_K_PCG_FUSED = 5,   /* fused PCG iterations: SpMV, updates and reductions in one launch */
  HYB_K_STEP = 6,        /* a whole batched step launched as one CUDA graph (hyb_batch_step) */
  HYB_K_COUNT = 7
};

/*
 * hyb_set_profiling -- enable (1) or disable (0) the launch profile and reset it.
 *  While enabled, every kernel launch of the context is bracketed by CUDA events
 *  recorded on the context stream; elapsed times are added up when each call
 *  synchronises. Costs about one event pair per launch.
 */
int hyb_set_profiling(hyb_ctx* ctx, int enable);

/*
 * hyb_get_profile -- host outputs for kernel class `kernel_class` (HYB_K_*):
 *  summed device time in milliseconds and number of launches since profiling
 *  was enabled. Either output may be NULL.
 */
int hyb_get_profile(const hyb_ctx* ctx, int kernel_class, double* total_ms, int64_t* launches);

/*
 * hyb_pcg_solve_noalloc -- the diagonal-preconditioned CG of hyb_solve_reduced on a
 *  caller-supplied CSR system, for callers that cannot allocate device memory: code
 *  whose device memory is entirely reserved by another allocator (a framework's
 *  caching pool, a fixed arena sized at start-up) or that must not make a call that
 *  can block the whole device the way cudaMalloc / cudaFree do. The paper has no
 *  counterpart; this is a deployment convenience.
 *  It allocates nothing: its solver scratch (four vectors of the row count, block
 *  partial sums, scalars and flags, about 16.8 MB) is one file-scope __device__
 *  array in the library, present on every GPU that loads the library until the
 *  process exits. Every call shares that array and leaves the last call's contents
 *  in it; calls that can overlap on the GPU (other streams, other host threads)
 *  race on it and must be serialised by the caller.
 *  The first call on a device looks up the array's device address
 *  (cudaGetSymbolAddress) and caches it per device. Every call copies the solver's
 *  flags to host memory and synchronises cuda_stream between chunks of iterations, so
 *  it must not be called while cuda_stream, or any stream capturing in global mode,
 *  is being captured into a CUDA graph.
 *  row_ptr (n+1 int64), col (nnz int32), val (nnz doubles), b (n doubles): device,
 *  the SPD system. x: device, n doubles, receives the solution (x0 = 0).
 *  n <= 524288 rows, else HYB_ERR_INVALID_ARG (nothing is enqueued).
 *  rows_per_face: 1 for any CSR matrix; (k+1)^2 for the reduced systems built by
 *  this library, whose (k+1)^2 consecutive rows share one column list.
 *  rtol, maxit, iters, rel_res and the return codes are those of hyb_solve_reduced.
 *  cuda_stream: the stream to run on; the call returns when its work is complete.
 */
int hyb_pcg_solve_noalloc(const int64_t* row_ptr, const int32_t* col, const double* val,
                          const double* b, double* x, int64_t n, int rows_per_face,
                          double rtol, int maxit, void* cuda_stream, int* iters, double* rel_res);

/*
 * hyb_measure_fma_peak -- measured FMA throughput of the current device in TFLOP/s
 *  (fp64 = 1: double, 0: float), from a grid of independent FMA chains timed with
 *  CUDA events on cuda_stream (best of 3). Used as the roofline denominator for
 *  kernels bound by arithmetic. Allocates and frees a small output buffer.
 */
int hyb_measure_fma_peak(int fp64, void* cuda_stream, double* tflops);

/*
 * hyb_rsqrt_probe -- the element kernels' pivot inverse square root (an FP32 seed built
 *  from the exponent and mantissa bits, then one third-order correction of the binomial
 *  series of (1 - e)^{-1/2}) and their pivot check, evaluated on n given doubles, for
 *  accuracy tests. Implementation check with no counterpart in the paper.
 *  x : device, n doubles; out : device, n doubles, receives the inverse square roots
 *  (meaningful where the check passes); positive_normal : device, n ints, receives 1 where
 *  x[i] is a positive normal double, else 0. Synchronises cuda_stream.
 *  HYB_ERR_INVALID_ARG for n < 0 or a null pointer with n > 0.
 */
int hyb_rsqrt_probe(int64_t n, const double* x, double* out, int* positive_normal, void* cuda_stream);

/* hyb_get_precision_split -- host outputs (any may be NULL): elements on the FP64 and the
 *  FP32 path and the contrast threshold in use (0 for HYB_FP64 contexts). */
int hyb_get_precision_split(const hyb_ctx* ctx, int64_t* n_fp64, int64_t* n_fp32, double* threshold);

/* hyb_get_sizes -- host outputs (any may be NULL): elements, n_loc, N_lambda, nnz. */
int hyb_get_sizes(const hyb_ctx* ctx, int64_t* n_elem, int* n_loc, int64_t* n_lambda, int64_t* nnz);

/* hyb_last_error_element -- element behind the last HYB_ERR_NOT_SPD / HYB_ERR_MESH, or -1. */
int hyb_last_error_element(const hyb_ctx* ctx, int64_t* element);

/* hyb_destroy -- free every buffer the context owns; NULL is a no-op. */
void hyb_destroy(hyb_ctx* ctx);

/* hyb_status_string -- static name of a status code. */
const char* hyb_status_string(int status);

/* ---------------------------------------------------------------------------------------
 * Batches: many independent problems of uneven mesh size and order in one context. Each
 * phase launches once per (order, colour, precision path) over all problems' elements, and
 * the reduced solves of all problems run as one batched PCG (every problem keeps its own
 * scalars and stopping test). Array-of-pointer arguments are HOST arrays of nprob DEVICE
 * pointers; per-problem conventions are those of the single-problem calls above.
 */
typedef struct hyb_batch hyb_batch;

/* hyb_setup_batch -- meshes, orders: host arrays of nprob; alphas, betas: host arrays of
 *  device pointers (kept until hyb_destroy_batch). precision / contrast_threshold as for
 *  hyb_setup. */
int hyb_setup_batch(int nprob, const hyb_mesh* meshes, const int* orders, const double* const* alphas,
                    const double* const* betas, int precision, double contrast_threshold, void* cuda_stream,
                    hyb_batch** out);

/* hyb_assemble_reduced_batch -- hyb_assemble_reduced for every problem (ess may be NULL). */
int hyb_assemble_reduced_batch(hyb_batch* b, const double* const* loads, const double* const* ess);

/* hyb_solve_reduced_batch -- diagonal PCG for every problem; iters, rel_res: host arrays of
 *  nprob or NULL. Returns HYB_ERR_NOT_CONVERGED if any problem hit maxit. */
int hyb_solve_reduced_batch(hyb_batch* b, double rtol, int maxit, double* const* lambdas, int* iters,
                            double* rel_res);

/* hyb_recover_batch -- hyb_recover for every problem. */
int hyb_recover_batch(hyb_batch* b, const double* const* lambdas, double* const* us);

/*
 * hyb_batch_step -- the whole hot path for every problem of the batch as ONE CUDA graph launch:
 *  the element phase of hyb_assemble_reduced_batch (both colours in order), the batched diagonal
 *  PCG of hyb_solve_reduced_batch (x0 = 0, ||r|| <= rtol ||r0|| per problem, at most maxit
 *  iterations) and hyb_recover_batch. The PCG loop runs on the device: it is a WHILE node of the
 *  graph whose body is a chunk of batched iterations followed by a one-block kernel that sets the
 *  node's condition from every problem's converged / broken-down flags and iteration count
 *  (cudaGraphSetConditional), so the host neither reads flags nor launches kernels between
 *  chunks. The graph is captured on the first call and again when rtol changes; loads, ess,
 *  lambdas, us and maxit go to device argument arrays that the graph reads, so they may change
 *  between calls. Paper: Thm 2.1 and eq. 2.4 per problem; the batching has no counterpart.
 *  loads, ess, lambdas, us : host arrays of nprob device pointers (ess may be NULL).
 *  iters, rel_res : host arrays of nprob or NULL.
 *  Returns the element phase's or the recovery's error first (HYB_ERR_NOT_SPD, ...), then
 *  HYB_ERR_BREAKDOWN or HYB_ERR_NOT_CONVERGED (outputs still written) as hyb_solve_reduced_batch.
 *  Synchronises the batch's stream. Afterwards the batch is in the assembled state
 *  (hyb_recover_batch, exports and hyb_refine on its contexts apply).
 */
int hyb_batch_step(hyb_batch* b, const double* const* loads, const double* const* ess, double rtol, int maxit,
                   double* const* lambdas, double* const* us, int* iters, double* rel_res);

/* hyb_batch_step_kernels -- host outputs (any may be NULL) describing the step graph: kernel nodes
 *  outside the PCG loop, kernel nodes of one pass of the loop body, and PCG iterations per pass.
 *  HYB_ERR_INVALID_ARG before the first hyb_batch_step. */
int hyb_batch_step_kernels(const hyb_batch* b, int64_t* outside_loop, int64_t* per_pass, int* iterations_per_pass);

/* hyb_batch_get_autotune -- the element-phase launch shape the set-up's autotuner chose for
 *  order bin `order` (0..3) and precision path (0 FP64, 1 FP32 mixed form), host outputs (any may
 *  be NULL): `multiple` of the CTAs resident on the GPU at once (1, 2, 4: persistent CTAs taking
 *  about elements / grid elements each) or 0 (one CTA per element), and the resulting grid (0 for
 *  one CTA per element). hyb_setup_batch times the candidates on a unit-cube problem of each
 *  order and path present (cached per device for the process). No counterpart in the paper. */
int hyb_batch_get_autotune(const hyb_batch* b, int order, int path, int* multiple, int* grid);

/* hyb_batch_context -- the single-problem context of problem i (owned by the batch; do not
 *  destroy), for sizes, exports and error queries. */
int hyb_batch_context(hyb_batch* b, int problem, hyb_ctx** ctx);

/*
 * hyb_batch_set_pcg_fused -- 1: hyb_solve_reduced_batch runs the fused PCG of
 *  hyb_solve_reduced on teams of blocks, one team per unconverged problem: per chunk of 64
 *  iterations the problems, sorted by size, go in groups to cooperative launches whose grid
 *  is split in proportion to their nonzeros. 0 (default): three launches per iteration over
 *  all problems (hyb_batch_set_graphs applies); on large batches those launches are big
 *  enough that launch and barrier costs do not matter, and non-cooperative blocks share the
 *  GPU among the problems better (256-problem benchmark: 5.3 s against 8.1 s).
 *  Implementation choice with no counterpart in the paper.
 */
int hyb_batch_set_pcg_fused(hyb_batch* b, int on);

/*
 * hyb_batch_set_graphs -- 1 (default): with the three-launch form (the default of
 *  hyb_batch_set_pcg_fused), hyb_solve_reduced_batch replays its 32-iteration chunk of batched PCG (96 launches)
 *  as one CUDA graph (captured on the first solve, and
 *  again when rtol changes; profiled as one HYB_K_PCG_FUSED launch); 0: direct launches.
 *  Implementation choice with no counterpart in the paper.
 */
int hyb_batch_set_graphs(hyb_batch* b, int on);

/* launch profile of the batch's own launches (see hyb_set_profiling / hyb_get_profile) */
int hyb_batch_set_profiling(hyb_batch* b, int enable);
int hyb_batch_get_profile(const hyb_batch* b, int kernel_class, double* total_ms, int64_t* launches);

/* hyb_destroy_batch -- free the batch and every per-problem context; NULL is a no-op. */
void hyb_destroy_batch(hyb_batch* b);

/*
 * hyb_two_level_layout -- multiplier layout of a two-level hexahedral mesh with master /
 *  slave interface dofs (Example 2.1: P = [I 0; 0 I; 0 W_sm], C = [0 -W_sm I_s]; Fig. 5.1,
 *  right). HOST memory only; no GPU work, no context.
 *  The mesh: a coarse nx x ny x nzc block (elements e = i + nx (j + ny l)) under a fine block of
 *  mx x my x nzf cells (elements nx ny nzc + i + mx (j + my l)), (mx, my) = (2 nx, 2 ny) when
 *  refine (each coarse top face is tiled by four fine bottom faces) or (nx, ny) (a conforming
 *  interface). Boundary faces carry no multiplier.
 *  Multiplier faces, each with (k+1)^2 multipliers (lower tangential axis fastest): the
 *  interior faces of the coarse block, then those of the fine block (each block numbered as
 *  the structured meshes above), then the interface faces grouped by coarse face: coarse face
 *  (I, J) owns faces F + r^2 (I + nx J) + a + r b for its sub-faces (a, b), r = 2 (refine) or 1,
 *  F the number of faces before them. Multiplier id = face id (k+1)^2 + node.
 *  nx, ny, nzc, nzf > 0 : block sizes; order : k (0..3); refine : 0 or 1.
 *  n_lambda, nnz : out, the number of multipliers and of nonzeros of H's pattern.
 *  elem_face : out or NULL, E x 6 int32: the face id of each local face (x0 x1 y0 y1 z0 z1) or
 *   -1 on the boundary; a coarse top face with refine gets the first of its four ids.
 *  W : out or NULL (written only with refine), 4 (k+1)^2 x (k+1)^2 doubles row-major: fine
 *   dof (sub-face a + 2b, node p) = sum_r W[.][r] coarse dof r, the coarse face's Q_k normal
 *   trace at the fine node times 1/4 (a dof is a flux density per unit reference area and a
 *   fine reference face is a quarter of the coarse one).
 *  row_ptr : out or NULL, n_lambda + 1 int64; col : out or NULL (needs row_ptr), nnz int32:
 *   H's pattern, multipliers coupled when one element carries both; the rows of a face share
 *   one sorted column list.
 *  Call once with NULL arrays for the sizes, then with arrays of those sizes.
 *  Errors: HYB_ERR_INVALID_ARG (non-positive sizes, null n_lambda / nnz, more than 2^31
 *  multipliers), HYB_ERR_UNSUPPORTED_ORDER.
 */
int hyb_two_level_layout(int nx, int ny, int nzc, int nzf, int order, int refine, int64_t* n_lambda,
                         int64_t* nnz, int32_t* elem_face, double* W, int64_t* row_ptr, int32_t* col);

#ifdef __cplusplus
}
#endif

#endif /* HYB_H */
