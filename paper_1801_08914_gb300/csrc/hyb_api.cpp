// Host side of libhyb: context, set-up of the reduced-system pattern and the
// C ABI entry points declared in include/hyb.h.
//
// Set-up derives, for a structured nx*ny*nz hex mesh, everything the element
// kernels need to scatter without atomics (arXiv:1801.08914, Sec. 5):
//   * interior-face (multiplier) numbering: faces by normal axis, then plane
//     index, then the lower and the higher tangential cell index;
//   * per element its six interior-face ids (-1 on the boundary);
//   * the CSR pattern of H: row (f, m) couples face f with every interior
//     face of its two neighbours (at most 11), columns sorted; every row of a
//     face has the same column list, so the rows of a face form one dense
//     (k+1)^2 x len block of the value array;
//   * per element the value offset of each face block (a, b);
//   * a two-colouring by (i + j + l) mod 2: the two neighbours of a face
//     always differ in colour.
#include <algorithm>
#include <cstdint>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "hyb_internal.h"

using namespace hyb;

namespace hyb {

struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> pool;              // event pairs: 2 t, 2 t + 1
  std::vector<int> cls;                       // class of pending pair t
  size_t used = 0;
  double ms[HYB_K_COUNT] = {0};
  int64_t launches[HYB_K_COUNT] = {0};
  bool failed = false;

  // Add up the pending pairs (call after the stream has synchronised).
  void collect() {
    for (size_t t = 0; t < used; ++t) {
      float v = 0.f;
      if (cudaEventElapsedTime(&v, pool[2 * t], pool[2 * t + 1]) == cudaSuccess) ms[cls[t]] += v;
      else failed = true;
    }
    used = 0;
  }
  void reset() {
    for (int c = 0; c < HYB_K_COUNT; ++c) { ms[c] = 0; launches[c] = 0; }
    used = 0;
  }
  ~Prof() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

int prof_begin(Prof* p, int c, cudaStream_t s) {
  if (!p || !p->on) return -1;
  p->launches[c] += 1;
  if (p->used * 2 + 2 > p->pool.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return -1; }
    p->pool.push_back(a);
    p->pool.push_back(b);
    p->cls.push_back(0);
  }
  const size_t t = p->used++;
  p->cls[t] = c;
  cudaEventRecord(p->pool[2 * t], s);
  return (int)t;
}

void prof_end(Prof* p, int token, cudaStream_t s) {
  if (!p || token < 0) return;
  cudaEventRecord(p->pool[2 * token + 1], s);
}

}  // namespace hyb

struct hyb_ctx {
  int nx = 0, ny = 0, nz = 0, k = 0;
  Sizes sz{};
  int64_t E = 0, n_lambda = 0, nnz = 0, n_ifaces = 0;
  int64_t n_iface_axis[3] = {0, 0, 0};
  cudaStream_t stream = nullptr;
  const double* vertices = nullptr;
  const double* alpha = nullptr;
  const double* beta = nullptr;
  int64_t* row_ptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
  double* rhs = nullptr;
  int32_t* elem_face = nullptr;
  int64_t* blockoff = nullptr;
  int32_t* colour_list[2] = {nullptr, nullptr};
  int64_t n_colour[2] = {0, 0};
  // mixed precision: element lists by (colour, path) and per-precision recovery lists
  int precision = HYB_FP64;
  double theta = 0.0;                      // contrast beta/alpha above which an element stays FP64
  int32_t* mlist[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [colour][0 = FP64, 1 = FP32]
  int64_t n_mlist[2][2] = {{0, 0}, {0, 0}};
  int32_t* plist[2] = {nullptr, nullptr};  // [path]: all elements of that path
  int64_t n_path[2] = {0, 0};
  int32_t* slot = nullptr;
  float* Lstore32 = nullptr;
  float* val32 = nullptr;                  // mixed: FP32 copy of the reduced-system values (PCG operator)
  float* z32 = nullptr;                    // mixed: FP32 copy of the scaled preconditioned residual
  double* dsq = nullptr;                   // mixed: sqrt of H's diagonal (scaling of the FP32 operator)
  int64_t* fptr32 = nullptr;               // mixed: the FP32 operator's padded face layout (F + 1 offsets)
  int32_t* col32 = nullptr;                // mixed: its padded column lists, one per face
  int op32 = 1;                            // mixed: PCG applies H from val32 (1) or from val (0)
  bool val32_ready = false;                // the FP32 operator matches the current assembly
  int pc = HYB_PC_JACOBI;                  // PCG preconditioner
  int pc_degree = 2, pc_coarsest = 512;    // multigrid: Chebyshev degree, coarsest-level size
  Amg* amg = nullptr;
  bool amg_ready = false;                  // the multigrid matches the current assembly
  std::vector<int32_t> h_list[2][2];       // host copies: [colour][path] (path 0 = FP64, 1 = FP32)
  double* Lstore = nullptr;
  double* zstore = nullptr;
  int* status = nullptr;
  long long* err_elem = nullptr;
  double *r = nullptr, *p = nullptr, *q = nullptr, *dinv = nullptr, *z = nullptr, *partial = nullptr,
         *scal = nullptr;
  int* flags = nullptr;
  int32_t* face_dof = nullptr;             // per interior face: 6 e + a of its low, then high side
  double* rho = nullptr;                   // refinement: normal jump C u, then the correction
  double* dlam = nullptr;
  double* rnorm = nullptr;                 // 2 doubles: ||rho||^2, ||g||^2
  unsigned long long* gridbar = nullptr;   // arrival counter of the fused PCG kernel's grid barrier
  int natural = 0;                         // boundary faces: essential (0) or natural (1)
  int fused = 1;                           // PCG: one cooperative launch per chunk (1) or 3 launches/iteration (0)
  int nblocks = 0;
  int mode = MODE_NONE;
  int64_t last_err_elem = -1;
  RefTables tabs[kMaxOrder + 1];
  std::vector<void*> allocs;
  Prof prof;
};

namespace {

template <class T>
int dalloc(hyb_ctx* c, T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) count = 1;
  void* p = nullptr;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return HYB_ERR_OOM;
  }
  c->allocs.push_back(p);
  *ptr = static_cast<T*>(p);
  return HYB_OK;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return HYB_OK;
  if (e == cudaErrorMemoryAllocation) return HYB_ERR_OOM;
  return HYB_ERR_CUDA;
}

// Read back and clear the device status word; records the element id.
int finish_phase(hyb_ctx* c) {
  int st = 0;
  long long el = -1;
  cudaError_t e = cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&el, c->err_elem, sizeof(long long), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  c->prof.collect();
  if (st != 0) c->last_err_elem = el;
  return st;
}

int reset_status(hyb_ctx* c) {
  cudaError_t e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->err_elem, 0xff, sizeof(long long), c->stream);
  return cuda_status(e);
}

// interior-face index of the axis-d face at plane pl with tangential cells (a, b), or -1
int64_t iface(const hyb_ctx* c, int d, int pl, int a, int b) {
  const int dims[3] = {c->nx, c->ny, c->nz};
  if (pl <= 0 || pl >= dims[d]) return -1;
  const int across0 = d == 0 ? c->ny : c->nx;
  int64_t off = 0;
  for (int t = 0; t < d; ++t) off += c->n_iface_axis[t];
  return off + (pl - 1) + (int64_t)(dims[d] - 1) * (a + (int64_t)across0 * b);
}

// the six interior-face ids of element (i, j, l) in local face order x0 x1 y0 y1 z0 z1
void element_faces(const hyb_ctx* c, int i, int j, int l, int64_t out[6]) {
  out[0] = iface(c, 0, i, j, l);
  out[1] = iface(c, 0, i + 1, j, l);
  out[2] = iface(c, 1, j, i, l);
  out[3] = iface(c, 1, j + 1, i, l);
  out[4] = iface(c, 2, l, i, j);
  out[5] = iface(c, 2, l + 1, i, j);
}

ElemArgs elem_args(hyb_ctx* c, const double* load, const double* ess, int colour) {
  ElemArgs a{};
  a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
  a.n_elem = c->E;
  a.vertices = c->vertices;
  a.alpha = c->alpha;
  a.beta = c->beta;
  a.load = load;
  a.ess = ess;
  a.elem_list = c->colour_list[colour];
  a.n_list = c->n_colour[colour];
  a.colour = colour;
  a.elem_face = c->elem_face;
  a.blockoff = c->blockoff;
  a.row_ptr = c->row_ptr;
  a.val = c->val;
  a.rhs = c->rhs;
  a.Lstore = c->Lstore;
  a.zstore = c->zstore;
  a.status = c->status;
  a.err_elem = c->err_elem;
  a.natural = c->natural;
  return a;
}

int autotune_theta(int order, cudaStream_t s, double* theta);

int setup_impl(hyb_ctx* c, const hyb_mesh* m, int order, const double* alpha, const double* beta, int precision,
               double theta) {
  c->nx = m->nx; c->ny = m->ny; c->nz = m->nz; c->k = order;
  c->sz = Sizes::of(order);
  c->vertices = m->vertices;
  c->alpha = alpha;
  c->beta = beta;
  const int nx = c->nx, ny = c->ny, nz = c->nz, nfn = c->sz.nfn;
  c->E = (int64_t)nx * ny * nz;
  c->n_iface_axis[0] = (int64_t)(nx - 1) * ny * nz;
  c->n_iface_axis[1] = (int64_t)nx * (ny - 1) * nz;
  c->n_iface_axis[2] = (int64_t)nx * ny * (nz - 1);
  c->n_ifaces = c->n_iface_axis[0] + c->n_iface_axis[1] + c->n_iface_axis[2];
  c->n_lambda = c->n_ifaces * nfn;
  const int64_t E = c->E;

  // element face table and colour lists
  std::vector<int32_t> elem_face(6 * E);
  std::vector<int32_t> lists[2];
  lists[0].reserve(E / 2 + 1);
  lists[1].reserve(E / 2 + 1);
  for (int l = 0; l < nz; ++l)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const int64_t e = i + (int64_t)nx * (j + (int64_t)ny * l);
        int64_t f[6];
        element_faces(c, i, j, l, f);
        for (int a = 0; a < 6; ++a) elem_face[6 * e + a] = (int32_t)f[a];
        lists[(i + j + l) & 1].push_back((int32_t)e);
      }

  // face adjacency: interior faces of the two neighbours, sorted, unique
  const int64_t F = c->n_ifaces;
  std::vector<int32_t> adj(11 * F, -1), adj_count(F, 0);
  std::vector<int64_t> nb(2 * F, -1);                 // low / high neighbour element
  std::vector<int32_t> face_dof(2 * F, 0);            // the same, as 6 e + local face
  for (int64_t e = 0; e < E; ++e)
    for (int a = 0; a < 6; ++a) {
      const int32_t f = elem_face[6 * e + a];
      if (f >= 0) {
        nb[2 * f + (a & 1 ? 0 : 1)] = e;   // face at x_hat = 1 of e: e is the low side
        face_dof[2 * f + (a & 1 ? 0 : 1)] = (int32_t)(6 * e + a);
      }
    }
  for (int64_t f = 0; f < F; ++f) {
    int32_t tmp[12];
    int n = 0;
    for (int s = 0; s < 2; ++s) {
      const int64_t e = nb[2 * f + s];
      for (int a = 0; a < 6; ++a) {
        const int32_t g = elem_face[6 * e + a];
        if (g >= 0) tmp[n++] = g;
      }
    }
    std::sort(tmp, tmp + n);
    const int u = (int)(std::unique(tmp, tmp + n) - tmp);
    for (int t = 0; t < u; ++t) adj[11 * f + t] = tmp[t];
    adj_count[f] = u;
  }
  // row pointers
  std::vector<int64_t> row_ptr(c->n_lambda + 1);
  row_ptr[0] = 0;
  for (int64_t f = 0; f < F; ++f)
    for (int mm = 0; mm < nfn; ++mm) {
      const int64_t r = f * nfn + mm;
      row_ptr[r + 1] = row_ptr[r] + (int64_t)adj_count[f] * nfn;
    }
  c->nnz = row_ptr[c->n_lambda];
  // block offsets: value index of (face a row node 0, column block of face b)
  std::vector<int64_t> blockoff(36 * E, -1);
  for (int64_t e = 0; e < E; ++e)
    for (int a = 0; a < 6; ++a) {
      const int32_t fa = elem_face[6 * e + a];
      if (fa < 0) continue;
      for (int b = 0; b < 6; ++b) {
        const int32_t fb = elem_face[6 * e + b];
        if (fb < 0) continue;
        const int32_t* lst = &adj[11 * (int64_t)fa];
        const int pos = (int)(std::lower_bound(lst, lst + adj_count[fa], fb) - lst);
        blockoff[36 * e + 6 * a + b] = row_ptr[(int64_t)fa * nfn] + (int64_t)pos * nfn;
      }
    }

  // device buffers
  int st;
  int32_t *d_adj = nullptr, *d_adjc = nullptr;
  const Sizes& s = c->sz;
  if ((st = dalloc(c, &c->row_ptr, c->n_lambda + 1))) return st;
  if ((st = dalloc(c, &c->col, c->nnz))) return st;
  if ((st = dalloc(c, &c->val, c->nnz))) return st;
  if ((st = dalloc(c, &c->rhs, c->n_lambda))) return st;
  if ((st = dalloc(c, &c->elem_face, 6 * E))) return st;
  if ((st = dalloc(c, &c->blockoff, 36 * E))) return st;
  for (int t = 0; t < 2; ++t) {
    c->n_colour[t] = (int64_t)lists[t].size();
    if ((st = dalloc(c, &c->colour_list[t], lists[t].size()))) return st;
  }
  // precision paths: FP64 for every element, or (mixed) FP64 only above the contrast threshold
  // (threshold 0: chosen by autotune_theta for this order on this device)
  c->precision = precision;
  if (precision == HYB_MIXED && !(theta > 0.0)) {
    if ((st = autotune_theta(order, c->stream, &theta))) return st;
  }
  c->theta = theta;
  std::vector<int32_t> slot_h(E, 0);
  if (precision == HYB_MIXED) {
    std::vector<double> ah(E), bh(E);
    cudaError_t e0 = cudaMemcpy(ah.data(), alpha, E * sizeof(double), cudaMemcpyDeviceToHost);
    if (e0 == cudaSuccess) e0 = cudaMemcpy(bh.data(), beta, E * sizeof(double), cudaMemcpyDeviceToHost);
    if (e0 != cudaSuccess) return cuda_status(e0);
    std::vector<int32_t> ml[2][2], pl[2];
    for (int col = 0; col < 2; ++col)
      for (int32_t el : lists[col]) {
        const int path = (bh[el] / ah[el] > c->theta) ? 0 : 1;
        slot_h[el] = (int32_t)pl[path].size();
        pl[path].push_back(el);
        ml[col][path].push_back(el);
      }
    for (int col = 0; col < 2; ++col)
      for (int path = 0; path < 2; ++path) c->h_list[col][path] = ml[col][path];
    for (int col = 0; col < 2; ++col)
      for (int path = 0; path < 2; ++path) {
        c->n_mlist[col][path] = (int64_t)ml[col][path].size();
        if ((st = dalloc(c, &c->mlist[col][path], ml[col][path].size()))) return st;
        if (!ml[col][path].empty() &&
            cudaMemcpy(c->mlist[col][path], ml[col][path].data(), ml[col][path].size() * sizeof(int32_t),
                       cudaMemcpyHostToDevice) != cudaSuccess)
          return HYB_ERR_CUDA;
      }
    for (int path = 0; path < 2; ++path) {
      c->n_path[path] = (int64_t)pl[path].size();
      if ((st = dalloc(c, &c->plist[path], pl[path].size()))) return st;
      if (!pl[path].empty() && cudaMemcpy(c->plist[path], pl[path].data(), pl[path].size() * sizeof(int32_t),
                                          cudaMemcpyHostToDevice) != cudaSuccess)
        return HYB_ERR_CUDA;
    }
    if ((st = dalloc(c, &c->slot, E))) return st;
    if (cudaMemcpy(c->slot, slot_h.data(), E * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
      return HYB_ERR_CUDA;
    if ((st = dalloc(c, &c->Lstore, (size_t)c->n_path[0] * (size_t)fp64_store_doubles(order)))) return st;
    if ((st = dalloc(c, &c->Lstore32, (size_t)c->n_path[1] * (size_t)mixed_store_floats(order)))) return st;
    // the FP32 operator's layout: every face's column list padded to a multiple of 8 entries
    std::vector<int64_t> fp32(F + 1, 0);
    for (int64_t f = 0; f < F; ++f) fp32[f + 1] = fp32[f] + ((int64_t)adj_count[f] * nfn + 7) / 8 * 8;
    if ((st = dalloc(c, &c->val32, (size_t)fp32[F] * nfn))) return st;
    if ((st = dalloc(c, &c->col32, (size_t)fp32[F]))) return st;
    if ((st = dalloc(c, &c->fptr32, (size_t)F + 1))) return st;
    if (cudaMemcpy(c->fptr32, fp32.data(), (F + 1) * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess)
      return HYB_ERR_CUDA;
    if ((st = dalloc(c, &c->z32, c->n_lambda))) return st;
    if ((st = dalloc(c, &c->dsq, c->n_lambda))) return st;
  } else {
    if ((st = dalloc(c, &c->Lstore, (size_t)E * (size_t)fp64_store_doubles(order)))) return st;
    for (int col = 0; col < 2; ++col) c->h_list[col][0] = lists[col];
  }
  if ((st = dalloc(c, &c->zstore, (size_t)E * s.n))) return st;
  if ((st = dalloc(c, &c->status, 1))) return st;
  if ((st = dalloc(c, &c->err_elem, 1))) return st;
  if ((st = dalloc(c, &d_adj, 11 * F))) return st;
  if ((st = dalloc(c, &d_adjc, F))) return st;
  c->nblocks = 152 * 8;
  if ((st = dalloc(c, &c->r, c->n_lambda))) return st;
  if ((st = dalloc(c, &c->p, c->n_lambda))) return st;
  if ((st = dalloc(c, &c->q, c->n_lambda))) return st;
  if ((st = dalloc(c, &c->dinv, c->n_lambda))) return st;
  if ((st = dalloc(c, &c->z, c->n_lambda))) return st;
  if ((st = dalloc(c, &c->partial, 2 * c->nblocks))) return st;
  if ((st = dalloc(c, &c->scal, 8))) return st;
  if ((st = dalloc(c, &c->flags, 4))) return st;
  if ((st = dalloc(c, &c->gridbar, 2))) return st;
  if ((st = dalloc(c, &c->face_dof, 2 * F))) return st;
  if ((st = dalloc(c, &c->rnorm, 2))) return st;

  cudaStream_t S = c->stream;
  cudaError_t e = cudaSuccess;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, S);
  };
  up(c->row_ptr, row_ptr.data(), row_ptr.size() * sizeof(int64_t));
  up(c->elem_face, elem_face.data(), elem_face.size() * sizeof(int32_t));
  up(c->face_dof, face_dof.data(), face_dof.size() * sizeof(int32_t));
  up(c->blockoff, blockoff.data(), blockoff.size() * sizeof(int64_t));
  up(c->colour_list[0], lists[0].data(), lists[0].size() * sizeof(int32_t));
  up(c->colour_list[1], lists[1].data(), lists[1].size() * sizeof(int32_t));
  up(d_adj, adj.data(), adj.size() * sizeof(int32_t));
  up(d_adjc, adj_count.data(), adj_count.size() * sizeof(int32_t));
  for (int t = 0; t <= kMaxOrder; ++t) build_ref_tables(t, &c->tabs[t]);
  if (e == cudaSuccess) e = upload_ref_tables(c->tabs, kMaxOrder + 1, S);
  if (e == cudaSuccess) e = upload_ref_tables_mixed(c->tabs, kMaxOrder + 1, S);
  if (e == cudaSuccess) e = launch_expand_cols(c->row_ptr, d_adj, d_adjc, F, nfn, c->col, S, &c->prof);
  if (e == cudaSuccess) e = cudaStreamSynchronize(S);   // host vectors die at return
  if (e != cudaSuccess) return cuda_status(e);
  if ((st = reset_status(c))) return st;
  ElemArgs a = elem_args(c, nullptr, nullptr, 0);
  if ((e = launch_check_geometry(order, a, S, &c->prof)) != cudaSuccess) return cuda_status(e);
  return finish_phase(c);
}

int assemble_impl(hyb_ctx* c, const double* load, const double* ess, int mode) {
  if (!c || !load) return HYB_ERR_INVALID_ARG;
  if (c->precision == HYB_MIXED && mode == MODE_SC) return HYB_ERR_INVALID_ARG;
  int st = reset_status(c);
  if (st) return st;
  c->mode = MODE_NONE;
  for (int colour = 0; colour < 2; ++colour) {
    ElemArgs a = elem_args(c, load, ess, colour);
    if (c->precision == HYB_MIXED) {
      // colour 0 of both paths completes before colour 1 starts (stream order)
      a.slot = c->slot;
      a.elem_list = c->mlist[colour][0];
      a.n_list = c->n_mlist[colour][0];
      cudaError_t e = launch_element(c->k, mode, a, c->stream, &c->prof);
      if (e != cudaSuccess) return cuda_status(e);
      a.elem_list = c->mlist[colour][1];
      a.n_list = c->n_mlist[colour][1];
      a.Lstore32 = c->Lstore32;
      e = launch_element_mixed(c->k, a, c->stream, &c->prof);
      if (e != cudaSuccess) return cuda_status(e);
      continue;
    }
    cudaError_t e = launch_element(c->k, mode, a, c->stream, &c->prof);
    if (e != cudaSuccess) return cuda_status(e);
  }
  c->val32_ready = false;                  // the FP32 operator is prepared by the next solve
  c->amg_ready = false;                    // and so is the multigrid
  st = finish_phase(c);
  if (st == HYB_OK) c->mode = mode;
  return st;
}

// ---- contrast-threshold autotuner. Speed: both element paths are timed on a unit-cube mesh
// of the same order (alpha = beta = 1, zero load; the element work does not depend on the
// values). Accuracy: on the faces, A_T^{-1} has a part of size 1 / alpha (divergence-free
// fields through the element) and a part of size 1 / beta; the FP32 mixed form obtains S_T as
// Y^T Y - V^T V, where the 1 / alpha parts cancel, so the 1 / beta part carries an absolute
// error of about u_32 / alpha, i.e. u_32 beta / alpha relative. Up to beta / alpha = 1e6 the
// FP64 refinement still converges (measured); at 1e8 (soft-hard test, Sec. 6.1, p = -8) the
// FP32 H of RT_1 is indefinite and the refinement of RT_2 / RT_3 stalls. So when FP32 is the
// faster path the threshold is kMixedContrastMax (elements above it stay FP64), else 0 (all
// FP64). Measured once per order and device, then cached for the process.
constexpr double kMixedContrastMax = 1e6;
std::mutex g_tune_mutex;
std::map<std::pair<int, int>, double> g_tuned;

int autotune_theta(int order, cudaStream_t s, double* theta) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HYB_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  const auto key = std::make_pair(dev, order);
  const auto it = g_tuned.find(key);
  if (it != g_tuned.end()) {
    *theta = it->second;
    return HYB_OK;
  }
  const int n = order >= 3 ? 12 : 16;
  const int64_t E = (int64_t)n * n * n, nv = (int64_t)(n + 1) * (n + 1) * (n + 1);
  const int nloc = Sizes::of(order).n;
  std::vector<double> vh(3 * nv);
  for (int l = 0; l <= n; ++l)
    for (int j = 0; j <= n; ++j)
      for (int i = 0; i <= n; ++i) {
        const int64_t v = i + (int64_t)(n + 1) * (j + (int64_t)(n + 1) * l);
        vh[3 * v] = (double)i / n;
        vh[3 * v + 1] = (double)j / n;
        vh[3 * v + 2] = (double)l / n;
      }
  std::vector<double> ones(E, 1.0);
  double* buf = nullptr;
  const size_t nd = 3 * nv + 2 * E + E * nloc;
  if (cudaMalloc(&buf, nd * sizeof(double)) != cudaSuccess) return HYB_ERR_OOM;
  double *verts = buf, *alpha = buf + 3 * nv, *beta = alpha + E, *load = beta + E;
  cudaError_t e = cudaMemcpyAsync(verts, vh.data(), vh.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(alpha, ones.data(), E * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(beta, ones.data(), E * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(load, 0, (size_t)E * nloc * sizeof(double), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int st = e == cudaSuccess ? HYB_OK : cuda_status(e);
  double ms[2] = {0.0, 0.0};
  hyb_mesh mesh{n, n, n, verts};
  for (int path = 0; path < 2 && st == HYB_OK; ++path) {
    hyb_ctx* t = new (std::nothrow) hyb_ctx();
    if (!t) { st = HYB_ERR_OOM; break; }
    t->stream = s;
    st = setup_impl(t, &mesh, order, alpha, beta, path ? HYB_MIXED : HYB_FP64, 1e300);
    if (st == HYB_OK) st = assemble_impl(t, load, nullptr, MODE_HYB);       // warm-up
    if (st == HYB_OK) {
      t->prof.reset();
      t->prof.on = true;
      for (int r = 0; r < 2 && st == HYB_OK; ++r) st = assemble_impl(t, load, nullptr, MODE_HYB);
      t->prof.collect();
      ms[path] = t->prof.ms[HYB_K_ELEMENT];
    }
    hyb_destroy(t);
  }
  cudaFree(buf);
  if (st != HYB_OK) return st;
  *theta = ms[1] < ms[0] ? kMixedContrastMax : 0.0;
  g_tuned[key] = *theta;
  return HYB_OK;
}

int recover_impl(hyb_ctx* c, const double* lam, double* u, int mode) {
  if (!c || !lam || !u) return HYB_ERR_INVALID_ARG;
  if (c->mode != mode) return HYB_ERR_INVALID_ARG;
  RecoverArgs a{};
  a.k = c->k;
  a.n_elem = c->E;
  a.mode = mode;
  a.elem_face = c->elem_face;
  a.lambda = lam;
  a.Lstore = c->Lstore;
  a.zstore = c->zstore;
  a.u = u;
  a.status = c->status;
  a.err_elem = c->err_elem;
  std::memcpy(a.wf, c->tabs[c->k].wf, sizeof(a.wf));
  if (c->precision == HYB_MIXED) {
    a.elem_list = c->plist[0];
    a.n_elem = c->n_path[0];
    a.slot = c->slot;
  }
  int st = reset_status(c);
  if (st) return st;
  cudaError_t e = launch_recover(a, c->stream, &c->prof);
  if (e != cudaSuccess) return cuda_status(e);
  if (c->precision == HYB_MIXED) {
    ElemArgs m = elem_args(c, nullptr, nullptr, 0);
    m.elem_list = c->plist[1];
    m.n_list = c->n_path[1];
    m.slot = c->slot;
    m.Lstore32 = c->Lstore32;
    e = launch_recover_mixed(c->k, m, lam, u, c->stream, &c->prof);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return finish_phase(c);
}

}  // namespace

extern "C" {

int hyb_setup(const hyb_mesh* m, int order, const double* alpha, const double* beta, int precision,
              double contrast_threshold, void* cuda_stream, hyb_ctx** out) {
  if (!out) return HYB_ERR_INVALID_ARG;
  *out = nullptr;
  if (!m || !m->vertices || !alpha || !beta) return HYB_ERR_INVALID_ARG;
  if (m->nx < 1 || m->ny < 1 || m->nz < 1) return HYB_ERR_INVALID_ARG;
  if ((int64_t)m->nx * m->ny * m->nz > INT32_MAX) return HYB_ERR_INVALID_ARG;
  if (order < 0 || order > kMaxOrder) return HYB_ERR_UNSUPPORTED_ORDER;
  if (precision != HYB_FP64 && precision != HYB_MIXED) return HYB_ERR_INVALID_ARG;
  if (!(contrast_threshold >= 0.0)) return HYB_ERR_INVALID_ARG;
  hyb_ctx* c = new (std::nothrow) hyb_ctx();
  if (!c) return HYB_ERR_OOM;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  int st;
  try {
    st = setup_impl(c, m, order, alpha, beta, precision, contrast_threshold);
  } catch (const std::bad_alloc&) {
    st = HYB_ERR_OOM;
  } catch (...) {
    st = HYB_ERR_CUDA;
  }
  if (st != HYB_OK && st != HYB_ERR_MESH) {
    hyb_destroy(c);
    return st;
  }
  *out = c;   // on HYB_ERR_MESH the context is returned so the element can be queried
  return st;
}

int hyb_assemble_reduced(hyb_ctx* ctx, const double* load, const double* ess) {
  return assemble_impl(ctx, load, ess, MODE_HYB);
}

int staticcond_assemble(hyb_ctx* ctx, const double* load, const double* ess) {
  if (ctx && ctx->natural) return HYB_ERR_INVALID_ARG;
  return assemble_impl(ctx, load, ess, MODE_SC);
}

namespace {

// Diagonal PCG on the assembled H (or S) with right-hand side b, x0 = 0.
// the FP32 operator of a mixed context applies (every element took the FP32 path; see solve_impl)
bool use_op32(const hyb_ctx* c) {
  return c->precision == HYB_MIXED && c->n_path[1] > 0 && c->n_path[0] == 0 && c->op32 && c->mode == MODE_HYB;
}

int prepare_op32(hyb_ctx* c) {
  if (c->val32_ready) return HYB_OK;
  cudaError_t e = launch_round_values(c->n_lambda, c->sz.nfn, c->row_ptr, c->col, c->val, c->fptr32, c->dsq,
                                      c->val32, c->col32, c->stream, &c->prof);
  if (e != cudaSuccess) return cuda_status(e);
  c->val32_ready = true;
  return HYB_OK;
}

// the multigrid of the current assembly (built on first use, its numeric part after every
// assembly); level 0 from the FP32 copy where the PCG uses it
int amg_prepare(hyb_ctx* c) {
  int st;
  if (!c->amg) {
    st = amg_create(c->nx, c->ny, c->nz, c->sz.nfn, c->pc_degree, c->pc_coarsest, c->row_ptr, c->col, c->val,
                    c->n_iface_axis, &c->amg);
    if (st) return st;
    c->amg_ready = false;
  }
  const bool want32 = use_op32(c);
  if (want32 && (st = prepare_op32(c))) return st;
  st = amg_set_fp32(c->amg, want32, c->val32, c->col32, c->fptr32, c->dsq);
  if (st < 0) return st;
  if (st == 1) c->amg_ready = false;
  if (!c->amg_ready) {
    if ((st = amg_numeric(c->amg, c->stream))) return st;
    c->amg_ready = true;
  }
  return HYB_OK;
}

int solve_impl(hyb_ctx* c, const double* b, double rtol, int maxit, double* lambda, int* iters, double* rel_res) {
  if (c->pc == HYB_PC_AMG) {
    // CG preconditioned by the aggregation multigrid (Sec. 4: H is H^1-like), FP64 values of H
    int st = amg_prepare(c);
    if (st) return st;
    const int tok = prof_begin(&c->prof, HYB_K_PCG_FUSED, c->stream);
    st = amg_pcg(c->amg, b, rtol, maxit, lambda, c->r, c->p, c->q, c->flags, c->scal, c->partial, c->stream, iters,
                 rel_res);
    prof_end(&c->prof, tok, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return HYB_ERR_CUDA;
    c->prof.collect();
    return st;
  }
  PcgArgs a{};
  a.n = c->n_lambda;
  a.row_ptr = c->row_ptr;
  a.col = c->col;
  a.val = c->val;
  a.b = b;
  a.x = lambda;
  a.r = c->r;
  a.p = c->p;
  a.q = c->q;
  a.dinv = c->dinv;
  a.z = c->fused ? c->z : nullptr;
  a.partial = c->partial;
  a.scal = c->scal;
  a.flags = c->flags;
  a.nblocks = c->nblocks;
  a.nfn = c->sz.nfn;
  // the FP32 operator only where every element took the FP32 path (contrast <= threshold
  // everywhere): an element above the threshold brings a near-null mode of H whose eigenvalue
  // the FP32 rounding cannot hold (soft-hard test, Sec. 6.1, mass 10^-8: PCG breakdown)
  if (use_op32(c) && c->fused) {
    // the solver's preparation of the operator, like D^-1 for the FP64 values: the scaled FP32
    // copy of H (H carries the FP32 elimination's error anyway; its FP64 values stay the
    // reference that hyb_refine's exact residual is measured against)
    int st = prepare_op32(c);
    if (st) return st;
    a.val32 = c->val32;
    a.z32 = c->z32;
    a.dsq = c->dsq;
    a.fptr32 = c->fptr32;
    a.col32 = c->col32;
  }
  cudaError_t e = pcg_init(a, c->stream, &c->prof);
  if (e != cudaSuccess) return cuda_status(e);
  int hf[4] = {0, 0, 0, 0};
  double hs[8] = {0};
  int done = 0;
  const int chunk = c->fused ? 64 : 32;
  for (;;) {
    e = cudaMemcpyAsync(hf, c->flags, sizeof(hf), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    c->prof.collect();
    done = hf[0];
    if (hf[1] || hf[2] || done >= maxit) break;
    const int n = std::min(chunk, maxit - done);
    if (c->fused) {
      e = cudaMemsetAsync(c->gridbar, 0, 2 * sizeof(unsigned long long), c->stream);
      if (e == cudaSuccess) e = pcg_iterations_fused(a, n, rtol, c->gridbar, c->stream, &c->prof);
    } else {
      e = pcg_iterations(a, n, rtol, c->stream, &c->prof);
    }
    if (e != cudaSuccess) return cuda_status(e);
  }
  e = cudaMemcpyAsync(hs, c->scal, sizeof(hs), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_status(e);
  if (iters) *iters = done;
  if (rel_res) *rel_res = hs[1] > 0.0 ? std::sqrt(hs[2] / hs[1]) : 0.0;
  if (hf[2] == 2) return HYB_ERR_TIMEOUT;
  if (hf[2]) return HYB_ERR_BREAKDOWN;
  if (!hf[1]) return HYB_ERR_NOT_CONVERGED;
  return HYB_OK;
}

}  // namespace

int hyb_solve_reduced(hyb_ctx* c, double rtol, int maxit, double* lambda, int* iters, double* rel_res) {
  if (!c || !lambda || maxit < 0 || !(rtol >= 0.0)) return HYB_ERR_INVALID_ARG;
  if (c->mode == MODE_NONE) return HYB_ERR_INVALID_ARG;
  return solve_impl(c, c->rhs, rtol, maxit, lambda, iters, rel_res);
}

int hyb_refine(hyb_ctx* c, int steps, double inner_rtol, int maxit, double* lambda, double* u, double* jump) {
  if (!c || !lambda || !u || steps < 0 || maxit < 0 || !(inner_rtol >= 0.0)) return HYB_ERR_INVALID_ARG;
  if (c->mode != MODE_HYB) return HYB_ERR_INVALID_ARG;
  int st;
  if (!c->rho) {
    if ((st = dalloc(c, &c->rho, c->n_lambda))) return st;
    if ((st = dalloc(c, &c->dlam, c->n_lambda))) return st;
  }
  JumpArgs j{};
  j.n_faces = c->n_ifaces;
  j.nfn = c->sz.nfn;
  j.n_loc = c->sz.n;
  j.ni = c->sz.ni;
  j.face_dof = c->face_dof;
  j.u = u;
  j.rho = c->rho;
  j.partial = c->partial;
  j.norm2 = c->rnorm;
  j.ticket = &c->flags[3];
  j.nblocks = c->nblocks;
  std::memcpy(j.wf, c->tabs[c->k].wf, sizeof(j.wf));
  cudaError_t e = launch_norm2(c->n_lambda, c->rhs, c->partial, c->nblocks, c->rnorm + 1, &c->flags[3], c->stream,
                               &c->prof);
  if (e != cudaSuccess) return cuda_status(e);
  for (int s = 0; s <= steps; ++s) {
    e = launch_face_jump(j, c->stream, &c->prof);
    if (e != cudaSuccess) return cuda_status(e);
    if (jump) {
      double hn[2] = {0, 0};
      e = cudaMemcpyAsync(hn, c->rnorm, sizeof(hn), cudaMemcpyDeviceToHost, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      if (e != cudaSuccess) return cuda_status(e);
      jump[s] = hn[1] > 0.0 ? std::sqrt(hn[0] / hn[1]) : std::sqrt(hn[0]);
    }
    if (s == steps) break;
    st = solve_impl(c, c->rho, inner_rtol, maxit, c->dlam, nullptr, nullptr);
    if (st != HYB_OK && st != HYB_ERR_NOT_CONVERGED) return st;
    e = launch_axpy(c->n_lambda, c->dlam, lambda, c->stream, &c->prof);
    if (e != cudaSuccess) return cuda_status(e);
    st = recover_impl(c, lambda, u, MODE_HYB);
    if (st != HYB_OK) return st;
  }
  e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? HYB_OK : cuda_status(e);
}

int hyb_set_natural_bc(hyb_ctx* c, int natural) {
  if (!c || (natural != 0 && natural != 1)) return HYB_ERR_INVALID_ARG;
  c->natural = natural;
  c->mode = MODE_NONE;                     // factors of the other reading are stale
  return HYB_OK;
}

int hyb_set_preconditioner(hyb_ctx* c, int kind, int chebyshev_degree, int coarsest) {
  if (!c || (kind != HYB_PC_JACOBI && kind != HYB_PC_AMG)) return HYB_ERR_INVALID_ARG;
  if (kind == HYB_PC_AMG && (chebyshev_degree < 1 || chebyshev_degree > 4 || coarsest < 1 || coarsest > 4096))
    return HYB_ERR_INVALID_ARG;
  if (kind == HYB_PC_AMG && (chebyshev_degree != c->pc_degree || coarsest != c->pc_coarsest)) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    amg_free(c->amg);
    c->amg = nullptr;
    c->amg_ready = false;
    c->pc_degree = chebyshev_degree;
    c->pc_coarsest = coarsest;
  }
  c->pc = kind;
  return HYB_OK;
}

int hyb_amg_apply(hyb_ctx* c, const double* r, double* z) {
  if (!c || !r || !z || c->mode == MODE_NONE || c->pc != HYB_PC_AMG) return HYB_ERR_INVALID_ARG;
  int st = amg_prepare(c);
  if (st) return st;
  if ((st = amg_apply(c->amg, r, z, c->stream))) return st;
  return cuda_status(cudaStreamSynchronize(c->stream));
}

int hyb_amg_info(hyb_ctx* c, int* levels, int64_t* sizes, double* lmax, int cap) {
  if (!c || !levels || cap < 0 || c->mode == MODE_NONE || c->pc != HYB_PC_AMG) return HYB_ERR_INVALID_ARG;
  int st = amg_prepare(c);
  if (st) return st;
  std::vector<int64_t> sz(64);
  *levels = amg_levels(c->amg, sz.data(), 64);
  for (int l = 0; l < *levels && l < cap; ++l) {
    if (sizes) sizes[l] = sz[l];
    if (lmax) lmax[l] = amg_lmax(c->amg, l);
  }
  return HYB_OK;
}

int hyb_set_mixed_operator(hyb_ctx* c, int fp32) {
  if (!c || (fp32 != 0 && fp32 != 1)) return HYB_ERR_INVALID_ARG;
  if (c->precision != HYB_MIXED) return HYB_ERR_INVALID_ARG;
  c->op32 = fp32;
  return HYB_OK;
}

int hyb_set_pcg_fused(hyb_ctx* c, int on) {
  if (!c || (on != 0 && on != 1)) return HYB_ERR_INVALID_ARG;
  if (on) {
    int dev = 0, coop = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (!coop) return HYB_ERR_INVALID_ARG;
  }
  c->fused = on;
  return HYB_OK;
}

int hyb_recover(hyb_ctx* ctx, const double* lambda, double* u) {
  return recover_impl(ctx, lambda, u, MODE_HYB);
}

int staticcond_recover(hyb_ctx* ctx, const double* u_face, double* u) {
  return recover_impl(ctx, u_face, u, MODE_SC);
}

int hyb_get_reduced(hyb_ctx* c, const int64_t** row_ptr, const int32_t** col, const double** val,
                    const double** rhs, int64_t* n, int64_t* nnz) {
  if (!c) return HYB_ERR_INVALID_ARG;
  if (row_ptr) *row_ptr = c->row_ptr;
  if (col) *col = c->col;
  if (val) *val = c->val;
  if (rhs) *rhs = c->rhs;
  if (n) *n = c->n_lambda;
  if (nnz) *nnz = c->nnz;
  return HYB_OK;
}

int hyb_export_reduced(hyb_ctx* c, int64_t* row_ptr, int32_t* col, double* val, double* rhs) {
  if (!c) return HYB_ERR_INVALID_ARG;
  cudaError_t e = cudaSuccess;
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    if (dst && e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream);
  };
  cp(row_ptr, c->row_ptr, (c->n_lambda + 1) * sizeof(int64_t));
  cp(col, c->col, c->nnz * sizeof(int32_t));
  cp(val, c->val, c->nnz * sizeof(double));
  cp(rhs, c->rhs, c->n_lambda * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_status(e);
}

int hyb_set_profiling(hyb_ctx* c, int enable) {
  if (!c) return HYB_ERR_INVALID_ARG;
  if (c->stream) cudaStreamSynchronize(c->stream);
  c->prof.collect();
  c->prof.reset();
  c->prof.on = enable != 0;
  return HYB_OK;
}

int hyb_get_profile(const hyb_ctx* c, int kernel_class, double* total_ms, int64_t* launches) {
  if (!c || kernel_class < 0 || kernel_class >= HYB_K_COUNT) return HYB_ERR_INVALID_ARG;
  if (total_ms) *total_ms = c->prof.ms[kernel_class];
  if (launches) *launches = c->prof.launches[kernel_class];
  return HYB_OK;
}

int hyb_get_precision_split(const hyb_ctx* c, int64_t* n_fp64, int64_t* n_fp32, double* threshold) {
  if (!c) return HYB_ERR_INVALID_ARG;
  const bool mixed = c->precision == HYB_MIXED;
  if (n_fp64) *n_fp64 = mixed ? c->n_path[0] : c->E;
  if (n_fp32) *n_fp32 = mixed ? c->n_path[1] : 0;
  if (threshold) *threshold = mixed ? c->theta : 0.0;
  return HYB_OK;
}

int hyb_get_sizes(const hyb_ctx* c, int64_t* n_elem, int* n_loc, int64_t* n_lambda, int64_t* nnz) {
  if (!c) return HYB_ERR_INVALID_ARG;
  if (n_elem) *n_elem = c->E;
  if (n_loc) *n_loc = c->sz.n;
  if (n_lambda) *n_lambda = c->n_lambda;
  if (nnz) *nnz = c->nnz;
  return HYB_OK;
}

int hyb_last_error_element(const hyb_ctx* c, int64_t* element) {
  if (!c || !element) return HYB_ERR_INVALID_ARG;
  *element = c->last_err_elem;
  return HYB_OK;
}

void hyb_destroy(hyb_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  amg_free(c->amg);
  for (void* p : c->allocs) cudaFree(p);
  delete c;
}

const char* hyb_status_string(int s) {
  switch (s) {
    case HYB_OK: return "HYB_OK";
    case HYB_ERR_INVALID_ARG: return "HYB_ERR_INVALID_ARG";
    case HYB_ERR_UNSUPPORTED_ORDER: return "HYB_ERR_UNSUPPORTED_ORDER";
    case HYB_ERR_MESH: return "HYB_ERR_MESH";
    case HYB_ERR_NOT_SPD: return "HYB_ERR_NOT_SPD";
    case HYB_ERR_NOT_CONVERGED: return "HYB_ERR_NOT_CONVERGED";
    case HYB_ERR_BREAKDOWN: return "HYB_ERR_BREAKDOWN";
    case HYB_ERR_CUDA: return "HYB_ERR_CUDA";
    case HYB_ERR_OOM: return "HYB_ERR_OOM";
    case HYB_ERR_TIMEOUT: return "HYB_ERR_TIMEOUT";
  }
  return "HYB_ERR_UNKNOWN";
}

}  // extern "C"

// ============================================================================================
// Batched problems: many independent meshes of uneven size and order. Set-up reuses the
// single-problem set-up per problem; every phase then launches once per (order, colour,
// precision path) over (problem, element) work items with per-problem arguments read from
// device arrays, and the reduced solves run as one batched PCG whose blocks are partitioned
// by problem (each problem keeps its own scalars, so its iterates equal a solo solve's).
struct hyb_batch {
  int nprob = 0;
  cudaStream_t stream = nullptr;
  int precision = HYB_FP64;
  std::vector<hyb_ctx*> ctx;
  std::vector<int> order;
  std::vector<ElemArgs> h_eargs;
  std::vector<RecoverArgs> h_rargs;
  std::vector<PcgArgs> h_pargs;
  ElemArgs* d_eargs = nullptr;
  RecoverArgs* d_rargs = nullptr;
  PcgArgs* d_pargs = nullptr;
  const double** d_lams = nullptr;
  double** d_us = nullptr;
  int egrid[kMaxOrder + 1][2] = {};         // [order][path]: CTAs of the element launch (0: one per element)
  int emult[kMaxOrder + 1][2] = {};         // the autotuned choice: multiple of the resident CTAs, 0 = per element
  int2* items[kMaxOrder + 1][2][2] = {};    // [order][colour][path]
  int64_t n_items[kMaxOrder + 1][2][2] = {};
  int2* ritems[kMaxOrder + 1][2] = {};      // [order][path]
  int64_t n_ritems[kMaxOrder + 1][2] = {};
  int32_t *spmv_prob = nullptr, *spmv_first = nullptr, *spmv_count = nullptr;
  int32_t *vec_prob = nullptr, *vec_first = nullptr, *vec_count = nullptr;
  int n_spmv = 0, n_vec = 0;
  int* flags_all = nullptr;
  double* scal_all = nullptr;
  int* status = nullptr;
  std::vector<void*> allocs;
  Prof prof;
  int mode = MODE_NONE;
  // the 32-iteration chunk of the batched PCG as a CUDA graph (captured on a private stream,
  // launched on `stream`); re-captured when rtol changes
  bool use_fused = false;                  // team-fused cooperative PCG, or three launches per iteration (default)
  int4* d_team = nullptr;                  // per-launch block tables of the team-fused form
  int team_cap = 0;
  bool use_graph = true;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  double graph_rtol = -1.0;
  // the whole step (hyb_batch_step) as one graph: element phase, PCG initialisation, the PCG
  // loop as a device-driven WHILE node, recovery; rebuilt when rtol or maxit changes
  cudaGraph_t step_graph = nullptr;
  cudaGraphExec_t step_exec = nullptr;
  double step_rtol = -1.0;
  int step_maxit = -1;
  int64_t step_kernels = 0;                // kernel nodes outside the loop body
  int64_t step_body_kernels = 0;           // kernel nodes of one pass of the loop body
  std::vector<PcgArgs> h_pargs_step;
};

namespace {

template <class T>
int balloc(hyb_batch* b, T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) count = 1;
  void* p = nullptr;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return HYB_ERR_OOM;
  }
  b->allocs.push_back(p);
  *ptr = static_cast<T*>(p);
  return HYB_OK;
}

template <class T>
int bupload(hyb_batch* b, T** dst, const std::vector<T>& src) {
  int st = balloc(b, dst, src.size());
  if (st) return st;
  if (!src.empty() &&
      cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
    return HYB_ERR_CUDA;
  return HYB_OK;
}

int batch_finish(hyb_batch* b) {
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  b->prof.collect();
  if (st != 0) {
    // the failing element's id is recorded by its own problem
    for (hyb_ctx* c : b->ctx) {
      long long el = -1;
      if (cudaMemcpy(&el, c->err_elem, sizeof(long long), cudaMemcpyDeviceToHost) == cudaSuccess && el >= 0)
        c->last_err_elem = el;
    }
  }
  return st;
}

int batch_reset(hyb_batch* b) {
  cudaError_t e = cudaMemsetAsync(b->status, 0, sizeof(int), b->stream);
  for (hyb_ctx* c : b->ctx)
    if (e == cudaSuccess) e = cudaMemsetAsync(c->err_elem, 0xff, sizeof(long long), b->stream);
  return cuda_status(e);
}

int setup_batch_impl(hyb_batch* b, const hyb_mesh* meshes, const int* orders, const double* const* alphas,
                     const double* const* betas, double theta) {
  int st;
  std::vector<int2> items[kMaxOrder + 1][2][2], ritems[kMaxOrder + 1][2];
  for (int p = 0; p < b->nprob; ++p) {
    if (orders[p] < 0 || orders[p] > kMaxOrder) return HYB_ERR_UNSUPPORTED_ORDER;
    hyb_ctx* c = new (std::nothrow) hyb_ctx();
    if (!c) return HYB_ERR_OOM;
    c->stream = b->stream;
    b->ctx.push_back(c);
    b->order.push_back(orders[p]);
    if ((st = setup_impl(c, &meshes[p], orders[p], alphas[p], betas[p], b->precision, theta))) return st;
    const int k = orders[p];
    for (int col = 0; col < 2; ++col)
      for (int path = 0; path < 2; ++path)
        for (int32_t e : c->h_list[col][path]) {
          items[k][col][path].push_back(make_int2(p, e));
          ritems[k][path].push_back(make_int2(p, e));
        }
  }
  if ((st = balloc(b, &b->status, 1))) return st;
  if ((st = balloc(b, &b->flags_all, 4 * (size_t)b->nprob))) return st;
  if ((st = balloc(b, &b->scal_all, 8 * (size_t)b->nprob))) return st;
  for (int k = 0; k <= kMaxOrder; ++k)
    for (int path = 0; path < 2; ++path) {
      for (int col = 0; col < 2; ++col) {
        b->n_items[k][col][path] = (int64_t)items[k][col][path].size();
        if ((st = bupload(b, &b->items[k][col][path], items[k][col][path]))) return st;
      }
      b->n_ritems[k][path] = (int64_t)ritems[k][path].size();
      if ((st = bupload(b, &b->ritems[k][path], ritems[k][path]))) return st;
    }
  // per-problem arguments (pointers that change per call are filled in by the phases)
  std::vector<int32_t> sp, sf, sc, vp, vf, vc;
  for (int p = 0; p < b->nprob; ++p) {
    hyb_ctx* c = b->ctx[p];
    ElemArgs a = elem_args(c, nullptr, nullptr, 0);
    a.slot = c->slot;
    a.Lstore32 = c->Lstore32;
    a.status = b->status;
    b->h_eargs.push_back(a);
    RecoverArgs r{};
    r.k = c->k;
    r.mode = MODE_HYB;
    r.elem_face = c->elem_face;
    r.Lstore = c->Lstore;
    r.zstore = c->zstore;
    r.slot = c->slot;
    r.status = b->status;
    r.err_elem = c->err_elem;
    std::memcpy(r.wf, c->tabs[c->k].wf, sizeof(r.wf));
    b->h_rargs.push_back(r);
    PcgArgs g{};
    g.n = c->n_lambda;
    g.row_ptr = c->row_ptr;
    g.col = c->col;
    g.val = c->val;
    g.b = c->rhs;
    g.r = c->r;
    g.p = c->p;
    g.q = c->q;
    g.dinv = c->dinv;
    g.z = c->z;                            // the team-fused form keeps z and a barrier counter per problem
    g.bar = c->gridbar;
    g.partial = c->partial;
    g.scal = b->scal_all + 8 * p;
    g.flags = b->flags_all + 4 * p;
    g.nblocks = c->nblocks;
    g.nfn = c->sz.nfn;
    b->h_pargs.push_back(g);
    // problem-aligned block ranges: about 64k nonzeros per SpMV block, 8k rows per vector block
    const int nbs = (int)std::max<int64_t>(1, std::min<int64_t>(c->nblocks * 5 / 8, (c->nnz + 65535) / 65536));
    const int nbv = (int)std::max<int64_t>(1, std::min<int64_t>(c->nblocks / 4, (c->n_lambda + 8191) / 8192));
    sf.push_back((int32_t)sp.size());
    sc.push_back(nbs);
    for (int i = 0; i < nbs; ++i) sp.push_back(p);
    vf.push_back((int32_t)vp.size());
    vc.push_back(nbv);
    for (int i = 0; i < nbv; ++i) vp.push_back(p);
  }
  b->n_spmv = (int)sp.size();
  b->n_vec = (int)vp.size();
  if ((st = bupload(b, &b->spmv_prob, sp)) || (st = bupload(b, &b->spmv_first, sf)) ||
      (st = bupload(b, &b->spmv_count, sc)) || (st = bupload(b, &b->vec_prob, vp)) ||
      (st = bupload(b, &b->vec_first, vf)) || (st = bupload(b, &b->vec_count, vc)))
    return st;
  if ((st = bupload(b, &b->d_eargs, b->h_eargs)) || (st = bupload(b, &b->d_rargs, b->h_rargs)) ||
      (st = bupload(b, &b->d_pargs, b->h_pargs)))
    return st;
  if ((st = balloc(b, &b->d_lams, b->nprob)) || (st = balloc(b, &b->d_us, b->nprob))) return st;
  return cuda_status(cudaStreamSynchronize(b->stream));
}

// ---- autotuner of the batched element launches: per (device, order, precision path) the grid
// as a multiple of the CTAs that fit on the GPU at once (1, 2 or 4: persistent CTAs, each taking
// about elements / grid elements in turn), or 0 (one CTA per element, the hardware scheduler
// balancing), whichever runs the element phase of a unit-cube problem of that order fastest
// (16^3 elements, RT_3 12^3; two colours, two repetitions after a warm-up). Cached per process.
std::mutex g_grid_mutex;
std::map<std::tuple<int, int, int>, int> g_grid_mult;

int batch_resident_ctas(int order, int path) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return sms * (path ? mixed_batch_ctas_per_sm(order) : element_batch_ctas_per_sm(order));
}

int autotune_batch_grid(int order, int path, cudaStream_t s, int* mult) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HYB_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_grid_mutex);
  const auto key = std::make_tuple(dev, order, path);
  const auto it = g_grid_mult.find(key);
  if (it != g_grid_mult.end()) {
    *mult = it->second;
    return HYB_OK;
  }
  const int n = order >= 3 ? 12 : 16;
  const int64_t E = (int64_t)n * n * n, nv = (int64_t)(n + 1) * (n + 1) * (n + 1);
  const int nloc = Sizes::of(order).n;
  std::vector<double> vh(3 * nv);
  for (int l = 0; l <= n; ++l)
    for (int j = 0; j <= n; ++j)
      for (int i = 0; i <= n; ++i) {
        const int64_t v = i + (int64_t)(n + 1) * (j + (int64_t)(n + 1) * l);
        vh[3 * v] = (double)i / n;
        vh[3 * v + 1] = (double)j / n;
        vh[3 * v + 2] = (double)l / n;
      }
  std::vector<double> ones(E, 1.0);
  double* buf = nullptr;
  if (cudaMalloc(&buf, (3 * nv + 2 * E + E * nloc) * sizeof(double)) != cudaSuccess) return HYB_ERR_OOM;
  double *verts = buf, *alpha = buf + 3 * nv, *beta = alpha + E, *load = beta + E;
  cudaError_t e = cudaMemcpyAsync(verts, vh.data(), vh.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(alpha, ones.data(), E * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(beta, ones.data(), E * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(load, 0, (size_t)E * nloc * sizeof(double), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int st = e == cudaSuccess ? HYB_OK : cuda_status(e);
  hyb_batch* t = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int best = 0;
  if (st == HYB_OK) {
    t = new (std::nothrow) hyb_batch();
    if (!t) st = HYB_ERR_OOM;
  }
  if (st == HYB_OK) {
    t->nprob = 1;
    t->stream = s;
    t->precision = path ? HYB_MIXED : HYB_FP64;
    hyb_mesh mesh{n, n, n, verts};
    const double* al = alpha;
    const double* be = beta;
    st = setup_batch_impl(t, &mesh, &order, &al, &be, path ? 1e300 : 0.0);
  }
  if (st == HYB_OK) {
    t->h_eargs[0].load = load;
    e = cudaMemcpyAsync(t->d_eargs, t->h_eargs.data(), sizeof(ElemArgs), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int resident = batch_resident_ctas(order, path);
    float best_ms = 0.0f;
    const int cand[4] = {0, 1, 2, 4};
    for (int c = 0; c < 4 && e == cudaSuccess && resident > 0; ++c) {
      const int grid = cand[c] * resident;
      auto run = [&]() {
        cudaError_t r = cudaSuccess;
        for (int col = 0; col < 2 && r == cudaSuccess; ++col)
          r = path ? launch_mixed_batch(order, t->d_eargs, t->items[order][col][1], t->n_items[order][col][1], col,
                                        false, nullptr, nullptr, grid, s, nullptr)
                   : launch_element_batch(order, MODE_HYB, t->d_eargs, t->items[order][col][0],
                                          t->n_items[order][col][0], col, grid, s, nullptr);
        return r;
      };
      e = run();                                       // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, s);
      for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = run();
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && (c == 0 || ms < best_ms)) {
        best_ms = ms;
        best = cand[c];
      }
    }
    if (e != cudaSuccess) st = cuda_status(e);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (t) hyb_destroy_batch(t);
  cudaFree(buf);
  if (st != HYB_OK) return st;
  g_grid_mult[key] = best;
  *mult = best;
  return HYB_OK;
}

// Batched PCG in the team-fused form: between chunks of 64 iterations the host reads every
// problem's flags, sorts the unconverged problems by size and runs them in groups of at most
// an eighth as many problems as the cooperative grid has blocks, one launch per group, the
// grid split in proportion to their nonzeros (at least one block each: with few problems per
// launch that floor costs little, and problems of similar size share a launch). The last,
// largest problems get the whole GPU.
int solve_batch_team(hyb_batch* b, double rtol, int maxit, int* iters, double* rel_res) {
  cudaError_t e = cudaSuccess;
  int st;
  constexpr int kSlots = 8;                        // block tables in flight per chunk
  if (!b->d_team) {
    if ((e = pcg_team_capacity(&b->team_cap)) != cudaSuccess) return cuda_status(e);
    if (b->team_cap < 1) return HYB_ERR_CUDA;
    if ((st = balloc(b, &b->d_team, (size_t)kSlots * b->team_cap))) return st;
  }
  const int cap = b->team_cap;
  std::vector<int> hf(4 * (size_t)b->nprob);
  std::vector<int4> table;
  for (;;) {
    e = cudaMemcpyAsync(hf.data(), b->flags_all, hf.size() * sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_status(e);
    b->prof.collect();
    int done = 0;
    std::vector<int> L;
    for (int p = 0; p < b->nprob; ++p) {
      done = std::max(done, hf[4 * p]);
      if (!hf[4 * p + 1] && !hf[4 * p + 2]) L.push_back(p);
    }
    if (L.empty() || done >= maxit) break;
    const int n = std::min(64, maxit - done);
    if ((e = pcg_zero_bars(b->d_pargs, b->nprob, b->stream)) != cudaSuccess) return cuda_status(e);
    std::sort(L.begin(), L.end(), [&](int x, int y) { return b->ctx[x]->nnz > b->ctx[y]->nnz; });
    int slot = 0;
    const size_t per_launch = (size_t)std::max(1, cap / 8);
    for (size_t g0 = 0; g0 < L.size(); g0 += per_launch) {
      const size_t g1 = std::min(L.size(), g0 + per_launch);
      const int m = (int)(g1 - g0);
      double wsum = 0.0;
      for (size_t i = g0; i < g1; ++i) wsum += (double)b->ctx[L[i]]->nnz;
      std::vector<int> nb(m, 1);
      int used = m;
      for (int i = 0; i < m; ++i) {                // one block each, the rest in proportion to nnz
        const int extra = (int)((double)(cap - m) * (double)b->ctx[L[g0 + i]]->nnz / wsum);
        nb[i] += extra;
        used += extra;
      }
      for (int i = 0; used < cap && i < m; ++i, ++used) nb[i] += 1;
      table.clear();
      for (int i = 0; i < m; ++i)
        for (int v = 0; v < nb[i]; ++v) table.push_back(make_int4(L[g0 + i], v, nb[i], 0));
      if (slot == kSlots) {                        // every table in use: let the launches drain
        if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return cuda_status(e);
        slot = 0;
      }
      int4* dt = b->d_team + (size_t)slot * cap;
      ++slot;
      e = cudaMemcpyAsync(dt, table.data(), table.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream);
      if (e == cudaSuccess) e = pcg_iterations_team(b->d_pargs, dt, (int)table.size(), n, rtol, b->stream, &b->prof);
      if (e != cudaSuccess) return cuda_status(e);
    }
  }
  std::vector<double> hs(8 * (size_t)b->nprob);
  e = cudaMemcpyAsync(hs.data(), b->scal_all, hs.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_status(e);
  st = HYB_OK;
  for (int p = 0; p < b->nprob; ++p) {
    if (iters) iters[p] = hf[4 * p];
    if (rel_res) rel_res[p] = hs[8 * p + 1] > 0.0 ? std::sqrt(hs[8 * p + 2] / hs[8 * p + 1]) : 0.0;
    if (hf[4 * p + 2] == 2) st = HYB_ERR_TIMEOUT;
    else if (hf[4 * p + 2] && st == HYB_OK) st = HYB_ERR_BREAKDOWN;
    else if (!hf[4 * p + 1] && st == HYB_OK) st = HYB_ERR_NOT_CONVERGED;
  }
  return st;
}

// Iterations per pass of the WHILE body of the batched step (the loop stops within a pass once
// every problem has converged: the kernels of a stopped problem return at once).
constexpr int kStepChunk = 16;

// Element phase of the batch on stream s (no profiling: it may be captured).
cudaError_t enqueue_batch_elements(hyb_batch* b, cudaStream_t s, int64_t* kernels) {
  cudaError_t e = cudaSuccess;
  for (int col = 0; col < 2 && e == cudaSuccess; ++col)
    for (int k = 0; k <= kMaxOrder && e == cudaSuccess; ++k) {
      if (b->n_items[k][col][0]) {
        e = launch_element_batch(k, MODE_HYB, b->d_eargs, b->items[k][col][0], b->n_items[k][col][0], col,
                                 b->egrid[k][0], s, nullptr);
        ++*kernels;
      }
      if (e == cudaSuccess && b->n_items[k][col][1]) {
        e = launch_mixed_batch(k, b->d_eargs, b->items[k][col][1], b->n_items[k][col][1], col, false, nullptr, nullptr,
                               b->egrid[k][1], s, nullptr);
        ++*kernels;
      }
    }
  return e;
}

cudaError_t enqueue_batch_recovery(hyb_batch* b, cudaStream_t s, int64_t* kernels) {
  cudaError_t e = cudaSuccess;
  for (int k = 0; k <= kMaxOrder && e == cudaSuccess; ++k) {
    if (b->n_ritems[k][0]) {
      e = launch_recover_batch(k, MODE_HYB, b->d_rargs, b->ritems[k][0], b->n_ritems[k][0], s, nullptr);
      ++*kernels;
    }
    if (e == cudaSuccess && b->n_ritems[k][1]) {
      e = launch_mixed_batch(k, b->d_eargs, b->ritems[k][1], b->n_ritems[k][1], 0, true, b->d_lams, b->d_us, 0, s,
                             nullptr);
      ++*kernels;
    }
  }
  return e;
}

void destroy_step_graph(hyb_batch* b) {
  if (b->step_exec) cudaGraphExecDestroy(b->step_exec);
  if (b->step_graph) cudaGraphDestroy(b->step_graph);
  b->step_exec = nullptr;
  b->step_graph = nullptr;
}

// Builds the step graph by capturing on a private stream into a graph made here:
//   [status resets, element launches (both colours in order), PCG flags reset, batched PCG
//    initialisation] -> WHILE(condition) { kStepChunk batched iterations; condition kernel }
//   -> [recovery launches].
// The WHILE condition starts at 1 and is rewritten by the last kernel of every pass.
int build_step_graph(hyb_batch* b, double rtol) {
  destroy_step_graph(b);
  cudaError_t e = cudaSuccess;
  if (!b->cap_stream) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  cudaGraph_t g = nullptr;
  if (e == cudaSuccess) e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return cuda_status(e);
  b->step_graph = g;
  cudaStream_t cs = b->cap_stream;
  PcgBatch pb{b->d_pargs, b->spmv_prob, b->spmv_first, b->spmv_count, b->vec_prob, b->vec_first, b->vec_count,
              b->n_spmv, b->n_vec};
  int64_t nk = 0, nbody = 0;
  std::vector<cudaGraphNode_t> tail;
  e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaError_t el = cudaMemsetAsync(b->status, 0, sizeof(int), cs);
    for (hyb_ctx* c : b->ctx)
      if (el == cudaSuccess) el = cudaMemsetAsync(c->err_elem, 0xff, sizeof(long long), cs);
    if (el == cudaSuccess) el = enqueue_batch_elements(b, cs, &nk);
    if (el == cudaSuccess) el = cudaMemsetAsync(b->flags_all, 0, 4 * (size_t)b->nprob * sizeof(int), cs);
    if (el == cudaSuccess) el = pcg_init_batch(pb, cs, nullptr);
    nk += 2;
    if (el == cudaSuccess) {
      cudaStreamCaptureStatus st;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      el = cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &deps, nullptr, &nd);
      if (el == cudaSuccess) tail.assign(deps, deps + nd);
    }
    e = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = el;
  }
  cudaGraphConditionalHandle h = 0;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cn = nullptr;
  if (e == cudaSuccess) e = cudaGraphAddNode(&cn, g, tail.data(), nullptr, tail.size(), &cp);
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaError_t el = pcg_iterations_batch(pb, kStepChunk, rtol, cs, nullptr);
      if (el == cudaSuccess) el = launch_pcg_continue(b->d_pargs, b->nprob, (unsigned long long)h, cs);
      nbody = 3 * kStepChunk + 1;
      e = cudaStreamEndCapture(cs, &body);
      if (e == cudaSuccess) e = el;
    }
  }
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, g, &cn, nullptr, 1, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaError_t el = enqueue_batch_recovery(b, cs, &nk);
    e = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = el;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->step_exec, g, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    destroy_step_graph(b);
    return cuda_status(e);
  }
  b->step_rtol = rtol;
  b->step_kernels = nk;
  b->step_body_kernels = nbody;
  return HYB_OK;
}

}  // namespace

extern "C" {

int hyb_setup_batch(int nprob, const hyb_mesh* meshes, const int* orders, const double* const* alphas,
                    const double* const* betas, int precision, double contrast_threshold, void* cuda_stream,
                    hyb_batch** out) {
  if (!out) return HYB_ERR_INVALID_ARG;
  *out = nullptr;
  if (nprob < 1 || !meshes || !orders || !alphas || !betas) return HYB_ERR_INVALID_ARG;
  if (precision != HYB_FP64 && precision != HYB_MIXED) return HYB_ERR_INVALID_ARG;
  if (!(contrast_threshold >= 0.0)) return HYB_ERR_INVALID_ARG;
  for (int p = 0; p < nprob; ++p) {
    if (!meshes[p].vertices || !alphas[p] || !betas[p]) return HYB_ERR_INVALID_ARG;
    if (meshes[p].nx < 1 || meshes[p].ny < 1 || meshes[p].nz < 1) return HYB_ERR_INVALID_ARG;
  }
  hyb_batch* b = new (std::nothrow) hyb_batch();
  if (!b) return HYB_ERR_OOM;
  b->nprob = nprob;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->precision = precision;
  int st;
  try {
    st = setup_batch_impl(b, meshes, orders, alphas, betas, contrast_threshold);
    // elements per CTA of every order bin and precision path present, autotuned per device
    for (int k = 0; k <= kMaxOrder && st == HYB_OK; ++k)
      for (int path = 0; path < 2 && st == HYB_OK; ++path) {
        if (!b->n_items[k][0][path] && !b->n_items[k][1][path]) continue;
        int mult = 0;
        st = autotune_batch_grid(k, path, b->stream, &mult);
        b->emult[k][path] = mult;
        b->egrid[k][path] = mult * batch_resident_ctas(k, path);
      }
  } catch (const std::bad_alloc&) {
    st = HYB_ERR_OOM;
  } catch (...) {
    st = HYB_ERR_CUDA;
  }
  if (st != HYB_OK) {
    hyb_destroy_batch(b);
    return st;
  }
  *out = b;
  return HYB_OK;
}

int hyb_assemble_reduced_batch(hyb_batch* b, const double* const* loads, const double* const* ess) {
  if (!b || !loads) return HYB_ERR_INVALID_ARG;
  for (int p = 0; p < b->nprob; ++p) {
    if (!loads[p]) return HYB_ERR_INVALID_ARG;
    b->h_eargs[p].load = loads[p];
    b->h_eargs[p].ess = ess ? ess[p] : nullptr;
  }
  cudaError_t e = cudaMemcpyAsync(b->d_eargs, b->h_eargs.data(), b->h_eargs.size() * sizeof(ElemArgs),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) return cuda_status(e);
  int st = batch_reset(b);
  if (st) return st;
  b->mode = MODE_NONE;
  for (int col = 0; col < 2; ++col)
    for (int k = 0; k <= kMaxOrder; ++k) {
      e = launch_element_batch(k, MODE_HYB, b->d_eargs, b->items[k][col][0], b->n_items[k][col][0], col,
                               b->egrid[k][0], b->stream, &b->prof);
      if (e == cudaSuccess && b->n_items[k][col][1])
        e = launch_mixed_batch(k, b->d_eargs, b->items[k][col][1], b->n_items[k][col][1], col, false, nullptr,
                               nullptr, b->egrid[k][1], b->stream, &b->prof);
      if (e != cudaSuccess) return cuda_status(e);
    }
  st = batch_finish(b);
  if (st == HYB_OK) {
    b->mode = MODE_HYB;
    for (hyb_ctx* c : b->ctx) c->mode = MODE_HYB;
  }
  return st;
}

int hyb_solve_reduced_batch(hyb_batch* b, double rtol, int maxit, double* const* lambdas, int* iters,
                            double* rel_res) {
  if (!b || !lambdas || maxit < 0 || !(rtol >= 0.0)) return HYB_ERR_INVALID_ARG;
  if (b->mode != MODE_HYB) return HYB_ERR_INVALID_ARG;
  cudaError_t e = cudaSuccess;
  for (int p = 0; p < b->nprob && e == cudaSuccess; ++p) {
    if (!lambdas[p]) return HYB_ERR_INVALID_ARG;
    b->h_pargs[p].x = lambdas[p];
    PcgArgs a = b->h_pargs[p];
    if (!b->use_fused) a.z = nullptr;
    e = pcg_init(a, b->stream, &b->prof);
  }
  if (b->use_fused && e == cudaSuccess) {
    e = cudaMemcpyAsync(b->d_pargs, b->h_pargs.data(), b->h_pargs.size() * sizeof(PcgArgs), cudaMemcpyHostToDevice,
                        b->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return solve_batch_team(b, rtol, maxit, iters, rel_res);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_pargs, b->h_pargs.data(), b->h_pargs.size() * sizeof(PcgArgs), cudaMemcpyHostToDevice,
                        b->stream);
  if (e != cudaSuccess) return cuda_status(e);
  PcgBatch pb{b->d_pargs, b->spmv_prob, b->spmv_first, b->spmv_count, b->vec_prob, b->vec_first, b->vec_count,
              b->n_spmv, b->n_vec};
  std::vector<int> hf(4 * (size_t)b->nprob);
  int done = 0;
  for (;;) {
    e = cudaMemcpyAsync(hf.data(), b->flags_all, hf.size() * sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_status(e);
    b->prof.collect();
    bool active = false;
    done = 0;
    for (int p = 0; p < b->nprob; ++p) {
      done = std::max(done, hf[4 * p]);
      if (!hf[4 * p + 1] && !hf[4 * p + 2]) active = true;
    }
    if (!active || done >= maxit) break;
    const int n = std::min(32, maxit - done);
    if (b->use_graph && n == 32) {
      if (!b->graph_exec || b->graph_rtol != rtol) {
        if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->graph_exec = nullptr;
        b->graph = nullptr;
        if (!b->cap_stream) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          const cudaError_t el = pcg_iterations_batch(pb, 32, rtol, b->cap_stream, nullptr);
          e = cudaStreamEndCapture(b->cap_stream, &b->graph);
          if (e == cudaSuccess) e = el;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph_exec, b->graph, 0);
        if (e != cudaSuccess) return cuda_status(e);
        b->graph_rtol = rtol;
      }
      const int tok = prof_begin(&b->prof, HYB_K_PCG_FUSED, b->stream);
      e = cudaGraphLaunch(b->graph_exec, b->stream);
      prof_end(&b->prof, tok, b->stream);
    } else {
      e = pcg_iterations_batch(pb, n, rtol, b->stream, &b->prof);
    }
    if (e != cudaSuccess) return cuda_status(e);
  }
  std::vector<double> hs(8 * (size_t)b->nprob);
  e = cudaMemcpyAsync(hs.data(), b->scal_all, hs.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_status(e);
  int st = HYB_OK;
  for (int p = 0; p < b->nprob; ++p) {
    if (iters) iters[p] = hf[4 * p];
    if (rel_res) rel_res[p] = hs[8 * p + 1] > 0.0 ? std::sqrt(hs[8 * p + 2] / hs[8 * p + 1]) : 0.0;
    if (hf[4 * p + 2]) st = HYB_ERR_BREAKDOWN;
    else if (!hf[4 * p + 1] && st == HYB_OK) st = HYB_ERR_NOT_CONVERGED;
  }
  return st;
}

int hyb_recover_batch(hyb_batch* b, const double* const* lambdas, double* const* us) {
  if (!b || !lambdas || !us) return HYB_ERR_INVALID_ARG;
  if (b->mode != MODE_HYB) return HYB_ERR_INVALID_ARG;
  for (int p = 0; p < b->nprob; ++p) {
    if (!lambdas[p] || !us[p]) return HYB_ERR_INVALID_ARG;
    b->h_rargs[p].lambda = lambdas[p];
    b->h_rargs[p].u = us[p];
  }
  cudaError_t e = cudaMemcpyAsync(b->d_rargs, b->h_rargs.data(), b->h_rargs.size() * sizeof(RecoverArgs),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_lams, lambdas, b->nprob * sizeof(double*), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_us, us, b->nprob * sizeof(double*), cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) return cuda_status(e);
  int st = batch_reset(b);
  if (st) return st;
  for (int k = 0; k <= kMaxOrder; ++k) {
    e = launch_recover_batch(k, MODE_HYB, b->d_rargs, b->ritems[k][0], b->n_ritems[k][0], b->stream, &b->prof);
    if (e == cudaSuccess && b->n_ritems[k][1])
      e = launch_mixed_batch(k, b->d_eargs, b->ritems[k][1], b->n_ritems[k][1], 0, true, b->d_lams, b->d_us, 0,
                             b->stream, &b->prof);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return batch_finish(b);
}

int hyb_batch_step(hyb_batch* b, const double* const* loads, const double* const* ess, double rtol, int maxit,
                   double* const* lambdas, double* const* us, int* iters, double* rel_res) {
  if (!b || !loads || !lambdas || !us || maxit < 1 || !(rtol >= 0.0)) return HYB_ERR_INVALID_ARG;
  for (int p = 0; p < b->nprob; ++p)
    if (!loads[p] || !lambdas[p] || !us[p]) return HYB_ERR_INVALID_ARG;
  b->h_pargs_step = b->h_pargs;
  for (int p = 0; p < b->nprob; ++p) {
    b->h_eargs[p].load = loads[p];
    b->h_eargs[p].ess = ess ? ess[p] : nullptr;
    PcgArgs& a = b->h_pargs_step[p];
    a.x = lambdas[p];
    a.z = nullptr;                               // the three-launch form keeps D^-1 r in q
    a.maxit = maxit;
    b->h_pargs[p].x = lambdas[p];
    b->h_rargs[p].lambda = lambdas[p];
    b->h_rargs[p].u = us[p];
  }
  cudaStream_t s = b->stream;
  cudaError_t e = cudaMemcpyAsync(b->d_eargs, b->h_eargs.data(), b->h_eargs.size() * sizeof(ElemArgs),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_pargs, b->h_pargs_step.data(), b->h_pargs_step.size() * sizeof(PcgArgs),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_rargs, b->h_rargs.data(), b->h_rargs.size() * sizeof(RecoverArgs),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_lams, lambdas, b->nprob * sizeof(double*), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_us, us, b->nprob * sizeof(double*), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the argument arrays are in place before any capture
  if (e != cudaSuccess) return cuda_status(e);
  int st;
  if (!b->step_exec || b->step_rtol != rtol) {
    if ((st = build_step_graph(b, rtol))) return st;
  }
  b->step_maxit = maxit;
  b->mode = MODE_NONE;
  for (hyb_ctx* c : b->ctx) c->mode = MODE_NONE;
  const int tok = prof_begin(&b->prof, HYB_K_STEP, s);
  e = cudaGraphLaunch(b->step_exec, s);
  prof_end(&b->prof, tok, s);
  if (e != cudaSuccess) return cuda_status(e);
  std::vector<int> hf(4 * (size_t)b->nprob);
  std::vector<double> hs(8 * (size_t)b->nprob);
  e = cudaMemcpyAsync(hf.data(), b->flags_all, hf.size() * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hs.data(), b->scal_all, hs.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_status(e);
  if ((st = batch_finish(b))) return st;         // synchronises; element or recovery errors first
  b->mode = MODE_HYB;
  for (hyb_ctx* c : b->ctx) c->mode = MODE_HYB;
  st = HYB_OK;
  for (int p = 0; p < b->nprob; ++p) {
    if (iters) iters[p] = hf[4 * p];
    if (rel_res) rel_res[p] = hs[8 * p + 1] > 0.0 ? std::sqrt(hs[8 * p + 2] / hs[8 * p + 1]) : 0.0;
    if (hf[4 * p + 2]) st = HYB_ERR_BREAKDOWN;
    else if (!hf[4 * p + 1] && st == HYB_OK) st = HYB_ERR_NOT_CONVERGED;
  }
  return st;
}

int hyb_batch_step_kernels(const hyb_batch* b, int64_t* outside_loop, int64_t* per_pass, int* iterations_per_pass) {
  if (!b || !b->step_exec) return HYB_ERR_INVALID_ARG;
  if (outside_loop) *outside_loop = b->step_kernels;
  if (per_pass) *per_pass = b->step_body_kernels;
  if (iterations_per_pass) *iterations_per_pass = kStepChunk;
  return HYB_OK;
}

int hyb_batch_get_autotune(const hyb_batch* b, int order, int path, int* multiple, int* grid) {
  if (!b || order < 0 || order > kMaxOrder || path < 0 || path > 1) return HYB_ERR_INVALID_ARG;
  if (multiple) *multiple = b->emult[order][path];
  if (grid) *grid = b->egrid[order][path];
  return HYB_OK;
}

int hyb_batch_context(hyb_batch* b, int problem, hyb_ctx** ctx) {
  if (!b || !ctx || problem < 0 || problem >= b->nprob) return HYB_ERR_INVALID_ARG;
  *ctx = b->ctx[problem];
  return HYB_OK;
}

int hyb_batch_set_profiling(hyb_batch* b, int enable) {
  if (!b) return HYB_ERR_INVALID_ARG;
  if (b->stream) cudaStreamSynchronize(b->stream);
  b->prof.collect();
  b->prof.reset();
  b->prof.on = enable != 0;
  return HYB_OK;
}

int hyb_batch_get_profile(const hyb_batch* b, int kernel_class, double* total_ms, int64_t* launches) {
  if (!b || kernel_class < 0 || kernel_class >= HYB_K_COUNT) return HYB_ERR_INVALID_ARG;
  if (total_ms) *total_ms = b->prof.ms[kernel_class];
  if (launches) *launches = b->prof.launches[kernel_class];
  return HYB_OK;
}

int hyb_batch_set_pcg_fused(hyb_batch* b, int on) {
  if (!b || (on != 0 && on != 1)) return HYB_ERR_INVALID_ARG;
  b->use_fused = on != 0;
  return HYB_OK;
}

int hyb_batch_set_graphs(hyb_batch* b, int on) {
  if (!b || (on != 0 && on != 1)) return HYB_ERR_INVALID_ARG;
  b->use_graph = on != 0;
  return HYB_OK;
}

void hyb_destroy_batch(hyb_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  destroy_step_graph(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (hyb_ctx* c : b->ctx) hyb_destroy(c);
  for (void* p : b->allocs) cudaFree(p);
  delete b;
}

}  // extern "C"
