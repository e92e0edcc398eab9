// Multiplier layout of a two-level hexahedral mesh: a coarse nx x ny x nzc block under a fine
// block of mx x my x nzf cells, (mx, my) = (2 nx, 2 ny) with a 2:1 non-conforming interface or
// (nx, ny) with a conforming one (arXiv:1801.08914, Example 2.1: master / slave interface dofs,
// C = [0 -W_sm I_s]; Fig. 5.1 right). Host logic only: the numbering of the multiplier faces,
// each element's face -> multiplier-block table, the interface map W and the CSR pattern of
// H = C A^{-1} C^T (two multipliers couple when one element carries both).

#include <algorithm>
#include <cstdint>
#include <vector>

#include "hyb.h"
#include "hyb_internal.h"

namespace hyb {
namespace {

struct TwoLevel {
  int nx, ny, nzc, nzf, mx, my, r;
  int64_t Ec, E;
  int64_t nface = 0;                  // multiplier faces
  std::vector<int32_t> ef;            // E x 6: face id or -1
  std::vector<std::vector<int64_t>> elems_of;   // face -> elements carrying it

  // face ids of the interior faces of one structured block, in the numbering of the structured
  // meshes (by normal axis; plane index along it fastest, then the lower, then the higher
  // tangential cell index), offset by base
  void block_faces(int ax, int ay, int az, int64_t e0, int64_t base, int64_t* count) {
    const int dims[3] = {ax, ay, az};
    int64_t id = base;
    for (int d = 0; d < 3; ++d) {
      const int t0 = d == 0 ? 1 : 0, t1 = d == 2 ? 1 : 2;
      for (int c1 = 0; c1 < dims[t1]; ++c1)
        for (int c0 = 0; c0 < dims[t0]; ++c0)
          for (int pl = 1; pl < dims[d]; ++pl, ++id) {
            int lo[3], hi[3];
            lo[d] = pl - 1; hi[d] = pl;
            lo[t0] = hi[t0] = c0;
            lo[t1] = hi[t1] = c1;
            const int64_t el = e0 + lo[0] + (int64_t)ax * (lo[1] + (int64_t)ay * lo[2]);
            const int64_t eh = e0 + hi[0] + (int64_t)ax * (hi[1] + (int64_t)ay * hi[2]);
            ef[el * 6 + 2 * d + 1] = (int32_t)id;
            ef[eh * 6 + 2 * d] = (int32_t)id;
          }
    }
    *count = id - base;
  }

  bool build(int nx_, int ny_, int nzc_, int nzf_, bool refine) {
    nx = nx_; ny = ny_; nzc = nzc_; nzf = nzf_;
    r = refine ? 2 : 1;
    mx = r * nx; my = r * ny;
    Ec = (int64_t)nx * ny * nzc;
    E = Ec + (int64_t)mx * my * nzf;
    ef.assign((size_t)E * 6, -1);
    int64_t nc = 0, nf = 0;
    block_faces(nx, ny, nzc, 0, 0, &nc);
    block_faces(mx, my, nzf, Ec, nc, &nf);
    // interface faces grouped by coarse face: coarse face (I, J) carries ids base + r^2 (I + nx J)
    // .. + r^2 - 1, fine sub-face (a, b) at + a + r b
    const int64_t base = nc + nf;
    for (int J = 0; J < ny; ++J)
      for (int I = 0; I < nx; ++I) {
        const int64_t first = base + (int64_t)r * r * (I + (int64_t)nx * J);
        ef[(I + (int64_t)nx * (J + (int64_t)ny * (nzc - 1))) * 6 + 5] = (int32_t)first;
        for (int b = 0; b < r; ++b)
          for (int a = 0; a < r; ++a)
            ef[(Ec + (r * I + a) + (int64_t)mx * (r * J + b)) * 6 + 4] = (int32_t)(first + a + r * b);
      }
    nface = base + (int64_t)r * r * nx * ny;
    if (nface > INT32_MAX) return false;
    elems_of.assign((size_t)nface, {});
    for (int64_t e = 0; e < E; ++e)
      for (int f = 0; f < 6; ++f) {
        const int32_t id = ef[e * 6 + f];
        if (id < 0) continue;
        const bool split = refine && is_top(e) && f == 5;
        for (int s = 0; s < (split ? 4 : 1); ++s) elems_of[id + s].push_back(e);
      }
    return true;
  }

  // a coarse element of the top layer (its z1 face lies on the interface)
  bool is_top(int64_t e) const { return e < Ec && e >= Ec - (int64_t)nx * ny; }

  // multiplier faces an element carries (its face ids, the four sub-faces of a split top face)
  void faces_of(int64_t e, std::vector<int64_t>& out) const {
    for (int f = 0; f < 6; ++f) {
      const int32_t id = ef[e * 6 + f];
      if (id < 0) continue;
      const bool split = r == 2 && is_top(e) && f == 5;
      for (int s = 0; s < (split ? 4 : 1); ++s) out.push_back(id + s);
    }
  }
};

}  // namespace
}  // namespace hyb

extern "C" int hyb_two_level_layout(int nx, int ny, int nzc, int nzf, int order, int refine, int64_t* n_lambda,
                                    int64_t* nnz, int32_t* elem_face, double* W, int64_t* row_ptr, int32_t* col) {
  using namespace hyb;
  if (nx <= 0 || ny <= 0 || nzc <= 0 || nzf <= 0 || !n_lambda || !nnz) return HYB_ERR_INVALID_ARG;
  if (order < 0 || order > kMaxOrder) return HYB_ERR_UNSUPPORTED_ORDER;
  const int64_t nfn = (int64_t)(order + 1) * (order + 1);
  TwoLevel m;
  if (!m.build(nx, ny, nzc, nzf, refine != 0) || m.nface * nfn > INT32_MAX) return HYB_ERR_INVALID_ARG;
  // column faces of every multiplier face: the faces of the elements carrying it
  std::vector<std::vector<int64_t>> cols((size_t)m.nface);
  std::vector<int64_t> tmp;
  int64_t total = 0;
  for (int64_t f = 0; f < m.nface; ++f) {
    tmp.clear();
    for (int64_t e : m.elems_of[f]) m.faces_of(e, tmp);
    std::sort(tmp.begin(), tmp.end());
    tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
    cols[f] = tmp;
    total += (int64_t)tmp.size() * nfn * nfn;
  }
  *n_lambda = m.nface * nfn;
  *nnz = total;
  if (elem_face) std::copy(m.ef.begin(), m.ef.end(), elem_face);
  if (W && refine) build_interface_w(order, W);
  if (row_ptr) {
    int64_t at = 0;
    for (int64_t f = 0; f < m.nface; ++f)
      for (int64_t q = 0; q < nfn; ++q) {
        row_ptr[f * nfn + q] = at;
        if (col)
          for (int64_t g : cols[f])
            for (int64_t c = 0; c < nfn; ++c) col[at++] = (int32_t)(g * nfn + c);
        else
          at += (int64_t)cols[f].size() * nfn;
      }
    row_ptr[m.nface * nfn] = at;
  }
  return HYB_OK;
}
