// Reference 1-D tables: Gauss-Legendre / Gauss-Lobatto rules and Lagrange bases.
//
// The element integrals of Sec. 2.1 are evaluated with the (k+2)-point
// Gauss-Legendre rule per direction; the RT_k basis is nodal on closed
// Gauss-Lobatto nodes (k+2) along its component and open Gauss-Legendre nodes
// (k+1) across it. Nodes come from Newton's method on Legendre polynomials
// (three-term recurrence), weights from the classical closed forms
// (Abramowitz & Stegun 25.4.29 and 25.4.32).
#include <cmath>
#include <cstring>

#include "hyb_internal.h"

namespace hyb {
namespace {

// P_n(x) and P_n'(x), |x| < 1.
void legendre_pd(int n, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int m = 1; m < n; ++m) {
    double p2 = ((2 * m + 1) * x * p1 - m * p0) / (m + 1);
    p0 = p1; p1 = p2;
  }
  *p = p1;
  *dp = n * (x * p1 - p0) / (x * x - 1.0);
}

// q-point Gauss-Legendre on [0,1], ascending.
void gauss_legendre01(int q, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < q; ++i) {
    double t = -std::cos(pi * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre_pd(q, t, &p, &dp);
      double d = p / dp;
      t -= d;
      if (std::fabs(d) < 1e-16) break;
    }
    double p, dp;
    legendre_pd(q, t, &p, &dp);
    x[i] = 0.5 * (t + 1.0);
    w[i] = 1.0 / ((1.0 - t * t) * dp * dp);   // half of 2/((1-t^2)P'^2)
  }
}

// q-point Gauss-Lobatto nodes on [0,1] (q >= 2): ends plus the roots of P_{q-1}'.
void gauss_lobatto01(int q, double* x) {
  const double pi = 3.14159265358979323846;
  const int n = q - 1;
  x[0] = 0.0;
  x[q - 1] = 1.0;
  for (int i = 1; i < q - 1; ++i) {
    double t = -std::cos(pi * i / n);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre_pd(n, t, &p, &dp);
      double d2p = (2.0 * t * dp - n * (n + 1) * p) / (1.0 - t * t);
      double d = dp / d2p;
      t -= d;
      if (std::fabs(d) < 1e-16) break;
    }
    x[i] = 0.5 * (t + 1.0);
  }
}

// Lagrange polynomial a on `nodes` (m of them) and its derivative at x.
void lagrange_at(const double* nodes, int m, int a, double x, double* v, double* dv) {
  double val = 1.0;
  for (int b = 0; b < m; ++b)
    if (b != a) val *= (x - nodes[b]) / (nodes[a] - nodes[b]);
  double der = 0.0;
  for (int d = 0; d < m; ++d) {
    if (d == a) continue;
    double t = 1.0 / (nodes[a] - nodes[d]);
    for (int b = 0; b < m; ++b)
      if (b != a && b != d) t *= (x - nodes[b]) / (nodes[a] - nodes[b]);
    der += t;
  }
  *v = val;
  *dv = der;
}

}  // namespace

void build_ref_tables(int k, RefTables* t) {
  std::memset(t, 0, sizeof(*t));
  const int Q = k + 2, P = k + 2, p = k + 1;
  gauss_legendre01(Q, t->qx, t->qw);
  double closed[kMaxClosed], open[kMaxOpen], ow[kMaxOpen];
  gauss_lobatto01(P, closed);
  gauss_legendre01(p, open, ow);
  for (int a = 0; a < P; ++a)
    for (int q = 0; q < Q; ++q) lagrange_at(closed, P, a, t->qx[q], &t->Vc[a][q], &t->Dc[a][q]);
  for (int a = 0; a < p; ++a)
    for (int q = 0; q < Q; ++q) {
      double dv;
      lagrange_at(open, p, a, t->qx[q], &t->Vo[a][q], &dv);
    }
  for (int s1 = 0; s1 < p; ++s1)
    for (int s0 = 0; s0 < p; ++s0) t->wf[s0 + p * s1] = ow[s0] * ow[s1];
  // div_hat of an RT_k basis function lies in Q_k; its value at the open node a along the
  // component's own axis is the closed-Lagrange derivative there (Kronecker across).
  for (int a = 0; a < P; ++a)
    for (int b = 0; b < p; ++b) {
      double v;
      lagrange_at(closed, P, a, open[b], &v, &t->DcO[a][b]);
    }
}

// Map from the (k+1)^2 dofs of a coarse face to those of the four fine faces that tile it on a
// 2:1 non-conforming interface (Example 2.1's W_sm; Fig. 5.1, right). A face dof is the normal
// flux density per unit reference area at a Gauss-Legendre node; fine sub-face (a, b) covers
// the coarse parameters [a/2, (a+1)/2] x [b/2, (b+1)/2], so its reference area is a quarter of
// the coarse one's and its dof at node (p0, p1) is 1/4 of the coarse Q_k trace there:
// W[(a + 2b) nfn + p0 + (k+1) p1][r0 + (k+1) r1] = L_r0((a + g_p0) / 2) L_r1((b + g_p1) / 2) / 4,
// with L the Lagrange basis on the k+1 Gauss-Legendre nodes g. Row-major, 4 nfn x nfn.
void build_interface_w(int k, double* W) {
  const int p = k + 1, nfn = p * p;
  double g[kMaxOpen], w[kMaxOpen];
  gauss_legendre01(p, g, w);
  for (int b = 0; b < 2; ++b)
    for (int a = 0; a < 2; ++a)
      for (int p1 = 0; p1 < p; ++p1)
        for (int p0 = 0; p0 < p; ++p0) {
          double* row = W + ((size_t)(a + 2 * b) * nfn + p0 + p * p1) * nfn;
          for (int r1 = 0; r1 < p; ++r1)
            for (int r0 = 0; r0 < p; ++r0) {
              double v0, v1, dv;
              lagrange_at(g, p, r0, 0.5 * (a + g[p0]), &v0, &dv);
              lagrange_at(g, p, r1, 0.5 * (b + g[p1]), &v1, &dv);
              row[r0 + p * r1] = 0.25 * v0 * v1;
            }
        }
}

}  // namespace hyb
