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

}  // namespace hyb
