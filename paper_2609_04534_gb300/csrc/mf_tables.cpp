// mf_tables.cpp -- 1D tables of the sum-factorised apply, computed once on the host in FP64.
//
// Basis: Lagrange polynomials on the k+1 Gauss-Lobatto-Legendre points of [0,1] (the nodal
// basis example of Sec. 3.1).  Quadrature: (k+1)-point Gauss-Legendre.  The sum-factorised
// pipeline of Sec. 3.1 needs, per direction, the basis values S and derivatives D at the
// Gauss points, the collocation derivative Dc on the Gauss points, and the 1D mass and
// stiffness matrices M = S^T W S and K = D^T W D of the Cartesian form Eq. (eval_pipeline).
#include <cmath>
#include <cstring>

#include "mf_internal.h"

namespace mf {

namespace {

// P_m(x) and P_{m-1}(x) by the three-term recurrence.
void legendre_pair(int m, double x, double* pm, double* pm1) {
  double a = 1.0, b = x; // P_0, P_1
  if (m == 0) { *pm = 1.0; *pm1 = 0.0; return; }
  for (int j = 2; j <= m; ++j) {
    const double c = ((2 * j - 1) * x * b - (j - 1) * a) / j;
    a = b;
    b = c;
  }
  *pm = b;
  *pm1 = a;
}

double legendre(int m, double x) {
  double p, q;
  legendre_pair(m, x, &p, &q);
  return p;
}

// GLL points on [-1,1]: the endpoints and the zeros of P_{k+1} - P_{k-1}, which is
// proportional to (1 - x^2) P_k'(x); its derivative is (2k+1) P_k.
void gll(int k, double* x) {
  x[0] = -1.0;
  x[k] = 1.0;
  for (int j = 1; j < k; ++j) {
    double t = -std::cos(M_PI * j / k);
    for (int it = 0; it < 60; ++it) {
      const double f = legendre(k + 1, t) - legendre(k - 1, t);
      const double df = (2 * k + 1) * legendre(k, t);
      const double dt = f / df;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    x[j] = t;
  }
}

// Gauss-Legendre on [-1,1]: zeros of P_n, weight 2 (1 - x^2) / (n P_{n-1})^2.
void gauss(int n, double* x, double* w) {
  for (int j = 0; j < n; ++j) {
    double t = -std::cos(M_PI * (4 * j + 3) / (4 * n + 2));
    for (int it = 0; it < 60; ++it) {
      double p, p1;
      legendre_pair(n, t, &p, &p1);
      const double dp = n * (p1 - t * p) / (1.0 - t * t);
      const double dt = p / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    double p, p1;
    legendre_pair(n, t, &p, &p1);
    x[j] = t;
    w[j] = 2.0 * (1.0 - t * t) / ((n * p1) * (n * p1));
  }
}

// Lagrange basis on nodes xn (size n): value and derivative of every basis function at s.
// phi_i(s) = prod_{m != i} (s - x_m)/(x_i - x_m);
// phi_i'(s) = sum_{m != i} 1/(x_i - x_m) prod_{l != i, m} (s - x_l)/(x_i - x_l).
void lagrange_at(int n, const double* xn, double s, double* v, double* d) {
  for (int i = 0; i < n; ++i) {
    double p = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != i) p *= (s - xn[m]) / (xn[i] - xn[m]);
    v[i] = p;
    double acc = 0.0;
    for (int m = 0; m < n; ++m) {
      if (m == i) continue;
      double term = 1.0 / (xn[i] - xn[m]);
      for (int l = 0; l < n; ++l)
        if (l != i && l != m) term *= (s - xn[l]) / (xn[i] - xn[l]);
      acc += term;
    }
    d[i] = acc;
  }
}

} // namespace

int make_host_tables(int degree, HostTables* t) {
  if (degree < 1 || degree + 1 > MAXN) return -1;
  std::memset(t, 0, sizeof(*t));
  const int n = degree + 1;
  t->n = n;
  double xg[MAXN], xq[MAXN], wq[MAXN];
  gll(degree, xg);
  gauss(n, xq, wq);
  for (int i = 0; i < n; ++i) {
    t->nodes[i] = 0.5 * (xg[i] + 1.0);
    t->qx[i] = 0.5 * (xq[i] + 1.0);
    t->qw[i] = 0.5 * wq[i];
  }
  for (int q = 0; q < n; ++q) {
    double v[MAXN], d[MAXN];
    lagrange_at(n, t->nodes, t->qx[q], v, d);
    for (int i = 0; i < n; ++i) { t->S[q * MAXN + i] = v[i]; t->D[q * MAXN + i] = d[i]; }
    // derivative of the Lagrange basis on the Gauss points, at Gauss point q
    lagrange_at(n, t->qx, t->qx[q], v, d);
    for (int r = 0; r < n; ++r) t->Dc[q * MAXN + r] = d[r];
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double m = 0.0, k = 0.0;
      for (int q = 0; q < n; ++q) {
        m += t->qw[q] * t->S[q * MAXN + i] * t->S[q * MAXN + j];
        k += t->qw[q] * t->D[q * MAXN + i] * t->D[q * MAXN + j];
      }
      t->M[i * MAXN + j] = m;
      t->K[i * MAXN + j] = k;
    }
  return 0;
}

} // namespace mf
