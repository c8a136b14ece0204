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

// Generalised symmetric eigenproblem K v = lam M v (M SPD) in long double: M = L L^T,
// C = L^-1 K L^-T, cyclic Jacobi rotations C = Q diag(lam) Q^T, V = L^-T Q (V^T M V = I),
// W = M V.  The pencil is centro-symmetric (J K J = K, J M J = M with the flip J), so every
// mode is symmetric or antisymmetric; the parity is imposed exactly and the modes are sorted
// symmetric first, each group by eigenvalue.
void fast_diag(int n, const double* Mm, const double* Km, double* Wout, double* lam_out) {
  typedef long double R;
  R L[MAXN][MAXN] = {}, C[MAXN][MAXN], Q[MAXN][MAXN], T[MAXN][MAXN];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      R s = Mm[i * MAXN + j];
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      L[i][j] = i == j ? std::sqrt(s) : s / L[j][j];
    }
  // T = L^-1 K (forward substitution per column), C = T L^-T = L^-1 (L^-1 K)^T
  for (int c = 0; c < n; ++c)
    for (int i = 0; i < n; ++i) {
      R s = Km[i * MAXN + c];
      for (int k = 0; k < i; ++k) s -= L[i][k] * T[k][c];
      T[i][c] = s / L[i][i];
    }
  for (int r = 0; r < n; ++r)
    for (int i = 0; i < n; ++i) {
      R s = T[r][i];
      for (int k = 0; k < i; ++k) s -= L[i][k] * C[r][k];
      C[r][i] = s / L[i][i];
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Q[i][j] = i == j ? 1 : 0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    R off = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += C[p][q] * C[p][q];
    if (off < 1e-60L) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (C[p][q] == 0) continue;
        const R th = (C[q][q] - C[p][p]) / (2 * C[p][q]);
        const R t = (th >= 0 ? 1 : -1) / (std::fabs(th) + std::sqrt(th * th + 1));
        const R cs = 1 / std::sqrt(t * t + 1), sn = t * cs;
        for (int k = 0; k < n; ++k) { // rotate columns p, q
          const R a = C[k][p], b = C[k][q];
          C[k][p] = cs * a - sn * b;
          C[k][q] = sn * a + cs * b;
        }
        for (int k = 0; k < n; ++k) { // rotate rows p, q
          const R a = C[p][k], b = C[q][k];
          C[p][k] = cs * a - sn * b;
          C[q][k] = sn * a + cs * b;
        }
        for (int k = 0; k < n; ++k) {
          const R a = Q[k][p], b = Q[k][q];
          Q[k][p] = cs * a - sn * b;
          Q[k][q] = sn * a + cs * b;
        }
      }
  }
  // V = L^-T Q (back substitution per column), W = M V
  R V[MAXN][MAXN], W[MAXN][MAXN];
  for (int m = 0; m < n; ++m)
    for (int i = n - 1; i >= 0; --i) {
      R s = Q[i][m];
      for (int k = i + 1; k < n; ++k) s -= L[k][i] * V[k][m];
      V[i][m] = s / L[i][i];
    }
  int par[MAXN];
  for (int m = 0; m < n; ++m) {
    R ds = 0, da = 0;
    for (int j = 0; j < n; ++j) {
      ds += std::fabs(V[j][m] - V[n - 1 - j][m]);
      da += std::fabs(V[j][m] + V[n - 1 - j][m]);
    }
    par[m] = da < ds ? 1 : 0; // 1: antisymmetric
    for (int j = 0; j < (n + 1) / 2; ++j) {
      const R a = V[j][m], b = V[n - 1 - j][m];
      if (par[m]) { V[j][m] = (a - b) / 2; V[n - 1 - j][m] = -(a - b) / 2; }
      else { V[j][m] = (a + b) / 2; V[n - 1 - j][m] = (a + b) / 2; }
      if (par[m] && j == n - 1 - j) V[j][m] = 0;
    }
  }
  for (int j = 0; j < n; ++j)
    for (int m = 0; m < n; ++m) {
      R s = 0;
      for (int k = 0; k < n; ++k) s += (R)Mm[j * MAXN + k] * V[k][m];
      W[j][m] = s;
    }
  for (int m = 0; m < n; ++m) // the parity of W's columns exactly as V's
    for (int j = 0; j < (n + 1) / 2; ++j) {
      const R a = W[j][m], b = W[n - 1 - j][m];
      if (par[m]) { W[j][m] = (a - b) / 2; W[n - 1 - j][m] = -(a - b) / 2; if (j == n - 1 - j) W[j][m] = 0; }
      else { W[j][m] = (a + b) / 2; W[n - 1 - j][m] = (a + b) / 2; }
    }
  // order: symmetric modes, then antisymmetric, each by eigenvalue
  int ord[MAXN], no = 0;
  for (int pass = 0; pass < 2; ++pass) {
    int sel[MAXN], ns = 0;
    for (int m = 0; m < n; ++m)
      if (par[m] == pass) sel[ns++] = m;
    for (int a = 0; a < ns; ++a)
      for (int b = a + 1; b < ns; ++b)
        if (C[sel[b]][sel[b]] < C[sel[a]][sel[a]]) { const int t = sel[a]; sel[a] = sel[b]; sel[b] = t; }
    for (int a = 0; a < ns; ++a) ord[no++] = sel[a];
  }
  for (int mm = 0; mm < n; ++mm) {
    const int m = ord[mm];
    lam_out[mm] = (double)C[m][m];
    for (int j = 0; j < n; ++j) Wout[j * MAXN + mm] = (double)W[j][m];
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
  fast_diag(n, t->M, t->K, t->Wfd, t->lam);
  return 0;
}

} // namespace mf
