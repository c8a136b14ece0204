/*
 * mf_oracle.c -- plain, slow FP64 CPU definition of the continuous Q_k operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this
 * file; only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (paper: Sec. 2 "Discontinuous Galerkin Discretization", Eq. (sipg),
 * first sum -- the cell-wise volume integral of grad u . grad v; the continuous space keeps
 * only this term):
 *
 *   A_K[i][j] = sum_q w_q |det J_q| ( c_m phi_i phi_j + (J_q^{-T} grad phi_i).(J_q^{-T} grad phi_j) )
 *   y = sum_K P_K^T A_K P_K x            (global numbering, ascending cell order)
 *
 * The element operator is applied as a loop over quadrature points and basis functions
 * of the whole cell -- no sum factorisation, no tensor-product contraction.  The basis is
 * the tensor-product Lagrange basis on the k+1 Gauss-Lobatto-Legendre nodes of [0,1]
 * (the nodal example of Sec. 3.1); quadrature is the (k+1)-point Gauss-Legendre rule per
 * direction.  The curved mesh uses the analytic Jacobian of the mapping at every
 * quadrature point (the "six metric entries plus det J per point" of Sec. 2).
 *
 * Dirichlet: the operator is P A P where P zeroes global nodes on the boundary of the
 * unit cube (homogeneous data, Sec. 2 model problem).
 *
 * Pins: tests/test_oracle_*.py check every function here against closed forms,
 * textbook stencils, exact polynomial energies, a brute-force assembled matrix and
 * manufactured-solution convergence rates.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXN 10
#define OR_PI 3.14159265358979323846264338327950288L

/* ---------------------------------------------------------------- 1D tables */

/* Legendre P_m(t) and P_m'(t) on [-1,1] by the three-term recurrence (long double). */
static void legendre(int m, long double t, long double* P, long double* dP) {
  long double p0 = 1.0L, p1 = t;
  if (m == 0) { *P = 1.0L; *dP = 0.0L; return; }
  for (int j = 2; j <= m; ++j) {
    long double p2 = ((2.0L * j - 1.0L) * t * p1 - (j - 1.0L) * p0) / j;
    p0 = p1; p1 = p2;
  }
  *P = p1;
  /* (1 - t^2) P_m' = m (P_{m-1} - t P_m) */
  *dP = (fabsl(1.0L - t * t) > 0.0L) ? m * (p0 - t * p1) / (1.0L - t * t)
                                     : 0.5L * m * (m + 1.0L) * (t > 0 ? 1.0L : ((m % 2) ? 1.0L : -1.0L));
}

/* Gauss-Lobatto-Legendre nodes of degree k (k+1 points) on [0,1], ascending.
 * Interior nodes are the roots of P_k'; Newton on q(t) = (1 - t^2) P_k'(t), whose
 * derivative follows from the Legendre equation: q'(t) = -k(k+1) P_k(t). */
int or_gll_nodes(int k, double* nodes) {
  if (k < 1 || k + 1 > OR_MAXN) return -1;
  long double t[OR_MAXN];
  t[0] = -1.0L; t[k] = 1.0L;
  for (int j = 1; j < k; ++j) {
    long double x = -cosl(OR_PI * j / k);
    for (int it = 0; it < 100; ++it) {
      long double P, dP;
      legendre(k, x, &P, &dP);
      long double q = (1.0L - x * x) * dP, dq = -k * (k + 1.0L) * P;
      long double dx = q / dq;
      x -= dx;
      if (fabsl(dx) < 1e-19L) break;
    }
    t[j] = x;
  }
  for (int j = 0; j <= k; ++j) nodes[j] = (double)(0.5L * (t[j] + 1.0L));
  return 0;
}

/* n-point Gauss-Legendre rule on [0,1]: roots of P_n by Newton, weights
 * 2 / ((1 - t^2) P_n'(t)^2) on [-1,1], halved for [0,1]. */
int or_gauss(int n, double* x, double* w) {
  if (n < 1 || n > 16) return -1;
  for (int j = 0; j < n; ++j) {
    long double t = -cosl(OR_PI * (j + 0.75L) / (n + 0.5L)), P, dP;
    for (int it = 0; it < 100; ++it) {
      legendre(n, t, &P, &dP);
      long double dt = P / dP;
      t -= dt;
      if (fabsl(dt) < 1e-19L) break;
    }
    legendre(n, t, &P, &dP);
    x[j] = (double)(0.5L * (t + 1.0L));
    w[j] = (double)(1.0L / ((1.0L - t * t) * dP * dP));
  }
  return 0;
}

/* Lagrange basis on the n given nodes, evaluated at s: phi_i(s) = prod_{m != i}
 * (s - x_m)/(x_i - x_m); derivative by the product rule. Long double throughout. */
void or_lagrange(int n, const double* nodes, double s, double* phi, double* dphi) {
  for (int i = 0; i < n; ++i) {
    long double v = 1.0L, d = 0.0L;
    for (int m = 0; m < n; ++m) {
      if (m == i) continue;
      long double den = (long double)nodes[i] - nodes[m];
      long double f = ((long double)s - nodes[m]) / den;
      d = d * f + v / den; /* (v*f)' = v'*f + v*f' */
      v = v * f;
    }
    phi[i] = (double)v;
    if (dphi) dphi[i] = (double)d;
  }
}

/* ---------------------------------------------------------------- mesh */

typedef struct {
  int nx, ny, nz;   /* cells per axis of the unit cube */
  int geom;         /* 0: affine x = A xh + b ; 1: curved xh + amp*s(xh)*(1,1,1) */
  double A[9];      /* row-major 3x3 (affine) */
  double b[3];
  double amp;       /* curved amplitude */
} or_mesh;

/* Mapping Phi(xh) and its gradient F[a][b] = d Phi_a / d xh_b.
 * Curved: Phi_a = xh_a + amp sin(pi xh_1) sin(pi xh_2) sin(pi xh_3) for a = 1,2,3. */
void or_map(const or_mesh* m, const double* xh, double* x, double* F) {
  if (m->geom == 0) {
    for (int a = 0; a < 3; ++a) {
      x[a] = m->b[a];
      for (int c = 0; c < 3; ++c) { x[a] += m->A[3 * a + c] * xh[c]; F[3 * a + c] = m->A[3 * a + c]; }
    }
  } else {
    double s[3], c[3];
    for (int d = 0; d < 3; ++d) { s[d] = sin(M_PI * xh[d]); c[d] = cos(M_PI * xh[d]); }
    double val = s[0] * s[1] * s[2];
    double g[3] = {M_PI * c[0] * s[1] * s[2], M_PI * s[0] * c[1] * s[2], M_PI * s[0] * s[1] * c[2]};
    for (int a = 0; a < 3; ++a) {
      x[a] = xh[a] + m->amp * val;
      for (int d = 0; d < 3; ++d) F[3 * a + d] = (a == d ? 1.0 : 0.0) + m->amp * g[d];
    }
  }
}

static double det3(const double* J) {
  return J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
         J[2] * (J[3] * J[7] - J[4] * J[6]);
}

static void inv3(const double* J, double det, double* Ji) {
  Ji[0] = (J[4] * J[8] - J[5] * J[7]) / det;
  Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
  Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
  Ji[3] = (J[5] * J[6] - J[3] * J[8]) / det;
  Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det;
  Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
  Ji[6] = (J[3] * J[7] - J[4] * J[6]) / det;
  Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
  Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
}

/* Jacobian of xi in [0,1]^3 of cell (cx,cy,cz) -> physical point:
 * J = F(xh) diag(1/nx, 1/ny, 1/nz), xh = ((cx+xi1)/nx, (cy+xi2)/ny, (cz+xi3)/nz). */
void or_cell_jacobian(const or_mesh* m, int cx, int cy, int cz, const double* xi, double* x, double* J) {
  double xh[3] = {(cx + xi[0]) / m->nx, (cy + xi[1]) / m->ny, (cz + xi[2]) / m->nz};
  double F[9];
  or_map(m, xh, x, F);
  double inv[3] = {1.0 / m->nx, 1.0 / m->ny, 1.0 / m->nz};
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) J[3 * a + d] = F[3 * a + d] * inv[d];
}

/* ---------------------------------------------------------------- operator */

typedef struct {
  or_mesh mesh;
  int k;        /* degree */
  double cm;    /* mass coefficient: 0 = Laplace, 1 = Helmholtz (M + K) */
  int bc;       /* 0 none, 1 homogeneous Dirichlet */
  int nq;       /* quadrature points per direction used by the operator (k+1) */
} or_op;

int64_t or_n_unique(const or_op* op) {
  int k = op->k;
  return (int64_t)(op->mesh.nx * k + 1) * (op->mesh.ny * k + 1) * (op->mesh.nz * k + 1);
}

/* global index of local node (i,j,l) of cell (cx,cy,cz); x fastest */
static int64_t gidx(const or_op* op, int cx, int cy, int cz, int i, int j, int l) {
  int k = op->k;
  int64_t NX = op->mesh.nx * k + 1, NY = op->mesh.ny * k + 1;
  int64_t I = (int64_t)cx * k + i, Jn = (int64_t)cy * k + j, L = (int64_t)cz * k + l;
  return I + NX * (Jn + NY * L);
}

static int on_boundary(const or_op* op, int64_t g) {
  int k = op->k;
  int64_t NX = op->mesh.nx * k + 1, NY = op->mesh.ny * k + 1, NZ = op->mesh.nz * k + 1;
  int64_t I = g % NX, Jn = (g / NX) % NY, L = g / (NX * NY);
  return I == 0 || I == NX - 1 || Jn == 0 || Jn == NY - 1 || L == 0 || L == NZ - 1;
}

typedef struct {
  int n, nq;
  double nodes[OR_MAXN], qx[16], qw[16];
  double phi[16][OR_MAXN], dphi[16][OR_MAXN]; /* phi[q][i] = phi_i(qx[q]) */
} or_tab;

static int make_tab(int k, int nq, or_tab* t) {
  t->n = k + 1; t->nq = nq;
  if (or_gll_nodes(k, t->nodes)) return -1;
  if (or_gauss(nq, t->qx, t->qw)) return -1;
  for (int q = 0; q < nq; ++q) or_lagrange(t->n, t->nodes, t->qx[q], t->phi[q], t->dphi[q]);
  return 0;
}

/* Local (split, unassembled) result y_K = A_K x_K of one cell, as a quadrature loop:
 * at each quadrature point evaluate u and its reference gradient from all n^3 basis
 * functions, map the gradient with J^{-T}, then test against every basis function. */
static void cell_apply(const or_op* op, const or_tab* t, int cx, int cy, int cz, const double* xK,
                       double* yK) {
  int n = t->n, nq = t->nq, n3 = n * n * n;
  for (int i = 0; i < n3; ++i) yK[i] = 0.0;
  for (int q3 = 0; q3 < nq; ++q3)
    for (int q2 = 0; q2 < nq; ++q2)
      for (int q1 = 0; q1 < nq; ++q1) {
        double xi[3] = {t->qx[q1], t->qx[q2], t->qx[q3]}, x[3], J[9], Ji[9];
        or_cell_jacobian(&op->mesh, cx, cy, cz, xi, x, J);
        double det = det3(J);
        inv3(J, det, Ji);
        double wdet = t->qw[q1] * t->qw[q2] * t->qw[q3] * fabs(det);
        double u = 0.0, gr[3] = {0.0, 0.0, 0.0};
        for (int l = 0; l < n; ++l)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
              double xv = xK[i + n * (j + n * l)];
              u += xv * t->phi[q1][i] * t->phi[q2][j] * t->phi[q3][l];
              gr[0] += xv * t->dphi[q1][i] * t->phi[q2][j] * t->phi[q3][l];
              gr[1] += xv * t->phi[q1][i] * t->dphi[q2][j] * t->phi[q3][l];
              gr[2] += xv * t->phi[q1][i] * t->phi[q2][j] * t->dphi[q3][l];
            }
        /* physical gradient: grad = J^{-T} grad_ref,  (J^{-T})[a][b] = Ji[b][a] */
        double pg[3];
        for (int a = 0; a < 3; ++a) pg[a] = Ji[a] * gr[0] + Ji[3 + a] * gr[1] + Ji[6 + a] * gr[2];
        for (int l = 0; l < n; ++l)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
              double v = t->phi[q1][i] * t->phi[q2][j] * t->phi[q3][l];
              double r0 = t->dphi[q1][i] * t->phi[q2][j] * t->phi[q3][l];
              double r1 = t->phi[q1][i] * t->dphi[q2][j] * t->phi[q3][l];
              double r2 = t->phi[q1][i] * t->phi[q2][j] * t->dphi[q3][l];
              double gv[3];
              for (int a = 0; a < 3; ++a) gv[a] = Ji[a] * r0 + Ji[3 + a] * r1 + Ji[6 + a] * r2;
              yK[i + n * (j + n * l)] +=
                  wdet * (op->cm * v * u + gv[0] * pg[0] + gv[1] * pg[1] + gv[2] * pg[2]);
            }
      }
}

/* Element matrix A_K (n^3 x n^3, row-major) by the explicit triple loop over
 * (quadrature point, test function, trial function). */
int or_element_matrix(const or_op* op, int cx, int cy, int cz, double* A) {
  or_tab t;
  if (make_tab(op->k, op->nq, &t)) return -1;
  int n = t.n, n3 = n * n * n, nq = t.nq;
  memset(A, 0, sizeof(double) * (size_t)n3 * n3);
  double* gphys = (double*)malloc(sizeof(double) * 4 * n3);
  for (int q3 = 0; q3 < nq; ++q3)
    for (int q2 = 0; q2 < nq; ++q2)
      for (int q1 = 0; q1 < nq; ++q1) {
        double xi[3] = {t.qx[q1], t.qx[q2], t.qx[q3]}, x[3], J[9], Ji[9];
        or_cell_jacobian(&op->mesh, cx, cy, cz, xi, x, J);
        double det = det3(J);
        inv3(J, det, Ji);
        double wdet = t.qw[q1] * t.qw[q2] * t.qw[q3] * fabs(det);
        for (int l = 0; l < n; ++l)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
              int a = i + n * (j + n * l);
              double r0 = t.dphi[q1][i] * t.phi[q2][j] * t.phi[q3][l];
              double r1 = t.phi[q1][i] * t.dphi[q2][j] * t.phi[q3][l];
              double r2 = t.phi[q1][i] * t.phi[q2][j] * t.dphi[q3][l];
              gphys[4 * a + 0] = t.phi[q1][i] * t.phi[q2][j] * t.phi[q3][l];
              for (int c = 0; c < 3; ++c) gphys[4 * a + 1 + c] = Ji[c] * r0 + Ji[3 + c] * r1 + Ji[6 + c] * r2;
            }
        for (int a = 0; a < n3; ++a)
          for (int b = 0; b < n3; ++b)
            A[(size_t)a * n3 + b] +=
                wdet * (op->cm * gphys[4 * a] * gphys[4 * b] + gphys[4 * a + 1] * gphys[4 * b + 1] +
                        gphys[4 * a + 2] * gphys[4 * b + 2] + gphys[4 * a + 3] * gphys[4 * b + 3]);
      }
  free(gphys);
  return 0;
}

/* Global indices of the n^3 local nodes of every cell (cell-major, local x fastest). */
void or_cell_dofs(const or_op* op, int64_t* out) {
  int n = op->k + 1;
  int64_t c = 0;
  for (int cz = 0; cz < op->mesh.nz; ++cz)
    for (int cy = 0; cy < op->mesh.ny; ++cy)
      for (int cx = 0; cx < op->mesh.nx; ++cx, ++c)
        for (int l = 0; l < n; ++l)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) out[c * n * n * n + i + n * (j + n * l)] = gidx(op, cx, cy, cz, i, j, l);
}

/* Unique -> cell-wise (canonical layout [cell][l][j][i]): the gather G. */
void or_scatter(const or_op* op, const double* xu, double* xcw) {
  int n = op->k + 1;
  int64_t c = 0;
  for (int cz = 0; cz < op->mesh.nz; ++cz)
    for (int cy = 0; cy < op->mesh.ny; ++cy)
      for (int cx = 0; cx < op->mesh.nx; ++cx, ++c)
        for (int l = 0; l < n; ++l)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) xcw[c * n * n * n + i + n * (j + n * l)] = xu[gidx(op, cx, cy, cz, i, j, l)];
}

/* Cell-wise split -> unique: the assembly G^T (ascending cell order). */
void or_assemble(const or_op* op, const double* ycw, double* yu) {
  int n = op->k + 1;
  memset(yu, 0, sizeof(double) * or_n_unique(op));
  int64_t c = 0;
  for (int cz = 0; cz < op->mesh.nz; ++cz)
    for (int cy = 0; cy < op->mesh.ny; ++cy)
      for (int cx = 0; cx < op->mesh.nx; ++cx, ++c)
        for (int l = 0; l < n; ++l)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) yu[gidx(op, cx, cy, cz, i, j, l)] += ycw[c * n * n * n + i + n * (j + n * l)];
}

/* Boundary mask on unique DoFs (1 = constrained node on the cube boundary). */
void or_boundary_mask(const or_op* op, uint8_t* mask) {
  int64_t N = or_n_unique(op);
  for (int64_t g = 0; g < N; ++g) mask[g] = (uint8_t)on_boundary(op, g);
}

/* Local results for a list of cells from a cell-wise (canonical) input: yloc[m] = A_K xcw[K]
 * for K = cells[m].  No Dirichlet mask (callers apply it).  Parallel over cells only. */
int or_apply_cells(const or_op* op, const double* xcw, int64_t ncell, const int64_t* cells, double* yloc,
                   int nthreads) {
  or_tab t;
  if (make_tab(op->k, op->nq, &t)) return -1;
  int n3 = t.n * t.n * t.n;
  int nx = op->mesh.nx, ny = op->mesh.ny;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (int64_t m = 0; m < ncell; ++m) {
    int64_t c = cells[m];
    int cx = (int)(c % nx), cy = (int)((c / nx) % ny), cz = (int)(c / ((int64_t)nx * ny));
    cell_apply(op, &t, cx, cy, cz, xcw + c * n3, yloc + m * n3);
  }
  return 0;
}

/* y = (P) A (P) x on unique DoFs: per cell gather, quadrature-loop apply, scatter-add in
 * ascending cell order; Dirichlet zeroes constrained entries of x before and y after. */
int or_apply(const or_op* op, const double* xu, double* yu, int nthreads) {
  or_tab t;
  if (make_tab(op->k, op->nq, &t)) return -1;
  int n = t.n, n3 = n * n * n;
  int64_t nc = (int64_t)op->mesh.nx * op->mesh.ny * op->mesh.nz, N = or_n_unique(op);
  double* xin = (double*)malloc(sizeof(double) * N);
  memcpy(xin, xu, sizeof(double) * N);
  if (op->bc)
    for (int64_t g = 0; g < N; ++g)
      if (on_boundary(op, g)) xin[g] = 0.0;
  double* ycw = (double*)malloc(sizeof(double) * nc * n3);
  double* xcw = (double*)malloc(sizeof(double) * nc * n3);
  or_scatter(op, xin, xcw);
  int nx = op->mesh.nx, ny = op->mesh.ny;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (int64_t c = 0; c < nc; ++c) {
    int cx = (int)(c % nx), cy = (int)((c / nx) % ny), cz = (int)(c / ((int64_t)nx * ny));
    cell_apply(op, &t, cx, cy, cz, xcw + c * n3, ycw + c * n3);
  }
  or_assemble(op, ycw, yu);
  if (op->bc)
    for (int64_t g = 0; g < N; ++g)
      if (on_boundary(op, g)) yu[g] = 0.0;
  free(xin); free(ycw); free(xcw);
  (void)n;
  return 0;
}

/* ---------------------------------------------------------------- CG */

static double dotu(const double* a, const double* b, int64_t N) {
  double s = 0.0;
  for (int64_t i = 0; i < N; ++i) s += a[i] * b[i];
  return s;
}

/* Textbook unpreconditioned CG on (P A P) x = P b from x = 0, over unique DoFs.
 * Stops after maxit iterations or when ||r|| <= rtol ||b||.  hist[m] = ||r_m|| / ||b||
 * for m = 0..iters.  Returns the number of iterations; -1 on breakdown (p^T A p <= 0). */
int or_cg(const or_op* op, const double* b_in, double* x, int maxit, double rtol, double* hist, int nthreads) {
  int64_t N = or_n_unique(op);
  double *b = (double*)malloc(8 * N), *r = (double*)malloc(8 * N), *p = (double*)malloc(8 * N),
         *q = (double*)malloc(8 * N);
  memcpy(b, b_in, 8 * N);
  if (op->bc)
    for (int64_t g = 0; g < N; ++g)
      if (on_boundary(op, g)) b[g] = 0.0;
  for (int64_t g = 0; g < N; ++g) { x[g] = 0.0; r[g] = b[g]; p[g] = b[g]; }
  double bn = sqrt(dotu(b, b, N)), rr = dotu(r, r, N);
  int it = 0, ret = 0;
  if (hist) hist[0] = bn > 0 ? sqrt(rr) / bn : 0.0;
  while (it < maxit && sqrt(rr) > rtol * bn) {
    or_apply(op, p, q, nthreads);
    double pq = dotu(p, q, N);
    if (!(pq > 0.0)) { ret = -1; break; }
    double alpha = rr / pq;
    for (int64_t g = 0; g < N; ++g) { x[g] += alpha * p[g]; r[g] -= alpha * q[g]; }
    double rr1 = dotu(r, r, N), beta = rr1 / rr;
    rr = rr1;
    for (int64_t g = 0; g < N; ++g) p[g] = r[g] + beta * p[g];
    ++it;
    if (hist) hist[it] = sqrt(rr) / bn;
  }
  free(b); free(r); free(p); free(q);
  return ret < 0 ? -1 : it;
}

/* ---------------------------------------------------------------- manufactured solution */

/* u = sin(f pi x) sin(f pi y) sin(f pi z), -Lap u = 3 f^2 pi^2 u */
static void exact_u(double f, const double* x, double* u, double* gu) {
  double s[3], c[3];
  for (int d = 0; d < 3; ++d) { s[d] = sin(f * M_PI * x[d]); c[d] = cos(f * M_PI * x[d]); }
  *u = s[0] * s[1] * s[2];
  if (gu) {
    gu[0] = f * M_PI * c[0] * s[1] * s[2];
    gu[1] = f * M_PI * s[0] * c[1] * s[2];
    gu[2] = f * M_PI * s[0] * s[1] * c[2];
  }
}

/* b_i = int f phi_i dx with f = (3 freq^2 pi^2 + cm) u, on unique DoFs, nqr-point Gauss rule. */
int or_rhs_manufactured(const or_op* op, double freq, int nqr, double* bu) {
  or_tab t;
  if (make_tab(op->k, nqr, &t)) return -1;
  int n = t.n, n3 = n * n * n;
  memset(bu, 0, sizeof(double) * or_n_unique(op));
  double* bK = (double*)malloc(sizeof(double) * n3);
  for (int cz = 0; cz < op->mesh.nz; ++cz)
    for (int cy = 0; cy < op->mesh.ny; ++cy)
      for (int cx = 0; cx < op->mesh.nx; ++cx) {
        for (int i = 0; i < n3; ++i) bK[i] = 0.0;
        for (int q3 = 0; q3 < nqr; ++q3)
          for (int q2 = 0; q2 < nqr; ++q2)
            for (int q1 = 0; q1 < nqr; ++q1) {
              double xi[3] = {t.qx[q1], t.qx[q2], t.qx[q3]}, x[3], J[9], u;
              or_cell_jacobian(&op->mesh, cx, cy, cz, xi, x, J);
              double wdet = t.qw[q1] * t.qw[q2] * t.qw[q3] * fabs(det3(J));
              exact_u(freq, x, &u, NULL);
              double f = (3.0 * freq * freq * M_PI * M_PI + op->cm) * u;
              for (int l = 0; l < n; ++l)
                for (int j = 0; j < n; ++j)
                  for (int i = 0; i < n; ++i)
                    bK[i + n * (j + n * l)] += wdet * f * t.phi[q1][i] * t.phi[q2][j] * t.phi[q3][l];
            }
        for (int l = 0; l < n; ++l)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) bu[gidx(op, cx, cy, cz, i, j, l)] += bK[i + n * (j + n * l)];
      }
  free(bK);
  return 0;
}

/* L2 and H1-seminorm errors of the unique-DoF FE function uh against the manufactured u. */
int or_errors(const or_op* op, double freq, const double* uh, int nqr, double* l2, double* h1) {
  or_tab t;
  if (make_tab(op->k, nqr, &t)) return -1;
  int n = t.n;
  double el2 = 0.0, eh1 = 0.0;
  for (int cz = 0; cz < op->mesh.nz; ++cz)
    for (int cy = 0; cy < op->mesh.ny; ++cy)
      for (int cx = 0; cx < op->mesh.nx; ++cx)
        for (int q3 = 0; q3 < nqr; ++q3)
          for (int q2 = 0; q2 < nqr; ++q2)
            for (int q1 = 0; q1 < nqr; ++q1) {
              double xi[3] = {t.qx[q1], t.qx[q2], t.qx[q3]}, x[3], J[9], Ji[9], u, gu[3];
              or_cell_jacobian(&op->mesh, cx, cy, cz, xi, x, J);
              double det = det3(J);
              inv3(J, det, Ji);
              double wdet = t.qw[q1] * t.qw[q2] * t.qw[q3] * fabs(det);
              exact_u(freq, x, &u, gu);
              double v = 0.0, gr[3] = {0.0, 0.0, 0.0};
              for (int l = 0; l < n; ++l)
                for (int j = 0; j < n; ++j)
                  for (int i = 0; i < n; ++i) {
                    double c = uh[gidx(op, cx, cy, cz, i, j, l)];
                    v += c * t.phi[q1][i] * t.phi[q2][j] * t.phi[q3][l];
                    gr[0] += c * t.dphi[q1][i] * t.phi[q2][j] * t.phi[q3][l];
                    gr[1] += c * t.phi[q1][i] * t.dphi[q2][j] * t.phi[q3][l];
                    gr[2] += c * t.phi[q1][i] * t.phi[q2][j] * t.dphi[q3][l];
                  }
              double pg[3];
              for (int a = 0; a < 3; ++a) pg[a] = Ji[a] * gr[0] + Ji[3 + a] * gr[1] + Ji[6 + a] * gr[2];
              el2 += wdet * (u - v) * (u - v);
              for (int a = 0; a < 3; ++a) eh1 += wdet * (gu[a] - pg[a]) * (gu[a] - pg[a]);
            }
  *l2 = sqrt(el2);
  *h1 = sqrt(eh1);
  return 0;
}

/* Nodal interpolant of the manufactured u on unique DoFs (node positions mapped by Phi). */
int or_interpolate_manufactured(const or_op* op, double freq, double* uu) {
  double nodes[OR_MAXN];
  int k = op->k;
  if (or_gll_nodes(k, nodes)) return -1;
  int n = k + 1;
  for (int cz = 0; cz < op->mesh.nz; ++cz)
    for (int cy = 0; cy < op->mesh.ny; ++cy)
      for (int cx = 0; cx < op->mesh.nx; ++cx)
        for (int l = 0; l < n; ++l)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
              double xi[3] = {nodes[i], nodes[j], nodes[l]}, x[3], J[9], u;
              or_cell_jacobian(&op->mesh, cx, cy, cz, xi, x, J);
              exact_u(freq, x, &u, NULL);
              uu[gidx(op, cx, cy, cz, i, j, l)] = u;
            }
  return 0;
}

/* Physical positions of the unique nodes (for polynomial-field pins): xyz[3*g + a]. */
int or_node_positions(const or_op* op, double* xyz) {
  double nodes[OR_MAXN];
  int k = op->k, n = k + 1;
  if (or_gll_nodes(k, nodes)) return -1;
  for (int cz = 0; cz < op->mesh.nz; ++cz)
    for (int cy = 0; cy < op->mesh.ny; ++cy)
      for (int cx = 0; cx < op->mesh.nx; ++cx)
        for (int l = 0; l < n; ++l)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
              double xi[3] = {nodes[i], nodes[j], nodes[l]}, x[3], J[9];
              or_cell_jacobian(&op->mesh, cx, cy, cz, xi, x, J);
              int64_t g = gidx(op, cx, cy, cz, i, j, l);
              xyz[3 * g] = x[0]; xyz[3 * g + 1] = x[1]; xyz[3 * g + 2] = x[2];
            }
  return 0;
}

/* Sum over all quadrature points of w |det J| (mesh volume as the operator integrates it). */
double or_volume(const or_op* op, int nqr) {
  or_tab t;
  if (make_tab(op->k, nqr, &t)) return -1.0;
  double v = 0.0;
  for (int cz = 0; cz < op->mesh.nz; ++cz)
    for (int cy = 0; cy < op->mesh.ny; ++cy)
      for (int cx = 0; cx < op->mesh.nx; ++cx)
        for (int q3 = 0; q3 < nqr; ++q3)
          for (int q2 = 0; q2 < nqr; ++q2)
            for (int q1 = 0; q1 < nqr; ++q1) {
              double xi[3] = {t.qx[q1], t.qx[q2], t.qx[q3]}, x[3], J[9];
              or_cell_jacobian(&op->mesh, cx, cy, cz, xi, x, J);
              v += t.qw[q1] * t.qw[q2] * t.qw[q3] * fabs(det3(J));
            }
  return v;
}

/* det J at one reference point of one cell (for the determinant pin). */
double or_cell_det(const or_mesh* m, int cx, int cy, int cz, const double* xi) {
  double x[3], J[9];
  or_cell_jacobian(m, cx, cy, cz, xi, x, J);
  return det3(J);
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
