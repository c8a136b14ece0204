// mf_internal.h -- internal types shared by the CUDA translation units of libmf.
//
// Native layout (the blocked [B, n_x, n_y, n_z, n_e] storage of Sec. 2, "storage layout as a
// free parameter"): cells are grouped in tiles of BL = 32 spatially adjacent cells (a
// TX x TY x TZ = 4 x 4 x 2 brick); inside a tile the cell lane is the fastest address, so a
// warp reading one local DoF of 32 cells touches 32 consecutive words (the coalescing rule
// of Sec. 6.3).  Element (tile t, local dof l, lane c) lives at (t * n^3 + l) * BL + c.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/mf.h"

namespace mf {

template <typename T>
struct CoefOf; // coefficient type of the 1D tables for a compute type (mf_dd.cuh)

constexpr int TX = 4, TY = 4, TZ = 2, BL = TX * TY * TZ;
constexpr int MAXN = 9;

enum Path { PATH_CARTESIAN = 0, PATH_AFFINE = 1, PATH_CURVED = 2 };

// Structured mesh + tile grid, passed by value to every kernel.
struct GridInfo {
  int nx, ny, nz;    // cells per axis
  int ntx, nty, ntz; // tiles per axis
  long long ntiles;
  int bc;            // 1: homogeneous Dirichlet on the cube boundary
};

// 1D tables on the reference interval [0,1] (n = k+1):
//   S[q][i]  = phi_i(x_q)             GLL Lagrange basis at Gauss points
//   Dc[q][r] = psi_r'(x_q)            derivative of the Gauss-point Lagrange basis (collocation)
//   W[q]                               Gauss weights
//   M[i][j] = sum_q W_q S[q][i] S[q][j],  K[i][j] = sum_q W_q D[q][i] D[q][j]  (1D mass, stiffness)
//
// Even-odd forms (for 1D contractions y = A x with A centro-symmetric, A[n-1-q][n-1-i] =
// A[q][i] -- S, S^T, M, K -- or centro-antisymmetric, A[n-1-q][n-1-i] = -A[q][i] -- Dc, Dc^T):
// with H = n/2, e_i = x_i + x_{n-1-i}, o_i = x_i - x_{n-1-i} (i < H) and e_H = x_H for odd n,
//   F[q][i] = (A[q][i] + A[q][n-1-i]) / 2 (i < H), F[q][H] = A[q][H];  G[q][i] = (A[q][i] - A[q][n-1-i]) / 2
// give u = F e and w = G o for q < H, and then y_q = u + w and y_{n-1-q} = u - w (symmetric)
// or w - u (antisymmetric); the middle output of odd n is Mid . e (symmetric, Mid = A[H][0..H])
// or Mid . o (antisymmetric, Mid = A[H][0..H-1]).
template <typename T, int N>
struct EoTab {
  static constexpr int H = N / 2, HE = (N + 1) / 2;
  T F[H * HE], G[H * H > 0 ? H * H : 1], Mid[HE];
};
// Fast diagonalisation of the 1D pencil (K, M): W = M V with V^T M V = I, V^T K V = diag(lam),
// so M = W W^T and K = W diag(lam) W^T.  Both matrices are centro-symmetric, so every column
// of W (mode) is symmetric or antisymmetric; the modes are stored with the HE symmetric ones
// first.  Forward z = W^T x on a folded pencil: z_s = Ff e (HE x HE), z_a = Gf o (H x H);
// backward y = W z: U = Fb z_s (HE outputs), V = Gb z_a (H outputs), y_j = U_j + V_j,
// y_(n-1-j) = U_j - V_j.  lam in the same mode order.
template <typename T, int N>
struct FdTab {
  static constexpr int H = N / 2, HE = (N + 1) / 2;
  T Ff[HE * HE], Gf[H * H > 0 ? H * H : 1], Fb[HE * HE], Gb[H * H > 0 ? H * H : 1], lam[N];
};
// What the apply kernels read: the Gauss weights and every 1D matrix in even-odd form.
template <typename T, int N>
struct Tab {
  T W[N];
  EoTab<T, N> eS, eSt, eD, eDt, eM, eK; // S, S^T, Dc, Dc^T, M, K
  FdTab<T, N> fd;                       // the Cartesian form's modes (fast diagonalisation)
};

// Precision views of an operator: storage type of the vectors / compute type of the apply.
// VK_DDS is VK_DD with double-float storage (the FP64 solver's internal vectors); it shares
// VK_DD's geometry and launch variant.
enum ViewKind { VK_F64 = 0, VK_DD = 1, VK_F32 = 2, VK_DDS = 3 };
// Element types of vectors: 8 double, 4 float, ELEM_DD double-float (8 bytes).
constexpr int ELEM_DD = 9;

// Device-resident CG scalars.
struct CgState {
  double rr;    // <r, r> (assembled): the convergence test
  double rz;    // <r, z>, z = M^-1 r (= rr without preconditioner): alpha and beta
  double pq;    // <p, A p>
  double alpha, beta;
  double bnorm; // ||b|| of this CG
  double tol2;  // (rtol * ||b||)^2
  int it;       // iterations done
  int flag;     // 0 running, 1 converged, 2 breakdown, 3 maxit
  int maxit;
  int pad;
};

// CG step carried by an apply launch (the split-dual iteration of Sec. 4): with st set, the
// apply writes the split product y = A_K p per cell (no duplicate summation) and each CTA
// writes its part of <p, y> over all copies -- the pairing of a consistent with a split
// vector, Lemma 1 -- to partials[blockIdx.x]; a one-CTA kernel then folds the partials and
// forms alpha = <r, r> / <p, y>.  The input is p = x; with update_p the apply instead reads r
// and the previous direction p and forms p = r + beta p at load (written back in place).
template <typename S>
struct CgFuse {
  S* p;
  const S* r;
  CgState* st;
  double* partials;
  int update_p;
};

// Everything an apply launch needs about one operator and one vector pair except the 1D
// tables (which depend only on the degree, so a batched launch over several requests of the
// same degree shares them in its parameters).
template <typename S, typename T>
struct ApplyJob {
  const S* __restrict__ x;
  S* __restrict__ y;
  const T* __restrict__ geom; // curved: [tile][comp][l][lane], 6 (Laplace) or 7 (Helmholtz) comps
  GridInfo g;
  T G[6];                     // affine: w-free metric w det J J^-1 J^-T (xx,xy,xz,yy,yz,zz)
  T mdet;                     // affine: mass_coeff * |det J|
  T gx, gy, gz, cmass;        // Cartesian: det/h_d^2 and mass_coeff * det
  // FP32 curved: the metric is computed per point from per-direction tables of
  // sin(pi xh), cos(pi xh) at the Gauss points of every cell layer ([(nx+ny+nz)*N][2]).
  const float* gtab;
  float amp, cm, h[3];
  CgFuse<S> cg; // cg.st == nullptr: plain apply
  // L2 prefetch distance in tiles (about one wave of resident CTAs ahead; 0 = off): the first
  // CTA of tile t prefetches the input and geometry of tile t + pf_tiles; pf_geom = 1 only
  // when geom is a streamed per-point metric of this operator's full tile range
  int pf_tiles, pf_geom;
};

template <typename S, typename T, int N>
struct ApplyArgs {
  ApplyJob<S, T> j;
  Tab<typename CoefOf<T>::type, N> tab;
};

// A batched apply over several requests of one degree, path and precision: CTA b belongs to
// job i with block0[i] <= b < block0[i + 1] and runs that job's CTA b - block0[i].
template <typename S, typename T, int N>
struct ApplyBatch {
  Tab<typename CoefOf<T>::type, N> tab;
  const ApplyJob<S, T>* jobs;
  const long long* block0; // njobs + 1 entries
  long long nunits;        // block0[njobs]: CTA-sized work units of all jobs
  int njobs;
};

// One request of a batched CG iteration (the serving loop): its operator and CG storage.
struct BatchMember {
  const mf_operator* op;
  void *x, *r, *p, *q; // CG vectors in the batch's element type
  CgState* st;
  double* apart;       // per-CTA <p, A p> partials of its apply
  void* sc;            // reduction scratch of its update
  double* hist;        // residual history (may be null)
  const float* dinv;   // Jacobi: inverse diagonal (null: no preconditioner)
};

// Host-side double tables (any n <= MAXN).
struct HostTables {
  int n;
  double nodes[MAXN], qx[MAXN], qw[MAXN];
  double S[MAXN * MAXN], D[MAXN * MAXN], Dc[MAXN * MAXN], M[MAXN * MAXN], K[MAXN * MAXN];
  // fast diagonalisation of (K, M): Wfd[j * MAXN + m] = W_jm for mode m (symmetric modes
  // first, each group by increasing eigenvalue), lam[m] its eigenvalue
  double Wfd[MAXN * MAXN], lam[MAXN];
};
int make_host_tables(int degree, HostTables* t);

// One precision "view" of an operator: element type, geometry pointer, constants.
struct View {
  int elem_bytes = 8;   // 8 double, 4 float
  void* geom = nullptr; // device, inside the caller workspace (curved only)
  size_t geom_bytes = 0;
};

} // namespace mf

struct mf_mesh {
  int nx, ny, nz, geom;
  double A[9], b[3], amp;
};

struct mf_operator {
  mf_mesh mesh;
  int degree, n, kind, precision, bc;
  double mass;
  int path;
  mf::GridInfo g;
  long long n_cellwise, n_unique, n_native;
  mf::HostTables tab;
  double G[6], mdet, gx, gy, gz, cmass; // affine / Cartesian constants (double)
  mf::View v64, v32;                    // v64 used by FP64 + MIXED, v32 by FP32 + MIXED
  void* workspace = nullptr;
  size_t workspace_bytes = 0;
  bool ready = false;
  // apply launch variant per ViewKind (autotuned); MF_VARIANT_TENSOR for the FP64 view of an
  // eligible Cartesian operator selects the tensor-core apply (mf_tc.cu)
  int variant[3] = {0, 0, 0};
  void* tc_table = nullptr;             // device: digit slices of the element matrix (workspace)
  int tc_fexp[64] = {0};                // per output row: biased exponent bound of its entries
  std::vector<unsigned short> tc_host;  // host copy of the digit slices (upload source)
};

namespace mf {

// error reporting (thread-local last error)
mf_status set_error(mf_status code, const char* fmt, ...);
mf_status cuda_check(cudaError_t e, const char* what);

// Per-precision dispatch entry points (defined in the per-degree instantiation units).
// elem: 8 or 4.  All return MF_OK or an error status.
// apply / geometry take a ViewKind; dss / layout / reductions take the element size.
mf_status launch_apply_split(const mf_operator* op, int vk, const void* x, void* y, cudaStream_t s);
// CG step apply (see CgFuse): p and r in the element type of the view vk; *nblocks = CTAs
// launched (the number of partials written)
mf_status launch_apply_cg(const mf_operator* op, int vk, void* p, const void* r, void* y, CgState* st, double* partials,
                          int update_p, long long* nblocks, cudaStream_t s);
// upper bound of the CTA count of any apply launch of op (size of CgFuse::partials)
long long apply_max_blocks(const mf_operator* op);
mf_status launch_dss(const mf_operator* op, int elem, void* y, cudaStream_t s);
mf_status launch_geometry(const mf_operator* op, int vk, void* geom, cudaStream_t s);
mf_status launch_layout(const mf_operator* op, int elem, int mode, const void* in, void* out, cudaStream_t s);

template <int N>
mf_status apply_split_n(const mf_operator* op, int vk, const void* x, void* y, cudaStream_t s);
template <int N>
mf_status apply_block_n(const mf_operator* op, int vk, int cells, const void* x, void* y, cudaStream_t s);
template <int N>
mf_status apply_cg_n(const mf_operator* op, int vk, void* p, const void* r, void* y, CgState* st, double* partials,
                     int update_p, long long* nblocks, cudaStream_t s);
template <int N>
mf_status dss_n(const mf_operator* op, int elem, void* y, cudaStream_t s);
template <int N>
mf_status make_consistent_n(const mf_operator* op, int elem, void* y, cudaStream_t s);
template <int N>
mf_status dss_atomic_n(const mf_operator* op, int elem, void* y, void* acc, cudaStream_t s);
template <int N>
mf_status stream_twin_n(const mf_operator* op, int vk, const void* x, void* y, const void* geom, int nc,
                        cudaStream_t s);
template <int N>
mf_status diagonal_n(const mf_operator* op, float* diag, float* gtab, cudaStream_t s);
// assembled diagonal (FP32, consistent, 0 on Dirichlet nodes); gtab: diag_table_bytes(op) bytes
mf_status launch_diagonal(const mf_operator* op, float* diag, float* gtab, cudaStream_t s);
inline size_t diag_table_bytes(const mf_operator* op) {
  return sizeof(float) * 2 * (size_t)(op->g.nx + op->g.ny + op->g.nz) * (size_t)op->n;
}
template <int N>
mf_status apply_batch_fill_n(const BatchMember* m, int n, int vk, void* jobs_host, long long* block0_host);
template <int N>
mf_status apply_batch_launch_n(const mf_operator* op0, int vk, const void* jobs_dev, const long long* block0_dev,
                               int njobs, long long blocks, cudaStream_t s);
// batched CG-step apply (mf_api.cu dispatch): all members share degree, path, kind and variant
mf_status apply_batch_fill(const BatchMember* m, int n, int vk, void* jobs_host, long long* block0_host);
mf_status apply_batch_launch(const mf_operator* op0, int vk, const void* jobs_dev, const long long* block0_dev,
                             int njobs, long long blocks, cudaStream_t s);
size_t apply_job_bytes(int vk); // size of one member's description
template <int N>
mf_status geometry_n(const mf_operator* op, int vk, void* geom, cudaStream_t s);
template <int N>
mf_status layout_n(const mf_operator* op, int elem, int mode, const void* in, void* out, cudaStream_t s);

// Tensor-core apply of the FP64 Cartesian operator (mf_tc.cu), degrees 1..3: launch variant
// MF_VARIANT_TENSOR (include/mf.h).
bool tc_eligible(const mf_operator* op);
size_t tc_table_bytes(const mf_operator* op);              // device bytes of its digit table
mf_status tc_setup(mf_operator* op, void* table_dev, cudaStream_t s); // builds and uploads it
mf_status tc_apply(const mf_operator* op, const void* x, void* y, cudaStream_t s);
int tc_read_error(int reset);                              // device error word (synchronous)

// CG preconditioned by degree-3 Chebyshev-accelerated Jacobi (mf_cheb.cu)
size_t cheb_workspace_bytes(const mf_operator* op);
mf_status cheb_solve(const mf_operator* op, const void* b, void* x, double rtol, int maxit, double ratio,
                     mf_solve_stats* stats, void* ws, size_t bytes, cudaStream_t s);

// layout modes
enum { LAYOUT_TO_NATIVE = 0, LAYOUT_FROM_NATIVE = 1, LAYOUT_SCATTER_UNIQUE = 2, LAYOUT_GATHER_UNIQUE = 3 };

// geometry components per point
inline int geom_comps(const mf_operator* op) { return op->kind == MF_HELMHOLTZ ? 7 : 6; }

// View kind of the FP64 apply, and the view kind matching an element size.  MF_FP64 computes
// in double-float.  MF_FP64_DFMA, and the FP64 view of MF_MIXED, use the native FP64 pipe:
// the mixed solver applies it only for the outer residual b - A x (a few times per solve),
// whose 53-bit evaluation keeps the true residual's floor well below the tolerances asked of
// it (double-float evaluation noise, about 2^-48 relative per value, left curved Q6 64^3
// requests stagnating near 1e-10).
inline int fp64_view(const mf_operator* op) {
  return (op->precision == MF_FP64_DFMA || op->precision == MF_MIXED) ? VK_F64 : VK_DD;
}
inline int view_of_elem(const mf_operator* op, int elem) { return elem == 8 ? fp64_view(op) : VK_F32; }

// Reductions and CG vector kernels (mf_cg.cu)
size_t reduce_scratch_bytes();
mf_status dot_launch(const mf_operator* op, int elem, const void* a, const void* b, int split, double* out,
                     void* scratch, cudaStream_t s);

} // namespace mf
