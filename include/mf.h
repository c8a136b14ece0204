/*
 * mf.h -- C ABI of the GB300 matrix-free Q_k operator library (libmf.so).
 *
 * The library evaluates y = A x for the continuous tensor-product Q_k finite-element
 * operator (Laplace, or Helmholtz = mass + Laplace) on a structured hexahedral mesh of the
 * unit cube, affine or curved, with the vector held in cell-wise storage: every cell owns
 * its (k+1)^3 nodal values and shared vertex/edge/face values are duplicated.  The apply
 * is the volume term of the paper's bilinear form (Sec. 2, Eq. (sipg), first sum) evaluated
 * by sum factorisation (Sec. 3.1, Eq. (eval_pipeline) for the Cartesian form), followed by
 * a deterministic summation of the duplicated values (the assembly G G^T of Sec. 4,
 * Eqs. (shadow_gather), (shadow_assembly)), organised as the dimension-split,
 * atomic-free sweeps of Sec. 3.
 *
 * Conventions for every entry point:
 *  - Return value: MF_OK (0) or a negative mf_status.  No entry point aborts.
 *  - Pointers named *_dev are device pointers owned by the caller (allocated e.g. through
 *    PyTorch).  The library never allocates, frees or retains device memory except inside
 *    a workspace the caller hands over (mf_operator_setup, mf_cg_solve, mf_server_create).
 *  - Pointers named *_host are host pointers owned by the caller.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).  Work is
 *    enqueued on it; the call returns before the GPU finishes unless stated otherwise.
 *  - Vectors in "native" layout have mf_info.n_native elements of the operator's element
 *    type (double for MF_FP64 and MF_MIXED, float for MF_FP32).  Native layout: tiles of
 *    32 cells (a 4x4x2 brick), element (tile, local dof l, lane) at (tile*n^3 + l)*32 + lane,
 *    l = i + n*(j + n*k) with x fastest.  Lanes of cells outside the mesh are padding: they
 *    are ignored on input and written as 0 on output.
 *  - "Canonical" cell-wise layout: [cell (x fastest)][k][j][i], n_cellwise elements.
 *  - "Unique" layout: global nodes (I,J,L), I = cx*k + i, lexicographic with x fastest,
 *    n_unique elements.
 *  - A cell-wise vector is consistent when all copies of each shared node are equal.
 */
#ifndef MF_H
#define MF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int mf_status;
#define MF_OK 0
#define MF_ERR_ARG (-1)           /* invalid argument, size or state */
#define MF_ERR_OOM (-2)           /* workspace or arena too small */
#define MF_ERR_CUDA (-3)          /* a CUDA call failed */
#define MF_ERR_NOT_CONVERGED (-4) /* solver reached maxit */
#define MF_ERR_BREAKDOWN (-5)     /* CG: p^T A p <= 0 or non-finite scalar */
#define MF_ERR_TIMEOUT (-6)       /* a bounded wait gave up */
#define MF_ERR_BUSY (-7)          /* request still pending / queue full */
#define MF_ERR_UNSUPPORTED (-8)   /* combination not built */
#define MF_ERR_CANCELLED (-9)     /* request cancelled before it finished */

enum { MF_AFFINE = 0, MF_CURVED_SIN = 1 };
enum { MF_LAPLACE = 0, MF_HELMHOLTZ = 1 };
/* MF_FP64: double vectors and geometry; the apply computes in double-float arithmetic on the
 *   FP32 pipe (about 48 significant bits, results within 1e-12 of FP64), because GB300 issues
 *   64x more FP32 than FP64 FMAs per clock.
 * MF_FP32: float vectors, geometry and arithmetic.
 * MF_MIXED: an FP32 view for the inner solver of mf_cg_solve(mixed = 1), and an FP64 view on
 *   the native FP64 pipe for its outer residual (as MF_FP64_DFMA).
 * MF_FP64_DFMA: as MF_FP64 but the apply uses the native FP64 FMA pipe. */
enum { MF_FP64 = 0, MF_FP32 = 1, MF_MIXED = 2, MF_FP64_DFMA = 3 };
enum { MF_BC_NONE = 0, MF_BC_DIRICHLET0 = 1 };

typedef struct mf_mesh mf_mesh;
typedef struct mf_operator mf_operator;
typedef struct mf_server mf_server;

/* Last error message of the calling thread (static storage, never NULL). */
const char* mf_last_error(void);

/* ------------------------------------------------------------------ mesh
 * nx*ny*nz cells of the unit cube.  geometry MF_AFFINE maps xh -> A xh + b with
 * affine_3x4 = {A row-major (9), b (3)} (NULL = identity).  MF_CURVED_SIN maps
 * xh -> xh + curve_amp * sin(pi xh1) sin(pi xh2) sin(pi xh3) on every coordinate; the
 * Jacobian is evaluated analytically at every Gauss point (Sec. 2: six metric entries and
 * det J per point).  Host-only object. */
mf_status mf_mesh_create(int nx, int ny, int nz, int geometry, const double* affine_3x4, double curve_amp,
                         mf_mesh** out);
void mf_mesh_destroy(mf_mesh* mesh);

/* ------------------------------------------------------------------ operator
 * degree k in 1..8 (n = k+1 GLL nodes and Gauss points per direction).  kind MF_LAPLACE or
 * MF_HELMHOLTZ (A = mass_coeff*M + K).  precision MF_FP64, MF_FP32 or MF_MIXED (FP64
 * vectors and geometry plus an FP32 copy of the geometry for the inner solver of
 * mf_cg_solve).  bc MF_BC_DIRICHLET0 applies P A P with P zeroing nodes on the cube
 * boundary.  Host-only until mf_operator_setup. */
mf_status mf_operator_create(const mf_mesh* mesh, int degree, int kind, double mass_coeff, int precision, int bc,
                             mf_operator** out);
void mf_operator_destroy(mf_operator* op);

typedef struct {
  int64_t n_cellwise;     /* cells * n^3 */
  int64_t n_unique;       /* (nx k+1)(ny k+1)(nz k+1) */
  int64_t n_native;       /* elements of a native vector (with padding lanes) */
  int64_t n_cells;
  int32_t degree, n, elem_bytes, path; /* path: 0 Cartesian, 1 affine general, 2 curved */
  size_t geom_bytes;      /* device bytes of per-point geometry (0 for affine paths) */
  size_t workspace_bytes; /* bytes mf_operator_setup needs (>= geom_bytes) */
  double algorithmic_bytes_per_apply; /* read x + write y + geometry, per apply */
} mf_info;
mf_status mf_operator_info(const mf_operator* op, mf_info* info);

/* Binds a caller-owned device workspace of >= info.workspace_bytes bytes (256-byte
 * aligned) and precomputes the per-point geometry into it on `stream`.  The workspace
 * must outlive the operator. */
mf_status mf_operator_setup(mf_operator* op, void* workspace_dev, size_t bytes, void* stream);

/* Autotuner: times each launch configuration of the apply kernel (variant 0: n^2 x CB
 * threads per CTA, registers capped for two CTAs per SM; variant 1: half the cells per CTA,
 * capped for three; variant 2: half the cells per CTA, no register cap; variant 3, for
 * MF_FP64 operators on an axis-aligned affine mesh of degree 1..3 only: the tensor-core
 * apply, see MF_VARIANT_TENSOR; variants 4 and 5, for MF_FP64 (double-float) operators
 * only: see MF_VARIANT_SMALL_CTA and MF_VARIANT_OCCUPANCY) with `reps` applies of x_dev into
 * y_dev (both native vectors
 * of this operator; y is overwritten) and keeps the fastest.  The choice is cached per
 * (device, degree, path, kind, precision, size class = floor(log2(cells))) for the life of
 * the process, so later operators of
 * the same class reuse it without timing, and persisted across processes in a JSON file keyed
 * by the GPU's name (MF_AUTOTUNE_CACHE, else $XDG_CACHE_HOME/libmf/autotune.json or
 * $HOME/.cache/libmf/autotune.json; MF_AUTOTUNE_CACHE=off disables the file): a stored choice
 * is used without timing.  Synchronises `stream` when it times.  Variants 0-2, 4 and 5 run the same
 * per-thread arithmetic and give bitwise equal results; variant 3 rounds differently (same
 * accuracy class), so its results agree with theirs within 1e-12 relative max-norm. */
mf_status mf_operator_autotune(mf_operator* op, const void* x_dev, void* y_dev, int reps, void* stream);
/* The tensor-core apply of the FP64 Cartesian operator (degree 1..3; the default launch
 * variant of such operators of degree 2 and 3).  All cells of an axis-aligned uniform mesh share one element
 * matrix A_e (the seven-contraction form of Sec. 3.1, Eq. (eval_pipeline), assembled per
 * element), so the local apply of 128 cells is the product X[128, n^3] A_e^T.  It runs on the
 * FP16 tensor cores (tcgen05) exactly: every value is cut into six balanced 8-bit integer
 * digits relative to its cell's (data) or row's (table) largest exponent, the 21 digit
 * products up to significance level 5 accumulate as exact integers in FP32, and the levels
 * are combined in 64-bit integers and rounded once to double (error-free splitting of
 * Ozaki et al., Numer. Algorithms 59, 2012).  Accuracy: a few 2^-48 relative to |A_e| |x|
 * per value.  A non-finite input value makes its cell's outputs NaN.  Needs
 * mf_operator_setup (the digit table lives in the operator workspace, at most 48 KB). */
#define MF_VARIANT_TENSOR 3
/* Half the cells per CTA of variant 0 (the B axis of the paper's block-size experiment,
 * Sec. 6; see mf_apply_split_block), with registers capped for 1.5x variant 0's resident
 * threads per SM.  Double-float view of MF_FP64 operators; same per-thread arithmetic as
 * variants 0-2 (bitwise equal results). */
#define MF_VARIANT_SMALL_CTA 4
/* Variant 0's cells per CTA with registers capped for three resident CTAs per SM instead of
 * two.  Double-float view of MF_FP64 operators; bitwise equal results. */
#define MF_VARIANT_OCCUPANCY 5
/* Forces a launch variant (0, 1 or 2) for every precision view, or MF_VARIANT_TENSOR /
 * MF_VARIANT_SMALL_CTA / MF_VARIANT_OCCUPANCY for the double-float view of an MF_FP64
 * operator (MF_ERR_UNSUPPORTED for an operator they do not cover); MF_ERR_ARG for any other
 * value. */
mf_status mf_operator_set_variant(mf_operator* op, int variant);
/* Variant in use for the operator's main precision view (-1 for a NULL operator). */
int mf_operator_get_variant(const mf_operator* op);

/* The library's device error word: nonzero when a bounded wait inside one of its kernels
 * (an mbarrier wait of the tensor-core apply) gave up; that kernel then left its outputs
 * incomplete.  Synchronous (reads device memory); reset != 0 clears the word. */
int mf_device_error(int reset);

/* ------------------------------------------------------------------ layout helpers */
/* canonical cell-wise -> native and back (device pointers, operator element type). */
mf_status mf_to_native(const mf_operator* op, const void* canonical_dev, void* native_dev, void* stream);
mf_status mf_from_native(const mf_operator* op, const void* native_dev, void* canonical_dev, void* stream);
/* unique -> native cell-wise copies (the gather G of Sec. 4, Eq. (shadow_gather)). */
mf_status mf_scatter_unique(const mf_operator* op, const void* unique_dev, void* native_dev, void* stream);
/* native consistent -> unique (reads one copy per node). */
mf_status mf_gather_unique(const mf_operator* op, const void* native_dev, void* unique_dev, void* stream);

/* ------------------------------------------------------------------ apply
 * y = G G^T A~ x: local sum-factorised apply of every cell followed by the deterministic
 * duplicate summation, so y is consistent; with MF_BC_DIRICHLET0, x is read as P x and y
 * is returned as P y.  x must be consistent.  x and y are native vectors and must not
 * overlap.  Summation order of duplicates: pairwise x, then y, then z
 * (((c000+c100)+(c010+c110))+((c001+c101)+(c011+c111)) for a vertex), independent of
 * tiling, so results are bitwise reproducible. */
mf_status mf_apply(const mf_operator* op, const void* x_dev, void* y_dev, void* stream);
/* y~ = A~ x: the split (unassembled) local results, no duplicate summation (Sec. 4,
 * Eq. (split_operator)). */
mf_status mf_apply_split(const mf_operator* op, const void* x_dev, void* y_dev, void* stream);
/* In-place duplicate summation y <- G G^T y (and P y for Dirichlet). */
mf_status mf_dss(const mf_operator* op, void* y_dev, void* stream);
/* In place: every copy of a shared node is replaced by the average of that node's copies,
 * y <- G diag(1/m) G^T y with m the multiplicity (1, 2, 4 or 8 copies), i.e. the assembly
 * G^T of Sec. 4, Eq. (shadow_assembly), divided by the number of cells sharing the node,
 * then the gather G of Eq. (shadow_gather).  Turns any cell-wise vector into a consistent
 * one (a projection: consistent vectors are left unchanged).  The copies are summed in the
 * canonical order of mf_dss and scaled by 1/m (exact), so all copies come out bitwise equal.
 * No Dirichlet mask is applied.  y_dev: native vector of the operator's element type,
 * caller-owned; padding lanes are left as they are.  Errors: MF_ERR_ARG (NULL argument),
 * MF_ERR_CUDA. */
mf_status mf_make_consistent(const mf_operator* op, void* y_dev, void* stream);
/* Ablation of the duplicate summation (a measurement entry; the paper compares its layer-
 * disjoint sweeps against an atomic variant in Sec. 6): every copy atomically adds its value
 * into an accumulator over unique nodes (scratch: mf_dss_atomic_workspace_bytes() device
 * bytes, 256-byte aligned), then every copy reads the sum back.  Consistent, but the order of
 * the atomic additions -- hence the last bits of the sums -- is not reproducible.  Same
 * precision as the operator's vectors; P y for Dirichlet. */
size_t mf_dss_atomic_workspace_bytes(const mf_operator* op);
mf_status mf_dss_atomic(const mf_operator* op, void* y_dev, void* scratch_dev, size_t scratch_bytes, void* stream);
/* Block-size sweep (a measurement entry: the paper sweeps the cells per thread block B of
 * its volume kernel, Sec. 6): mf_apply_split with cells_per_cta = B in {4, 8, 16, 32} cells
 * per CTA -- divisors of the 32-cell layout tile -- instead of the launch variant's.
 * Registers are capped so that every B keeps launch variant 0's resident threads per SM.
 * Same result as mf_apply_split with launch variant 0 (the arithmetic of a cell does not
 * depend on B), no duplicate summation.  Built for degree 3 on every path with MF_FP64
 * (double-float) and MF_FP32 operators, and for the Cartesian path of MF_FP64 operators at
 * every degree; n^2 B threads must lie in 32..1024.  x_dev, y_dev: device, n_native elements
 * of the operator's vector precision, caller-owned, distinct.  Errors: MF_ERR_ARG (NULL
 * operator or vectors, B not one of the four, operator not ready), MF_ERR_UNSUPPORTED (a
 * combination not built; MF_FP64_DFMA and MF_MIXED, whose double vectors take the native
 * FP64 apply), MF_ERR_CUDA. */
mf_status mf_apply_split_block(const mf_operator* op, int cells_per_cta, const void* x_dev, void* y_dev, void* stream);
/* Stream twin of the apply kernel (a measurement entry: the paper times kernels that keep a
 * kernel's memory accesses and drop its arithmetic, Sec. 6, as the ceiling of its access
 * pattern).  One launch with the apply's grid and cells per CTA (the operator's launch
 * variant) and its global accesses: the cell-wise x tile of every CTA is read; for a curved
 * mesh in an FP64 precision the per-point metric (6 words per point, 7 for Helmholtz, 8 bytes
 * each) is read as the apply streams it; y is written by x-pencils.  No contraction and no
 * duplicate summation.  y_dev receives a bit-copy of x_dev, not an operator result.
 * x_dev, y_dev: device, n_native elements of the operator's vector precision, caller-owned,
 * distinct.  Errors: MF_ERR_ARG (NULL or equal vectors, operator not ready), MF_ERR_CUDA. */
mf_status mf_apply_stream_twin(const mf_operator* op, const void* x_dev, void* y_dev, void* stream);
/* The assembled diagonal of the operator (P A P for Dirichlet: 0 on constrained nodes), as a
 * consistent native vector of FP32 values (n_native floats), computed from the same
 * quadrature and metric as the apply, for Jacobi preconditioning of CG (the paper's smoother,
 * Sec. 5.2, is a Chebyshev-accelerated block Jacobi inside multigrid).  Scratch:
 * mf_diagonal_workspace_bytes() device bytes. */
size_t mf_diagonal_workspace_bytes(const mf_operator* op);
mf_status mf_diagonal(const mf_operator* op, float* diag_dev, void* scratch_dev, size_t scratch_bytes, void* stream);
/* End to end from host memory: copies canonical x_host to the device, applies, copies the
 * canonical result to y_host and synchronises `stream`.  Uses the caller's device
 * workspace of >= mf_apply_host_workspace_bytes() bytes. */
size_t mf_apply_host_workspace_bytes(const mf_operator* op);
mf_status mf_apply_host(const mf_operator* op, const void* x_host, void* y_host, void* workspace_dev, size_t bytes,
                        void* stream);

/* ------------------------------------------------------------------ manufactured workload
 * u = sin(freq pi x) sin(freq pi y) sin(freq pi z) on the unit cube (homogeneous Dirichlet data
 * for integer freq), f = -Lap u + c_m u.  mf_rhs_manufactured writes the consistent assembled
 * load vector b_i = int f phi_i (Gauss rule of the operator, k+1 points per direction; masked
 * for MF_BC_DIRICHLET0).  mf_error_manufactured writes sum_K int_K (u - u_h)^2 (the squared L2
 * error of the native vector u_h) to *l2sq_dev.  Both evaluate u at the physical quadrature
 * points in double-float arithmetic and need mf_manufactured_workspace_bytes() of scratch.
 * Affine maps must be axis-aligned (MF_ERR_UNSUPPORTED otherwise). */
size_t mf_manufactured_workspace_bytes(const mf_operator* op);
mf_status mf_rhs_manufactured(const mf_operator* op, double freq, void* b_dev, void* scratch_dev, size_t scratch_bytes,
                              void* stream);
mf_status mf_error_manufactured(const mf_operator* op, double freq, const void* u_dev, double* l2sq_dev,
                                void* scratch_dev, size_t scratch_bytes, void* stream);

/* ------------------------------------------------------------------ reductions
 * Assembled inner product of two consistent native vectors (each unique node counted once:
 * copies weighted by 1/multiplicity, powers of two, so exact), accumulated in FP64 in a
 * fixed order; result written to *result_dev (one double, device).  With split=1 the
 * first vector is a split dual and the pairing is the flat sum over all copies (Lemma 1,
 * Eq. (shadow_pairing)).  Needs mf_reduce_workspace_bytes() of scratch. */
size_t mf_reduce_workspace_bytes(const mf_operator* op);
mf_status mf_dot(const mf_operator* op, const void* a_dev, const void* b_dev, int split, double* result_dev,
                 void* scratch_dev, size_t scratch_bytes, void* stream);

/* Allocation-free variant of mf_dot (the paper has no counterpart: it is a service for
 * callers that may not allocate device memory where they reduce, e.g. a solver inside a
 * host application whose device memory belongs to another allocator, or a time-critical
 * loop that avoids cudaMalloc because it may synchronise the device).  Same result as
 * mf_dot within rounding (same weights, FP64 accumulation, fixed order; a different CTA
 * split).  Its scratch is a 512 KiB static device array inside libmf (held by every GPU
 * that loads the library until exit): vectors with n_native > 134,217,728 elements are
 * rejected with MF_ERR_ARG, as is an operator that has not been set up (mf_operator_setup),
 * both before any CUDA call.  The first successful call on a device looks up that array's
 * address with the device current and caches it per device for the life of the process
 * (a failed lookup is not cached: the next call retries); make that first call before any
 * stream capture.  The cached address is invalid after cudaDeviceReset.  All calls share the
 * array: calls that overlap on the GPU race, so serialise them.  Calls no allocating
 * routine. */
mf_status mf_dot_noalloc(const mf_operator* op, const void* a_dev, const void* b_dev, int split, double* result_dev,
                         void* stream);

/* ------------------------------------------------------------------ CG solver
 * CG (unpreconditioned unless mf_cg_solve_ex asks for Jacobi) on (P A P) x = P b from x = 0 for
 * consistent native b, to
 * ||b - A x|| <= rtol ||b|| (assembled Euclidean norm = the pairing <r, r> of Sec. 4) or
 * maxit iterations.  mixed = 0: FP64 (or FP32 for an MF_FP32 operator) CG; for MF_FP64 and
 * MF_MIXED operators its iteration keeps x, r, p and A p as double-float pairs (about 48
 * significant bits, FP32-pipe arithmetic; b enters scaled by the power of two of max|b|, x
 * leaves scaled back), MF_FP64_DFMA keeps doubles.  mixed = 1
 * (operator MF_MIXED): FP64 defect correction -- outer residual r = b - A x, the update and
 * all dot products in FP64, inner CG with the FP32 apply.  Without a preconditioner the inner
 * CG is not restarted at a defect-correction step but continued with reliable updates (Clark
 * et al. 2010): its residual is replaced by the FP64 one (scaled by 1/||b|| throughout), its
 * search direction kept, p = r^ + beta p with beta = <r^, r^> / <r_k, r_k>, and its tolerance
 * reset to inner_rtol ||r^||; mf_solve_options.mixed_restart = 1 restarts it from p = r^
 * instead (the Jacobi-preconditioned solve always restarts).  Synchronous.  Workspace:
 * mf_cg_workspace_bytes(op, mixed) device bytes. */
typedef struct {
  int32_t iterations;       /* total CG iterations (inner iterations for mixed) */
  int32_t outer_iterations; /* defect-correction steps (mixed) */
  double rel_residual;      /* final ||b - A x|| / ||b|| in FP64 */
  double seconds;           /* wall time of the solve */
  int32_t status;           /* MF_OK, MF_ERR_NOT_CONVERGED, MF_ERR_BREAKDOWN */
  int32_t check_every;      /* iterations between host residual checks */
} mf_solve_stats;
size_t mf_cg_workspace_bytes(const mf_operator* op, int mixed);
mf_status mf_cg_solve(const mf_operator* op, const void* b_dev, void* x_dev, double rtol, int maxit, int mixed,
                      mf_solve_stats* stats, void* workspace_dev, size_t bytes, void* stream);
/* End to end from host memory: copies the canonical cell-wise right-hand side b_host
 * (n_cellwise elements of the operator's element type, consistent) to the device, converts
 * it to the native layout, runs mf_cg_solve from x = 0, and copies the canonical solution
 * to x_host; synchronises `stream` before it returns.  Host buffers are the caller's (pinned
 * memory makes the copies asynchronous DMA; pageable memory works, more slowly).  Device
 * workspace: mf_cg_solve_host_workspace_bytes(op, mixed) bytes, 256-byte aligned.  Returns
 * what mf_cg_solve returns (x_host is written for MF_ERR_NOT_CONVERGED and MF_ERR_BREAKDOWN
 * too), or MF_ERR_ARG / MF_ERR_OOM / MF_ERR_CUDA. */
size_t mf_cg_solve_host_workspace_bytes(const mf_operator* op, int mixed);
mf_status mf_cg_solve_host(const mf_operator* op, const void* b_host, void* x_host, double rtol, int maxit, int mixed,
                           mf_solve_stats* stats, void* workspace_dev, size_t bytes, void* stream);
/* mf_cg_solve with options (0 fields keep the defaults): inner_rtol of the FP32 CG in
 * defect correction (default 0.1 with reliable updates -- Q4 curved 96^3: 1e-3 took 23770
 * inner iterations, 0.1 2579 -- and 1e-3 restarted), CG iterations per graph launch (default 20), cap on
 * defect-correction steps (default 60), and the form of the CG iteration:
 *   MF_CG_SPLIT_DUAL (default) -- the Krylov loop on split data of Sec. 4: the apply leaves
 *     A p split (no duplicate summation) and forms <p, A p> -- the pairing of the consistent p
 *     with the split product over all copies (Lemma 1) -- as the sum over quadrature points
 *     of grad u . G grad u; the duplicate summation is folded into the update of x and r;
 *     then p = r + beta p.  Four kernels per iteration (apply, alpha, update, direction).
 *   MF_CG_ASSEMBLED -- apply, duplicate summation, then the vector kernels on assembled
 *     vectors (five kernels per iteration).
 *   MF_CG_SPLIT_DUAL_FUSED -- MF_CG_SPLIT_DUAL with p = r + beta p formed by the apply at
 *     load (three kernels per iteration).
 * All compute the same iterates up to rounding (only <p, A p> is summed differently). */
enum { MF_CG_DEFAULT = 0, MF_CG_SPLIT_DUAL = 1, MF_CG_ASSEMBLED = 2, MF_CG_SPLIT_DUAL_FUSED = 3 };
/* Preconditioner (mf_solve_options.precond): none (default), Jacobi -- z = r / diag(P A P)
 * with the assembled diagonal of mf_diagonal (0 on Dirichlet nodes); split-dual form only --
 * or the degree-3 Chebyshev-accelerated Jacobi method of Sec. 5.2 (the paper's smoother as a
 * CG preconditioner): z = M^-1 r is three Richardson updates z <- z + w_j D^-1 (r - A z) from
 * z = 0 with the weights of Eq. (chebyshev_weights) on [b / cheb_ratio, b], b = 1.1 times a
 * 12-step power-iteration estimate of the largest eigenvalue of D^-1 A; M is symmetric positive
 * definite.  Each CG iteration then applies the operator three times (iterations in
 * mf_solve_stats are CG iterations); assembled vectors of the operator's element type, MF_FP64
 * and MF_FP32 operators, mixed = 0 only; workspace mf_cg_workspace_bytes_ex().  The
 * convergence test stays ||r|| <= rtol ||b||; alpha and beta use <r, z>. */
enum { MF_PRECOND_NONE = 0, MF_PRECOND_JACOBI = 1, MF_PRECOND_CHEBYSHEV = 2 };
typedef struct {
  double inner_rtol;
  int32_t chunk_iterations;
  int32_t max_outer;
  int32_t cg_form; /* MF_CG_* */
  int32_t precond; /* MF_PRECOND_* */
  double cheb_ratio; /* MF_PRECOND_CHEBYSHEV: b / a of the target interval (0: 30) */
  int32_t mixed_restart; /* mixed, unpreconditioned: 0 reliable updates, 1 restarted inner CG */
  int32_t reserved;      /* 0 */
} mf_solve_options;
/* Workspace of mf_cg_solve_ex with these options (opts may be NULL: mf_cg_workspace_bytes). */
size_t mf_cg_workspace_bytes_ex(const mf_operator* op, int mixed, const mf_solve_options* opts);
mf_status mf_cg_solve_ex(const mf_operator* op, const void* b_dev, void* x_dev, double rtol, int maxit, int mixed,
                         const mf_solve_options* opts, mf_solve_stats* stats, void* workspace_dev, size_t bytes,
                         void* stream);
/* Kernel timing of the CG iteration (a measurement helper; the paper has no counterpart):
 * runs `iterations` FP64 (FP32 for an MF_FP32 operator) CG iterations from x = 0 on b, of the
 * form cg_form (MF_CG_*), launching every kernel directly (no graph) with CUDA events around
 * each kernel group on `stream`, and writes the mean durations in milliseconds:
 * ms_out[0] the apply kernel (split-dual forms: the apply and the one-CTA alpha kernel after it),
 * ms_out[1] the duplicate
 * summation (assembled form; 0 for split-dual), ms_out[2] the vector kernels, ms_out[3] the
 * whole iteration.  1 <= iterations <= 1000.  Same workspace as mf_cg_solve (mixed = 0).
 * Synchronous. */
mf_status mf_cg_profile(const mf_operator* op, const void* b_dev, void* x_dev, int iterations, int cg_form,
                        void* workspace_dev, size_t bytes, void* stream, double* ms_out);
/* Records up to `cap` relative residual norms (one per iteration, FP64) of the next
 * mf_cg_solve on this thread into hist_host; pass NULL to stop recording. */
mf_status mf_cg_record_history(double* hist_host, int cap);

/* ------------------------------------------------------------------ serving
 * Continuous-batching solve server.  Requests are queued by mf_batch_submit and admitted in
 * arrival order whenever one of max_slots slots and enough of the caller's device arena are
 * free (a request that does not fit yet does not block smaller ones behind it).  An admitted
 * request keeps its geometry, vectors and CG state resident in its arena block.  Its set-up,
 * the outer steps of defect correction and its finish run on its slot's CUDA stream; its CG
 * iterations run in a continuous batch: every active request of the same degree, path,
 * operator kind, vector precision and launch variant takes part in one batched launch per
 * kernel of the (split-dual) CG iteration -- apply, alpha, update, direction -- in chunks of
 * chunk_iterations, and requests join and leave the batch between chunks.  The batched apply
 * is one persistent launch: the CTAs that fit the GPU at once loop over the CTA-sized work
 * units of all members.  Requests whose own apply takes more than 1024 CTAs run their own
 * graph chunks (they fill the GPU alone).  Each request's
 * arithmetic (its CTAs, reductions and their order) is exactly that of its own solo launch,
 * so its result does not depend on what else is in the batch.  batching = -1 runs every
 * request as separate graph chunks on its own stream instead.  A native scheduler thread
 * advances requests when their scalars have landed and admits new ones as slots and memory
 * free up.  Every request solves the homogeneous Dirichlet problem on the unit cube with the
 * given operator; mixed = 1 runs FP32 applies inside FP64 defect correction (else FP64 CG).
 * The arena is the only device memory used (pinned host memory holds per-slot scalars and
 * batch descriptors); it must outlive the server. */
enum { MF_RHS_MANUFACTURED = 0, MF_RHS_RANDOM = 1 };

typedef struct {
  int32_t max_slots;        /* concurrent requests (default 32, at most 256) */
  int32_t queue_capacity;   /* pending requests before MF_ERR_BUSY (default 100000) */
  int32_t chunk_iterations; /* CG iterations per graph launch (default 10) */
  int32_t autotune;         /* 1: autotune the apply of each new operator class */
  double inner_rtol;        /* mixed: inner FP32 CG tolerance (default 0.1, reliable updates) */
  int32_t batching;         /* 0 / 1: continuous batches of CG iterations (default); -1: off */
  int32_t mixed_restart;    /* mixed: 0 reliable updates (default), 1 restarted inner CG */
} mf_server_config;

typedef struct {
  int32_t nx, ny, nz, degree, kind, geometry;
  double mass_coeff, curve_amp;
  int32_t rhs;              /* MF_RHS_MANUFACTURED (u = prod sin(freq pi x_d)) or MF_RHS_RANDOM */
  double freq;              /* manufactured frequency */
  uint64_t seed;            /* random right-hand side: splitmix64 stream on unique DoFs */
  double rtol;              /* relative residual target (assembled Euclidean norm) */
  int32_t maxit;            /* CG iterations cap (inner iterations for mixed) */
  int32_t mixed;
  double* x_out_host;       /* optional: receives the solution on unique DoFs (n_unique doubles) */
} mf_request;

typedef struct {
  int32_t status;           /* MF_ERR_BUSY while queued or running; then the solve status */
  int32_t iterations, outer_iterations;
  double rel_residual;
  double l2_error;          /* manufactured right-hand side: ||u - u_h||_L2, else -1 */
  double t_submit, t_admit, t_done, latency; /* seconds since server creation; latency = done - submit */
  int64_t n_cellwise, n_unique;
  size_t device_bytes;      /* arena bytes the request held */
} mf_result;

typedef struct {
  int64_t pending, active, admitted, completed;
  size_t arena_bytes, arena_used, arena_peak;
} mf_server_stats_t;

mf_status mf_server_create(const mf_server_config* cfg, void* arena_dev, size_t arena_bytes, mf_server** out);
/* Validates and queues a request; MF_ERR_OOM if it can never fit in the arena, MF_ERR_BUSY if
 * the queue is full. */
mf_status mf_batch_submit(mf_server* server, const mf_request* req, uint64_t* ticket);
/* MF_ERR_BUSY (res->status too) while pending; MF_OK once finished, after which the ticket
 * is forgotten (res->status holds the solve's own status). */
mf_status mf_batch_poll(mf_server* server, uint64_t ticket, mf_result* res);
/* Marks a request cancelled: dropped if still queued, stopped at its next chunk if running
 * (final status MF_ERR_CANCELLED). */
mf_status mf_batch_cancel(mf_server* server, uint64_t ticket);
/* Waits (bounded) until no request is queued or running; MF_ERR_TIMEOUT otherwise. */
mf_status mf_server_drain(mf_server* server, double timeout_s);
mf_status mf_server_stats(mf_server* server, mf_server_stats_t* out);
/* Cancels outstanding work, waits for the slot streams and frees host resources. */
void mf_server_destroy(mf_server* server);

#ifdef __cplusplus
}
#endif
#endif /* MF_H */
