// mf_api.cu -- C ABI: mesh and operator handles, workspace binding, layout helpers, apply.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>

#include <sys/stat.h>
#include <unistd.h>

#include "mf_dd.cuh"
#include "mf_internal.h"

namespace mf {

static thread_local char g_err[512] = "";

mf_status set_error(mf_status code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

mf_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MF_OK;
  return set_error(MF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define MF_DISPATCH_N(n, fn, ...)                                                   \
  switch (n) {                                                                      \
    case 2: return fn<2>(__VA_ARGS__);                                              \
    case 3: return fn<3>(__VA_ARGS__);                                              \
    case 4: return fn<4>(__VA_ARGS__);                                              \
    case 5: return fn<5>(__VA_ARGS__);                                              \
    case 6: return fn<6>(__VA_ARGS__);                                              \
    case 7: return fn<7>(__VA_ARGS__);                                              \
    case 8: return fn<8>(__VA_ARGS__);                                              \
    case 9: return fn<9>(__VA_ARGS__);                                              \
    default: return set_error(MF_ERR_UNSUPPORTED, "degree %d not built", (n) - 1);  \
  }

mf_status launch_apply_split(const mf_operator* op, int elem, const void* x, void* y, cudaStream_t s) {
  MF_DISPATCH_N(op->n, apply_split_n, op, elem, x, y, s);
}
mf_status launch_apply_cg(const mf_operator* op, int vk, void* p, const void* r, void* y, CgState* st, double* partials,
                          int update_p, long long* nblocks, cudaStream_t s) {
  MF_DISPATCH_N(op->n, apply_cg_n, op, vk, p, r, y, st, partials, update_p, nblocks, s);
}
mf_status apply_batch_fill(const BatchMember* m, int n, int vk, void* jobs_host, long long* block0_host) {
  MF_DISPATCH_N(m[0].op->n, apply_batch_fill_n, m, n, vk, jobs_host, block0_host);
}
mf_status apply_batch_launch(const mf_operator* op0, int vk, const void* jobs_dev, const long long* block0_dev,
                             int njobs, long long blocks, cudaStream_t s) {
  MF_DISPATCH_N(op0->n, apply_batch_launch_n, op0, vk, jobs_dev, block0_dev, njobs, blocks, s);
}
size_t apply_job_bytes(int vk) {
  // the description layout depends only on the element types, not on the degree
  return vk == VK_F32 ? sizeof(ApplyJob<float, FP32C>)
                      : (vk == VK_DDS ? sizeof(ApplyJob<dd, dd>)
                                      : (vk == VK_DD ? sizeof(ApplyJob<double, dd>) : sizeof(ApplyJob<double, double>)));
}
mf_status launch_diagonal(const mf_operator* op, float* diag, float* gtab, cudaStream_t s) {
  MF_DISPATCH_N(op->n, diagonal_n, op, diag, gtab, s);
}
// every launch variant puts at least 4 cells of a 32-cell tile in one CTA
long long apply_max_blocks(const mf_operator* op) { return op->g.ntiles * (BL / 4); }
mf_status launch_dss(const mf_operator* op, int elem, void* y, cudaStream_t s) {
  MF_DISPATCH_N(op->n, dss_n, op, elem, y, s);
}
mf_status launch_geometry(const mf_operator* op, int elem, void* geom, cudaStream_t s) {
  MF_DISPATCH_N(op->n, geometry_n, op, elem, geom, s);
}
mf_status launch_layout(const mf_operator* op, int elem, int mode, const void* in, void* out, cudaStream_t s) {
  MF_DISPATCH_N(op->n, layout_n, op, elem, mode, in, out, s);
}

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

} // namespace mf

using namespace mf;

extern "C" {

const char* mf_last_error(void) { return g_err; }

mf_status mf_mesh_create(int nx, int ny, int nz, int geometry, const double* affine_3x4, double curve_amp,
                         mf_mesh** out) {
  if (!out) return set_error(MF_ERR_ARG, "mf_mesh_create: out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) return set_error(MF_ERR_ARG, "mf_mesh_create: cell counts must be >= 1");
  if ((long long)nx * ny * nz > (1LL << 31)) return set_error(MF_ERR_ARG, "mf_mesh_create: too many cells");
  if (geometry != MF_AFFINE && geometry != MF_CURVED_SIN)
    return set_error(MF_ERR_ARG, "mf_mesh_create: unknown geometry %d", geometry);
  mf_mesh* m = new (std::nothrow) mf_mesh;
  if (!m) return set_error(MF_ERR_OOM, "mf_mesh_create: host allocation failed");
  m->nx = nx; m->ny = ny; m->nz = nz; m->geom = geometry; m->amp = curve_amp;
  for (int i = 0; i < 9; ++i) m->A[i] = (i % 4 == 0) ? 1.0 : 0.0;
  for (int i = 0; i < 3; ++i) m->b[i] = 0.0;
  if (geometry == MF_AFFINE && affine_3x4) {
    for (int i = 0; i < 9; ++i) m->A[i] = affine_3x4[i];
    for (int i = 0; i < 3; ++i) m->b[i] = affine_3x4[9 + i];
  }
  if (geometry == MF_CURVED_SIN) {
    // det of the map is 1 + amp*pi*(c s s + s c s + s s c) >= 1 - amp*pi*sqrt(3)*... ; require
    // a strictly positive Jacobian everywhere: |amp| * pi * 3 < 1 is sufficient.
    if (!(std::fabs(curve_amp) * M_PI * 3.0 < 1.0)) {
      delete m;
      return set_error(MF_ERR_ARG, "mf_mesh_create: curve_amp %g may fold the mesh", curve_amp);
    }
  }
  *out = m;
  return MF_OK;
}

void mf_mesh_destroy(mf_mesh* mesh) { delete mesh; }

mf_status mf_operator_create(const mf_mesh* mesh, int degree, int kind, double mass_coeff, int precision, int bc,
                             mf_operator** out) {
  if (!out || !mesh) return set_error(MF_ERR_ARG, "mf_operator_create: NULL argument");
  *out = nullptr;
  if (degree < 1 || degree > 8) return set_error(MF_ERR_ARG, "mf_operator_create: degree %d not in 1..8", degree);
  if (kind != MF_LAPLACE && kind != MF_HELMHOLTZ) return set_error(MF_ERR_ARG, "mf_operator_create: kind %d", kind);
  if (precision != MF_FP64 && precision != MF_FP32 && precision != MF_MIXED && precision != MF_FP64_DFMA)
    return set_error(MF_ERR_ARG, "mf_operator_create: precision %d", precision);
  if (bc != MF_BC_NONE && bc != MF_BC_DIRICHLET0) return set_error(MF_ERR_ARG, "mf_operator_create: bc %d", bc);
  mf_operator* op = new (std::nothrow) mf_operator;
  if (!op) return set_error(MF_ERR_OOM, "mf_operator_create: host allocation failed");
  op->mesh = *mesh;
  op->degree = degree;
  op->n = degree + 1;
  op->kind = kind;
  op->mass = (kind == MF_HELMHOLTZ) ? mass_coeff : 0.0;
  op->precision = precision;
  op->bc = bc;
  if (make_host_tables(degree, &op->tab)) {
    delete op;
    return set_error(MF_ERR_ARG, "mf_operator_create: table construction failed");
  }
  GridInfo& g = op->g;
  g.nx = mesh->nx; g.ny = mesh->ny; g.nz = mesh->nz;
  g.ntx = (g.nx + TX - 1) / TX; g.nty = (g.ny + TY - 1) / TY; g.ntz = (g.nz + TZ - 1) / TZ;
  g.ntiles = (long long)g.ntx * g.nty * g.ntz;
  g.bc = bc;
  const long long n3 = (long long)op->n * op->n * op->n;
  op->n_cellwise = (long long)g.nx * g.ny * g.nz * n3;
  op->n_unique = (long long)(g.nx * degree + 1) * (g.ny * degree + 1) * (g.nz * degree + 1);
  op->n_native = g.ntiles * n3 * BL;
  // affine constants: J = A diag(1/nx, 1/ny, 1/nz) is the same on every cell
  for (int m = 0; m < 6; ++m) op->G[m] = 0.0;
  op->mdet = op->gx = op->gy = op->gz = op->cmass = 0.0;
  if (mesh->geom == MF_AFFINE) {
    double J[9];
    const double h[3] = {1.0 / g.nx, 1.0 / g.ny, 1.0 / g.nz};
    for (int r = 0; r < 3; ++r)
      for (int d = 0; d < 3; ++d) J[3 * r + d] = mesh->A[3 * r + d] * h[d];
    const double det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                       J[2] * (J[3] * J[7] - J[4] * J[6]);
    if (!(std::fabs(det) > 0.0)) {
      delete op;
      return set_error(MF_ERR_ARG, "mf_operator_create: singular affine map");
    }
    double Ji[9];
    Ji[0] = (J[4] * J[8] - J[5] * J[7]) / det; Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
    Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det; Ji[3] = (J[5] * J[6] - J[3] * J[8]) / det;
    Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det; Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
    Ji[6] = (J[3] * J[7] - J[4] * J[6]) / det; Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
    Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
    const int pr[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    const double ad = std::fabs(det);
    for (int m = 0; m < 6; ++m) {
      const int r = pr[m][0], s = pr[m][1];
      op->G[m] = ad * (Ji[3 * r] * Ji[3 * s] + Ji[3 * r + 1] * Ji[3 * s + 1] + Ji[3 * r + 2] * Ji[3 * s + 2]);
    }
    op->mdet = op->mass * ad;
    const bool diag = J[1] == 0.0 && J[2] == 0.0 && J[3] == 0.0 && J[5] == 0.0 && J[6] == 0.0 && J[7] == 0.0;
    if (diag) {
      op->path = PATH_CARTESIAN;
      op->gx = op->G[0]; op->gy = op->G[3]; op->gz = op->G[5];
      op->cmass = op->mdet;
    } else {
      op->path = PATH_AFFINE;
    }
  } else {
    op->path = PATH_CURVED;
  }
  const size_t npts = (size_t)op->n_native; // points per tile equal dofs per tile
  op->v64.elem_bytes = 8;
  op->v32.elem_bytes = 4;
  if (op->path == PATH_CURVED) {
    const size_t comps = (size_t)geom_comps(op);
    op->v64.geom_bytes = (precision == MF_FP32) ? 0 : comps * npts * 8;
    // the FP32 view computes its metric per point from small sin/cos tables
    const size_t tab = sizeof(float) * 2 * (size_t)(g.nx + g.ny + g.nz) * op->n;
    op->v32.geom_bytes = (precision == MF_FP64 || precision == MF_FP64_DFMA) ? 0 : tab;
  }
  // the FP64 view of a Cartesian operator of degree 2 or 3 applies on the tensor cores by
  // default (at degree 1 the double-float kernel is faster; the autotuner can still pick it)
  if (tc_eligible(op) && op->n >= 3) op->variant[VK_DD] = MF_VARIANT_TENSOR;
  *out = op;
  return MF_OK;
}

void mf_operator_destroy(mf_operator* op) { delete op; }

mf_status mf_operator_info(const mf_operator* op, mf_info* info) {
  if (!op || !info) return set_error(MF_ERR_ARG, "mf_operator_info: NULL argument");
  std::memset(info, 0, sizeof(*info));
  info->n_cellwise = op->n_cellwise;
  info->n_unique = op->n_unique;
  info->n_native = op->n_native;
  info->n_cells = (long long)op->g.nx * op->g.ny * op->g.nz;
  info->degree = op->degree;
  info->n = op->n;
  info->elem_bytes = (op->precision == MF_FP32) ? 4 : 8;
  info->path = op->path;
  info->geom_bytes = op->v64.geom_bytes + op->v32.geom_bytes;
  info->workspace_bytes = align256(op->v64.geom_bytes) + align256(op->v32.geom_bytes) + align256(tc_table_bytes(op)) + 256;
  const double e = info->elem_bytes;
  double per_dof = 2.0 * e;
  if (op->path == PATH_CURVED && op->precision != MF_FP32) per_dof += geom_comps(op) * e; // FP32: no stream
  info->algorithmic_bytes_per_apply = per_dof * (double)op->n_cellwise;
  return MF_OK;
}

mf_status mf_operator_setup(mf_operator* op, void* workspace_dev, size_t bytes, void* stream) {
  if (!op) return set_error(MF_ERR_ARG, "mf_operator_setup: NULL operator");
  mf_info info;
  mf_operator_info(op, &info);
  if (info.workspace_bytes > 256 && (!workspace_dev || bytes < info.workspace_bytes))
    return set_error(MF_ERR_OOM, "mf_operator_setup: workspace of %zu bytes < %zu", bytes, info.workspace_bytes);
  if (workspace_dev && (reinterpret_cast<uintptr_t>(workspace_dev) & 255))
    return set_error(MF_ERR_ARG, "mf_operator_setup: workspace not 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(workspace_dev);
  op->v64.geom = nullptr;
  op->v32.geom = nullptr;
  if (op->v64.geom_bytes) { op->v64.geom = w; w += align256(op->v64.geom_bytes); }
  if (op->v32.geom_bytes) { op->v32.geom = w; w += align256(op->v32.geom_bytes); }
  op->tc_table = nullptr;
  if (tc_table_bytes(op)) {
    mf_status st = tc_setup(op, w, s);
    if (st) return st;
    w += align256(tc_table_bytes(op));
  }
  op->workspace = workspace_dev;
  op->workspace_bytes = bytes;
  if (op->path == PATH_CURVED) {
    if (op->v64.geom) { mf_status st = launch_geometry(op, fp64_view(op), op->v64.geom, s); if (st) return st; }
    if (op->v32.geom) { mf_status st = launch_geometry(op, VK_F32, op->v32.geom, s); if (st) return st; }
  }
  op->ready = true;
  return MF_OK;
}

static mf_status check_ready(const mf_operator* op, const char* who) {
  if (!op) return set_error(MF_ERR_ARG, "%s: NULL operator", who);
  if (!op->ready) return set_error(MF_ERR_ARG, "%s: operator not set up (mf_operator_setup)", who);
  return MF_OK;
}

static int elem_of(const mf_operator* op) { return op->precision == MF_FP32 ? 4 : 8; }

mf_status mf_to_native(const mf_operator* op, const void* canonical_dev, void* native_dev, void* stream) {
  if (!op || !canonical_dev || !native_dev) return set_error(MF_ERR_ARG, "mf_to_native: NULL argument");
  return launch_layout(op, elem_of(op), LAYOUT_TO_NATIVE, canonical_dev, native_dev, static_cast<cudaStream_t>(stream));
}
mf_status mf_from_native(const mf_operator* op, const void* native_dev, void* canonical_dev, void* stream) {
  if (!op || !canonical_dev || !native_dev) return set_error(MF_ERR_ARG, "mf_from_native: NULL argument");
  return launch_layout(op, elem_of(op), LAYOUT_FROM_NATIVE, native_dev, canonical_dev, static_cast<cudaStream_t>(stream));
}
mf_status mf_scatter_unique(const mf_operator* op, const void* unique_dev, void* native_dev, void* stream) {
  if (!op || !unique_dev || !native_dev) return set_error(MF_ERR_ARG, "mf_scatter_unique: NULL argument");
  return launch_layout(op, elem_of(op), LAYOUT_SCATTER_UNIQUE, unique_dev, native_dev, static_cast<cudaStream_t>(stream));
}
mf_status mf_gather_unique(const mf_operator* op, const void* native_dev, void* unique_dev, void* stream) {
  if (!op || !unique_dev || !native_dev) return set_error(MF_ERR_ARG, "mf_gather_unique: NULL argument");
  return launch_layout(op, elem_of(op), LAYOUT_GATHER_UNIQUE, native_dev, unique_dev, static_cast<cudaStream_t>(stream));
}

mf_status mf_apply_split(const mf_operator* op, const void* x_dev, void* y_dev, void* stream) {
  mf_status st = check_ready(op, "mf_apply_split");
  if (st) return st;
  if (!x_dev || !y_dev || x_dev == y_dev) return set_error(MF_ERR_ARG, "mf_apply_split: bad vectors");
  return launch_apply_split(op, view_of_elem(op, elem_of(op)), x_dev, y_dev, static_cast<cudaStream_t>(stream));
}

mf_status mf_apply_split_block(const mf_operator* op, int cells_per_cta, const void* x_dev, void* y_dev,
                               void* stream) {
  if (!op) return set_error(MF_ERR_ARG, "mf_apply_split_block: NULL operator");
  if (cells_per_cta != 4 && cells_per_cta != 8 && cells_per_cta != 16 && cells_per_cta != 32)
    return set_error(MF_ERR_ARG, "mf_apply_split_block: cells per CTA must be 4, 8, 16 or 32");
  mf_status st = check_ready(op, "mf_apply_split_block");
  if (st) return st;
  if (!x_dev || !y_dev || x_dev == y_dev) return set_error(MF_ERR_ARG, "mf_apply_split_block: bad vectors");
  MF_DISPATCH_N(op->n, apply_block_n, op, view_of_elem(op, elem_of(op)), cells_per_cta, x_dev, y_dev,
                static_cast<cudaStream_t>(stream));
}

mf_status mf_dss(const mf_operator* op, void* y_dev, void* stream) {
  if (!op || !y_dev) return set_error(MF_ERR_ARG, "mf_dss: NULL argument");
  return launch_dss(op, elem_of(op), y_dev, static_cast<cudaStream_t>(stream));
}

mf_status mf_make_consistent(const mf_operator* op, void* y_dev, void* stream) {
  if (!op || !y_dev) return set_error(MF_ERR_ARG, "mf_make_consistent: NULL argument");
  MF_DISPATCH_N(op->n, make_consistent_n, op, elem_of(op), y_dev, static_cast<cudaStream_t>(stream));
}

size_t mf_diagonal_workspace_bytes(const mf_operator* op) { return op ? diag_table_bytes(op) : 0; }

mf_status mf_diagonal(const mf_operator* op, float* diag_dev, void* scratch_dev, size_t scratch_bytes, void* stream) {
  if (!op || !diag_dev) return set_error(MF_ERR_ARG, "mf_diagonal: NULL argument");
  if (!scratch_dev || scratch_bytes < diag_table_bytes(op))
    return set_error(MF_ERR_OOM, "mf_diagonal: scratch %zu < %zu bytes", scratch_bytes, diag_table_bytes(op));
  return launch_diagonal(op, diag_dev, static_cast<float*>(scratch_dev), static_cast<cudaStream_t>(stream));
}

size_t mf_dss_atomic_workspace_bytes(const mf_operator* op) {
  return op ? (size_t)op->n_unique * (size_t)elem_of(op) : 0;
}

mf_status mf_dss_atomic(const mf_operator* op, void* y_dev, void* scratch_dev, size_t scratch_bytes, void* stream) {
  if (!op || !y_dev) return set_error(MF_ERR_ARG, "mf_dss_atomic: NULL argument");
  if (!scratch_dev || scratch_bytes < mf_dss_atomic_workspace_bytes(op))
    return set_error(MF_ERR_OOM, "mf_dss_atomic: scratch %zu < %zu bytes", scratch_bytes,
                     mf_dss_atomic_workspace_bytes(op));
  if (reinterpret_cast<uintptr_t>(scratch_dev) & 255) return set_error(MF_ERR_ARG, "mf_dss_atomic: scratch alignment");
  MF_DISPATCH_N(op->n, dss_atomic_n, op, elem_of(op), y_dev, scratch_dev, static_cast<cudaStream_t>(stream));
}

mf_status mf_apply_stream_twin(const mf_operator* op, const void* x_dev, void* y_dev, void* stream) {
  mf_status st = check_ready(op, "mf_apply_stream_twin");
  if (st) return st;
  if (!x_dev || !y_dev || x_dev == y_dev) return set_error(MF_ERR_ARG, "mf_apply_stream_twin: bad vectors");
  const int vk = view_of_elem(op, elem_of(op));
  const void* geom = (vk != VK_F32 && op->path == PATH_CURVED) ? op->v64.geom : nullptr;
  const int nc = geom ? geom_comps(op) : 0;
  MF_DISPATCH_N(op->n, stream_twin_n, op, vk, x_dev, y_dev, geom, nc, static_cast<cudaStream_t>(stream));
}

mf_status mf_apply(const mf_operator* op, const void* x_dev, void* y_dev, void* stream) {
  mf_status st = mf_apply_split(op, x_dev, y_dev, stream);
  if (st) return st;
  return launch_dss(op, elem_of(op), y_dev, static_cast<cudaStream_t>(stream));
}

size_t mf_apply_host_workspace_bytes(const mf_operator* op) {
  if (!op) return 0;
  const size_t e = (size_t)elem_of(op);
  return 2 * align256((size_t)op->n_native * e) + align256((size_t)op->n_cellwise * e);
}

mf_status mf_apply_host(const mf_operator* op, const void* x_host, void* y_host, void* workspace_dev, size_t bytes,
                        void* stream) {
  mf_status st = check_ready(op, "mf_apply_host");
  if (st) return st;
  if (!x_host || !y_host) return set_error(MF_ERR_ARG, "mf_apply_host: NULL host buffer");
  const size_t need = mf_apply_host_workspace_bytes(op);
  if (!workspace_dev || bytes < need) return set_error(MF_ERR_OOM, "mf_apply_host: workspace %zu < %zu", bytes, need);
  const size_t e = (size_t)elem_of(op);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(workspace_dev);
  void* xn = w;
  void* yn = w + align256((size_t)op->n_native * e);
  void* can = w + 2 * align256((size_t)op->n_native * e);
  const size_t cbytes = (size_t)op->n_cellwise * e;
  if ((st = cuda_check(cudaMemcpyAsync(can, x_host, cbytes, cudaMemcpyHostToDevice, s), "mf_apply_host H2D"))) return st;
  if ((st = mf_to_native(op, can, xn, stream))) return st;
  if ((st = mf_apply(op, xn, yn, stream))) return st;
  if ((st = mf_from_native(op, yn, can, stream))) return st;
  if ((st = cuda_check(cudaMemcpyAsync(y_host, can, cbytes, cudaMemcpyDeviceToHost, s), "mf_apply_host D2H"))) return st;
  return cuda_check(cudaStreamSynchronize(s), "mf_apply_host sync");
}

static std::mutex g_tune_mu;
// (device, n, path, kind, view, size class) -> variant
static std::map<std::tuple<int, int, int, int, int, int>, int> g_tune_cache;
// Size class of an operator for the autotuner: floor(log2(cells)).  The best launch shape
// depends on how many waves of CTAs the mesh makes, so a choice timed on a small mesh is not
// reused for a large one.
static int tune_size_class(const mf_operator* op) {
  const long long cells = (long long)op->g.nx * op->g.ny * op->g.nz;
  int c = 0;
  while (c < 62 && (2LL << c) <= cells) ++c;
  return c;
}

// The autotuner's choices persist across processes in a JSON object of "key": variant
// entries, one per line, with key "<GPU name>|lib=2|n=<n>|path=<p>|kind=<k>|view=<v>".  The
// file is MF_AUTOTUNE_CACHE if set ("off" disables it), else $XDG_CACHE_HOME/libmf/
// autotune.json or $HOME/.cache/libmf/autotune.json.  It is read once per process (entries of
// other GPUs are kept and written back) and rewritten through a temporary file after each new
// choice; a missing or unreadable file only means the variants are timed again.
static std::map<std::string, int> g_tune_file;
static bool g_tune_file_loaded = false;

static std::string tune_file_path() {
  const char* e = std::getenv("MF_AUTOTUNE_CACHE");
  if (e && *e) return std::strcmp(e, "off") == 0 ? std::string() : std::string(e);
  const char* x = std::getenv("XDG_CACHE_HOME");
  if (x && *x) return std::string(x) + "/libmf/autotune.json";
  const char* h = std::getenv("HOME");
  if (h && *h) return std::string(h) + "/.cache/libmf/autotune.json";
  return std::string();
}

static void tune_file_load(const std::string& path) {
  g_tune_file_loaded = true;
  if (path.empty()) return;
  FILE* f = std::fopen(path.c_str(), "r");
  if (!f) return;
  char line[1024];
  while (std::fgets(line, sizeof(line), f)) {
    const char* q0 = std::strchr(line, '"');
    if (!q0) continue;
    const char* q1 = std::strchr(q0 + 1, '"');
    if (!q1) continue;
    const char* colon = std::strchr(q1, ':');
    if (!colon) continue;
    int v = -1;
    if (std::sscanf(colon + 1, " %d", &v) == 1 && v >= 0 && v <= MF_VARIANT_OCCUPANCY)
      g_tune_file[std::string(q0 + 1, q1)] = v;
  }
  std::fclose(f);
}

static void tune_file_store(const std::string& path) {
  if (path.empty()) return;
  const std::string dir = path.substr(0, path.find_last_of('/'));
  if (!dir.empty() && dir != path) {
    // create the directory chain (best effort)
    for (size_t i = 1; i <= dir.size(); ++i)
      if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
  }
  const std::string tmp = path + "." + std::to_string((long long)getpid()) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "{\n");
  size_t i = 0;
  for (const auto& kv : g_tune_file) {
    std::string k;
    for (char ch : kv.first) k += (ch == '"' || ch == '\\') ? '_' : ch;
    std::fprintf(f, "  \"%s\": %d%s\n", k.c_str(), kv.second, ++i < g_tune_file.size() ? "," : "");
  }
  std::fprintf(f, "}\n");
  const bool ok = std::fclose(f) == 0;
  if (ok) std::rename(tmp.c_str(), path.c_str());
  else std::remove(tmp.c_str());
}

static std::string tune_key(int dev, const mf_operator* op, int vk) {
  cudaDeviceProp prop;
  std::string name = "unknown";
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
  char buf[160];
  std::snprintf(buf, sizeof(buf), "|lib=4|n=%d|path=%d|kind=%d|view=%d|cells=2^%d", op->n, op->path, op->kind, vk,
                tune_size_class(op));
  return name + buf;
}

mf_status mf_operator_autotune(mf_operator* op, const void* x_dev, void* y_dev, int reps, void* stream) {
  mf_status st = check_ready(op, "mf_operator_autotune");
  if (st) return st;
  if (!x_dev || !y_dev || x_dev == y_dev) return set_error(MF_ERR_ARG, "mf_operator_autotune: bad vectors");
  if (reps < 1) reps = 3;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  if ((st = cuda_check(cudaGetDevice(&dev), "cudaGetDevice"))) return st;
  const int vk = view_of_elem(op, elem_of(op));
  const auto key = std::make_tuple(dev, op->n, op->path, op->kind, vk, tune_size_class(op));
  const std::string fkey = tune_key(dev, op, vk);
  const std::string fpath = tune_file_path();
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      op->variant[vk] = it->second;
      return MF_OK;
    }
    if (!g_tune_file_loaded) tune_file_load(fpath);
    auto ft = g_tune_file.find(fkey);
    // a stored choice is used if it is valid for this operator (the tensor-core variant only
    // where it is built, the small-CTA one on the double-float view)
    if (ft != g_tune_file.end() &&
        (ft->second < MF_VARIANT_TENSOR || (ft->second == MF_VARIANT_TENSOR && vk == VK_DD && tc_eligible(op)) ||
         ((ft->second == MF_VARIANT_SMALL_CTA || ft->second == MF_VARIANT_OCCUPANCY) && vk == VK_DD))) {
      op->variant[vk] = ft->second;
      g_tune_cache[key] = ft->second;
      return MF_OK;
    }
  }
  cudaEvent_t e0, e1;
  if ((st = cuda_check(cudaEventCreate(&e0), "event"))) return st;
  if ((st = cuda_check(cudaEventCreate(&e1), "event"))) { cudaEventDestroy(e0); return st; }
  float best = 1e30f;
  int best_v = 0;
  // candidates: 0-2 everywhere, the small-CTA and occupancy variants on the double-float
  // view, the tensor-core apply where it is built
  int cand[6], nvar = 0;
  for (int v = 0; v < 3; ++v) cand[nvar++] = v;
  if (vk == VK_DD) {
    cand[nvar++] = MF_VARIANT_SMALL_CTA;
    cand[nvar++] = MF_VARIANT_OCCUPANCY;
  }
  if (vk == VK_DD && tc_eligible(op)) cand[nvar++] = MF_VARIANT_TENSOR;
  for (int ci = 0; ci < nvar && st == MF_OK; ++ci) {
    const int v = cand[ci];
    op->variant[vk] = v;
    st = launch_apply_split(op, vk, x_dev, y_dev, s); // warm-up
    if (st) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && st == MF_OK; ++r) st = launch_apply_split(op, vk, x_dev, y_dev, s);
    cudaEventRecord(e1, s);
    if (st) break;
    if ((st = cuda_check(cudaEventSynchronize(e1), "autotune sync"))) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; best_v = v; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  op->variant[vk] = best_v;
  if (st) return st;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = best_v;
  g_tune_file[fkey] = best_v;
  tune_file_store(fpath);
  return MF_OK;
}

mf_status mf_operator_set_variant(mf_operator* op, int variant) {
  if (!op || variant < 0 || variant > MF_VARIANT_OCCUPANCY)
    return set_error(MF_ERR_ARG, "mf_operator_set_variant: bad argument");
  if (variant == MF_VARIANT_SMALL_CTA || variant == MF_VARIANT_OCCUPANCY) {
    if (view_of_elem(op, elem_of(op)) != VK_DD)
      return set_error(MF_ERR_UNSUPPORTED, "mf_operator_set_variant: variants 4 and 5 cover the double-float "
                                           "view of MF_FP64 operators");
    op->variant[VK_DD] = variant;
    return MF_OK;
  }
  if (variant == MF_VARIANT_TENSOR) {
    if (!tc_eligible(op))
      return set_error(MF_ERR_UNSUPPORTED, "mf_operator_set_variant: the tensor-core apply covers FP64 Cartesian "
                                           "operators of degree 1..3");
    op->variant[VK_DD] = MF_VARIANT_TENSOR;
    return MF_OK;
  }
  op->variant[VK_F64] = op->variant[VK_DD] = op->variant[VK_F32] = variant;
  return MF_OK;
}

int mf_device_error(int reset) { return tc_read_error(reset); }

int mf_operator_get_variant(const mf_operator* op) {
  return op ? op->variant[view_of_elem(op, elem_of(op))] : -1;
}

} // extern "C"
