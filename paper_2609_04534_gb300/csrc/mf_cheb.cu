// mf_cheb.cu -- CG preconditioned by the degree-3 Chebyshev-accelerated point Jacobi method
// (mf_solve_options.precond = MF_PRECOND_CHEBYSHEV).
//
// The preconditioner is the paper's smoother (Sec. 5.2) with the point-Jacobi diagonal D of the
// assembled operator P A P as its block: for a target interval [a, b] of the spectrum of
// D^-1 A, with c = (a + b) / 2, d = (b - a) / 2 and the weights of Eq. (chebyshev_weights),
//   w_j = 1 / (c - d cos((2j - 1) pi / 6)),  j = 1, 2, 3,
// z = M^-1 r is three Richardson updates from z = 0 in the factorised form of
// Eq. (chebyshev_richardson),
//   z <- z + w_j D^-1 (r - A z),
// whose error polynomial p_3(l) = prod_j (1 - w_j l) is the scaled Chebyshev polynomial
// T_3((c - l) / d) / T_3(c / d) of Eq. (chebyshev_error_polynomial).  M^-1 = q(D^-1 A) D^-1
// with q(l) = (1 - p_3(l)) / l > 0 for l > 0, so M is symmetric positive definite and CG with
// it is well defined.  The first stage needs no apply (z = 0): two applies per preconditioner,
// three per CG iteration.
//
// b is 1.1 times a power-iteration estimate of the largest eigenvalue of D^-1 A (12 applies
// from the masked right-hand side); a = b / ratio (mf_solve_options.cheb_ratio, default 30).
// The iteration is the textbook preconditioned CG on assembled (consistent) vectors of the
// operator's element type: every apply is the local apply plus the duplicate summation, the
// dots are the assembled products of Sec. 4, alpha and beta are formed on the device, and the
// host reads <r, r> every 10 iterations for the convergence test.
#include <cmath>
#include <cstring>

#include "mf_kernels.cuh"

namespace mf {
namespace {

constexpr int CHEB_CHECK = 10; // iterations between host convergence checks
constexpr int CHEB_POWER = 12; // power iterations for the largest eigenvalue of D^-1 A

// device scalars of the solve
struct ChebScal {
  double rz, rz_old, pq, rr, alpha, beta, bb, nrm;
};

unsigned cheb_blocks(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

// r = P b (zero on the cube boundary with Dirichlet, and on padding lanes); x = 0; p = 0
template <typename T, int N>
__global__ void cheb_init_kernel(const T* __restrict__ b, T* __restrict__ r, T* __restrict__ x, T* __restrict__ p,
                                 long long n, GridInfo g) {
  constexpr int N2 = N * N, N3 = N2 * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int lane = (int)(e & (BL - 1));
    const int l = (int)((e >> 5) % N3);
    const long long t = (e >> 5) / N3;
    int cx, cy, cz;
    cell_of(g, t, lane, cx, cy, cz);
    const bool valid = cx < g.nx && cy < g.ny && cz < g.nz;
    const bool bnd = g.bc && on_cube_boundary<N>(g, cx, cy, cz, l % N, (l / N) % N, l / N2);
    r[e] = (valid && !bnd) ? b[e] : T(0);
    x[e] = T(0);
    p[e] = T(0);
  }
}

// dinv = 1 / diag where diag > 0 (0 on Dirichlet nodes and padding)
__global__ void cheb_dinv_kernel(float* __restrict__ d, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float v = d[e];
    d[e] = v > 0.0f ? 1.0f / v : 0.0f;
  }
}

// z = w D^-1 r (first stage, z = 0 before) or z = z + w D^-1 (r - t)
template <typename T>
__global__ void cheb_stage_kernel(T* __restrict__ z, const T* __restrict__ r, const T* __restrict__ t,
                                  const float* __restrict__ dinv, double w, long long n, int first) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const T dw = (T)(w * (double)dinv[e]);
    z[e] = first ? dw * r[e] : z[e] + dw * (r[e] - t[e]);
  }
}

// power iteration: v = D^-1 (A v) in place of the applied vector
template <typename T>
__global__ void cheb_scale_kernel(T* __restrict__ v, const float* __restrict__ dinv, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    v[e] = v[e] * (T)dinv[e];
}
// v = w / sqrt(<w, w>) (norm from the device scalars)
template <typename T>
__global__ void cheb_normalize_kernel(T* __restrict__ v, const T* __restrict__ w, const ChebScal* sc, long long n) {
  const double nv = sc->nrm;
  const T s = (T)(nv > 0.0 && isfinite(nv) ? 1.0 / sqrt(nv) : 0.0);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    v[e] = w[e] * s;
}

// beta = <r, z> / <r, z>_old (0 at the first iteration)
__global__ void cheb_beta_kernel(ChebScal* sc, int first) {
  sc->beta = first ? 0.0 : sc->rz / sc->rz_old;
  sc->rz_old = sc->rz;
}
// alpha = <r, z> / <p, A p>
__global__ void cheb_alpha_kernel(ChebScal* sc) { sc->alpha = sc->pq > 0.0 ? sc->rz / sc->pq : 0.0; }

// p = z + beta p
template <typename T>
__global__ void cheb_p_kernel(T* __restrict__ p, const T* __restrict__ z, const ChebScal* sc, long long n) {
  const T be = (T)sc->beta;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    p[e] = z[e] + be * p[e];
}
// x += alpha p ; r -= alpha q
template <typename T>
__global__ void cheb_xr_kernel(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ q,
                               const ChebScal* sc, long long n) {
  const T al = (T)sc->alpha;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    x[e] = x[e] + al * p[e];
    r[e] = r[e] - al * q[e];
  }
}

size_t a256(size_t b) { return (b + 255) & ~size_t(255); }

struct ChebWs {
  ChebScal* sc;
  void* red;
  float *dinv, *dtab;
  void *r, *p, *q, *z, *t;
};
size_t cheb_layout(const mf_operator* op, char* base, ChebWs* w) {
  const size_t n = (size_t)op->n_native, e = op->precision == MF_FP32 ? 4 : 8;
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* { char* p = base ? base + off : nullptr; off += a256(bytes); return p; };
  ChebWs t;
  t.sc = (ChebScal*)take(sizeof(ChebScal));
  t.red = take(reduce_scratch_bytes());
  t.dinv = (float*)take(sizeof(float) * n);
  t.dtab = (float*)take(diag_table_bytes(op));
  t.r = take(n * e);
  t.p = take(n * e);
  t.q = take(n * e);
  t.z = take(n * e);
  t.t = take(n * e);
  if (w) *w = t;
  return off;
}

template <int N>
mf_status cheb_init_n(const mf_operator* op, int elem, const void* b, void* r, void* x, void* p, cudaStream_t s) {
  const long long n = op->n_native;
  if (elem == 8)
    cheb_init_kernel<double, N><<<cheb_blocks(n), 256, 0, s>>>((const double*)b, (double*)r, (double*)x, (double*)p, n,
                                                               op->g);
  else
    cheb_init_kernel<float, N><<<cheb_blocks(n), 256, 0, s>>>((const float*)b, (float*)r, (float*)x, (float*)p, n,
                                                              op->g);
  return cuda_check(cudaGetLastError(), "chebyshev init");
}
mf_status cheb_init(const mf_operator* op, int elem, const void* b, void* r, void* x, void* p, cudaStream_t s) {
  switch (op->n) {
    case 2: return cheb_init_n<2>(op, elem, b, r, x, p, s);
    case 3: return cheb_init_n<3>(op, elem, b, r, x, p, s);
    case 4: return cheb_init_n<4>(op, elem, b, r, x, p, s);
    case 5: return cheb_init_n<5>(op, elem, b, r, x, p, s);
    case 6: return cheb_init_n<6>(op, elem, b, r, x, p, s);
    case 7: return cheb_init_n<7>(op, elem, b, r, x, p, s);
    case 8: return cheb_init_n<8>(op, elem, b, r, x, p, s);
    case 9: return cheb_init_n<9>(op, elem, b, r, x, p, s);
    default: return set_error(MF_ERR_UNSUPPORTED, "n=%d not built", op->n);
  }
}

// the assembled operator: local apply and duplicate summation (P A P with Dirichlet)
mf_status cheb_apply(const mf_operator* op, int elem, const void* x, void* y, cudaStream_t s) {
  mf_status st = launch_apply_split(op, view_of_elem(op, elem), x, y, s);
  if (st) return st;
  return launch_dss(op, elem, y, s);
}

template <typename T>
mf_status cheb_solve_t(const mf_operator* op, const void* b, void* x, double rtol, int maxit, double ratio,
                       mf_solve_stats* stats, const ChebWs& w, cudaStream_t s) {
  const long long n = op->n_native;
  const int elem = sizeof(T);
  const unsigned nb = cheb_blocks(n);
  mf_status st;
  T *r = (T*)w.r, *p = (T*)w.p, *q = (T*)w.q, *z = (T*)w.z, *t = (T*)w.t, *xx = (T*)x;
  ChebScal* sc = w.sc;
  auto dot = [&](const T* a, const T* bb, double* out) { return dot_launch(op, elem, a, bb, 0, out, w.red, s); };
  if ((st = cuda_check(cudaMemsetAsync(w.red, 0, 256, s), "chebyshev scratch"))) return st;
  if ((st = cheb_init(op, elem, b, r, x, p, s))) return st;
  // D^-1 of the assembled diagonal (FP32, consistent, 0 on Dirichlet nodes)
  if ((st = launch_diagonal(op, w.dinv, w.dtab, s))) return st;
  cheb_dinv_kernel<<<nb, 256, 0, s>>>(w.dinv, n);
  if ((st = dot(r, r, &sc->bb))) return st;
  // largest eigenvalue of D^-1 A by power iteration from the normalised right-hand side
  if ((st = dot(r, r, &sc->nrm))) return st;
  cheb_normalize_kernel<T><<<nb, 256, 0, s>>>(z, r, sc, n);
  for (int i = 0; i < CHEB_POWER; ++i) {
    if ((st = cheb_apply(op, elem, z, t, s))) return st;
    cheb_scale_kernel<T><<<nb, 256, 0, s>>>(t, w.dinv, n);
    if ((st = dot(t, t, &sc->nrm))) return st;
    if (i + 1 < CHEB_POWER) cheb_normalize_kernel<T><<<nb, 256, 0, s>>>(z, t, sc, n);
  }
  ChebScal h;
  if ((st = cuda_check(cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, s), "chebyshev D2H"))) return st;
  if ((st = cuda_check(cudaStreamSynchronize(s), "chebyshev sync"))) return st;
  const double bnorm2 = h.bb;
  stats->iterations = 0;
  stats->outer_iterations = 0;
  stats->rel_residual = 0.0;
  stats->status = MF_OK;
  stats->check_every = CHEB_CHECK;
  if (!(bnorm2 > 0.0) || !std::isfinite(bnorm2)) {
    stats->status = std::isfinite(bnorm2) ? MF_OK : MF_ERR_BREAKDOWN;
    return stats->status;
  }
  const double lmax = std::sqrt(h.nrm); // ||D^-1 A v|| for the normalised iterate v
  if (!(lmax > 0.0) || !std::isfinite(lmax)) return set_error(MF_ERR_BREAKDOWN, "chebyshev: eigenvalue estimate");
  const double bb = 1.1 * lmax, aa = bb / ratio, c = 0.5 * (aa + bb), d = 0.5 * (bb - aa);
  double wj[3];
  for (int j = 1; j <= 3; ++j) wj[j - 1] = 1.0 / (c - d * std::cos((2 * j - 1) * M_PI / 6.0));
  const double tol2 = rtol * rtol * bnorm2;
  int it = 0;
  for (; it < maxit;) {
    // z = M^-1 r: three Richardson stages from z = 0 (Eq. (chebyshev_richardson))
    cheb_stage_kernel<T><<<nb, 256, 0, s>>>(z, r, nullptr, w.dinv, wj[0], n, 1);
    for (int j = 1; j < 3; ++j) {
      if ((st = cheb_apply(op, elem, z, t, s))) return st;
      cheb_stage_kernel<T><<<nb, 256, 0, s>>>(z, r, t, w.dinv, wj[j], n, 0);
    }
    if ((st = dot(r, z, &sc->rz))) return st;
    cheb_beta_kernel<<<1, 1, 0, s>>>(sc, it == 0);
    cheb_p_kernel<T><<<nb, 256, 0, s>>>(p, z, sc, n);
    if ((st = cheb_apply(op, elem, p, q, s))) return st;
    if ((st = dot(p, q, &sc->pq))) return st;
    cheb_alpha_kernel<<<1, 1, 0, s>>>(sc);
    cheb_xr_kernel<T><<<nb, 256, 0, s>>>(xx, r, p, q, sc, n);
    if ((st = dot(r, r, &sc->rr))) return st;
    ++it;
    if (it % CHEB_CHECK == 0 || it == maxit) {
      if ((st = cuda_check(cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, s), "chebyshev D2H"))) return st;
      if ((st = cuda_check(cudaStreamSynchronize(s), "chebyshev sync"))) return st;
      if (!std::isfinite(h.rr) || !(h.pq > 0.0)) {
        stats->iterations = it;
        stats->rel_residual = std::sqrt(h.rr / bnorm2);
        stats->status = MF_ERR_BREAKDOWN;
        return MF_ERR_BREAKDOWN;
      }
      if (h.rr <= tol2) break;
    }
  }
  if ((st = cuda_check(cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, s), "chebyshev D2H"))) return st;
  if ((st = cuda_check(cudaStreamSynchronize(s), "chebyshev sync"))) return st;
  stats->iterations = it;
  stats->rel_residual = std::sqrt(h.rr / bnorm2);
  stats->status = h.rr <= tol2 ? MF_OK : MF_ERR_NOT_CONVERGED;
  return stats->status;
}

} // namespace

size_t cheb_workspace_bytes(const mf_operator* op) { return cheb_layout(op, nullptr, nullptr); }

mf_status cheb_solve(const mf_operator* op, const void* b, void* x, double rtol, int maxit, double ratio,
                     mf_solve_stats* stats, void* ws, size_t bytes, cudaStream_t s) {
  if (op->precision == MF_MIXED) return set_error(MF_ERR_UNSUPPORTED, "chebyshev: MF_FP64 or MF_FP32 operators");
  if (bytes < cheb_workspace_bytes(op)) return set_error(MF_ERR_OOM, "chebyshev: workspace %zu < %zu", bytes,
                                                         cheb_workspace_bytes(op));
  if (!(ratio > 1.0)) ratio = 30.0;
  ChebWs w;
  cheb_layout(op, static_cast<char*>(ws), &w);
  if (op->precision == MF_FP32) return cheb_solve_t<float>(op, b, x, rtol, maxit, ratio, stats, w, s);
  return cheb_solve_t<double>(op, b, x, rtol, maxit, ratio, stats, w, s);
}

} // namespace mf
