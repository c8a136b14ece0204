// mf_rhs.cu -- manufactured-solution workload on the device: right-hand side b_i = int f phi_i
// and the L2 error of a discrete solution, for u = prod_d sin(freq pi x_d) on the unit cube
// (the model problem of Sec. 2, with the manufactured solution of Sec. 6.1 at a chosen
// frequency), f = -Lap u + c_m u = (3 freq^2 pi^2 + c_m) u.
//
// Both use the operator's (k+1)-point Gauss rule and the sum factorisation of the apply
// (S^T sweeps for b, S sweeps for u_h).  Point values are evaluated in double-float:
//  - per direction, sin/cos(pi xh) and sin/cos(freq pi x) at the Gauss points of every cell
//    layer are tabulated once in FP64 into the caller's scratch;
//  - Cartesian map: u at a point is a product of three table entries;
//  - curved map x_d = xh_d + amp s(xh): sin(freq pi x_d) = sin(a) cos(th) + cos(a) sin(th) with
//    a = freq pi xh_d tabulated and th = freq pi amp s(xh) (|th| <= freq pi |amp|) from a dd
//    Taylor series; |det J| = h^3 |1 + amp (ds/dxh_1 + ds/dxh_2 + ds/dxh_3)| (rank-one update).
// b is written as local integrals and made consistent (and masked) by the duplicate summation.
#include <cmath>

#include "mf_dd.cuh"
#include "mf_internal.h"

namespace mf {
namespace {

constexpr int TAYLOR = 13; // terms of the sin / cos series: |th| <= 2 gives error < 1e-17

struct Series {
  dd s[TAYLOR], c[TAYLOR]; // (-1)^m/(2m+1)!, (-1)^m/(2m)!
};

template <typename T, int N>
struct RhsArgs {
  GridInfo g;
  int curved;
  double amp, coef, freq;
  double scale[3], shift[3]; // Cartesian affine: x_d = scale_d xh_d + shift_d
  double qx[MAXN], qw[MAXN];
  dd S[N * N];
  Series ser;
  const dd* tab;             // [(nx+ny+nz) * N][4]
  const T* u;                // error mode: discrete solution (native layout)
  T* b;                      // rhs mode: output (native layout, split)
  struct RedPart* red;
  double* out;
};

struct RedPart {
  unsigned int counter;
  unsigned int pad[63];
  double partial[65536];
};

__device__ __forceinline__ dd ddv(double v) { return dd_from_double(v); }
__device__ __forceinline__ dd dd_abs(dd a) { return a.hi < 0.0f ? dd(-a.hi, -a.lo) : a; }

template <int N>
__global__ void rhs_tables_kernel(dd* tab, GridInfo g, double freq, int curved, double3 scale, double3 shift,
                                  RhsArgs<double, N> qa) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int total = (g.nx + g.ny + g.nz) * N;
  if (e >= total) return;
  const int r = e / N, q = e - r * N;
  int d, c;
  if (r < g.nx) { d = 0; c = r; }
  else if (r < g.nx + g.ny) { d = 1; c = r - g.nx; }
  else { d = 2; c = r - g.nx - g.ny; }
  const int nd = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
  const double xh = (c + qa.qx[q]) / nd;
  double sp, cp, sf, cf;
  sincospi(xh, &sp, &cp);
  const double sc = d == 0 ? scale.x : (d == 1 ? scale.y : scale.z);
  const double sh = d == 0 ? shift.x : (d == 1 ? shift.y : shift.z);
  const double xd = curved ? xh : sc * xh + sh;
  sincospi(freq * xd, &sf, &cf);
  const double v[4] = {sp, cp, sf, cf};
  for (int m = 0; m < 4; ++m) {
    const float h = __double2float_rn(v[m]);
    tab[4 * (size_t)e + m] = dd(h, __double2float_rn(v[m] - (double)h));
  }
}

__device__ __forceinline__ void dd_sincos_small(dd t, const Series& ser, dd& sv, dd& cv) {
  const dd t2 = t * t;
  dd ps = ser.s[TAYLOR - 1], pc = ser.c[TAYLOR - 1];
#pragma unroll
  for (int m = TAYLOR - 2; m >= 0; --m) {
    ps = finish(fma(ps, t2, ser.s[m]));
    pc = finish(fma(pc, t2, ser.c[m]));
  }
  sv = ps * t;
  cv = pc;
}

// u(x_q) and w_q |det J_q| at Gauss point (i, j, k) of cell (cx, cy, cz).
template <typename T, int N>
__device__ __forceinline__ dd point_u(const RhsArgs<T, N>& a, int cx, int cy, int cz, int i, int j, int k, dd* wdet) {
  const dd* tx = a.tab + 4 * (size_t)(cx * N + i);
  const dd* ty = a.tab + 4 * (size_t)((a.g.nx + cy) * N + j);
  const dd* tz = a.tab + 4 * (size_t)((a.g.nx + a.g.ny + cz) * N + k);
  const double hx = 1.0 / a.g.nx, hy = 1.0 / a.g.ny, hz = 1.0 / a.g.nz;
  const double w = a.qw[i] * a.qw[j] * a.qw[k];
  if (!a.curved) {
    *wdet = ddv(w * fabs(a.scale[0] * a.scale[1] * a.scale[2]) * hx * hy * hz);
    return (tx[2] * ty[2]) * tz[2];
  }
  const dd pi = dd(3.14159274101257324f, -8.74227766e-08f);
  const dd sxy = tx[0] * ty[0];
  const dd s = sxy * tz[0];
  const dd g1 = ((pi * tx[1]) * ty[0]) * tz[0];
  const dd g2 = ((pi * tx[0]) * ty[1]) * tz[0];
  const dd g3 = (pi * sxy) * tz[1];
  const dd amp = ddv(a.amp);
  const dd jac = finish(fma(amp, (g1 + g2) + g3, dd(1)));
  *wdet = ddv(w * hx * hy * hz) * dd_abs(jac);
  const dd th = (ddv(a.freq) * pi) * (amp * s);
  dd st, ct;
  dd_sincos_small(th, a.ser, st, ct);
  const dd ux = finish(fma(tx[2], ct, tx[3] * st));
  const dd uy = finish(fma(ty[2], ct, ty[3] * st));
  const dd uz = finish(fma(tz[2], ct, tz[3] * st));
  return (ux * uy) * uz;
}

template <int N>
struct RCfg {
  static constexpr int CB = (N <= 4) ? 32 : (N <= 6) ? 16 : 8;
  static constexpr int NT = N * N * CB;
};

// b_K = (S^T (x) S^T (x) S^T) (w |det J| f) per cell, written split (before the DSS).
template <typename T, int N>
__global__ void __launch_bounds__(RCfg<N>::NT) rhs_kernel(RhsArgs<T, N> a) {
  constexpr int CB = RCfg<N>::CB, N2 = N * N, N3 = N2 * N, GPT = BL / CB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dd* buf = reinterpret_cast<dd*>(smem_raw);
  const int t = (int)(blockIdx.x / GPT);
  const int lane0 = (blockIdx.x % GPT) * CB;
  const int c = threadIdx.x % CB, p = threadIdx.x / CB, pa = p % N, pb = p / N;
  const int lane = lane0 + c;
  const int txy = a.g.ntx * a.g.nty, tz = t / txy, rr = t - tz * txy, ty = rr / a.g.ntx, tx = rr - ty * a.g.ntx;
  const int cx = tx * TX + (lane & 3), cy = ty * TY + ((lane >> 2) & 3), cz = tz * TZ + (lane >> 4);
  const bool valid = cx < a.g.nx && cy < a.g.ny && cz < a.g.nz;
  dd v[N];
  const dd coef = ddv(a.coef);
#pragma unroll
  for (int q = 0; q < N; ++q) {
    if (valid) {
      dd wd;
      const dd u = point_u<T, N>(a, cx, cy, cz, pa, pb, q, &wd);
      v[q] = (coef * u) * wd;
    } else {
      v[q] = dd(0);
    }
  }
#pragma unroll
  for (int kk = 0; kk < N; ++kk) { // S^T along z, pencil (i=pa, j=pb)
    dd s = dd(0);
#pragma unroll
    for (int q = 0; q < N; ++q) s = fma(a.S[q * N + kk], v[q], s);
    buf[(pa + N * pb + N2 * kk) * CB + c] = finish(s);
  }
  __syncthreads();
  { // S^T along y, pencil (i=pa, k=pb)
    dd in[N];
#pragma unroll
    for (int q = 0; q < N; ++q) in[q] = buf[(pa + N * q + N2 * pb) * CB + c];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      dd s = dd(0);
#pragma unroll
      for (int q = 0; q < N; ++q) s = fma(a.S[q * N + j], in[q], s);
      buf[(pa + N * j + N2 * pb) * CB + c] = finish(s);
    }
  }
  __syncthreads();
  { // S^T along x, pencil (j=pa, k=pb) -> global
    dd in[N];
#pragma unroll
    for (int q = 0; q < N; ++q) in[q] = buf[(q + N * pa + N2 * pb) * CB + c];
    const long long base = (long long)t * N3 * BL + lane;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      dd s = dd(0);
#pragma unroll
      for (int q = 0; q < N; ++q) s = fma(a.S[q * N + i], in[q], s);
      s = finish(s);
      a.b[base + (long long)(i + N * pa + N2 * pb) * BL] = valid ? (T)dd_to_double(s) : T(0);
    }
  }
}

// Fixed-order block sum valid for any block size (CTAs of n^2 * CB threads need not be a
// multiple of 32): every thread parks its value in shared memory, warp 0 folds the array
// with a stride of 32 and finishes with shuffles.  Result valid in thread 0.
__device__ __forceinline__ double block_sum_d(double v, int nthreads) {
  __shared__ double park[1024];
  park[threadIdx.x] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    for (int i = threadIdx.x; i < nthreads; i += 32) s += park[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  __syncthreads();
  return s;
}

// sum over cells and Gauss points of w |det J| (u - u_h)^2; u_h by S sweeps of the cell values.
template <typename T, int N>
__global__ void __launch_bounds__(RCfg<N>::NT) err_kernel(RhsArgs<T, N> a) {
  constexpr int CB = RCfg<N>::CB, NT = RCfg<N>::NT, N2 = N * N, N3 = N2 * N, GPT = BL / CB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dd* buf = reinterpret_cast<dd*>(smem_raw);
  const int t = (int)(blockIdx.x / GPT);
  const int lane0 = (blockIdx.x % GPT) * CB;
  const long long base = (long long)t * N3 * BL + lane0;
  for (int idx = threadIdx.x; idx < N3 * CB; idx += NT) {
    const int l = idx / CB, cc = idx - l * CB;
    buf[idx] = to_compute<dd, double>((double)a.u[base + (long long)l * BL + cc]);
  }
  __syncthreads();
  const int c = threadIdx.x % CB, p = threadIdx.x / CB, pa = p % N, pb = p / N;
  const int lane = lane0 + c;
  const int txy = a.g.ntx * a.g.nty, tz = t / txy, rr = t - tz * txy, ty = rr / a.g.ntx, tx = rr - ty * a.g.ntx;
  const int cx = tx * TX + (lane & 3), cy = ty * TY + ((lane >> 2) & 3), cz = tz * TZ + (lane >> 4);
  const bool valid = cx < a.g.nx && cy < a.g.ny && cz < a.g.nz;
  { // x sweep, pencil (j=pa, k=pb)
    dd in[N];
#pragma unroll
    for (int i = 0; i < N; ++i) in[i] = buf[(i + N * pa + N2 * pb) * CB + c];
#pragma unroll
    for (int q = 0; q < N; ++q) {
      dd s = dd(0);
#pragma unroll
      for (int i = 0; i < N; ++i) s = fma(a.S[q * N + i], in[i], s);
      buf[(q + N * pa + N2 * pb) * CB + c] = finish(s);
    }
  }
  __syncthreads();
  { // y sweep, pencil (i=pa, k=pb)
    dd in[N];
#pragma unroll
    for (int j = 0; j < N; ++j) in[j] = buf[(pa + N * j + N2 * pb) * CB + c];
#pragma unroll
    for (int q = 0; q < N; ++q) {
      dd s = dd(0);
#pragma unroll
      for (int j = 0; j < N; ++j) s = fma(a.S[q * N + j], in[j], s);
      buf[(pa + N * q + N2 * pb) * CB + c] = finish(s);
    }
  }
  __syncthreads();
  double acc = 0.0;
  { // z sweep in registers, then the point errors
    dd in[N];
#pragma unroll
    for (int k = 0; k < N; ++k) in[k] = buf[(pa + N * pb + N2 * k) * CB + c];
#pragma unroll
    for (int q = 0; q < N; ++q) {
      dd s = dd(0);
#pragma unroll
      for (int k = 0; k < N; ++k) s = fma(a.S[q * N + k], in[k], s);
      if (valid) {
        dd wd;
        const dd u = point_u<T, N>(a, cx, cy, cz, pa, pb, q, &wd);
        const dd e = finish(fma(dd(-1), finish(s), u));
        acc += dd_to_double((e * e) * wd);
      }
    }
  }
  acc = block_sum_d(acc, NT);
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    a.red->partial[blockIdx.x] = acc;
    __threadfence();
    am_last = (atomicAdd(&a.red->counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  double tot = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += NT) tot += ((volatile double*)a.red->partial)[b];
  tot = block_sum_d(tot, NT);
  if (threadIdx.x == 0) {
    *a.out = tot;
    a.red->counter = 0;
  }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

size_t table_bytes(const mf_operator* op) {
  return align256(sizeof(dd) * 4 * (size_t)(op->g.nx + op->g.ny + op->g.nz) * op->n);
}

template <typename T, int N>
mf_status fill(const mf_operator* op, double freq, RhsArgs<T, N>& a, dd* tab) {
  if (op->path == PATH_AFFINE) return set_error(MF_ERR_UNSUPPORTED, "manufactured solution: sheared affine maps not supported");
  a.g = op->g;
  a.curved = op->path == PATH_CURVED;
  a.amp = op->mesh.amp;
  a.freq = freq;
  a.coef = 3.0 * freq * freq * M_PI * M_PI + (op->kind == MF_HELMHOLTZ ? op->mass : 0.0);
  for (int d = 0; d < 3; ++d) { a.scale[d] = op->mesh.A[4 * d]; a.shift[d] = op->mesh.b[d]; }
  for (int q = 0; q < N; ++q) {
    a.qx[q] = op->tab.qx[q];
    a.qw[q] = op->tab.qw[q];
    for (int i = 0; i < N; ++i) a.S[q * N + i] = host_from_double<dd>(op->tab.S[q * MAXN + i]);
  }
  long double fs = 1.0L, fc = 1.0L; // (2m+1)!, (2m)!
  for (int m = 0; m < TAYLOR; ++m) {
    if (m > 0) { fc = fs * (2 * m); fs = fc * (2 * m + 1); }
    const double cs = (double)(((m & 1) ? -1.0L : 1.0L) / fs);
    const double cc = (double)(((m & 1) ? -1.0L : 1.0L) / fc);
    a.ser.s[m] = host_from_double<dd>(cs);
    a.ser.c[m] = host_from_double<dd>(cc);
  }
  if (a.curved && std::fabs(freq * M_PI * op->mesh.amp) > 2.0)
    return set_error(MF_ERR_UNSUPPORTED, "manufactured solution: freq*pi*amp beyond the series range");
  a.tab = tab;
  return MF_OK;
}

template <typename T, int N>
mf_status tables(const mf_operator* op, const RhsArgs<T, N>& a, dd* tab, cudaStream_t s) {
  RhsArgs<double, N> qa;
  for (int q = 0; q < N; ++q) qa.qx[q] = a.qx[q];
  const int total = (op->g.nx + op->g.ny + op->g.nz) * N;
  rhs_tables_kernel<N><<<(total + 127) / 128, 128, 0, s>>>(tab, op->g, a.freq, a.curved,
                                                           make_double3(a.scale[0], a.scale[1], a.scale[2]),
                                                           make_double3(a.shift[0], a.shift[1], a.shift[2]), qa);
  return cuda_check(cudaGetLastError(), "manufactured tables launch");
}

// static shared memory of the RHS / error kernels (the 1024-double reduction park and a
// flag): static + dynamic above 48 KB needs the opt-in
constexpr size_t STATIC_SMEM_ALLOWANCE = 1024 * sizeof(double) + 256;

template <typename T, int N>
mf_status rhs_t(const mf_operator* op, double freq, void* b, char* scratch, cudaStream_t s) {
  RhsArgs<T, N> a;
  dd* tab = reinterpret_cast<dd*>(scratch);
  mf_status st = fill<T, N>(op, freq, a, tab);
  if (st) return st;
  if ((st = tables<T, N>(op, a, tab, s))) return st;
  a.b = static_cast<T*>(b);
  const size_t smem = sizeof(dd) * N * N * N * RCfg<N>::CB;
  if (smem + STATIC_SMEM_ALLOWANCE > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(rhs_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(e, "rhs attribute");
  }
  const long long blocks = op->g.ntiles * (BL / RCfg<N>::CB);
  rhs_kernel<T, N><<<(unsigned)blocks, RCfg<N>::NT, smem, s>>>(a);
  return cuda_check(cudaGetLastError(), "rhs launch");
}

template <typename T, int N>
mf_status err_t(const mf_operator* op, double freq, const void* u, double* out, char* scratch, cudaStream_t s) {
  RhsArgs<T, N> a;
  dd* tab = reinterpret_cast<dd*>(scratch);
  mf_status st = fill<T, N>(op, freq, a, tab);
  if (st) return st;
  if ((st = tables<T, N>(op, a, tab, s))) return st;
  a.u = static_cast<const T*>(u);
  a.red = reinterpret_cast<RedPart*>(scratch + table_bytes(op));
  a.out = out;
  const long long blocks = op->g.ntiles * (BL / RCfg<N>::CB);
  if (blocks > 65536) return set_error(MF_ERR_UNSUPPORTED, "manufactured error: mesh too large (%lld CTAs)", blocks);
  if ((st = cuda_check(cudaMemsetAsync(&a.red->counter, 0, sizeof(unsigned), s), "err memset"))) return st;
  const size_t smem = sizeof(dd) * N * N * N * RCfg<N>::CB;
  if (smem + STATIC_SMEM_ALLOWANCE > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(err_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(e, "err attribute");
  }
  err_kernel<T, N><<<(unsigned)blocks, RCfg<N>::NT, smem, s>>>(a);
  return cuda_check(cudaGetLastError(), "err launch");
}

#define MF_RHS_SWITCH(fn, T, ...)                                                          \
  switch (op->n) {                                                                        \
    case 2: return fn<T, 2>(__VA_ARGS__);                                                 \
    case 3: return fn<T, 3>(__VA_ARGS__);                                                 \
    case 4: return fn<T, 4>(__VA_ARGS__);                                                 \
    case 5: return fn<T, 5>(__VA_ARGS__);                                                 \
    case 6: return fn<T, 6>(__VA_ARGS__);                                                 \
    case 7: return fn<T, 7>(__VA_ARGS__);                                                 \
    case 8: return fn<T, 8>(__VA_ARGS__);                                                 \
    case 9: return fn<T, 9>(__VA_ARGS__);                                                 \
    default: return set_error(MF_ERR_UNSUPPORTED, "n=%d not built", op->n);               \
  }

mf_status rhs_dispatch(const mf_operator* op, double freq, void* b, char* sc, cudaStream_t s) {
  if (op->precision == MF_FP32) { MF_RHS_SWITCH(rhs_t, float, op, freq, b, sc, s); }
  MF_RHS_SWITCH(rhs_t, double, op, freq, b, sc, s);
}
mf_status err_dispatch(const mf_operator* op, double freq, const void* u, double* out, char* sc, cudaStream_t s) {
  if (op->precision == MF_FP32) { MF_RHS_SWITCH(err_t, float, op, freq, u, out, sc, s); }
  MF_RHS_SWITCH(err_t, double, op, freq, u, out, sc, s);
}

} // namespace
} // namespace mf

using namespace mf;

extern "C" {

size_t mf_manufactured_workspace_bytes(const mf_operator* op) {
  if (!op) return 0;
  return table_bytes(op) + align256(sizeof(RedPart));
}

mf_status mf_rhs_manufactured(const mf_operator* op, double freq, void* b_dev, void* scratch_dev, size_t scratch_bytes,
                              void* stream) {
  if (!op || !b_dev) return set_error(MF_ERR_ARG, "mf_rhs_manufactured: NULL argument");
  if (!op->ready) return set_error(MF_ERR_ARG, "mf_rhs_manufactured: operator not set up");
  if (!scratch_dev || scratch_bytes < mf_manufactured_workspace_bytes(op))
    return set_error(MF_ERR_OOM, "mf_rhs_manufactured: scratch too small");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mf_status st = rhs_dispatch(op, freq, b_dev, static_cast<char*>(scratch_dev), s);
  if (st) return st;
  return mf_dss(op, b_dev, stream);
}

mf_status mf_error_manufactured(const mf_operator* op, double freq, const void* u_dev, double* l2sq_dev,
                                void* scratch_dev, size_t scratch_bytes, void* stream) {
  if (!op || !u_dev || !l2sq_dev) return set_error(MF_ERR_ARG, "mf_error_manufactured: NULL argument");
  if (!scratch_dev || scratch_bytes < mf_manufactured_workspace_bytes(op))
    return set_error(MF_ERR_OOM, "mf_error_manufactured: scratch too small");
  return err_dispatch(op, freq, u_dev, l2sq_dev, static_cast<char*>(scratch_dev), static_cast<cudaStream_t>(stream));
}

} // extern "C"
