// mf_cg.cu -- deterministic reductions, fused CG vector kernels and the CG / defect-correction
// drivers.
//
// CG structure (Sec. 4, "the Krylov loop on split data" and the pairing of Lemma 1): the
// iterate x and search direction p are consistent cell-wise vectors; every scalar is an
// inner product of two cell-wise vectors taken so that each global node counts once (copies
// weighted by 1/multiplicity, a power of two, so the weighting is exact).  With z = r (no
// preconditioner) the monitored quantity <r, z>^{1/2} is the assembled Euclidean residual
// norm.  Reductions run in FP64 in a fixed order (block tree, then the last block sums the
// block partials in index order), so every scalar is bitwise reproducible.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "mf_dd.cuh"
#include "mf_internal.h"
#include "mf_reduce.cuh"
#include "mf_solver.h"

namespace mf {

constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 2048;
constexpr int HIST_CAP = 65536;

// Scratch of one reduction: a done-counter and the block partials.
struct RedScratch {
  unsigned int counter;
  unsigned int pad[63];
  double partial[RED_MAX_BLOCKS];
  double partial2[RED_MAX_BLOCKS]; // a second sum reduced alongside (the update's <r, z>)
};

size_t reduce_scratch_bytes() { return sizeof(RedScratch); }



// Weight of native element e in an assembled inner product: 0 for padding, otherwise
// 1 / (number of cells sharing the node).  split = 1: 1 for every real copy.
template <int N>
__device__ __forceinline__ float node_weight(const GridInfo& g, long long e, int split) {
  constexpr int N2 = N * N, N3 = N2 * N;
  // tile indices fit in 32 bits (n_native < 2^31 * 32): keep the divisions 32-bit
  const int lane = (int)(e & (BL - 1));
  const unsigned row = (unsigned)(e >> 5);
  const int t = (int)(row / (unsigned)N3);
  const int l = (int)(row - (unsigned)t * (unsigned)N3);
  const int txy = g.ntx * g.nty;
  const int tz = t / txy;
  const int r = t - tz * txy;
  const int ty = r / g.ntx;
  const int tx = r - ty * g.ntx;
  const int cx = tx * TX + (lane & 3), cy = ty * TY + ((lane >> 2) & 3), cz = tz * TZ + (lane >> 4);
  if (cx >= g.nx || cy >= g.ny || cz >= g.nz) return 0.0f;
  if (split) return 1.0f;
  const int i = l % N, j = (l / N) % N, k = l / N2;
  const int sh = (((i == 0 && cx > 0) || (i == N - 1 && cx < g.nx - 1)) ? 1 : 0) +
                 (((j == 0 && cy > 0) || (j == N - 1 && cy < g.ny - 1)) ? 1 : 0) +
                 (((k == 0 && cz > 0) || (k == N - 1 && cz < g.nz - 1)) ? 1 : 0);
  // 1 / multiplicity = 2^-sh, selected (a division would cost far more)
  return sh == 0 ? 1.0f : (sh == 1 ? 0.5f : (sh == 2 ? 0.25f : 0.125f));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block tree sum; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[RED_THREADS / 32];
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  if (ln == 0) ws[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = (ln < RED_THREADS / 32) ? ws[ln] : 0.0;
    s = warp_sum(s);
  }
  __syncthreads();
  return s;
}

// Called by every thread of every block after the block partial is known.  Returns true
// in thread 0 of the last block to finish, with *total = sum of partials in index order.
// Two sums reduced together (partial and partial2), one counter; the last CTA gets both.
__device__ __forceinline__ bool last_block_total2(RedScratch* sc, double part, double part2, double* total,
                                                  double* total2, int cta, int ncta) {
  __shared__ bool am_last2;
  if (threadIdx.x == 0) {
    sc->partial[cta] = part;
    sc->partial2[cta] = part2;
    __threadfence();
    const unsigned prev = atomicAdd(&sc->counter, 1u);
    am_last2 = (prev == (unsigned)ncta - 1);
  }
  __syncthreads();
  if (!am_last2) return false;
  __threadfence();
  double s = 0.0, s2 = 0.0;
  for (int b = threadIdx.x; b < ncta; b += RED_THREADS) {
    s += ((volatile double*)sc->partial)[b];
    s2 += ((volatile double*)sc->partial2)[b];
  }
  s = block_sum(s);
  s2 = block_sum(s2);
  if (threadIdx.x == 0) {
    sc->counter = 0;
    *total = s;
    *total2 = s2;
  }
  return threadIdx.x == 0;
}

// cta / ncta: the CTA's index and the CTA count of its reduction (a batched launch runs
// several reductions, each over its own CTA range and scratch).
__device__ __forceinline__ bool last_block_total(RedScratch* sc, double part, double* total, int cta, int ncta) {
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    sc->partial[cta] = part;
    __threadfence();
    const unsigned prev = atomicAdd(&sc->counter, 1u);
    am_last = (prev == (unsigned)ncta - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double s = 0.0;
  for (int b = threadIdx.x; b < ncta; b += RED_THREADS) s += ((volatile double*)sc->partial)[b];
  s = block_sum(s);
  if (threadIdx.x == 0) {
    sc->counter = 0; // self-cleaning for the next launch
    *total = s;
  }
  return threadIdx.x == 0;
}

static int red_blocks(long long n) {
  long long b = (n + (long long)RED_THREADS * 8 - 1) / ((long long)RED_THREADS * 8);
  if (b < 1) b = 1;
  if (b > RED_MAX_BLOCKS) b = RED_MAX_BLOCKS;
  return (int)b;
}

template <typename T, int N>
__global__ void __launch_bounds__(RED_THREADS) dot_kernel(const T* __restrict__ a, const T* __restrict__ b, long long n,
                                                          GridInfo g, int split, RedScratch* sc, double* out) {
  typename AccOf<T>::type acc;
  for (long long e = blockIdx.x * (long long)RED_THREADS + threadIdx.x; e < n; e += (long long)gridDim.x * RED_THREADS)
    acc.add(node_weight<N>(g, e, split), a[e], b[e]);
  const double s = block_sum(acc.value());
  double tot;
  if (last_block_total(sc, s, &tot, blockIdx.x, gridDim.x)) *out = tot;
}

// alpha = rr / <p, q>
template <typename T, int N>
__global__ void __launch_bounds__(RED_THREADS) cg_pq_kernel(const T* __restrict__ p, const T* __restrict__ q, long long n,
                                                            GridInfo g, RedScratch* sc, CgState* st) {
  typename AccOf<T>::type acc;
  for (long long e = blockIdx.x * (long long)RED_THREADS + threadIdx.x; e < n; e += (long long)gridDim.x * RED_THREADS)
    acc.add(node_weight<N>(g, e, 0), p[e], q[e]);
  const double s = block_sum(acc.value());
  double tot;
  if (last_block_total(sc, s, &tot, blockIdx.x, gridDim.x)) {
    if (st->flag == 0) {
      st->pq = tot;
      if (!(tot > 0.0) || !isfinite(tot)) { st->flag = 2; st->alpha = 0.0; }
      else st->alpha = st->rr / tot;
    } else {
      st->alpha = 0.0;
    }
  }
}

// x += alpha p ; r -= alpha q ; rr_new = <r, r> ; beta = rr_new / rr
template <typename T, int N>
__global__ void __launch_bounds__(RED_THREADS) cg_xr_kernel(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                                            const T* __restrict__ q, long long n, GridInfo g,
                                                            RedScratch* sc, CgState* st, double* hist) {
  const T al = (T)st->alpha; // float vectors: FP32 updates (the inner CG of defect correction)
  const bool run = st->flag == 0;
  typename AccOf<T>::type acc;
  for (long long e = blockIdx.x * (long long)RED_THREADS + threadIdx.x; e < n; e += (long long)gridDim.x * RED_THREADS) {
    T rv = r[e];
    if (run) {
      x[e] = fma(al, p[e], x[e]);
      rv = fma(-al, q[e], rv);
      r[e] = rv;
    }
    acc.add(node_weight<N>(g, e, 0), rv, rv);
  }
  const double s = block_sum(acc.value());
  double tot;
  if (last_block_total(sc, s, &tot, blockIdx.x, gridDim.x)) {
    if (st->flag == 0) {
      st->beta = tot / st->rr;
      st->rr = tot;
      st->rz = tot;
      st->it += 1;
      if (hist && st->it < HIST_CAP) hist[st->it] = sqrt(tot) / st->bnorm;
      if (tot <= st->tol2) st->flag = 1;
      else if (!isfinite(tot)) st->flag = 2;
      else if (st->it >= st->maxit) st->flag = 3;
    } // stopped: beta stays that of the last step (a reliable update continues from it)
  }
}

// z = M^-1 r of Jacobi preconditioning: the element-wise product with the inverse diagonal
__device__ __forceinline__ double precond_z(double r, float d) { return r * (double)d; }
__device__ __forceinline__ float precond_z(float r, float d) { return r * d; }
__device__ __forceinline__ dd precond_z(dd r, float d) { return finish(mul0(r, dd(d, 0.0f))); }

// Four consecutive vector elements (16 bytes of floats, 32 of doubles / double-floats): the
// streaming kernels move them with 16-byte accesses.  Native vectors hold a multiple of 32
// elements and start 256-byte aligned.
template <typename T>
struct alignas(4 * sizeof(T) < 16 ? 16 : 4 * sizeof(T)) Quad {
  T v[4];
};

// p = r + beta p, two quads per thread and trip so that four 16-byte loads are in flight
// p = z + beta p, z = r or, with dinv, z = r / diag(A)
template <typename T>
__device__ __forceinline__ void cg_p_body(const T* __restrict__ r, T* __restrict__ p, const float* __restrict__ dinv,
                                          long long n, const CgState* st, long long cta, long long ncta) {
  const T be = scalar_from_double<T>(st->beta);
  // stopped (converged, broken down or at maxit): the direction stays the last one applied,
  // which a reliable update of the mixed solver continues from
  if (st->flag != 0) return;
  const long long nq = n / 4;
  const Quad<T>* __restrict__ rq = reinterpret_cast<const Quad<T>*>(r);
  Quad<T>* __restrict__ pq = reinterpret_cast<Quad<T>*>(p);
  const long long stride = ncta * blockDim.x;
  for (long long i = cta * (long long)blockDim.x + threadIdx.x; i < nq; i += 2 * stride) {
    const bool two = i + stride < nq;
    Quad<T> a = pq[i], b = rq[i], c, d;
    if (two) { c = pq[i + stride]; d = rq[i + stride]; }
    if (dinv) {
      const float4 d0 = reinterpret_cast<const float4*>(dinv)[i];
      b.v[0] = precond_z(b.v[0], d0.x); b.v[1] = precond_z(b.v[1], d0.y);
      b.v[2] = precond_z(b.v[2], d0.z); b.v[3] = precond_z(b.v[3], d0.w);
      if (two) {
        const float4 d1 = reinterpret_cast<const float4*>(dinv)[i + stride];
        d.v[0] = precond_z(d.v[0], d1.x); d.v[1] = precond_z(d.v[1], d1.y);
        d.v[2] = precond_z(d.v[2], d1.z); d.v[3] = precond_z(d.v[3], d1.w);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) a.v[j] = finish(fma(be, a.v[j], b.v[j]));
    pq[i] = a;
    if (two) {
#pragma unroll
      for (int j = 0; j < 4; ++j) c.v[j] = finish(fma(be, c.v[j], d.v[j]));
      pq[i + stride] = c;
    }
  }
}
template <typename T>
__global__ void cg_p_kernel(const T* __restrict__ r, T* __restrict__ p, const float* __restrict__ dinv, long long n,
                            const CgState* st) {
  cg_p_body<T>(r, p, dinv, n, st, blockIdx.x, gridDim.x);
}

// Split-dual CG update (Sec. 4: the Krylov loop on split data).  q~ = A_K p is the split
// product written by the apply; its assembled value q = G G^T q~ is formed here, per copy, as
// the sum of the copies of the node in the canonical order of the duplicate summation (pairs
// along x, then the pair sums along y, then along z -- the same expression in every copy, so
// q is consistent bitwise and equal to what the separate duplicate summation writes).  Then
// x += alpha p, r -= alpha q, and <r, r> (copies weighted by 1/multiplicity) gives
// beta = <r,r>_new / <r,r> and the convergence test.
//
// Work unit: one x-pencil (tile t, local j, k) of the 32 cells of a tile; a warp takes a unit,
// lane = cell, so each of its accesses is one contiguous 32-element row.  Every load of the
// unit (the pencil's x, p, r, q~, and the q~ of the neighbour copies along y / z and of the
// x-neighbours at both pencil ends) is issued before any sum, so a thread keeps up to 7n + 8
// loads in flight.
template <typename T, int N>
__device__ __forceinline__ void cg_update_body(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                               const T* __restrict__ q, const float* __restrict__ dinv,
                                               const GridInfo& g, RedScratch* sc, CgState* st, double* hist, int cta,
                                               int ncta) {
  constexpr int N2 = N * N, N3 = N2 * N, K = N - 1;
  if (st->flag != 0) return; // uniform: converged or stopped, nothing changes
  const T al = scalar_from_double<T>(st->alpha);
  const long long tile_el = (long long)N3 * BL;                 // elements of one tile
  const long long ty_step = (long long)g.ntx * tile_el;         // one tile row along y
  const long long tz_step = (long long)g.ntx * g.nty * tile_el; // one tile layer along z
  const int lane = threadIdx.x & 31;
  const int lx = lane & 3, ly = (lane >> 2) & 3, lz = lane >> 4;
  // element distance to the neighbour copy across each face of the cell
  const long long dxm = lx > 0 ? (long long)K * BL - 1 : (long long)K * BL - tile_el + (TX - 1);
  const long long dxp = lx < TX - 1 ? -(long long)K * BL + 1 : tile_el - (long long)K * BL - (TX - 1);
  const long long dym = ly > 0 ? (long long)K * N * BL - TX : (long long)K * N * BL - ty_step + TX * (TY - 1);
  const long long dyp = ly < TY - 1 ? -(long long)K * N * BL + TX : ty_step - (long long)K * N * BL - TX * (TY - 1);
  const long long dzm = lz > 0 ? (long long)K * N2 * BL - TX * TY : (long long)K * N2 * BL - tz_step + TX * TY * (TZ - 1);
  const long long dzp =
      lz < TZ - 1 ? -(long long)K * N2 * BL + TX * TY : tz_step - (long long)K * N2 * BL - TX * TY * (TZ - 1);
  const long long units = g.ntiles * N2;
  const long long warps = (long long)ncta * (RED_THREADS / 32);
  typename AccOf<T>::type acc, accz; // <r, r> and (preconditioned) <r, z>
  for (long long u = cta * (long long)(RED_THREADS / 32) + (threadIdx.x >> 5); u < units; u += warps) {
    const long long t = u / N2;
    const int jk = (int)(u - t * N2);
    const int j = jk % N, k = jk / N;
    const int txy = g.ntx * g.nty;
    const int tz = (int)(t / txy);
    const int rm = (int)(t - (long long)tz * txy);
    const int ty = rm / g.ntx, tx = rm - ty * g.ntx;
    const int cx = tx * TX + lx, cy = ty * TY + ly, cz = tz * TZ + lz;
    if (cx >= g.nx || cy >= g.ny || cz >= g.nz) continue; // padding lane: nothing to update
    const bool hxm = cx > 0, hxp = cx < g.nx - 1;
    const bool ym = j == 0 && cy > 0, yp = j == K && cy < g.ny - 1;
    const bool zm = k == 0 && cz > 0, zp = k == K && cz < g.nz - 1;
    const int my = (ym || yp) ? 2 : 1, mz = (zm || zp) ? 2 : 1;
    // copy offsets along y and z: index 0 = low copy, 1 = high copy (0 = this copy)
    const long long oy[2] = {ym ? dym : 0, yp ? dyp : 0};
    const long long oz[2] = {zm ? dzm : 0, zp ? dzp : 0};
    const long long e0 = t * tile_el + (long long)(N * j + N2 * k) * BL + lane;
    T Q[2][2][N], XM[2][2], XP[2][2];
#pragma unroll
    for (int zz = 0; zz < 2; ++zz)
#pragma unroll
      for (int yy = 0; yy < 2; ++yy)
        if (zz < mz && yy < my) {
          const long long o = e0 + oz[zz] + oy[yy];
#pragma unroll
          for (int i = 0; i < N; ++i) Q[zz][yy][i] = q[o + (long long)i * BL];
          if (hxm) XM[zz][yy] = q[o + dxm];
          if (hxp) XP[zz][yy] = q[o + (long long)K * BL + dxp];
        }
    T xv[N], pv[N], rv[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      xv[i] = x[e0 + (long long)i * BL];
      pv[i] = p[e0 + (long long)i * BL];
      rv[i] = r[e0 + (long long)i * BL];
    }
    const int shyz = (my - 1) + (mz - 1);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const bool xl = i == 0 && hxm, xh = i == K && hxp;
      T sz[2];
#pragma unroll
      for (int zz = 0; zz < 2; ++zz)
        if (zz < mz) {
          T sy[2];
#pragma unroll
          for (int yy = 0; yy < 2; ++yy)
            if (yy < my) {
              T v = Q[zz][yy][i];
              if (xl) v = XM[zz][yy] + v;
              else if (xh) v = v + XP[zz][yy];
              sy[yy] = v;
            }
          sz[zz] = my == 2 ? sy[0] + sy[1] : sy[0];
        }
      const T qv = mz == 2 ? sz[0] + sz[1] : sz[0];
      const long long e = e0 + (long long)i * BL;
      x[e] = finish(fma(al, pv[i], xv[i]));
      const T rn = finish(fma(-al, qv, rv[i]));
      r[e] = rn;
      const int sh = shyz + ((xl || xh) ? 1 : 0);
      const float w = sh == 0 ? 1.0f : (sh == 1 ? 0.5f : (sh == 2 ? 0.25f : 0.125f));
      acc.add(w, rn, rn);
      if (dinv) accz.add(w, rn, precond_z(rn, dinv[e]));
    }
  }
  const double s = block_sum(acc.value());
  const double sz = dinv ? block_sum(accz.value()) : 0.0;
  double tot, totz;
  if (last_block_total2(sc, s, sz, &tot, &totz, cta, ncta)) {
    const double rz = dinv ? totz : tot;
    st->beta = rz / st->rz;
    st->rz = rz;
    st->rr = tot;
    st->it += 1;
    if (hist && st->it < HIST_CAP) hist[st->it] = sqrt(tot) / st->bnorm;
    if (tot <= st->tol2) st->flag = 1;
    else if (!isfinite(tot)) st->flag = 2;
    else if (st->it >= st->maxit) st->flag = 3;
  }
}
template <typename T, int N>
__global__ void __launch_bounds__(RED_THREADS) cg_update_kernel(T* __restrict__ x, T* __restrict__ r,
                                                                const T* __restrict__ p, const T* __restrict__ q,
                                                                const float* __restrict__ dinv, GridInfo g,
                                                                RedScratch* sc, CgState* st, double* hist) {
  cg_update_body<T, N>(x, r, p, q, dinv, g, sc, st, hist, blockIdx.x, gridDim.x);
}

// alpha = <r, r> / <p, A p> from the apply's per-CTA partials of <p, A p>, folded in a fixed
// order (breakdown when <p, A p> is not positive and finite).
__device__ __forceinline__ void alpha_body(const double* __restrict__ partials, long long nparts, CgState* st) {
  __shared__ double park[1024];
  if (st->flag != 0) return; // uniform
  double s = 0.0;
  for (long long i = threadIdx.x; i < nparts; i += blockDim.x) s += partials[i];
  s = block_park_sum(s, park);
  if (threadIdx.x == 0) {
    st->pq = s;
    if (!(s > 0.0) || !isfinite(s)) {
      st->flag = 2;
      st->alpha = 0.0;
    } else {
      st->alpha = st->rz / s;
    }
  }
}
__global__ void __launch_bounds__(1024) alpha_kernel(const double* __restrict__ partials, long long nparts,
                                                     CgState* st) {
  alpha_body(partials, nparts, st);
}

// ---------------------------------------------------------------------------------------
// Batched CG iteration (the serving loop's continuous batch): one launch per kernel for all
// members; member i owns CTAs [block0[i], block0[i+1]) of the update and direction launches,
// exactly the CTA count its own launch would use, so every member computes bitwise what it
// would compute alone.
// ---------------------------------------------------------------------------------------
struct VecJob {
  void *x, *r, *p, *q;
  const float* dinv; // Jacobi: inverse diagonal (null: no preconditioner)
  GridInfo g;
  RedScratch* sc;
  CgState* st;
  double* hist;
  double* apart;
  long long n;                  // native elements
  long long apply_blocks;       // CTAs of its apply (partials to fold)
  long long up0, up1, pp0, pp1; // its CTA ranges in the update and direction launches
};

__device__ __forceinline__ int find_member(const VecJob* jobs, int njobs, bool update) {
  int lo = 0, hi = njobs - 1; // largest i whose range starts at or before blockIdx.x
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((update ? jobs[mid].up0 : jobs[mid].pp0) <= (long long)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
__global__ void __launch_bounds__(1024) alpha_batch_kernel(const VecJob* __restrict__ jobs) {
  const VecJob& j = jobs[blockIdx.x];
  alpha_body(j.apart, j.apply_blocks, j.st);
}
template <typename T, int N>
__global__ void __launch_bounds__(RED_THREADS) cg_update_batch_kernel(const VecJob* __restrict__ jobs, int njobs) {
  const VecJob& j = jobs[find_member(jobs, njobs, true)];
  cg_update_body<T, N>((T*)j.x, (T*)j.r, (const T*)j.p, (const T*)j.q, j.dinv, j.g, j.sc, j.st, j.hist,
                       (int)((long long)blockIdx.x - j.up0), (int)(j.up1 - j.up0));
}
template <typename T>
__global__ void cg_p_batch_kernel(const VecJob* __restrict__ jobs, int njobs) {
  const VecJob& j = jobs[find_member(jobs, njobs, false)];
  cg_p_body<T>((const T*)j.r, (T*)j.p, j.dinv, j.n, j.st, (long long)blockIdx.x - j.pp0, j.pp1 - j.pp0);
}

// Small element-wise kernels of the drivers.
template <typename T>
__global__ void copy_kernel(const T* __restrict__ a, T* __restrict__ b, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) b[e] = a[e];
}
template <typename T>
__global__ void zero_kernel(T* __restrict__ a, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) a[e] = T(0);
}
// r = b - q (FP64)
__global__ void sub_kernel(const double* __restrict__ b, const double* __restrict__ q, double* __restrict__ r, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) r[e] = b[e] - q[e];
}
// r32 = r64 * scale
__global__ void to32_kernel(const double* __restrict__ r, float* __restrict__ o, const double* rn2, long long n) {
  const double sc = (*rn2 > 0.0) ? 1.0 / sqrt(*rn2) : 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) o[e] = (float)(r[e] * sc);
}
// Reliable update of the mixed solver's inner CG (its residual r_k+1 replaced by the FP64
// one, r^): beta = <r^, r^> / <r_k, r_k> = beta_k <r^, r^> / <r_k+1, r_k+1> (Clark et al.'s
// reliable-update CG), the state restarted on <r^, r^>.  When the recursive residual has
// drifted from the true one by more than RELIABLE_DRIFT ||r^||, the kept direction carries
// little information and the CG restarts from p = r^ (beta = 0) instead.
constexpr double RELIABLE_DRIFT = 0.1;
__global__ void reliable_state_kernel(CgState* st, const double* rr_new, const double* cross, double inner_rtol,
                                      int maxit) {
  const double rr = *rr_new;
  CgState h = *st;
  const double drift2 = rr - 2.0 * *cross + h.rr; // ||r^ - r_k+1||^2
  const bool keep = h.rz > 0.0 && isfinite(h.rz) && drift2 <= RELIABLE_DRIFT * RELIABLE_DRIFT * rr;
  h.beta = keep ? h.beta * rr / h.rz : 0.0;
  h.rr = h.rz = rr;
  h.bnorm = sqrt(rr);
  h.tol2 = inner_rtol * inner_rtol * rr;
  h.pq = h.alpha = 0.0;
  h.it = 0;
  h.maxit = maxit;
  h.flag = !isfinite(rr) ? 2 : ((rr == 0.0) ? 1 : (maxit <= 0 ? 3 : 0));
  *st = h;
}
// x += sqrt(rn2) * d
__global__ void axpy64_kernel(double* __restrict__ x, const float* __restrict__ d, const double* rn2, long long n) {
  const double sc = sqrt(*rn2);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) x[e] += sc * (double)d[e];
}
// Jacobi: d <- 1 / d where positive (Dirichlet nodes and padding keep 0)
__global__ void invert_diag_kernel(float* __restrict__ d, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    d[e] = d[e] > 0.0f ? 1.0f / d[e] : 0.0f;
}
// p = z = r / diag (the first search direction of the preconditioned CG)
template <typename T>
__global__ void precond_copy_kernel(const T* __restrict__ r, T* __restrict__ p, const float* __restrict__ dinv,
                                    long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    p[e] = precond_z(r[e], dinv[e]);
}

// FP64 solver with double-float vectors: r = b 2^-s as double-float, where 2^s is the power of
// two of max|b| (so every value of the iteration stays well inside the float exponent range,
// for right-hand sides anywhere in the double range); the solution is converted back with
// x = 2^s x~ at the end.  max|b| is an integer max over the bit patterns of |b| (order-free,
// so deterministic); *amax must be zero before the launch.
__global__ void absmax_bits_kernel(const double* __restrict__ b, unsigned long long* amax, long long n) {
  unsigned long long m = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    m = max(m, (unsigned long long)__double_as_longlong(b[e]) & 0x7fffffffffffffffull);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(amax, m);
}
// 2^s from the bits of max|b|: s = its unbiased exponent; 1 for zero, subnormal or non-finite
__device__ __forceinline__ double pow2_of_bits(unsigned long long bits) {
  const int e = (int)((bits >> 52) & 0x7ff);
  if (e == 0 || e == 0x7ff) return 1.0;
  return __longlong_as_double((long long)e << 52); // 2^(e - 1023)
}
__device__ __forceinline__ double inv_pow2_of_bits(unsigned long long bits) {
  const int e = (int)((bits >> 52) & 0x7ff);
  if (e == 0 || e == 0x7ff) return 1.0;
  const int f = 2046 - e; // biased exponent of 2^(1023 - e); 0 means 2^-1023, a subnormal
  return f > 0 ? __longlong_as_double((long long)f << 52) : __longlong_as_double(1ll << 51);
}
__global__ void to_dd_scaled_kernel(const double* __restrict__ b, dd* __restrict__ r, const unsigned long long* amax,
                                    long long n) {
  const double isc = inv_pow2_of_bits(*amax);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    r[e] = dd_from_double(b[e] * isc);
}
__global__ void from_dd_scaled_kernel(const dd* __restrict__ x, double* __restrict__ o, const unsigned long long* amax,
                                      long long n) {
  const double sc = pow2_of_bits(*amax);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    o[e] = dd_to_double(x[e]) * sc;
}

// Dirichlet mask P b (zero constrained copies) -- used on the right-hand side
template <typename T, int N>
__global__ void mask_kernel(const T* __restrict__ b, T* __restrict__ o, long long n, GridInfo g) {
  constexpr int N2 = N * N, N3 = N2 * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int lane = (int)(e & (BL - 1));
    const unsigned row = (unsigned)(e >> 5);
    const int t = (int)(row / (unsigned)N3);
    const int l = (int)(row - (unsigned)t * (unsigned)N3);
    const int txy = g.ntx * g.nty;
    const int tz = t / txy;
    const int rr = t - tz * txy;
    const int ty = rr / g.ntx, tx = rr - ty * g.ntx;
    const int cx = tx * TX + (lane & 3), cy = ty * TY + ((lane >> 2) & 3), cz = tz * TZ + (lane >> 4);
    const int i = l % N, j = (l / N) % N, k = l / N2;
    const bool valid = cx < g.nx && cy < g.ny && cz < g.nz;
    const bool bnd = g.bc && ((cx == 0 && i == 0) || (cx == g.nx - 1 && i == N - 1) || (cy == 0 && j == 0) ||
                              (cy == g.ny - 1 && j == N - 1) || (cz == 0 && k == 0) || (cz == g.nz - 1 && k == N - 1));
    o[e] = (valid && !bnd) ? b[e] : T(0);
  }
}

static unsigned ew_blocks(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// ------------------------------------------------------------------ typed dispatch helpers
template <int N>
static mf_status dot_n(const mf_operator* op, int elem, const void* a, const void* b, int split, double* out,
                       RedScratch* sc, cudaStream_t s) {
  const long long n = op->n_native;
  const int bl = red_blocks(n);
  if (elem == 8)
    dot_kernel<double, N><<<bl, RED_THREADS, 0, s>>>((const double*)a, (const double*)b, n, op->g, split, sc, out);
  else if (elem == ELEM_DD)
    dot_kernel<dd, N><<<bl, RED_THREADS, 0, s>>>((const dd*)a, (const dd*)b, n, op->g, split, sc, out);
  else
    dot_kernel<float, N><<<bl, RED_THREADS, 0, s>>>((const float*)a, (const float*)b, n, op->g, split, sc, out);
  return cuda_check(cudaGetLastError(), "dot launch");
}

#define MF_SWITCH_N(n, fn, ...)                                          \
  switch (n) {                                                           \
    case 2: return fn<2>(__VA_ARGS__);                                   \
    case 3: return fn<3>(__VA_ARGS__);                                   \
    case 4: return fn<4>(__VA_ARGS__);                                   \
    case 5: return fn<5>(__VA_ARGS__);                                   \
    case 6: return fn<6>(__VA_ARGS__);                                   \
    case 7: return fn<7>(__VA_ARGS__);                                   \
    case 8: return fn<8>(__VA_ARGS__);                                   \
    case 9: return fn<9>(__VA_ARGS__);                                   \
    default: return set_error(MF_ERR_UNSUPPORTED, "n=%d not built", n);  \
  }

mf_status dot_launch(const mf_operator* op, int elem, const void* a, const void* b, int split, double* out, void* scratch,
                     cudaStream_t s) {
  MF_SWITCH_N(op->n, dot_n, op, elem, a, b, split, out, (RedScratch*)scratch, s);
}

template <typename T, int N>
static mf_status mask_n(const mf_operator* op, const void* b, void* o, cudaStream_t s) {
  const long long n = op->n_native;
  mask_kernel<T, N><<<ew_blocks(n), 256, 0, s>>>((const T*)b, (T*)o, n, op->g);
  return cuda_check(cudaGetLastError(), "mask launch");
}
template <int N>
static mf_status mask_e(const mf_operator* op, int elem, const void* b, void* o, cudaStream_t s) {
  return elem == 8 ? mask_n<double, N>(op, b, o, s) : mask_n<float, N>(op, b, o, s);
}
static mf_status launch_mask(const mf_operator* op, int elem, const void* b, void* o, cudaStream_t s) {
  MF_SWITCH_N(op->n, mask_e, op, elem, b, o, s);
}

// One CG iteration's vector kernels (after q = A p).
template <typename T, int N>
static mf_status cg_vec_n(const mf_operator* op, T* x, T* r, T* p, T* q, RedScratch* sc1, RedScratch* sc2, CgState* st,
                          double* hist, cudaStream_t s) {
  const long long n = op->n_native;
  const int bl = red_blocks(n);
  cg_pq_kernel<T, N><<<bl, RED_THREADS, 0, s>>>(p, q, n, op->g, sc1, st);
  cg_xr_kernel<T, N><<<bl, RED_THREADS, 0, s>>>(x, r, p, q, n, op->g, sc2, st, hist);
  cg_p_kernel<T><<<ew_blocks(n), 256, 0, s>>>(r, p, nullptr, n, st);
  return cuda_check(cudaGetLastError(), "cg vector launch");
}
template <int N>
static mf_status cg_vec_e(const mf_operator* op, int elem, void* x, void* r, void* p, void* q, RedScratch* sc1,
                          RedScratch* sc2, CgState* st, double* hist, cudaStream_t s) {
  if (elem == 8) return cg_vec_n<double, N>(op, (double*)x, (double*)r, (double*)p, (double*)q, sc1, sc2, st, hist, s);
  return cg_vec_n<float, N>(op, (float*)x, (float*)r, (float*)p, (float*)q, sc1, sc2, st, hist, s);
}
static mf_status launch_cg_vec(const mf_operator* op, int elem, void* x, void* r, void* p, void* q, RedScratch* sc1,
                               RedScratch* sc2, CgState* st, double* hist, cudaStream_t s) {
  MF_SWITCH_N(op->n, cg_vec_e, op, elem, x, r, p, q, sc1, sc2, st, hist, s);
}

template <int N>
static mf_status cg_update_e(const mf_operator* op, int elem, void* x, void* r, void* p, void* q, const SolveWs& w,
                             CgState* st, double* hist, cudaStream_t s) {
  const float* dinv = w.dinv_active;
  // one warp per x-pencil unit, at most RED_MAX_BLOCKS CTAs (warps loop over further units)
  long long bl = (op->g.ntiles * (long long)N * N + RED_THREADS / 32 - 1) / (RED_THREADS / 32);
  if (bl > RED_MAX_BLOCKS) bl = RED_MAX_BLOCKS;
  if (bl < 1) bl = 1;
  if (elem == 8)
    cg_update_kernel<double, N><<<(unsigned)bl, RED_THREADS, 0, s>>>((double*)x, (double*)r, (const double*)p,
                                                                      (const double*)q, dinv, op->g, w.sc2, st, hist);
  else if (elem == ELEM_DD)
    cg_update_kernel<dd, N><<<(unsigned)bl, RED_THREADS, 0, s>>>((dd*)x, (dd*)r, (const dd*)p, (const dd*)q, dinv,
                                                                  op->g, w.sc2, st, hist);
  else
    cg_update_kernel<float, N><<<(unsigned)bl, RED_THREADS, 0, s>>>((float*)x, (float*)r, (const float*)p,
                                                                     (const float*)q, dinv, op->g, w.sc2, st, hist);
  return cuda_check(cudaGetLastError(), "cg update launch");
}
static mf_status launch_cg_update(const mf_operator* op, int elem, void* x, void* r, void* p, void* q, const SolveWs& w,
                                  CgState* st, double* hist, cudaStream_t s) {
  MF_SWITCH_N(op->n, cg_update_e, op, elem, x, r, p, q, w, st, hist, s);
}
template <int N>
static mf_status cg_p_e(const mf_operator* op, int elem, const void* r, void* p, const float* dinv, CgState* st,
                        cudaStream_t s) {
  const long long n = op->n_native;
  if (elem == 8) cg_p_kernel<double><<<ew_blocks(n), 256, 0, s>>>((const double*)r, (double*)p, dinv, n, st);
  else if (elem == ELEM_DD) cg_p_kernel<dd><<<ew_blocks(n), 256, 0, s>>>((const dd*)r, (dd*)p, dinv, n, st);
  else cg_p_kernel<float><<<ew_blocks(n), 256, 0, s>>>((const float*)r, (float*)p, dinv, n, st);
  return cuda_check(cudaGetLastError(), "cg p launch");
}
static mf_status launch_cg_p(const mf_operator* op, int elem, const void* r, void* p, const float* dinv, CgState* st,
                             cudaStream_t s) {
  MF_SWITCH_N(op->n, cg_p_e, op, elem, r, p, dinv, st, s);
}
// apply with <p, A_K p> partials, then alpha
static mf_status launch_apply_alpha(const mf_operator* op, int elem, void* p, const void* r, void* q, const SolveWs& w,
                                   CgState* st, int fused_p, cudaStream_t s) {
  const int vk = elem == ELEM_DD ? VK_DDS : view_of_elem(op, elem);
  long long nb = 0;
  mf_status rc = launch_apply_cg(op, vk, p, r, q, st, w.apart, fused_p, &nb, s);
  if (rc) return rc;
  alpha_kernel<<<1, 1024, 0, s>>>(w.apart, nb, st);
  return cuda_check(cudaGetLastError(), "alpha launch");
}
// One split-dual iteration: apply with <p, A_K p> (alpha), update (q = G G^T q~, x, r, beta),
// then p = z + beta p -- or, with fused_p, the apply forms p = r + beta p itself at load.
static mf_status launch_cg_split(const mf_operator* op, int elem, void* x, void* r, void* p, void* q, const SolveWs& w,
                                 CgState* st, double* hist, int fused_p, cudaStream_t s) {
  mf_status rc = launch_apply_alpha(op, elem, p, r, q, w, st, fused_p, s);
  if (rc) return rc;
  if ((rc = launch_cg_update(op, elem, x, r, p, q, w, st, hist, s))) return rc;
  return fused_p ? MF_OK : launch_cg_p(op, elem, r, p, w.dinv_active, st, s);
}

// apply + duplicate summation with a given element type (selects the FP64 or FP32 view)
static mf_status apply_elem(const mf_operator* op, int elem, const void* x, void* y, cudaStream_t s) {
  mf_status st = launch_apply_split(op, view_of_elem(op, elem), x, y, s);
  if (st) return st;
  return launch_dss(op, elem, y, s);
}

static size_t a256(size_t b) { return (b + 255) & ~size_t(255); }

static thread_local double* g_hist_host = nullptr;
static thread_local int g_hist_cap = 0;

size_t solve_ws_layout(const mf_operator* op, int mixed, char* base, SolveWs* w) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* { char* p = base ? base + off : nullptr; off += a256(bytes); return p; };
  const size_t n = (size_t)op->n_native;
  const int elem = mixed ? 4 : (op->precision == MF_FP32 ? 4 : 8);
  SolveWs t;
  t.st = (CgState*)take(sizeof(CgState));
  t.sc1 = (RedScratch*)take(sizeof(RedScratch));
  t.sc2 = (RedScratch*)take(sizeof(RedScratch));
  t.sc3 = (RedScratch*)take(sizeof(RedScratch));
  t.hist = (double*)take(sizeof(double) * HIST_CAP);
  t.scal = (double*)take(sizeof(double) * 16);
  t.apart = (double*)take(sizeof(double) * (size_t)apply_max_blocks(op));
  t.dinv = (float*)take(sizeof(float) * n);        // Jacobi: inverse of the assembled diagonal
  t.dtab = (float*)take(diag_table_bytes(op));     //   and the diagonal's sin / cos tables
  t.dinv_active = nullptr;
  t.r = take(n * elem);
  t.p = take(n * elem);
  t.q = take(n * elem);
  t.r64 = t.q64 = t.b64 = t.d32 = t.xdd = nullptr;
  if (!mixed && elem == 8 && fp64_view(op) == VK_DD) t.xdd = take(n * 8); // double-float iterate
  if (mixed) {
    t.r64 = take(n * 8);
    t.q64 = take(n * 8);
    t.b64 = take(n * 8);
    t.d32 = take(n * 4);
  }
  if (w) *w = t;
  return off;
}

// CG state from the first residual norm (kept on the device: no host round trip).
__global__ void init_state_kernel(CgState* st, const double* rr0, const double* rz0, double rtol, int maxit) {
  const double rr = *rr0;
  CgState h;
  h.rr = rr;
  h.rz = *rz0;
  h.pq = h.alpha = h.beta = 0.0;
  h.bnorm = sqrt(rr);
  h.tol2 = (rtol * h.bnorm) * (rtol * h.bnorm);
  h.it = 0;
  h.maxit = maxit;
  h.pad = 0;
  h.flag = !isfinite(rr) || !isfinite(h.rz) ? 2 : ((rr <= h.tol2 || rr == 0.0) ? 1 : (maxit <= 0 ? 3 : 0));
  *st = h;
}

// ---------------------------------------------------------------- solver engine
// Phase machine shared by the synchronous mf_cg_solve and the server.  Every phase enqueues
// its GPU work and one small device-to-host copy into the host mirror; the caller advances
// the engine once that copy has landed (stream synchronise, or an event recorded after it).

// start an inner (or plain) CG on rhs (already masked) into x_in with tolerance rtol
static mf_status eng_inner_start(SolverEngine* e, const void* rhs, void* x_in, double rtol, int maxit) {
  const long long n = e->op->n_native;
  cudaStream_t s = e->s;
  const int el = e->vt;
  mf_status st;
  // p = r; with the direction update fused into the apply: p = 0 and beta = 0, so the first
  // apply forms p = r + 0 p = r
  if (el == ELEM_DD) {
    // double-float vectors (8 bytes like a double; zero is all-zero bits in both): r = b 2^-s
    unsigned long long* amax = reinterpret_cast<unsigned long long*>(e->w.scal + 3);
    if ((st = cuda_check(cudaMemsetAsync(amax, 0, sizeof(*amax), s), "max clear"))) return st;
    absmax_bits_kernel<<<ew_blocks(n), 256, 0, s>>>((const double*)rhs, amax, n);
    zero_kernel<double><<<ew_blocks(n), 256, 0, s>>>((double*)x_in, n);
    to_dd_scaled_kernel<<<ew_blocks(n), 256, 0, s>>>((const double*)rhs, (dd*)e->w.r, amax, n);
    if (e->form == MF_CG_SPLIT_DUAL_FUSED) zero_kernel<double><<<ew_blocks(n), 256, 0, s>>>((double*)e->w.p, n);
    else copy_kernel<double><<<ew_blocks(n), 256, 0, s>>>((const double*)e->w.r, (double*)e->w.p, n);
  } else if (el == 8) {
    zero_kernel<double><<<ew_blocks(n), 256, 0, s>>>((double*)x_in, n);
    copy_kernel<double><<<ew_blocks(n), 256, 0, s>>>((const double*)rhs, (double*)e->w.r, n);
    if (e->form == MF_CG_SPLIT_DUAL_FUSED) zero_kernel<double><<<ew_blocks(n), 256, 0, s>>>((double*)e->w.p, n);
    else copy_kernel<double><<<ew_blocks(n), 256, 0, s>>>((const double*)rhs, (double*)e->w.p, n);
  } else {
    zero_kernel<float><<<ew_blocks(n), 256, 0, s>>>((float*)x_in, n);
    copy_kernel<float><<<ew_blocks(n), 256, 0, s>>>((const float*)rhs, (float*)e->w.r, n);
    if (e->form == MF_CG_SPLIT_DUAL_FUSED) zero_kernel<float><<<ew_blocks(n), 256, 0, s>>>((float*)e->w.p, n);
    else copy_kernel<float><<<ew_blocks(n), 256, 0, s>>>((const float*)rhs, (float*)e->w.p, n);
  }
  if ((st = cuda_check(cudaGetLastError(), "cg init"))) return st;
  if ((st = dot_launch(e->op, el, e->w.r, e->w.r, 0, e->w.scal, e->w.sc3, s))) return st;
  const double* rz0 = e->w.scal;
  if (e->w.dinv_active) { // preconditioned: p = z = r / diag, <r, z>
    if (el == 8) precond_copy_kernel<double><<<ew_blocks(n), 256, 0, s>>>((const double*)e->w.r, (double*)e->w.p, e->w.dinv_active, n);
    else if (el == ELEM_DD) precond_copy_kernel<dd><<<ew_blocks(n), 256, 0, s>>>((const dd*)e->w.r, (dd*)e->w.p, e->w.dinv_active, n);
    else precond_copy_kernel<float><<<ew_blocks(n), 256, 0, s>>>((const float*)e->w.r, (float*)e->w.p, e->w.dinv_active, n);
    if ((st = cuda_check(cudaGetLastError(), "precond init"))) return st;
    if ((st = dot_launch(e->op, el, e->w.r, e->w.p, 0, e->w.scal + 5, e->w.sc3, s))) return st;
    rz0 = e->w.scal + 5;
  }
  init_state_kernel<<<1, 1, 0, s>>>(e->w.st, e->w.scal, rz0, rtol, maxit);
  if ((st = cuda_check(cudaGetLastError(), "init state"))) return st;
  e->phase = PH_INNER;
  return cuda_check(cudaMemcpyAsync(&e->hm->st, e->w.st, sizeof(CgState), cudaMemcpyDeviceToHost, s), "state D2H");
}

static mf_status eng_chunk(SolverEngine* e) {
  cudaStream_t s = e->s;
  mf_status st;
  if (!e->exec) {
    if ((st = cuda_check(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "capture begin"))) return st;
    mf_status cst = MF_OK;
    for (int c = 0; c < e->chunk && cst == MF_OK; ++c) {
      if (e->form != MF_CG_ASSEMBLED) {
        cst = launch_cg_split(e->op, e->vt, e->x_in, e->w.r, e->w.p, e->w.q, e->w, e->w.st, e->w.hist,
                              e->form == MF_CG_SPLIT_DUAL_FUSED, s);
      } else {
        cst = apply_elem(e->op, e->elem_in, e->w.p, e->w.q, s);
        if (cst == MF_OK)
          cst = launch_cg_vec(e->op, e->elem_in, e->x_in, e->w.r, e->w.p, e->w.q, e->w.sc1, e->w.sc2, e->w.st,
                              e->w.hist, s);
      }
    }
    cudaError_t ce = cudaStreamEndCapture(s, &e->graph);
    if (cst) {
      if (e->graph) { cudaGraphDestroy(e->graph); e->graph = nullptr; }
      return cst;
    }
    if ((st = cuda_check(ce, "capture end"))) return st;
    if ((st = cuda_check(cudaGraphInstantiate(&e->exec, e->graph, 0), "graph instantiate"))) return st;
  }
  if ((st = cuda_check(cudaGraphLaunch(e->exec, s), "graph launch"))) return st;
  return cuda_check(cudaMemcpyAsync(&e->hm->st, e->w.st, sizeof(CgState), cudaMemcpyDeviceToHost, s), "state D2H");
}

// mixed: r64 = b - A x (or b when x = 0); ||b||^2 and ||r||^2 to the host mirror
static mf_status eng_outer_residual(SolverEngine* e, bool first) {
  const long long n = e->op->n_native;
  cudaStream_t s = e->s;
  mf_status st;
  double* b = (double*)e->w.b64;
  double* r = (double*)e->w.r64;
  if (first) {
    copy_kernel<double><<<ew_blocks(n), 256, 0, s>>>(b, r, n);
    if ((st = dot_launch(e->op, 8, b, b, 0, e->w.scal + 1, e->w.sc3, s))) return st;
  } else {
    if ((st = apply_elem(e->op, 8, e->x, e->w.q64, s))) return st;
    sub_kernel<<<ew_blocks(n), 256, 0, s>>>(b, (const double*)e->w.q64, r, n);
  }
  if ((st = dot_launch(e->op, 8, r, r, 0, e->w.scal + 2, e->w.sc3, s))) return st;
  e->phase = PH_OUTER;
  return cuda_check(cudaMemcpyAsync(&e->hm->bn2, e->w.scal + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, s),
                    "residual D2H");
}

mf_status engine_init(SolverEngine* e, const mf_operator* op, int mixed, const void* b, void* x, double rtol, int maxit,
                      void* ws, cudaStream_t s, HostMirror* hm) {
  e->op = op;
  e->mixed = mixed;
  e->elem_in = mixed ? 4 : (op->precision == MF_FP32 ? 4 : 8);
  e->s = s;
  solve_ws_layout(op, mixed, static_cast<char*>(ws), &e->w);
  e->b = b;
  e->x = x;
  e->x_in = mixed ? e->w.d32 : x;
  e->rtol = rtol;
  e->maxit = maxit;
  e->hm = hm;
  e->phase = 0;
  e->total_it = e->outer = 0;
  e->bn = e->rel = 0.0;
  e->status = MF_OK;
  e->exec = nullptr;
  e->graph = nullptr;
  e->cancel = false;
  return MF_OK;
}

mf_status engine_start(SolverEngine* e) {
  mf_status st;
  const long long n = e->op->n_native;
  // the reductions find their last CTA with a counter that must start at zero (it resets
  // itself after every launch); the workspace may hold anything
  for (RedScratch* sc : {e->w.sc1, e->w.sc2, e->w.sc3})
    if ((st = cuda_check(cudaMemsetAsync(sc, 0, sizeof(unsigned) * 64, e->s), "counter clear"))) return st;
  // The FP64 solver of a double-float operator keeps its split-dual iteration's vectors in
  // double-float as well: every vector operation then runs on the FP32 pipe (GB300's FP64 pipe
  // could not keep up with HBM even for the vector updates).  b is scaled by a power of two
  // near 1/||b|| on entry and x converted back on exit.
  e->w.dinv_active = nullptr;
  if (e->precond != MF_PRECOND_NONE) e->reliable = false; // Jacobi: restarted inner CG
  if (!(e->inner_rtol > 0.0)) e->inner_rtol = e->reliable ? 0.1 : 1e-3;
  if (e->precond == MF_PRECOND_JACOBI) {
    if ((st = launch_diagonal(e->op, e->w.dinv, e->w.dtab, e->s))) return st;
    invert_diag_kernel<<<ew_blocks(n), 256, 0, e->s>>>(e->w.dinv, n);
    if ((st = cuda_check(cudaGetLastError(), "diagonal inverse"))) return st;
    e->w.dinv_active = e->w.dinv;
  }
  e->vt = e->elem_in;
  if (!e->mixed && e->elem_in == 8 && fp64_view(e->op) == VK_DD && e->form != MF_CG_ASSEMBLED && e->w.xdd) {
    e->vt = ELEM_DD;
    e->x_in = e->w.xdd;
  }
  if (!e->mixed) {
    if ((st = launch_mask(e->op, e->elem_in, e->b, e->w.q, e->s))) return st;
    return eng_inner_start(e, e->w.q, e->x_in, e->rtol, e->maxit);
  }
  if ((st = launch_mask(e->op, 8, e->b, e->w.b64, e->s))) return st;
  zero_kernel<double><<<ew_blocks(n), 256, 0, e->s>>>((double*)e->x, n);
  return eng_outer_residual(e, true);
}

static void eng_record_history(SolverEngine* e, int it) {
  if (!e->record || !g_hist_host) return;
  int take = it;
  if (take > HIST_CAP - 1) take = HIST_CAP - 1;
  if (e->hist_off + take + 1 > g_hist_cap) take = g_hist_cap - e->hist_off - 1;
  if (e->hist_off < g_hist_cap) g_hist_host[e->hist_off] = 1.0;
  if (take > 0) cudaMemcpy(g_hist_host + e->hist_off + 1, e->w.hist + 1, sizeof(double) * take, cudaMemcpyDeviceToHost);
  e->hist_off += take + 1;
}

static mf_status eng_finish(SolverEngine* e, mf_status st) {
  e->status = st;
  e->phase = PH_DONE;
  return MF_OK;
}

mf_status engine_advance(SolverEngine* e) {
  e->idle = false;
  if (e->phase == PH_DONE) return MF_OK;
  mf_status st;
  const long long n = e->op->n_native;
  if (e->phase == PH_INNER) {
    const CgState& h = e->hm->st;
    if (h.flag == 0 && !e->cancel) {
      if (!e->external) return eng_chunk(e);
      e->idle = true; // the batch runs the iterations
      return MF_OK;
    }
    eng_record_history(e, h.it);
    e->total_it += h.it;
    if (!e->mixed) {
      if (e->vt == ELEM_DD) { // x = 2^s x~
        from_dd_scaled_kernel<<<ew_blocks(n), 256, 0, e->s>>>(
            (const dd*)e->w.xdd, (double*)e->x, reinterpret_cast<const unsigned long long*>(e->w.scal + 3), n);
        if ((st = cuda_check(cudaGetLastError(), "solution conversion"))) return st;
      }
      e->rel = (h.bnorm > 0) ? std::sqrt(h.rr) / h.bnorm : 0.0;
      if (e->cancel) return eng_finish(e, MF_ERR_BUSY);
      if (h.flag == 2)
        return eng_finish(e, set_error(MF_ERR_BREAKDOWN, "CG breakdown (p^T A p <= 0 or non-finite) at iteration %d", h.it));
      return eng_finish(e, h.flag == 3 ? MF_ERR_NOT_CONVERGED : MF_OK);
    }
    if (h.flag == 2) return eng_finish(e, set_error(MF_ERR_BREAKDOWN, "inner CG breakdown at iteration %d", h.it));
    // the inner unknowns are scaled by 1/||b|| (reliable updates) or 1/||r|| of the step
    axpy64_kernel<<<ew_blocks(n), 256, 0, e->s>>>((double*)e->x, (const float*)e->w.d32,
                                                  e->w.scal + (e->reliable ? 1 : 2), n);
    e->outer += 1;
    return eng_outer_residual(e, false);
  }
  if (e->phase == PH_OUTER) {
    const double bn2 = e->hm->bn2, rn2 = e->hm->rn2;
    if (!std::isfinite(bn2) || !std::isfinite(rn2))
      return eng_finish(e, set_error(MF_ERR_BREAKDOWN, "mf_cg_solve: non-finite residual"));
    e->bn = std::sqrt(bn2);
    e->rel = e->bn > 0 ? std::sqrt(rn2) / e->bn : 0.0;
    if (e->rel <= e->rtol || e->bn == 0.0) return eng_finish(e, MF_OK);
    if (e->cancel) return eng_finish(e, MF_ERR_BUSY);
    if (e->outer >= e->max_outer || e->total_it >= e->maxit) return eng_finish(e, MF_ERR_NOT_CONVERGED);
    to32_kernel<<<ew_blocks(n), 256, 0, e->s>>>((const double*)e->w.r64, (float*)e->w.q,
                                                e->w.scal + (e->reliable ? 1 : 2), n);
    if ((st = cuda_check(cudaGetLastError(), "to32"))) return st;
    if (!e->reliable || e->outer == 0)
      return eng_inner_start(e, e->w.q, e->w.d32, e->inner_rtol, e->maxit - e->total_it);
    // reliable update: <r^, r^> and <r^, r_k+1> (the drift test), then r = r^, p = r + beta p,
    // d = 0, inner state restarted
    if ((st = dot_launch(e->op, 4, e->w.q, e->w.q, 0, e->w.scal, e->w.sc3, e->s))) return st;
    if ((st = dot_launch(e->op, 4, e->w.q, e->w.r, 0, e->w.scal + 6, e->w.sc3, e->s))) return st;
    copy_kernel<float><<<ew_blocks(n), 256, 0, e->s>>>((const float*)e->w.q, (float*)e->w.r, n);
    zero_kernel<float><<<ew_blocks(n), 256, 0, e->s>>>((float*)e->w.d32, n);
    if ((st = cuda_check(cudaGetLastError(), "reliable update"))) return st;
    reliable_state_kernel<<<1, 1, 0, e->s>>>(e->w.st, e->w.scal, e->w.scal + 6, e->inner_rtol,
                                             e->maxit - e->total_it);
    if ((st = cuda_check(cudaGetLastError(), "reliable state"))) return st;
    if (e->form == MF_CG_SPLIT_DUAL_FUSED) {
      // the fused apply forms p = r + beta p at its load
    } else if ((st = launch_cg_p(e->op, 4, e->w.r, e->w.p, nullptr, e->w.st, e->s))) {
      return st;
    }
    e->phase = PH_INNER;
    return cuda_check(cudaMemcpyAsync(&e->hm->st, e->w.st, sizeof(CgState), cudaMemcpyDeviceToHost, e->s),
                      "state D2H");
  }
  return set_error(MF_ERR_ARG, "solver engine: advance before start");
}

// ---------------------------------------------------------------- continuous batches
BatchMember engine_batch_member(const SolverEngine* e) {
  BatchMember m;
  m.op = e->op;
  m.x = e->x_in;
  m.r = e->w.r;
  m.p = e->w.p;
  m.q = e->w.q;
  m.st = e->w.st;
  m.apart = e->w.apart;
  m.sc = e->w.sc2;
  m.hist = nullptr;
  m.dinv = e->w.dinv_active;
  return m;
}

size_t batch_plan_bytes(int n, int vk) {
  return a256((size_t)n * apply_job_bytes(vk)) + a256(sizeof(long long) * (size_t)(n + 1)) +
         a256(sizeof(VecJob) * (size_t)n);
}

static int update_blocks(const mf_operator* op) {
  long long bl = (op->g.ntiles * (long long)op->n * op->n + RED_THREADS / 32 - 1) / (RED_THREADS / 32);
  if (bl > RED_MAX_BLOCKS) bl = RED_MAX_BLOCKS;
  if (bl < 1) bl = 1;
  return (int)bl;
}

mf_status batch_plan_build(BatchPlan* plan, const BatchMember* m, int n, int elem, void* dev, void* host_stage,
                           cudaStream_t s) {
  if (n <= 0) return set_error(MF_ERR_ARG, "batch: no members");
  const mf_operator* op0 = m[0].op;
  const int vk = elem == ELEM_DD ? VK_DDS : view_of_elem(op0, elem);
  for (int i = 1; i < n; ++i) {
    const mf_operator* o = m[i].op;
    if (o->n != op0->n || o->path != op0->path || o->kind != op0->kind ||
        o->variant[vk == VK_DDS ? VK_DD : vk] != op0->variant[vk == VK_DDS ? VK_DD : vk])
      return set_error(MF_ERR_ARG, "batch: members of different classes");
  }
  BatchPlan p;
  p.n = n;
  p.elem = elem;
  p.vk = vk;
  p.op0 = op0;
  p.dev = static_cast<char*>(dev);
  p.jobs_off = 0;
  p.block0_off = a256((size_t)n * apply_job_bytes(vk));
  p.vec_off = p.block0_off + a256(sizeof(long long) * (size_t)(n + 1));
  char* h = static_cast<char*>(host_stage);
  long long* block0 = reinterpret_cast<long long*>(h + p.block0_off);
  mf_status st = apply_batch_fill(m, n, vk, h + p.jobs_off, block0);
  if (st) return st;
  p.apply_blocks = block0[n];
  VecJob* vj = reinterpret_cast<VecJob*>(h + p.vec_off);
  long long up = 0, pp = 0;
  for (int i = 0; i < n; ++i) {
    const mf_operator* o = m[i].op;
    VecJob& v = vj[i];
    v.x = m[i].x;
    v.dinv = m[i].dinv;
    v.r = m[i].r;
    v.p = m[i].p;
    v.q = m[i].q;
    v.g = o->g;
    v.sc = static_cast<RedScratch*>(m[i].sc);
    v.st = m[i].st;
    v.hist = m[i].hist;
    v.apart = m[i].apart;
    v.n = o->n_native;
    v.apply_blocks = block0[i + 1] - block0[i];
    v.up0 = up;
    up += update_blocks(o);
    v.up1 = up;
    v.pp0 = pp;
    pp += ew_blocks(o->n_native);
    v.pp1 = pp;
  }
  p.up_blocks = up;
  p.pp_blocks = pp;
  if (up > 0x7fffffffLL || pp > 0x7fffffffLL) return set_error(MF_ERR_UNSUPPORTED, "batch too large");
  if ((st = cuda_check(cudaMemcpyAsync(dev, host_stage, batch_plan_bytes(n, vk), cudaMemcpyHostToDevice, s),
                       "batch descriptors H2D")))
    return st;
  *plan = p;
  return MF_OK;
}

template <int N>
static mf_status batch_vec_n(const BatchPlan& p, cudaStream_t s) {
  const VecJob* vj = reinterpret_cast<const VecJob*>(p.dev + p.vec_off);
  alpha_batch_kernel<<<p.n, 1024, 0, s>>>(vj);
  if (p.elem == 8) {
    cg_update_batch_kernel<double, N><<<(unsigned)p.up_blocks, RED_THREADS, 0, s>>>(vj, p.n);
    cg_p_batch_kernel<double><<<(unsigned)p.pp_blocks, 256, 0, s>>>(vj, p.n);
  } else if (p.elem == ELEM_DD) {
    cg_update_batch_kernel<dd, N><<<(unsigned)p.up_blocks, RED_THREADS, 0, s>>>(vj, p.n);
    cg_p_batch_kernel<dd><<<(unsigned)p.pp_blocks, 256, 0, s>>>(vj, p.n);
  } else {
    cg_update_batch_kernel<float, N><<<(unsigned)p.up_blocks, RED_THREADS, 0, s>>>(vj, p.n);
    cg_p_batch_kernel<float><<<(unsigned)p.pp_blocks, 256, 0, s>>>(vj, p.n);
  }
  return cuda_check(cudaGetLastError(), "batched CG launch");
}

mf_status batch_iteration(const BatchPlan& p, cudaStream_t s) {
  mf_status st = apply_batch_launch(p.op0, p.vk, p.dev + p.jobs_off, reinterpret_cast<const long long*>(p.dev + p.block0_off),
                                    p.n, p.apply_blocks, s);
  if (st) return st;
  MF_SWITCH_N(p.op0->n, batch_vec_n, p, s);
}

__global__ void gather_states_kernel(const VecJob* __restrict__ jobs, int n, CgState* __restrict__ out) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = *jobs[i].st;
}
mf_status batch_gather_states(const BatchPlan& p, CgState* states_dev, cudaStream_t s) {
  gather_states_kernel<<<1, 256, 0, s>>>(reinterpret_cast<const VecJob*>(p.dev + p.vec_off), p.n, states_dev);
  return cuda_check(cudaGetLastError(), "state gather");
}

void engine_release(SolverEngine* e) {
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->graph) cudaGraphDestroy(e->graph);
  e->exec = nullptr;
  e->graph = nullptr;
}

} // namespace mf

using namespace mf;

extern "C" {

size_t mf_reduce_workspace_bytes(const mf_operator* op) { return op ? sizeof(RedScratch) : 0; }

mf_status mf_dot(const mf_operator* op, const void* a_dev, const void* b_dev, int split, double* result_dev,
                 void* scratch_dev, size_t scratch_bytes, void* stream) {
  if (!op || !a_dev || !b_dev || !result_dev) return set_error(MF_ERR_ARG, "mf_dot: NULL argument");
  if (!scratch_dev || scratch_bytes < sizeof(RedScratch))
    return set_error(MF_ERR_OOM, "mf_dot: scratch %zu < %zu bytes", scratch_bytes, sizeof(RedScratch));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mf_status st = cuda_check(cudaMemsetAsync(scratch_dev, 0, sizeof(unsigned) * 64, s), "mf_dot memset");
  if (st) return st;
  return dot_launch(op, op->precision == MF_FP32 ? 4 : 8, a_dev, b_dev, split ? 1 : 0, result_dev, scratch_dev, s);
}

mf_status mf_cg_record_history(double* hist_host, int cap) {
  g_hist_host = hist_host;
  g_hist_cap = hist_host ? cap : 0;
  return MF_OK;
}

size_t mf_cg_workspace_bytes(const mf_operator* op, int mixed) {
  if (!op) return 0;
  return solve_ws_layout(op, mixed ? 1 : 0, nullptr, nullptr);
}

size_t mf_cg_workspace_bytes_ex(const mf_operator* op, int mixed, const mf_solve_options* opts) {
  if (!op) return 0;
  if (opts && opts->precond == MF_PRECOND_CHEBYSHEV) return cheb_workspace_bytes(op);
  return mf_cg_workspace_bytes(op, mixed);
}

mf_status mf_cg_solve(const mf_operator* op, const void* b_dev, void* x_dev, double rtol, int maxit, int mixed,
                      mf_solve_stats* stats, void* workspace_dev, size_t bytes, void* stream) {
  return mf_cg_solve_ex(op, b_dev, x_dev, rtol, maxit, mixed, nullptr, stats, workspace_dev, bytes, stream);
}

static size_t host_align(size_t b) { return (b + 255) & ~size_t(255); }

size_t mf_cg_solve_host_workspace_bytes(const mf_operator* op, int mixed) {
  if (!op) return 0;
  const size_t e = op->precision == MF_FP32 ? 4 : 8;
  return host_align(mf_cg_workspace_bytes(op, mixed)) + 2 * host_align((size_t)op->n_native * e) +
         host_align((size_t)op->n_cellwise * e);
}

mf_status mf_cg_solve_host(const mf_operator* op, const void* b_host, void* x_host, double rtol, int maxit, int mixed,
                           mf_solve_stats* stats, void* workspace_dev, size_t bytes, void* stream) {
  if (!op || !b_host || !x_host) return set_error(MF_ERR_ARG, "mf_cg_solve_host: NULL argument");
  if (!op->ready) return set_error(MF_ERR_ARG, "mf_cg_solve_host: operator not set up");
  const size_t need = mf_cg_solve_host_workspace_bytes(op, mixed);
  if (!workspace_dev || bytes < need) return set_error(MF_ERR_OOM, "mf_cg_solve_host: workspace %zu < %zu", bytes, need);
  if (reinterpret_cast<uintptr_t>(workspace_dev) & 255)
    return set_error(MF_ERR_ARG, "mf_cg_solve_host: workspace alignment");
  const size_t e = op->precision == MF_FP32 ? 4 : 8;
  const size_t cgb = host_align(mf_cg_workspace_bytes(op, mixed)), nb = host_align((size_t)op->n_native * e);
  char* w = static_cast<char*>(workspace_dev);
  void* bn = w + cgb;
  void* xn = w + cgb + nb;
  void* can = w + cgb + 2 * nb;
  const size_t cbytes = (size_t)op->n_cellwise * e;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mf_status st = cuda_check(cudaMemcpyAsync(can, b_host, cbytes, cudaMemcpyHostToDevice, s), "mf_cg_solve_host H2D");
  if (st) return st;
  if ((st = mf_to_native(op, can, bn, stream))) return st;
  const mf_status solve = mf_cg_solve_ex(op, bn, xn, rtol, maxit, mixed, nullptr, stats, w, cgb, stream);
  if (solve != MF_OK && solve != MF_ERR_NOT_CONVERGED && solve != MF_ERR_BREAKDOWN) return solve;
  if ((st = mf_from_native(op, xn, can, stream))) return st;
  if ((st = cuda_check(cudaMemcpyAsync(x_host, can, cbytes, cudaMemcpyDeviceToHost, s), "mf_cg_solve_host D2H")))
    return st;
  if ((st = cuda_check(cudaStreamSynchronize(s), "mf_cg_solve_host sync"))) return st;
  return solve;
}

mf_status mf_cg_solve_ex(const mf_operator* op, const void* b_dev, void* x_dev, double rtol, int maxit, int mixed,
                         const mf_solve_options* opts, mf_solve_stats* stats, void* workspace_dev, size_t bytes,
                         void* stream) {
  if (!op || !b_dev || !x_dev) return set_error(MF_ERR_ARG, "mf_cg_solve: NULL argument");
  if (opts && ((opts->inner_rtol != 0.0 && !(opts->inner_rtol > 0.0 && opts->inner_rtol < 1.0)) ||
               opts->chunk_iterations < 0 || opts->max_outer < 0 || opts->cg_form < 0 ||
               opts->cg_form > MF_CG_SPLIT_DUAL_FUSED || opts->precond < 0 || opts->precond > MF_PRECOND_CHEBYSHEV ||
               (opts->precond == MF_PRECOND_JACOBI && opts->cg_form > MF_CG_SPLIT_DUAL) ||
               opts->mixed_restart < 0 || opts->mixed_restart > 1 || opts->reserved != 0 ||
               (opts->precond == MF_PRECOND_CHEBYSHEV && (mixed || opts->cheb_ratio < 0.0 ||
                                                         (opts->cheb_ratio != 0.0 && !(opts->cheb_ratio > 1.0))))))
    return set_error(MF_ERR_ARG, "mf_cg_solve_ex: bad options");
  if (!op->ready) return set_error(MF_ERR_ARG, "mf_cg_solve: operator not set up");
  if (maxit < 0 || !(rtol >= 0.0)) return set_error(MF_ERR_ARG, "mf_cg_solve: bad rtol/maxit");
  if (mixed && op->precision != MF_MIXED) return set_error(MF_ERR_ARG, "mf_cg_solve: mixed needs an MF_MIXED operator");
  if (opts && opts->precond == MF_PRECOND_CHEBYSHEV) {
    if (!workspace_dev || (reinterpret_cast<uintptr_t>(workspace_dev) & 255))
      return set_error(MF_ERR_ARG, "mf_cg_solve: workspace NULL or not 256-byte aligned");
    const auto t0 = std::chrono::steady_clock::now();
    mf_solve_stats local;
    mf_solve_stats* sp = stats ? stats : &local;
    std::memset(sp, 0, sizeof(*sp));
    mf_status rc = cheb_solve(op, b_dev, x_dev, rtol, maxit, opts->cheb_ratio, sp, workspace_dev, bytes,
                              static_cast<cudaStream_t>(stream));
    sp->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return rc;
  }
  const size_t need = mf_cg_workspace_bytes(op, mixed);
  if (!workspace_dev || bytes < need) return set_error(MF_ERR_OOM, "mf_cg_solve: workspace %zu < %zu", bytes, need);
  if (reinterpret_cast<uintptr_t>(workspace_dev) & 255) return set_error(MF_ERR_ARG, "mf_cg_solve: workspace alignment");
  // CUDA graph capture is not allowed on the legacy default stream: run on a private
  // blocking stream (implicitly ordered with the legacy stream) when none is given.
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStream_t own = nullptr;
  if (s == nullptr) {
    mf_status cs = cuda_check(cudaStreamCreateWithFlags(&own, cudaStreamDefault), "mf_cg_solve stream");
    if (cs) return cs;
    s = own;
  }
  struct StreamGuard {
    cudaStream_t st;
    ~StreamGuard() {
      if (st) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
    }
  } guard{own};
  const auto t0 = std::chrono::steady_clock::now();
  HostMirror hm;
  std::memset(&hm, 0, sizeof(hm));
  SolverEngine e;
  engine_init(&e, op, mixed ? 1 : 0, b_dev, x_dev, rtol, maxit, workspace_dev, s, &hm);
  if (opts) {
    if (opts->inner_rtol > 0.0) e.inner_rtol = opts->inner_rtol;
    if (opts->chunk_iterations > 0) e.chunk = opts->chunk_iterations;
    if (opts->max_outer > 0) e.max_outer = opts->max_outer;
    if (opts->cg_form != MF_CG_DEFAULT) e.form = opts->cg_form;
    e.precond = opts->precond;
    e.reliable = opts->mixed_restart == 0;
  }
  e.record = g_hist_host != nullptr;
  mf_status st = engine_start(&e);
  // every advance either finishes or moves the iteration count forward by a chunk; bound the
  // host loop anyway so that a device state that stops changing cannot spin it forever
  const long long max_steps = 2LL * ((long long)maxit / e.chunk + 2) * (e.max_outer + 2) + 16;
  long long steps = 0;
  while (st == MF_OK && e.phase != PH_DONE) {
    if ((st = cuda_check(cudaStreamSynchronize(s), "mf_cg_solve sync"))) break;
    if (++steps > max_steps) {
      st = set_error(MF_ERR_TIMEOUT, "mf_cg_solve: no progress after %lld steps", steps);
      break;
    }
    st = engine_advance(&e);
  }
  engine_release(&e);
  cudaStreamSynchronize(s);
  if (st == MF_OK) st = e.status;
  mf_solve_stats out;
  std::memset(&out, 0, sizeof(out));
  out.iterations = e.total_it;
  out.outer_iterations = mixed ? e.outer : 1;
  out.rel_residual = e.rel;
  out.check_every = e.chunk;
  out.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  out.status = st;
  if (stats) *stats = out;
  if (st == MF_ERR_NOT_CONVERGED) set_error(st, "mf_cg_solve: not converged after %d iterations", out.iterations);
  return st;
}

mf_status mf_cg_profile(const mf_operator* op, const void* b_dev, void* x_dev, int iterations, int cg_form,
                        void* workspace_dev, size_t bytes, void* stream, double* ms_out) {
  if (!op || !b_dev || !x_dev || !ms_out) return set_error(MF_ERR_ARG, "mf_cg_profile: NULL argument");
  if (!op->ready) return set_error(MF_ERR_ARG, "mf_cg_profile: operator not set up");
  if (iterations < 1 || iterations > 1000 || cg_form < 0 || cg_form > MF_CG_SPLIT_DUAL_FUSED)
    return set_error(MF_ERR_ARG, "mf_cg_profile: iterations must be in [1, 1000], cg_form an MF_CG_* value");
  const size_t need = mf_cg_workspace_bytes(op, 0);
  if (!workspace_dev || bytes < need) return set_error(MF_ERR_OOM, "mf_cg_profile: workspace %zu < %zu", bytes, need);
  if (reinterpret_cast<uintptr_t>(workspace_dev) & 255) return set_error(MF_ERR_ARG, "mf_cg_profile: workspace alignment");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  HostMirror hm;
  std::memset(&hm, 0, sizeof(hm));
  SolverEngine e;
  // one untimed iteration first: it loads the kernels (lazy module loading) and warms the caches
  engine_init(&e, op, 0, b_dev, x_dev, 0.0, iterations + 1, workspace_dev, s, &hm);
  if (cg_form != MF_CG_DEFAULT) e.form = cg_form;
  mf_status st = engine_start(&e);
  if (st) return st;
  std::vector<cudaEvent_t> ev(4 * (size_t)iterations, nullptr);
  for (auto& x : ev)
    if ((st = cuda_check(cudaEventCreate(&x), "mf_cg_profile event"))) break;
  const int el = e.vt;
  for (int it = -1; it < iterations && st == MF_OK; ++it) {
    cudaEvent_t* E = &ev[4 * (size_t)(it < 0 ? 0 : it)];
    if (it == 0 && (st = cuda_check(cudaStreamSynchronize(s), "mf_cg_profile warm-up"))) break;
    cudaEventRecord(E[0], s);
    if (e.form != MF_CG_ASSEMBLED) {
      const int fp = e.form == MF_CG_SPLIT_DUAL_FUSED;
      st = launch_apply_alpha(op, el, e.w.p, e.w.r, e.w.q, e.w, e.w.st, fp, s);
      cudaEventRecord(E[1], s);
      cudaEventRecord(E[2], s);
      if (st == MF_OK) st = launch_cg_update(op, el, e.x_in, e.w.r, e.w.p, e.w.q, e.w, e.w.st, nullptr, s);
      if (st == MF_OK && !fp) st = launch_cg_p(op, el, e.w.r, e.w.p, e.w.dinv_active, e.w.st, s);
    } else {
      st = launch_apply_split(op, view_of_elem(op, el), e.w.p, e.w.q, s);
      cudaEventRecord(E[1], s);
      if (st == MF_OK) st = launch_dss(op, el, e.w.q, s);
      cudaEventRecord(E[2], s);
      if (st == MF_OK)
        st = launch_cg_vec(op, el, e.x_in, e.w.r, e.w.p, e.w.q, e.w.sc1, e.w.sc2, e.w.st, nullptr, s);
    }
    cudaEventRecord(E[3], s);
  }
  if (st == MF_OK) st = cuda_check(cudaStreamSynchronize(s), "mf_cg_profile sync");
  double acc[4] = {0, 0, 0, 0};
  for (int it = 0; it < iterations && st == MF_OK; ++it) {
    cudaEvent_t* E = &ev[4 * (size_t)it];
    float a = 0, b = 0, c = 0, d = 0;
    cudaEventElapsedTime(&a, E[0], E[1]);
    cudaEventElapsedTime(&b, E[1], E[2]);
    cudaEventElapsedTime(&c, E[2], E[3]);
    cudaEventElapsedTime(&d, E[0], E[3]);
    acc[0] += a; acc[1] += b; acc[2] += c; acc[3] += d;
  }
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  if (st) return st;
  for (int i = 0; i < 4; ++i) ms_out[i] = acc[i] / iterations;
  if (e.form != MF_CG_ASSEMBLED) ms_out[1] = 0.0;
  return MF_OK;
}

} // extern "C"
