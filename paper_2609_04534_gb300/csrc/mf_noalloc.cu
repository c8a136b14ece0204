// mf_noalloc.cu -- mf_dot_noalloc: the assembled dot product of mf_dot without any
// caller-provided scratch and without any allocation.
//
// Why it exists: some callers of this library cannot allocate device memory at the point
// where they need a reduction -- for example a solver embedded in a host application whose
// device memory is owned by another allocator (a framework's caching pool or a fixed arena
// it must not bypass), or a time-critical loop that must not call cudaMalloc because an
// allocation may synchronise the whole device.  For them the reduction scratch (one FP64
// partial per CTA plus a done-counter) lives in a file-scope static device array instead.
//
// Limits and behaviour:
//  - Each CTA reduces a fixed chunk of 2048 elements, so the reduction needs
//    ceil(n_native / 2048) partials; the static array holds 65536 of them (512 KiB + 256 B,
//    held by every GPU that loads the library until the process exits).  Vectors longer than
//    65536 * 2048 = 134,217,728 elements are rejected with MF_ERR_ARG before any GPU work.
//  - An operator that has not been set up is rejected (after the size check, before any
//    CUDA call), so a call with a bad operator never reaches a launch.
//  - The first successful call on each device resolves the array's device address with
//    cudaGetSymbolAddress while that device is current and caches it per device; later calls
//    on that device reuse it.  A failed lookup is not cached: the next call retries it.  Make
//    that first call before any stream capture.  The cached address is invalid after
//    cudaDeviceReset (the module, and with it the array, is reloaded).
//  - Every call shares the one array: the done-counter is cleared (cudaMemsetAsync) at the
//    start of each call, and the partials are rewritten before they are read.  Calls whose
//    executions overlap on the GPU (on different streams, or on different host threads)
//    race on the array and give wrong results; serialise them.
//  - No cudaMalloc, cudaFree or allocating library routine is called.
#include <mutex>

#include "mf_internal.h"

namespace mf {
namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PER_THREAD = 8;
constexpr long long NA_CHUNK = (long long)NA_THREADS * NA_PER_THREAD;
constexpr int NA_MAX_PARTIALS = 65536;

struct NoAllocScratch {
  unsigned int counter;
  unsigned int pad[63];
  double partial[NA_MAX_PARTIALS];
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int NA_MAX_DEVICES = 64;
NoAllocScratch* g_scratch_ptr[NA_MAX_DEVICES]; // resolved addresses (null: not resolved yet)
std::mutex g_scratch_mu;

// The array's device address on the current device `dev`, resolved on first use; only a
// successful lookup is cached.
cudaError_t scratch_address(int dev, NoAllocScratch** out) {
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (!p) return cudaErrorInvalidSymbol;
    g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Weight of native element e in the assembled pairing: 1/multiplicity of its node (exact,
// a power of two), 1 for every real copy when split, 0 for padding lanes.
template <int N>
__device__ __forceinline__ double na_weight(const GridInfo& g, long long e, int split) {
  constexpr int N2 = N * N, N3 = N2 * N;
  const int lane = (int)(e & (BL - 1));
  const long long row = e >> 5;
  const int l = (int)(row % N3);
  const int t = (int)(row / N3);
  const int txy = g.ntx * g.nty;
  const int tz = t / txy, r = t - tz * txy, ty = r / g.ntx, tx = r - ty * g.ntx;
  const int cx = tx * TX + (lane & 3), cy = ty * TY + ((lane >> 2) & 3), cz = tz * TZ + (lane >> 4);
  if (cx >= g.nx || cy >= g.ny || cz >= g.nz) return 0.0;
  if (split) return 1.0;
  const int i = l % N, j = (l / N) % N, k = l / N2;
  const int m = (((i == 0 && cx > 0) || (i == N - 1 && cx < g.nx - 1)) ? 2 : 1) *
                (((j == 0 && cy > 0) || (j == N - 1 && cy < g.ny - 1)) ? 2 : 1) *
                (((k == 0 && cz > 0) || (k == N - 1 && cz < g.nz - 1)) ? 2 : 1);
  return 1.0 / m;
}

__device__ __forceinline__ double na_block_sum(double v) {
  __shared__ double ws[NA_THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  if (ln == 0) ws[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = (ln < NA_THREADS / 32) ? ws[ln] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  __syncthreads();
  return s;
}

template <typename T, int N>
__global__ void __launch_bounds__(NA_THREADS) dot_noalloc_kernel(const T* __restrict__ a, const T* __restrict__ b,
                                                                 long long n, GridInfo g, int split,
                                                                 NoAllocScratch* sc, double* out) {
  const long long base = blockIdx.x * NA_CHUNK;
  double s = 0.0;
#pragma unroll
  for (int r = 0; r < NA_PER_THREAD; ++r) {
    const long long e = base + (long long)r * NA_THREADS + threadIdx.x;
    if (e < n) s += na_weight<N>(g, e, split) * ((double)a[e] * (double)b[e]);
  }
  s = na_block_sum(s);
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    sc->partial[blockIdx.x] = s;
    __threadfence();
    am_last = (atomicAdd(&sc->counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += NA_THREADS) t += ((volatile double*)sc->partial)[i];
  t = na_block_sum(t);
  if (threadIdx.x == 0) {
    *out = t;
    sc->counter = 0;
  }
}

template <int N>
mf_status na_launch(const mf_operator* op, int elem, const void* a, const void* b, int split, double* out,
                    NoAllocScratch* sc, unsigned blocks, cudaStream_t s) {
  if (elem == 8)
    dot_noalloc_kernel<double, N><<<blocks, NA_THREADS, 0, s>>>((const double*)a, (const double*)b, op->n_native,
                                                                op->g, split, sc, out);
  else
    dot_noalloc_kernel<float, N><<<blocks, NA_THREADS, 0, s>>>((const float*)a, (const float*)b, op->n_native,
                                                               op->g, split, sc, out);
  return cuda_check(cudaGetLastError(), "mf_dot_noalloc launch");
}

} // namespace
} // namespace mf

using namespace mf;

extern "C" mf_status mf_dot_noalloc(const mf_operator* op, const void* a_dev, const void* b_dev, int split,
                                    double* result_dev, void* stream) {
  if (!op || !a_dev || !b_dev || !result_dev) return set_error(MF_ERR_ARG, "mf_dot_noalloc: NULL argument");
  const long long blocks = (op->n_native + NA_CHUNK - 1) / NA_CHUNK;
  if (blocks > NA_MAX_PARTIALS)
    return set_error(MF_ERR_ARG,
                     "mf_dot_noalloc: vector of %lld elements exceeds the %lld-element limit of the static "
                     "reduction scratch (use mf_dot with caller scratch)",
                     op->n_native, (long long)NA_MAX_PARTIALS * NA_CHUNK);
  if (blocks == 0) return set_error(MF_ERR_ARG, "mf_dot_noalloc: empty vector");
  if (!op->ready) return set_error(MF_ERR_ARG, "mf_dot_noalloc: operator not set up (mf_operator_setup)");
  int dev = -1;
  mf_status st = cuda_check(cudaGetDevice(&dev), "mf_dot_noalloc: cudaGetDevice");
  if (st) return st;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return set_error(MF_ERR_ARG, "mf_dot_noalloc: device %d not supported", dev);
  NoAllocScratch* sc = nullptr;
  if ((st = cuda_check(scratch_address(dev, &sc), "mf_dot_noalloc: cudaGetSymbolAddress"))) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = cuda_check(cudaMemsetAsync(&sc->counter, 0, sizeof(unsigned int), s), "mf_dot_noalloc: clear counter")))
    return st;
  const int elem = op->precision == MF_FP32 ? 4 : 8;
  const unsigned nb = (unsigned)blocks;
  const int sp = split ? 1 : 0;
  switch (op->n) {
    case 2: return na_launch<2>(op, elem, a_dev, b_dev, sp, result_dev, sc, nb, s);
    case 3: return na_launch<3>(op, elem, a_dev, b_dev, sp, result_dev, sc, nb, s);
    case 4: return na_launch<4>(op, elem, a_dev, b_dev, sp, result_dev, sc, nb, s);
    case 5: return na_launch<5>(op, elem, a_dev, b_dev, sp, result_dev, sc, nb, s);
    case 6: return na_launch<6>(op, elem, a_dev, b_dev, sp, result_dev, sc, nb, s);
    case 7: return na_launch<7>(op, elem, a_dev, b_dev, sp, result_dev, sc, nb, s);
    case 8: return na_launch<8>(op, elem, a_dev, b_dev, sp, result_dev, sc, nb, s);
    case 9: return na_launch<9>(op, elem, a_dev, b_dev, sp, result_dev, sc, nb, s);
    default: return set_error(MF_ERR_UNSUPPORTED, "mf_dot_noalloc: n=%d not built", op->n);
  }
}
