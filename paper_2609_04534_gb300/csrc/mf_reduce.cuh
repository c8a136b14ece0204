// mf_reduce.cuh -- per-thread accumulators and fixed-order block / grid reductions shared by
// the CG vector kernels and the apply kernel's fused CG epilogue.  Every reduction here sums
// in an order that depends only on the launch shape, never on timing, so scalars are bitwise
// reproducible.
#pragma once
#include <cuda_runtime.h>

#include "mf_dd.cuh"

namespace mf {

// Per-thread accumulation of w a b (w = 1/multiplicity, a power of two, so scaling by it is
// exact).  GB300 issues 64x fewer FP64 than FP32 instructions, and a bandwidth-bound vector
// kernel that spent two FP64 operations per element on its dot product would be bound by the
// FP64 pipe instead of HBM; so products are formed and summed on the FP32 pipe: each operand
// is split into float parts by integer bit operations, the leading product is exact by
// TwoProd, the first-order cross terms are added, and the thread's sum is kept in
// double-float (TwoSum on the leading part).  About 2^-44 relative per product, far below
// what the CG scalars need.  Operands outside [2^-60, 2^60] in magnitude (where the float
// parts or their products would leave the float range) take an FP64 FMA instead, so the
// double range is kept.  The thread's value enters the FP64 block reduction once.
struct AccD {
  float hi = 0.0f, lo = 0.0f;
  double wide = 0.0;
  __device__ __forceinline__ void add2(float pw, float ew) {
    const float s = hi + pw;
    const float v = s - hi;
    const float t = (hi - (s - v)) + (pw - v);
    hi = s;
    lo += t + ew;
  }
  // biased exponent of a double within [1023 - 60, 1023 + 60]
  __device__ __forceinline__ static bool in_window(double a) {
    const unsigned e = ((unsigned)__double2hiint(a) >> 20) & 0x7ffu;
    return e - 963u <= 120u;
  }
  __device__ __forceinline__ void add(float w, double a, double b) {
    if (in_window(a) && in_window(b)) {
      const dd x = dd_from_double(a), y = dd_from_double(b);
      const float p = x.hi * y.hi;
      float e = fmaf(x.hi, y.hi, -p);
      e = fmaf(x.hi, y.lo, e);
      e = fmaf(x.lo, y.hi, e);
      add2(p * w, e * w);
    } else if ((__double_as_longlong(a) << 1) != 0 && (__double_as_longlong(b) << 1) != 0) { // both nonzero
      wide = ::fma((double)w * a, b, wide);
    }
  }
  __device__ __forceinline__ void add(double a, double b) { add(1.0f, a, b); }
  __device__ __forceinline__ double value() const { return ((double)hi + (double)lo) + wide; }
};
struct AccF {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add2(float pw, float ew) {
    const float s = hi + pw;
    const float v = s - hi;
    const float t = (hi - (s - v)) + (pw - v);
    hi = s;
    lo += t + ew;
  }
  __device__ __forceinline__ void add(float w, float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    add2(p * w, e * w);
  }
  __device__ __forceinline__ void add(float a, float b) { add(1.0f, a, b); }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
// Double-float operands (the FP64 solver's vectors): the same exact leading product and
// first-order cross terms, summed in double-float.
struct AccDD {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float w, dd a, dd b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float pw = p * w, ew = e * w;
    const float s = hi + pw;
    const float v = s - hi;
    const float t = (hi - (s - v)) + (pw - v);
    hi = s;
    lo += t + ew;
  }
  __device__ __forceinline__ void add(dd a, dd b) { add(1.0f, a, b); }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
template <typename T>
struct AccOf;
template <>
struct AccOf<double> { using type = AccD; };
template <>
struct AccOf<float> { using type = AccF; };
template <>
struct AccOf<dd> { using type = AccDD; };

// Sum of v over the CTA in a fixed order for any block size of at least 32 threads: every
// thread parks its value in park[threadIdx.x] (blockDim.x doubles of shared memory), warp 0
// folds the park with stride 32 and then by a shuffle tree.  Result valid in thread 0.  Ends
// with a barrier, so park may be reused afterwards.
__device__ __forceinline__ double block_park_sum(double v, double* park) {
  park[threadIdx.x] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    for (int i = threadIdx.x; i < (int)blockDim.x; i += 32) s += park[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  __syncthreads();
  return s;
}

} // namespace mf
