// mf_dd.cuh -- double-float ("dd") arithmetic: a value is the unevaluated sum hi + lo of two
// floats (about 48 significant bits).  GB300's FP32 pipe issues 64x more FMAs per clock than
// its FP64 pipe, so FP64-accurate sum factorisation runs faster in dd than in native double.
//
// Building blocks are the classical error-free transformations: Knuth's TwoSum
// (s + e = a + b exactly) and the FMA-based TwoProd (p + e = a * b exactly, e = fma(a, b, -p)).
// fma() below accumulates a*b + c without renormalising; finish() renormalises a chain result
// with Dekker's FastTwoSum.  Conversions to and from double split the IEEE bit pattern with
// integer operations, so the hot loop issues no FP64 instruction except one add per stored
// value.
#pragma once
#include <cstring>

#include <cuda_runtime.h>

namespace mf {

// bit casts that also compile for the host (the conversions below are tested on the CPU)
__host__ __device__ __forceinline__ unsigned fbits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned u;
  std::memcpy(&u, &f, sizeof(u));
  return u;
#endif
}
__host__ __device__ __forceinline__ double dbl_of_bits(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  std::memcpy(&d, &b, sizeof(d));
  return d;
#endif
}

struct __align__(8) dd {
  float hi, lo;
  __host__ __device__ dd() {}
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit constexpr dd(int v) : hi((float)v), lo(0.0f) {}
};

// Native overloads so that unqualified fma() inside namespace mf also serves double / float.
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }

// a*b + c.  TwoProd of the leading parts, first-order cross terms, TwoSum with c.hi; the
// rounding errors collect in lo (not renormalised: call finish() at the end of a chain).
__device__ __forceinline__ dd fma(dd a, dd b, dd c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float s = c.hi + p;
  const float v = s - c.hi;
  const float t = (c.hi - (s - v)) + (p - v);
  return dd(s, t + (c.lo + e));
}

// a*b as the first term of a chain: TwoProd of the leading parts plus the cross terms, not
// renormalised (an fma() into a zero accumulator would spend a TwoSum on the zero).
__device__ __forceinline__ dd mul0(dd a, dd b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return dd(p, e);
}
__device__ __forceinline__ double mul0(double a, double b) { return a * b; }
__device__ __forceinline__ float mul0(float a, float b) { return a * b; }

__device__ __forceinline__ dd finish(dd a) {
  const float h = a.hi + a.lo;
  return dd(h, a.lo - (h - a.hi));
}
__device__ __forceinline__ double finish(double a) { return a; }
__device__ __forceinline__ float finish(float a) { return a; }

__device__ __forceinline__ dd operator*(dd a, dd b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return finish(dd(p, e));
}

__host__ __device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }

__device__ __forceinline__ dd operator+(dd a, dd b) {
  const float s = a.hi + b.hi;
  const float v = s - a.hi;
  const float t = (a.hi - (s - v)) + (b.hi - v);
  return finish(dd(s, t + (a.lo + b.lo)));
}

// double -> dd: hi keeps the leading 24 significant bits (truncated), lo the remaining 29
// bits rounded to 24.  Magnitudes below 2^-126 flush to zero; inf/nan go through hi.
__device__ __forceinline__ dd dd_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi32 = (unsigned)(b >> 32), lo32 = (unsigned)b;
  const int e = (int)((hi32 >> 20) & 0x7ffu);
  const unsigned sign = hi32 & 0x80000000u;
  const int ef = e - 896; // float biased exponent of the same power of two
  if (e == 0x7ff) return dd(__double2float_rn(x), 0.0f);
  if (ef <= 0) return dd(0.0f, 0.0f);
  if (ef >= 255) return dd(__uint_as_float(sign | 0x7f800000u), 0.0f);
  const unsigned mant = ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);
  const float h = __uint_as_float(sign | ((unsigned)ef << 23) | mant);
  const unsigned r = lo32 & 0x1fffffffu;
  const int es = e - 948; // float biased exponent of 2^(e - 1075)
  float l = (es > 0) ? __uint2float_rn(r) * __uint_as_float((unsigned)es << 23) : 0.0f;
  return dd(h, sign ? -l : l);
}

// float -> double by bit manipulation (normal numbers; zero and subnormals give zero).
__host__ __device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = fbits(f);
  const unsigned ex = (u >> 23) & 0xffu;
  if (ex == 0u) return 0.0;
  if (ex == 0xffu) return (double)f;
  const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long de = (unsigned long long)(ex - 127u + 1023u) << 52;
  const unsigned long long m = (unsigned long long)(u & 0x7fffffu) << 29;
  return dbl_of_bits(s | de | m);
}

// dd -> double: exact sum of the two parts (one FP64 add, rounded to nearest).  A subnormal lo
// flushes to zero, as in dd_from_double.  (An integer-only form of this conversion, lo added
// as a count of ulps of hi's double, was measured: 20 integer instructions cost the
// issue-bound apply kernels more than the FP64 add, 3-6%.)
__host__ __device__ __forceinline__ double dd_to_double(dd a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

// Two FP32 values of neighbouring cells processed by one thread (the FP32 apply): every
// operation acts on both lanes; table coefficients stay scalar floats.
struct __align__(8) f2 {
  float x, y;
  __host__ __device__ f2() {}
  __host__ __device__ constexpr f2(float a, float b) : x(a), y(b) {}
  __host__ __device__ explicit constexpr f2(int v) : x((float)v), y((float)v) {}
};
__device__ __forceinline__ f2 fma(float c, f2 a, f2 b) { return f2(fmaf(c, a.x, b.x), fmaf(c, a.y, b.y)); }
__device__ __forceinline__ f2 fma(f2 c, f2 a, f2 b) { return f2(fmaf(c.x, a.x, b.x), fmaf(c.y, a.y, b.y)); }
__device__ __forceinline__ f2 mul0(float c, f2 a) { return f2(c * a.x, c * a.y); }
__device__ __forceinline__ f2 mul0(f2 c, f2 a) { return f2(c.x * a.x, c.y * a.y); }
__device__ __forceinline__ f2 finish(f2 a) { return a; }
__device__ __forceinline__ f2 operator*(float c, f2 a) { return f2(c * a.x, c * a.y); }
__device__ __forceinline__ f2 operator*(f2 c, f2 a) { return f2(c.x * a.x, c.y * a.y); }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ f2 operator-(f2 a) { return f2(-a.x, -a.y); }

// Coefficient type of the 1D tables for a compute type, and cells per compute value.
template <typename T>
struct CoefOf { using type = T; };
template <>
struct CoefOf<f2> { using type = float; };
template <typename T>
struct CellsPer { static constexpr int value = 1; };
template <>
struct CellsPer<f2> { static constexpr int value = 2; };
template <typename T>
struct IsF32 { static constexpr bool value = false; };
template <>
struct IsF32<float> { static constexpr bool value = true; };
template <>
struct IsF32<f2> { static constexpr bool value = true; };

// Compute type of the FP32 view: pairs of cells per thread (MF_FP32_PAIRS=0: one cell).
#ifndef MF_FP32_PAIRS
#define MF_FP32_PAIRS 1
#endif
#if MF_FP32_PAIRS
using FP32C = f2;
#else
using FP32C = float;
#endif

// A double scalar (a CG coefficient) in a vector element type.
template <typename S>
__device__ __forceinline__ S scalar_from_double(double v) { return (S)v; }
template <>
__device__ __forceinline__ dd scalar_from_double<dd>(double v) { return dd_from_double(v); }

// storage <-> compute conversions used by the kernels
template <typename C, typename S>
__device__ __forceinline__ C to_compute(S v) { return (C)v; }
template <>
__device__ __forceinline__ dd to_compute<dd, double>(double v) { return dd_from_double(v); }

template <typename S, typename C>
__device__ __forceinline__ S to_storage(C v) { return (S)v; }
template <>
__device__ __forceinline__ double to_storage<double, dd>(dd v) { return dd_to_double(v); }

// host: double -> compute type
template <typename C>
inline C host_from_double(double v) { return (C)v; }
template <>
inline f2 host_from_double<f2>(double v) { return f2((float)v, (float)v); }
template <>
inline dd host_from_double<dd>(double v) {
  const float h = (float)v;
  return dd(h, (float)(v - (double)h));
}

} // namespace mf
