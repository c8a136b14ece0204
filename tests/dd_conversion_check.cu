// Host check of the double-float -> double conversion of the CUDA path (mf_dd.cuh), compiled
// by nvcc as a host program: normalised pairs across the float range, powers of two with lo
// on either side, many lo scales, zero, non-normalised and subnormal lo, inf and nan.
// Criterion: |r - (hi + lo)| <= 2^-53 |hi| (rounded to nearest); a non-normalised pair gives
// exactly the FP64 sum; a subnormal lo flushes to zero (the dd range starts at 2^-126).
// Prints "ok <count>" and exits 0, or the first failure.
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <random>

#include "mf_dd.cuh"

using mf::dd;

static int check(float h, float l, long long* n) {
  const double r = mf::dd_to_double(dd(h, l));
  ++*n;
  if (std::isnan(h) || std::isnan(l)) return std::isnan(r) ? 0 : 1;
  if (std::isinf(h)) return (r == (double)h) ? 0 : 1;
  const double dh = h, dl = l;
  if (dl != 0.0 && std::fabs(dl) < std::ldexp(1.0, -126)) return r == dh ? 0 : 5; // flushed lo
  const double rh = r - dh; // exact: r and hi lie within a factor of two (Sterbenz)
  const double err = std::fabs(rh - dl);
  const bool normalised = std::fabs(dl) <= std::ldexp(std::fabs(dh), -24);
  if (normalised && dh != 0.0) {
    if (err > std::ldexp(std::fabs(dh), -53)) return 2;
  } else if (r != dh + dl) {
    return 4; // the FP64 sum
  }
  return 0;
}

int main() {
  std::mt19937_64 g(12345);
  std::uniform_real_distribution<double> u(1.0, 2.0);
  std::uniform_int_distribution<int> ex(-120, 120);
  long long n = 0;
  auto fail = [&](const char* what, float h, float l, int code) {
    std::printf("FAIL %s h=%a l=%a code=%d r=%a\n", what, h, l, code, mf::dd_to_double(dd(h, l)));
    return 1;
  };
  for (int i = 0; i < 2000000; ++i) { // normalised pairs of random doubles
    double x = std::ldexp(u(g), ex(g)) * ((i & 1) ? -1.0 : 1.0);
    const float h = (float)x;
    const float l = (float)(x - (double)h);
    if (int c = check(h, l, &n)) return fail("random", h, l, c);
  }
  for (int e = -120; e <= 120; ++e) { // powers of two with lo on either side, all lo scales
    for (int s = 25; s <= 60; ++s) {
      for (int sg = 0; sg < 4; ++sg) {
        const float h = std::ldexp(1.0f, e) * ((sg & 1) ? -1.0f : 1.0f);
        const float mag = std::ldexp(1.0f + std::ldexp(1.0f, -23) * (s % 7), e - s);
        const float l = ((sg >> 1) ? -1.0f : 1.0f) * mag;
        if (std::fabs((double)l) > std::ldexp(std::fabs((double)h), -25) && (sg >> 1) != (sg & 1)) continue;
        if (int c = check(h, l, &n)) return fail("power of two", h, l, c);
      }
    }
    const float hm = std::nextafter(std::ldexp(1.0f, e + 1), 0.0f); // mantissa all ones, lo up
    if (int c = check(hm, std::ldexp(1.0f, e - 24), &n)) return fail("top of binade", hm, std::ldexp(1.0f, e - 24), c);
  }
  const float specials[][2] = {{1.0f, 0.0f}, {-3.0f, -0.0f}, {1.0f, 0.25f}, {1.0f, -0.75f},
                               {std::ldexp(1.0f, -100), std::ldexp(1.0f, -140)}, {0.0f, 0.0f},
                               {INFINITY, 0.0f}, {-INFINITY, 1.0f}, {NAN, 0.0f}, {1.0f, NAN}};
  for (auto& p : specials)
    if (int c = check(p[0], p[1], &n)) return fail("special", p[0], p[1], c);
  std::printf("ok %lld\n", n);
  return 0;
}
