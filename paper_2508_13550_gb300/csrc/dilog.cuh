// dilog.cuh -- the dilogarithm dilog(x) = Li2(x) = -int_0^x log(1 - t)/t dt,
// 0 <= x <= 1, of the spherical biharmonic Green's function (Sec. 2, Eq. G_B:
// G_B = (1/4pi) dilog((1 + x.y)/2) = (1/4pi) Li2(1 - d^2/4)).
//
// Method: the Bernoulli-number expansion Li2 = sum_{n>=0} B_n u^(n+1)/(n+1)!
// in u = -log(1 - x), which converges for |u| < 2 pi and is used for
// x <= 1/2 (u <= log 2), with Euler's reflection
// Li2(x) = pi^2/6 - log(x) log(1 - x) - Li2(1 - x) for x > 1/2.
#pragma once

#include <math.h>

namespace csfmm {

// sum_{n>=0} B_n u^(n+1)/(n+1)! for 0 <= u <= log 2, in FP64 (terms through
// B_20, below 1e-18 relative there), Horner in u^2.
__device__ __forceinline__ double li2_bernoulli(double u) {
  const double u2 = u * u;
  double s = -174611.0 / 330.0 / 51090942171709440000.0;  // B_20 / 21!
  s = fma(s, u2, 43867.0 / 798.0 / 121645100408832000.0);  // B_18 / 19!
  s = fma(s, u2, -3617.0 / 510.0 / 355687428096000.0);     // B_16 / 17!
  s = fma(s, u2, 7.0 / 6.0 / 1307674368000.0);              // B_14 / 15!
  s = fma(s, u2, -691.0 / 2730.0 / 6227020800.0);           // B_12 / 13!
  s = fma(s, u2, 5.0 / 66.0 / 39916800.0);                  // B_10 / 11!
  s = fma(s, u2, -1.0 / 30.0 / 362880.0);                   // B_8 / 9!
  s = fma(s, u2, 1.0 / 42.0 / 5040.0);                      // B_6 / 7!
  s = fma(s, u2, -1.0 / 30.0 / 120.0);                      // B_4 / 5!
  s = fma(s, u2, 1.0 / 6.0 / 6.0);                          // B_2 / 3!
  return u + u2 * fma(u, s, -0.25);                         // B_0 u + B_1 u^2/2 + ...
}

__device__ __forceinline__ double dilog64(double x) {
  constexpr double kPi2Over6 = 1.6449340668482264365;
  if (x <= 0.5) return li2_bernoulli(-log1p(-x));
  if (x >= 1.0) return kPi2Over6;
  return kPi2Over6 - log(x) * log1p(-x) - li2_bernoulli(-log(x));
}

// Li2(1 - z) for 0 <= z <= 1 in FP32 (z = d^2/4): two MUFU logarithms on the
// near branch, one on the far branch, series through B_6 (truncation below
// 1e-8 relative for u <= log 2).  `lg2` is the base-2 logarithm to use.
template <typename Lg2>
__device__ __forceinline__ float li2_one_minus(float z, Lg2 lg2) {
  constexpr float kLn2 = 0.69314718055994531f;
  constexpr float kPi2Over6 = 1.6449340668482264f;
  auto series = [](float u) {
    const float u2 = u * u;
    float s = fmaf(u2, 1.0f / 211680.0f, -1.0f / 3600.0f);
    s = fmaf(s, u2, 1.0f / 36.0f);
    return fmaf(u2, fmaf(u, s, -0.25f), u);
  };
  const float lz = lg2(z) * kLn2;  // log(1 - x), x = 1 - z
  if (z >= 0.5f) return series(-lz);
  const float lx = lg2(1.0f - z) * kLn2;  // log(x)
  return kPi2Over6 - lx * lz - series(-lx);
}

}  // namespace csfmm
