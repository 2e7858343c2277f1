// fp32_math.cuh -- FP32 arithmetic shared by the FP32-bulk interaction
// kernels (interact32.cu) and the FP32 tree-code kernels (cstc.cu): the
// one-instruction kernel factors, packed f32x2 operations, two-sum
// accumulation and the per-cell weight totals of the log kernel.
#pragma once

#include <math.h>

#include "csfmm_internal.cuh"
#include "dilog.cuh"

namespace csfmm {

// Kernel factor f(d2) (Laplace: log2 d2, Newton: 1/sqrt d2, Biot-Savart: 1/d2:
// one MUFU instruction each; biharmonic: dilog(1 - d2/4), one or two).  Flush-to-zero is safe: d2 of two distinct
// points on the unit sphere is far above the FP32 denormal range.
__device__ __forceinline__ float mufu_rsqrt(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mufu_lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mufu_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// SAL kernel coefficients from the Love number fit a1 = -2.7, b0 = -6.21196,
// b1 = 6.1: (1 - b0) and -(a1 - b1) ln 2 (for the log2 form).
constexpr float kSalC1 = 7.21196f;
constexpr float kSalC2Log2 = (float)(8.8 * 0.69314718055994530942);

template <int KID>
__device__ __forceinline__ float kfactor(float d2) {
  if constexpr (KID == CSFMM_KERNEL_LAPLACE) return mufu_lg2(d2);
  else if constexpr (KID == CSFMM_KERNEL_NEWTON) return mufu_rsqrt(d2);
  else if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) return mufu_rcp(d2);
  else if constexpr (KID == CSFMM_KERNEL_BIHARMONIC)
    return li2_one_minus(0.25f * d2, [](float v) { return mufu_lg2(v); });
  else if constexpr (KID == CSFMM_KERNEL_SAL) {
    // (1 - b0)/g - (a1 - b1) ln(t + t^2), g = sqrt(d2), t = g/2: one rsqrt and
    // one log2 (the log's argument t(1 + t) is formed exactly enough in FP32)
    const float r = mufu_rsqrt(d2);
    const float t = 0.5f * (d2 * r);
    return fmaf(kSalC1, r, kSalC2Log2 * mufu_lg2(fmaf(t, t, t)));
  }
  else return 1.0f;
}

// Log kernel: a list entry (target cell c, source cell s) scales its
// pair-relative coordinates by sigma = 2^e, exact in FP32, with 2^-e of the
// order of the distance between the two cells (or of the source radius), so
// that log2(sigma^2 d^2) stays near zero.  The FP32 sums of w log2(sigma^2 d^2)
// then have small partial sums; the shift 2 e sum(w) is removed in FP64.
__device__ __forceinline__ int log_scale_exp(const PlanView &v, int c, int s) {
  const double dx = v.ccentre[3 * c] - v.ccentre[3 * s];
  const double dy = v.ccentre[3 * c + 1] - v.ccentre[3 * s + 1];
  const double dz = v.ccentre[3 * c + 2] - v.ccentre[3 * s + 2];
  const double ref = fmax(fmax(sqrt(dx * dx + dy * dy + dz * dz), v.cradius[s]), 1e-18);
  return -ilogb(ref);
}
__device__ __forceinline__ float exp2i(int e) { return __int_as_float((127 + e) << 23); }

// Packed pairs of FP32 values in one 64-bit register (Blackwell f32x2 math).
typedef unsigned long long f2x;
__device__ __forceinline__ f2x f2_sub(f2x a, f2x b) {
  f2x d;
  asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x f2_mul(f2x a, f2x b) {
  f2x d;
  asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x f2_fma(f2x a, f2x b, f2x c) {
  f2x d;
  asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2x f2_add(f2x a, f2x b) {
  f2x d;
  asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x f2_pack(float lo, float hi) {
  f2x d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void f2_unpack(f2x a, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a));
}

// Accumulation of a tile: FP32 sums over chunks of kChunk sources, each chunk
// folded into an unevaluated FP32 pair (hi, lo) by Knuth's two-sum, so that
// the rounding error of a tile sum is that of a kChunk-term sum rather than
// of a kTile-term one (errors of long same-signed FP32 sums do not average
// out across targets that share the same tile geometry).
#ifndef CSFMM_CHUNK
#define CSFMM_CHUNK 32
#endif
constexpr int kChunk = CSFMM_CHUNK;
__device__ __forceinline__ void two_sum_fold(float &hi, float &lo, float c) {
  const float s = hi + c;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (c - bb);
  hi = s;
}
__device__ __forceinline__ void two_sum_fold(f2x &hi, f2x &lo, f2x c) {
  const f2x s = f2_add(hi, c);
  const f2x bb = f2_sub(s, hi);
  lo = f2_add(lo, f2_add(f2_sub(hi, f2_sub(s, bb)), f2_sub(c, bb)));
  hi = s;
}
__device__ __forceinline__ double f2_total(f2x hi, f2x lo, int h) {
  float a0, a1, b0, b1;
  f2_unpack(hi, a0, a1);
  f2_unpack(lo, b0, b1);
  return h == 0 ? (double)a0 + (double)b0 : (double)a1 + (double)b1;
}
// Weight total of source cell s for right-hand side r: particles (kind 0, a
// leaf's weights) or proxies (kind 1), as an FP32 pair.
__device__ __forceinline__ float2 weight_total(const PlanView &v, int s, int r, int kind) {
  return v.wtot[((int64_t)s * v.wtot_ld + r) * 2 + kind];
}
// (hi, lo) -= (t.x, t.y) for both halves of a packed pair.
__device__ __forceinline__ void fold_minus(f2x &hi, f2x &lo, float2 t) {
  two_sum_fold(hi, lo, f2_pack(-t.x, -t.x));
  lo = f2_add(lo, f2_pack(-t.y, -t.y));
}
__device__ __forceinline__ void fold_minus(float &hi, float &lo, float2 t) {
  two_sum_fold(hi, lo, -t.x);
  lo -= t.y;
}

}  // namespace csfmm
