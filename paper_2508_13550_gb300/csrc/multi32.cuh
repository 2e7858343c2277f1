// multi32.cuh -- FP32-bulk interactions for several right-hand sides
// (NR = 8 or 16, scalar kernels; Sec. 5, Eqs. PP, PC, CP, CC): the kernel
// factor of a (target, source) pair is computed once and applied to every
// right-hand side with packed FMAs over pairs of right-hand sides.  Used for
// both the near field (targets = particles of a leaf, PP and PC sources) and
// the far field (targets = proxies of a cell, CP and CC sources), by the
// per-phase kernel of interact32.cu and by the persistent kernel of
// persistent.cu.
#pragma once

#include "csfmm_internal.cuh"
#include "fp32_math.cuh"

namespace csfmm {

// Sources staged per shared-memory tile.
constexpr int kMultiTile = 256;

// Targets per thread and threads per block of the multi-right-hand-side
// kernel.  The kernel is bound by shared-memory loads (one coordinate and four
// weight vectors per source); two targets per thread halve them per target
// (measured at 16 RHS, N = 1.57M Poisson: near field 20.5 ms with one target,
// 16.2 ms with two at 128 threads, 17.4 ms with two at 64 threads).
#ifndef CSFMM_MULTI_NT
#define CSFMM_MULTI_NT 2
#endif
#ifndef CSFMM_MULTI_THREADS
#define CSFMM_MULTI_THREADS 128
#endif
static_assert(CSFMM_MULTI_THREADS % 32 == 0 && CSFMM_MULTI_THREADS <= 1024, "block size");

// Barrier of the nth threads taking part in one item: barrier 0 with the
// whole block is __syncthreads; barriers 1, 2, ... let two halves of a block
// work on different cells.
__device__ __forceinline__ void group_sync(int bar, int nth) {
  asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nth) : "memory");
}

template <int KID, int NT, int NR, bool SELF>
__device__ __forceinline__ void eval_multi(const float4 *__restrict__ sp,
                                           const ulonglong2 *__restrict__ sw4, int j,
                                           const float (&tx)[NT], const float (&ty)[NT],
                                           const float (&tz)[NT], const int (&self)[NT],
                                           f2x (&acc)[NT][NR / 2]) {
  const float4 s = sp[j];
  f2x w2[NR / 2];
#pragma unroll
  for (int q = 0; q < NR / 4; ++q) {
    const ulonglong2 u = sw4[j * (NR / 4) + q];
    w2[2 * q] = u.x;
    w2[2 * q + 1] = u.y;
  }
#pragma unroll
  for (int k = 0; k < NT; ++k) {
    const float rx = tx[k] - s.x, ry = ty[k] - s.y, rz = tz[k] - s.z;
    const float d2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
    float f = kfactor<KID>(d2);
    if constexpr (SELF) f = (j == self[k]) ? 0.0f : f;
    const f2x ff = f2_pack(f, f);
#pragma unroll
    for (int q = 0; q < NR / 2; ++q) acc[k][q] = f2_fma(w2[q], ff, acc[k][q]);
  }
}

// Sums of one staged tile in FP32 over chunks of CH sources, each chunk
// folded into the (hi, lo) totals by two-sum.
template <int KID, int NT, int NR, bool SELF, int CH>
__device__ __forceinline__ void tile_sum_multi(const float4 *__restrict__ sp,
                                               const ulonglong2 *__restrict__ sw4, int nj,
                                               const float (&tx)[NT], const float (&ty)[NT],
                                               const float (&tz)[NT], const int (&self)[NT],
                                               f2x (&hi)[NT][NR / 2], f2x (&lo)[NT][NR / 2]) {
  constexpr int kChunk = CH;
  for (int jc = 0; jc < nj; jc += kChunk) {
    f2x acc[NT][NR / 2];
#pragma unroll
    for (int k = 0; k < NT; ++k)
#pragma unroll
      for (int q = 0; q < NR / 2; ++q) acc[k][q] = 0ull;
    if (jc + kChunk <= nj) {  // full chunk: constant trip count
#pragma unroll 2
      for (int jj = 0; jj < kChunk; ++jj)
        eval_multi<KID, NT, NR, SELF>(sp, sw4, jc + jj, tx, ty, tz, self, acc);
    } else {
#pragma unroll 2
      for (int j = jc; j < nj; ++j) eval_multi<KID, NT, NR, SELF>(sp, sw4, j, tx, ty, tz, self, acc);
    }
#pragma unroll
    for (int k = 0; k < NT; ++k)
#pragma unroll
      for (int q = 0; q < NR / 2; ++q) two_sum_fold(hi[k][q], lo[k][q], acc[k][q]);
  }
}

// FAR = false: near field of leaf c into phi (FP64); FAR = true: far field of
// cell c into psi (FP64; a cell without CP/CC entries gets zeros).  nth
// threads (tid = 0 .. nth-1, synchronised by barrier `bar`) share the item,
// NT targets per thread strided by nth; every target keeps FP32 (hi, lo)
// running totals per right-hand side over the whole list, summing tiles in
// chunks of CH sources, and writes FP64 once.  sp [kMultiTile] and sw4
// [(NR/4) kMultiTile] are this group's shared memory.
template <int KID, int NR, bool FAR, int NT = CSFMM_MULTI_NT, int CH = kChunk>
__device__ __forceinline__ void multi32_item(const PlanView &v, int c, const float *wsf,
                                             const float *wbar, int ldr, int r0, double *phi,
                                             double *psi, float4 *sp, ulonglong2 *sw4, int tid,
                                             int nth, int bar) {
  if (!cell_ok(v, c)) return;
  const int P = v.P;
  const int tb = FAR ? 0 : v.cbegin[c];
  const int te = FAR ? P : v.cend[c];
  const int64_t po = (int64_t)c * 3 * P;
  float *swf = reinterpret_cast<float *>(sw4);
  for (int i0 = tb; i0 < te; i0 += nth * NT) {
    float ox[NT], oy[NT], oz[NT];
    // running totals over all list entries, FP32 (hi, lo) pairs per pair of
    // right-hand sides; the log kernel holds sum w (log2 d2 - 1)
    f2x hi[NT][NR / 2], lo[NT][NR / 2];
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      const int i = i0 + tid + k * nth;
      const int ii = i < te ? i : tb;
      if (FAR) {
        ox[k] = v.proxy32[po + ii]; oy[k] = v.proxy32[po + P + ii]; oz[k] = v.proxy32[po + 2 * P + ii];
      } else {
        const float4 o = v.off32[ii];
        ox[k] = o.x; oy[k] = o.y; oz[k] = o.z;
      }
#pragma unroll
      for (int q = 0; q < NR / 2; ++q) hi[k][q] = lo[k][q] = 0ull;
    }
    for (int pass = 0; pass < 2; ++pass) {
      const int type = FAR ? (pass == 0 ? CSFMM_LIST_CP : CSFMM_LIST_CC)
                           : (pass == 0 ? CSFMM_LIST_PP : CSFMM_LIST_PC);
      const bool particles = type == CSFMM_LIST_PP || type == CSFMM_LIST_CP;
      const int e0 = v.loff[type][c], e1 = v.loff[type][c + 1];
      for (int ee = e0; ee < e1; ++ee) {
        const int s = v.lsrc[type][ee];
        if (!cell_ok(v, s)) continue;
        const float4 dcv = v.ldc[type][ee];
        const float dcx = dcv.x, dcy = dcv.y, dcz = dcv.z;
        float tx[NT], ty[NT], tz[NT];
#pragma unroll
        for (int k = 0; k < NT; ++k) {
          tx[k] = ox[k] + dcx;
          ty[k] = oy[k] + dcy;
          tz[k] = oz[k] + dcz;
        }
        const int sb = particles ? v.cbegin[s] : 0;
        const int nsrc = particles ? v.cend[s] - sb : P;
        const bool self_tile = !FAR && type == CSFMM_LIST_PP && s == c;
        if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
          // -(1/4pi) sum w ln(d2/2) = -(ln2/4pi) (sum w log2 d2 - sum w); the
          // target's own weight is not part of the sum over the self leaf
#pragma unroll
          for (int q = 0; q < NR / 2; ++q) {
            const float2 W0 = weight_total(v, s, r0 + 2 * q, particles ? 0 : 1);
            const float2 W1 = weight_total(v, s, r0 + 2 * q + 1, particles ? 0 : 1);
#pragma unroll
            for (int k = 0; k < NT; ++k) {
              two_sum_fold(hi[k][q], lo[k][q], f2_pack(-W0.x, -W1.x));
              lo[k][q] = f2_add(lo[k][q], f2_pack(-W0.y, -W1.y));
              const int i = i0 + tid + k * nth;
              if (self_tile && i < te)
                two_sum_fold(hi[k][q], lo[k][q], f2_pack(wsf[(int64_t)(r0 + 2 * q) * v.N + i],
                                                         wsf[(int64_t)(r0 + 2 * q + 1) * v.N + i]));
            }
          }
        }
        for (int j0 = 0; j0 < nsrc; j0 += kMultiTile) {
          const int nj = min(kMultiTile, nsrc - j0);
          group_sync(bar, nth);
          for (int t = tid; t < nj; t += nth) {
            float wv[NR];
            if (particles) {
              const int j = sb + j0 + t;
              sp[t] = v.off32[j];
#pragma unroll
              for (int q = 0; q < NR; ++q) wv[q] = wsf[(int64_t)(r0 + q) * v.N + j];
            } else {
              const int64_t so = (int64_t)s * 3 * P;
              const int k = j0 + t;
              sp[t] = make_float4(v.proxy32[so + k], v.proxy32[so + P + k], v.proxy32[so + 2 * P + k], 0.f);
#pragma unroll
              for (int q = 0; q < NR; ++q) wv[q] = wbar[((int64_t)s * ldr + r0 + q) * P + k];
            }
#pragma unroll
            for (int q = 0; q < NR / 4; ++q)
              reinterpret_cast<float4 *>(swf)[t * (NR / 4) + q] =
                  make_float4(wv[4 * q], wv[4 * q + 1], wv[4 * q + 2], wv[4 * q + 3]);
          }
          group_sync(bar, nth);
          int self[NT];
#pragma unroll
          for (int k = 0; k < NT; ++k) self[k] = (i0 + tid + k * nth) - (sb + j0);
          if (self_tile)
            tile_sum_multi<KID, NT, NR, true, CH>(sp, sw4, nj, tx, ty, tz, self, hi, lo);
          else
            tile_sum_multi<KID, NT, NR, false, CH>(sp, sw4, nj, tx, ty, tz, self, hi, lo);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      const int i = i0 + tid + k * nth;
      if (i >= te) continue;
#pragma unroll
      for (int q = 0; q < NR / 2; ++q)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int qq = 2 * q + h;
          double val = f2_total(hi[k][q], lo[k][q], h);
          if constexpr (KID == CSFMM_KERNEL_LAPLACE) val *= -(0.69314718055994530942 * kInv4Pi);
          if constexpr (KID == CSFMM_KERNEL_BIHARMONIC) val *= kInv4Pi;
          if (FAR) psi[((int64_t)c * ldr + r0 + qq) * P + i] = val;
          else phi[(int64_t)(r0 + qq) * v.N + i] = val;
        }
    }
  }
}

}  // namespace csfmm
