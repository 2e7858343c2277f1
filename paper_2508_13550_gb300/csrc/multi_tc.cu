// multi_tc.cu -- near field of 16 right-hand sides with the kernel-matrix
// products on the tensor cores (Sec. 5, Eqs. PP and PC; CSFMM_SCHED_TENSOR_NEAR).
//
// For a target leaf T and one list entry S the near field of all right-hand
// sides is the product  Phi[i][r] += sum_j K(x_i, y_j) W[j][r]  of the kernel
// matrix (formed on the fly, as in every FP32 kernel: pair-relative FP32
// coordinates, one MUFU operation per value) with the sources' weight matrix.
// The product runs on the tensor cores with warp-level mma.sync m16n8k8 in
// TF32 (FP32 accumulation): each of K and W is split into a TF32 head and a
// remainder, K W = Kh Wh + Kh Wl + Kl Wh (three products; the dropped Kl Wl
// is about 2^-22 of the product), so that the products keep nearly FP32
// accuracy.  The A fragment of an mma is exactly the four kernel values the
// thread computes (rows g and g + 8 of a 16-target tile, sources t and t + 4
// of an 8-source step; g = lane / 4, t = lane % 4), so the kernel matrix never
// leaves registers; the weights are staged per source tile in shared memory
// already split and laid out as B fragments.  Each list entry's tile sums are
// folded into FP32 (hi, lo) running totals by two-sum, as in the FP32 kernels.
//
// One block of 8 warps per target leaf, two 16-target row tiles per warp (256
// targets per pass).  Per kernel value: 7 FP32 lane-ops, 4 integer operations
// for the TF32 rounding, one MUFU operation; per 16 x 8 tile and 8 right-hand
// sides, 3 mma.sync.
//
// Measured (16 RHS, N = 1.57M Poisson, n = 10; tensor-core TF32 mma.sync at
// 300 TFLOP/s on this GPU): near field 15.8 ms against 16.9 ms for the FP32
// pipe's per-phase kernel (about 112 issued instructions per warp and 256
// kernel values, issue-bound near 9 values per clock per SM, reaching 3.1),
// and the error against the FP64 direct sum 2.2e-7 against 5.1e-8.  The
// tensor cores' FP32 accumulation does not round to nearest: on random TF32
// operands 34% of the m16n8k8 results came out smaller in magnitude than the
// exact sum rounded to nearest (mean -0.39 ulp), a bias toward zero that a
// uniform grid's recurring kernel values do not average out.  The FP32 pipe
// stays the default.
#include "csfmm_internal.cuh"
#include "fp32_math.cuh"

namespace csfmm {

namespace {

constexpr int kTcWarps = 8;
constexpr int kTcThreads = 32 * kTcWarps;
constexpr int kTcRT = 2;                         // 16-row tiles per warp
constexpr int kTcTargets = kTcWarps * kTcRT * 16;  // targets per pass
constexpr int kTcTile = 256;                     // sources per staged tile
static_assert(kTcTile % 8 == 0, "whole 8-source steps");

// x rounded to TF32 (11 significant bits, half away from zero on the bit
// pattern; a carry into the exponent is the correct rounding).  The tensor
// cores ignore the 13 low bits of a TF32 operand, i.e. truncate toward zero,
// which on a uniform grid (the same kernel values recurring) would bias the
// sums, so both parts are rounded here.
__device__ __forceinline__ uint32_t tf32_round(float x) {
  return (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
}
// TF32 head of x and the remainder x - head (exact in FP32), rounded to TF32.
__device__ __forceinline__ void tf32_split(float x, uint32_t &hi, uint32_t &lo) {
  hi = tf32_round(x);
  lo = tf32_round(__fsub_rn(x, __uint_as_float(hi)));
}

// D += A B for one m16n8k8 TF32 tile (A row-major 16 x 8, B column-major 8 x 8).
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void two_sum_fold1(float &hi, float &lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bb = __fsub_rn(s, hi);
  lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb)));
  hi = s;
}

template <int KID>
__device__ __forceinline__ float kval(float tx, float ty, float tz, const float4 &s) {
  const float rx = tx - s.x, ry = ty - s.y, rz = tz - s.z;
  return kfactor<KID>(fmaf(rz, rz, fmaf(ry, ry, rx * rx)));
}

// Accumulator element e (0..3) of n-tile nt belongs to row g + 8 (e / 2) of
// the tile and right-hand side 8 nt + 2 t + (e % 2).
template <int KID>
__global__ void __launch_bounds__(kTcThreads, 2) near16_tc_kernel(PlanView v, const int32_t *leaves,
                                                                 const float *wsf, const float *wbar,
                                                                 int ldr, int r0, double *phi) {
  __shared__ float4 sp[kTcTile];
  // B fragments [k-step][n-tile][lane]: (b0 head, b1 head, b0 rest, b1 rest)
  __shared__ uint4 sB[(kTcTile / 8) * 2 * 32];
  const int c = leaves[blockIdx.x];
  if (!cell_ok(v, c)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int tb = v.cbegin[c], te = v.cend[c], P = v.P;
  for (int i0 = tb; i0 < te; i0 += kTcTargets) {
    float ox[kTcRT][2], oy[kTcRT][2], oz[kTcRT][2];
    int ti[kTcRT][2];
#pragma unroll
    for (int rt = 0; rt < kTcRT; ++rt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = i0 + (warp * kTcRT + rt) * 16 + g + 8 * h;
        ti[rt][h] = i;
        const float4 o = v.off32[i < te ? i : tb];
        ox[rt][h] = o.x; oy[rt][h] = o.y; oz[rt][h] = o.z;
      }
    float hi[kTcRT][2][4], lo[kTcRT][2][4];
#pragma unroll
    for (int rt = 0; rt < kTcRT; ++rt)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) hi[rt][nt][e] = lo[rt][nt][e] = 0.f;
    for (int pass = 0; pass < 2; ++pass) {
      const int type = pass == 0 ? CSFMM_LIST_PP : CSFMM_LIST_PC;
      const bool particles = type == CSFMM_LIST_PP;
      const int e0 = v.loff[type][c], e1 = v.loff[type][c + 1];
      for (int ee = e0; ee < e1; ++ee) {
        const int s = v.lsrc[type][ee];
        if (!cell_ok(v, s)) continue;
        const float4 dcv = v.ldc[type][ee];
        float tx[kTcRT][2], ty[kTcRT][2], tz[kTcRT][2];
#pragma unroll
        for (int rt = 0; rt < kTcRT; ++rt)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            tx[rt][h] = ox[rt][h] + dcv.x;
            ty[rt][h] = oy[rt][h] + dcv.y;
            tz[rt][h] = oz[rt][h] + dcv.z;
          }
        const int sb = particles ? v.cbegin[s] : 0;
        const int nsrc = particles ? v.cend[s] - sb : P;
        const bool self_tile = particles && s == c;
        if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
          // -(1/4pi) sum w ln(d2/2) = -(ln2/4pi) (sum w log2 d2 - sum w); the
          // target's own weight is not part of the sum over the self leaf
#pragma unroll
          for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int r = r0 + 8 * nt + 2 * t + u;
              const float2 W = weight_total(v, s, r, particles ? 0 : 1);
#pragma unroll
              for (int rt = 0; rt < kTcRT; ++rt)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  const int e = 2 * h + u;
                  two_sum_fold1(hi[rt][nt][e], lo[rt][nt][e], -W.x);
                  lo[rt][nt][e] = __fadd_rn(lo[rt][nt][e], -W.y);
                  const int i = ti[rt][h];
                  if (self_tile && i < te)
                    two_sum_fold1(hi[rt][nt][e], lo[rt][nt][e], wsf[(int64_t)r * v.N + i]);
                }
            }
        }
        for (int j0 = 0; j0 < nsrc; j0 += kTcTile) {
          const int nj = min(kTcTile, nsrc - j0);
          const int njp = (nj + 7) & ~7;
          __syncthreads();
          for (int j = threadIdx.x; j < njp; j += kTcThreads) {
            float4 o = make_float4(1.0e4f, 1.0e4f, 1.0e4f, 0.f);  // padding: far away, no weight
            if (j < nj) {
              if (particles) {
                o = v.off32[sb + j0 + j];
              } else {
                const int64_t so = (int64_t)s * 3 * P;
                o = make_float4(v.proxy32[so + j0 + j], v.proxy32[so + P + j0 + j],
                                v.proxy32[so + 2 * P + j0 + j], 0.f);
              }
            }
            sp[j] = o;
          }
#pragma unroll 4
          for (int r = 0; r < 16; ++r)
          for (int j = threadIdx.x; j < njp; j += kTcThreads) {
            float w = 0.f;
            if (j < nj)
              w = particles ? wsf[(int64_t)(r0 + r) * v.N + sb + j0 + j]
                            : wbar[((int64_t)s * ldr + r0 + r) * P + j0 + j];
            uint32_t wh, wl;
            tf32_split(w, wh, wl);
            const int ks = j >> 3, k = j & 7, which = k >> 2;
            const int ln = (r & 7) * 4 + (k & 3);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&sB[(ks * 2 + (r >> 3)) * 32 + ln]);
            dst[which] = wh;
            dst[2 + which] = wl;
          }
          __syncthreads();
          // head products and cross products in separate accumulators (two
          // independent mma chains per output tile)
          float acc[kTcRT][2][4], acx[kTcRT][2][4];
#pragma unroll
          for (int rt = 0; rt < kTcRT; ++rt)
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
              for (int e = 0; e < 4; ++e) acc[rt][nt][e] = acx[rt][nt][e] = 0.f;
          const int self0 = sb + j0;  // point index of staged source 0
#pragma unroll 2
          for (int ks = 0; ks < njp / 8; ++ks) {
            const float4 sa = sp[ks * 8 + t], sc = sp[ks * 8 + t + 4];
            const uint4 b0 = sB[(ks * 2) * 32 + lane], b1 = sB[(ks * 2 + 1) * 32 + lane];
#pragma unroll
            for (int rt = 0; rt < kTcRT; ++rt) {
              float k4[4];
              k4[0] = kval<KID>(tx[rt][0], ty[rt][0], tz[rt][0], sa);
              k4[1] = kval<KID>(tx[rt][1], ty[rt][1], tz[rt][1], sa);
              k4[2] = kval<KID>(tx[rt][0], ty[rt][0], tz[rt][0], sc);
              k4[3] = kval<KID>(tx[rt][1], ty[rt][1], tz[rt][1], sc);
              if (self_tile) {
                const int ja = self0 + ks * 8 + t, jc = ja + 4;
                if (ti[rt][0] == ja) k4[0] = 0.f;
                if (ti[rt][1] == ja) k4[1] = 0.f;
                if (ti[rt][0] == jc) k4[2] = 0.f;
                if (ti[rt][1] == jc) k4[3] = 0.f;
              }
              uint32_t ah[4], al[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) tf32_split(k4[q], ah[q], al[q]);
              mma_tf32(acc[rt][0], ah, b0.x, b0.y);
              mma_tf32(acc[rt][1], ah, b1.x, b1.y);
              mma_tf32(acx[rt][0], ah, b0.z, b0.w);
              mma_tf32(acx[rt][1], ah, b1.z, b1.w);
              mma_tf32(acx[rt][0], al, b0.x, b0.y);
              mma_tf32(acx[rt][1], al, b1.x, b1.y);
            }
          }
#pragma unroll
          for (int rt = 0; rt < kTcRT; ++rt)
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                two_sum_fold1(hi[rt][nt][e], lo[rt][nt][e], acc[rt][nt][e]);
                lo[rt][nt][e] = __fadd_rn(lo[rt][nt][e], acx[rt][nt][e]);
              }
        }
      }
    }
#pragma unroll
    for (int rt = 0; rt < kTcRT; ++rt)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = ti[rt][e >> 1];
          if (i >= te) continue;
          const int r = r0 + 8 * nt + 2 * t + (e & 1);
          double val = (double)hi[rt][nt][e] + (double)lo[rt][nt][e];
          if constexpr (KID == CSFMM_KERNEL_LAPLACE) val *= -(0.69314718055994530942 * kInv4Pi);
          if constexpr (KID == CSFMM_KERNEL_BIHARMONIC) val *= kInv4Pi;
          phi[(int64_t)r * v.N + i] = val;
        }
  }
}

}  // namespace

void launch_near16_tc(const PlanView &v, int nleaves, const int32_t *leaves, const float *wsf,
                      const float *wbar, int ldr, int r0, double *phi, cudaStream_t st) {
  switch (v.kernel_id) {
    case CSFMM_KERNEL_LAPLACE: near16_tc_kernel<CSFMM_KERNEL_LAPLACE><<<nleaves, kTcThreads, 0, st>>>(v, leaves, wsf, wbar, ldr, r0, phi); break;
    case CSFMM_KERNEL_NEWTON: near16_tc_kernel<CSFMM_KERNEL_NEWTON><<<nleaves, kTcThreads, 0, st>>>(v, leaves, wsf, wbar, ldr, r0, phi); break;
    case CSFMM_KERNEL_SAL: near16_tc_kernel<CSFMM_KERNEL_SAL><<<nleaves, kTcThreads, 0, st>>>(v, leaves, wsf, wbar, ldr, r0, phi); break;
    case CSFMM_KERNEL_BIHARMONIC: near16_tc_kernel<CSFMM_KERNEL_BIHARMONIC><<<nleaves, kTcThreads, 0, st>>>(v, leaves, wsf, wbar, ldr, r0, phi); break;
    default: near16_tc_kernel<CSFMM_KERNEL_ONE><<<nleaves, kTcThreads, 0, st>>>(v, leaves, wsf, wbar, ldr, r0, phi); break;
  }
}

}  // namespace csfmm
