// near32.cu -- the FP32-bulk near field: PP and PC potentials at the target
// particles of every leaf (Sec. 5, Eqs. PP and PC):
//     phi(x_i) = sum_{S in PP(T)} sum_{y_j in S, j != i} K(x_i, y_j) w_j
//              + sum_{S in PC(T)} sum_k K(x_i, s_k) wbar_k(S)
//
// This is the hot loop of the evaluation (82% of the kernel evaluations of
// the N = 6.3M workload).  It is bound by the arithmetic pipes, not by memory:
// per evaluation 7 FP32 operations (3 for the pair-relative difference, 3 for
// |r|^2, 1 to accumulate) and one MUFU operation (rsqrt, lg2 or rcp).
//
// Layout: one thread block (kThreads threads) per target leaf; each thread
// owns NT targets (strided by kThreads, coalesced loads) and reuses every
// source it reads from shared memory NT times.  Sources of one list entry (a
// leaf's particles or a cell's proxies) are staged through shared memory as
// float4 (offset from the source cell centre, weight) tiles of kTile.
// Coordinates are pair-relative: t_i = (x_i - c_T) + (c_T - c_S) with the
// centre difference formed in FP64 and rounded once, so that r = t_i - s_j is
// accurate to FP32 rounding of |x_i - c_T| + |c_T - c_S| without cancellation
// against |x|=1.  Sums over one tile are FP32; the per-target total is FP64.
// The i = j term only exists when S = T; that tile runs a variant that masks
// r = 0, every other tile runs unmasked.
#include <math.h>

#include "csfmm_internal.cuh"

namespace csfmm {

namespace {

constexpr int kThreads = 64;
constexpr int kTile = 256;

template <int KID>
__host__ __device__ constexpr int kdim32() {
  return KID == CSFMM_KERNEL_BIOT_SAVART ? 3 : 1;
}

// Kernel factor f(d2) (Laplace: log2 d2, Newton: 1/sqrt d2, Biot-Savart: 1/d2).
template <int KID>
__device__ __forceinline__ float kfactor(float d2) {
  if constexpr (KID == CSFMM_KERNEL_LAPLACE) return __log2f(d2);
  else if constexpr (KID == CSFMM_KERNEL_NEWTON) return rsqrtf(d2);
  else if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) return __frcp_rn(d2);
  else return 1.0f;
}

template <int KID, int NT, int NR, bool SELF>
__device__ __forceinline__ void tile_sum(const float4 *__restrict__ sp, const float *__restrict__ sw,
                                         int nj, const float (&tx)[NT], const float (&ty)[NT],
                                         const float (&tz)[NT], const int (&self)[NT],
                                         float (&a)[NT][NR][3]) {
#pragma unroll 4
  for (int j = 0; j < nj; ++j) {
    const float4 s = sp[j];
    float wq[NR];
    wq[0] = s.w;
#pragma unroll
    for (int q = 1; q < NR; ++q) wq[q] = sw[q * kTile + j];
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      const float rx = tx[k] - s.x, ry = ty[k] - s.y, rz = tz[k] - s.z;
      const float d2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
      float f = kfactor<KID>(d2);
      if constexpr (SELF) f = (j == self[k]) ? 0.0f : f;
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) {
          const float g = wq[q] * f;
          a[k][q][0] = fmaf(g, rx, a[k][q][0]);
          a[k][q][1] = fmaf(g, ry, a[k][q][1]);
          a[k][q][2] = fmaf(g, rz, a[k][q][2]);
        } else {
          a[k][q][0] = fmaf(wq[q], f, a[k][q][0]);
        }
      }
    }
  }
}

template <int KID, int NT, int NR>
__global__ void __launch_bounds__(kThreads) near32_kernel(PlanView v, const int32_t *leaves,
                                                          const float *wsf, int ldw,
                                                          const float *wbar, int ldr, int r0,
                                                          double *phi) {
  constexpr int DIM = kdim32<KID>();
  __shared__ float4 sp[kTile];
  __shared__ float sw[NR * kTile];
  __shared__ float wsum[NR][kThreads / 32];
  const int c = leaves[blockIdx.x];
  const int b = v.cbegin[c], e = v.cend[c], P = v.P;
  const double cTx = v.ccentre[3 * c], cTy = v.ccentre[3 * c + 1], cTz = v.ccentre[3 * c + 2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i0 = b; i0 < e; i0 += kThreads * NT) {
    float ox[NT], oy[NT], oz[NT];
    double xa[NT][3];   // absolute target position (Biot-Savart cross product)
    bool act[NT];
    double out[NT][NR][DIM];
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      const int i = i0 + threadIdx.x + k * kThreads;
      act[k] = i < e;
      const int ii = act[k] ? i : b;
      const float4 o = v.off32[ii];
      ox[k] = o.x; oy[k] = o.y; oz[k] = o.z;
      if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) {
        xa[k][0] = v.x[ii]; xa[k][1] = v.x[v.N + ii]; xa[k][2] = v.x[2 * (int64_t)v.N + ii];
      }
#pragma unroll
      for (int q = 0; q < NR; ++q)
#pragma unroll
        for (int d = 0; d < DIM; ++d) out[k][q][d] = 0.0;
    }
    for (int pass = 0; pass < 2; ++pass) {
      const int type = pass == 0 ? CSFMM_LIST_PP : CSFMM_LIST_PC;
      const int e0 = v.loff[type][c], e1 = v.loff[type][c + 1];
      for (int ee = e0; ee < e1; ++ee) {
        const int s = v.lsrc[type][ee];
        const float dcx = (float)(cTx - v.ccentre[3 * s]);
        const float dcy = (float)(cTy - v.ccentre[3 * s + 1]);
        const float dcz = (float)(cTz - v.ccentre[3 * s + 2]);
        float tx[NT], ty[NT], tz[NT];
#pragma unroll
        for (int k = 0; k < NT; ++k) {
          tx[k] = ox[k] + dcx;
          ty[k] = oy[k] + dcy;
          tz[k] = oz[k] + dcz;
        }
        const bool pp = type == CSFMM_LIST_PP;
        const int sb = pp ? v.cbegin[s] : 0;
        const int nsrc = pp ? v.cend[s] - sb : P;
        const bool self_tile = pp && s == c;
        for (int j0 = 0; j0 < nsrc; j0 += kTile) {
          const int nj = min(kTile, nsrc - j0);
          __syncthreads();
          float part[NR];
#pragma unroll
          for (int q = 0; q < NR; ++q) part[q] = 0.f;
          for (int t = threadIdx.x; t < nj; t += kThreads) {
            float4 val;
            float wv[NR];
            if (pp) {
              const int j = sb + j0 + t;
              val = v.off32[j];
#pragma unroll
              for (int q = 0; q < NR; ++q) wv[q] = wsf[(int64_t)(r0 + q) * ldw + j];
            } else {
              const int64_t so = (int64_t)s * 3 * P;
              const int k = j0 + t;
              val = make_float4(v.proxy32[so + k], v.proxy32[so + P + k], v.proxy32[so + 2 * P + k], 0.f);
#pragma unroll
              for (int q = 0; q < NR; ++q) wv[q] = wbar[((int64_t)s * ldr + r0 + q) * P + k];
            }
            val.w = wv[0];
            sp[t] = val;
#pragma unroll
            for (int q = 1; q < NR; ++q) sw[q * kTile + t] = wv[q];
#pragma unroll
            for (int q = 0; q < NR; ++q) part[q] += wv[q];
          }
          if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
#pragma unroll
            for (int q = 0; q < NR; ++q) {
              float x = part[q];
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
              if (lane == 0) wsum[q][warp] = x;
            }
          }
          __syncthreads();
          float a[NT][NR][3];
#pragma unroll
          for (int k = 0; k < NT; ++k)
#pragma unroll
            for (int q = 0; q < NR; ++q) a[k][q][0] = a[k][q][1] = a[k][q][2] = 0.f;
          int self[NT];
#pragma unroll
          for (int k = 0; k < NT; ++k) self[k] = (i0 + (int)threadIdx.x + k * kThreads) - (sb + j0);
          if (self_tile)
            tile_sum<KID, NT, NR, true>(sp, sw, nj, tx, ty, tz, self, a);
          else
            tile_sum<KID, NT, NR, false>(sp, sw, nj, tx, ty, tz, self, a);
#pragma unroll
          for (int k = 0; k < NT; ++k) {
#pragma unroll
            for (int q = 0; q < NR; ++q) {
              if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
                // -(1/4pi) sum w ln(d2/2) = -(ln2/4pi) (sum w log2 d2 - sum w)
                float tot = 0.f;
#pragma unroll
                for (int u = 0; u < kThreads / 32; ++u) tot += wsum[q][u];
                if (self_tile && self[k] >= 0 && self[k] < nj)
                  tot -= (q == 0) ? sp[self[k]].w : sw[q * kTile + self[k]];
                out[k][q][0] += -(0.69314718055994530942 * kInv4Pi) * ((double)a[k][q][0] - (double)tot);
              } else if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) {
                const double b0 = a[k][q][0], b1 = a[k][q][1], b2 = a[k][q][2];
                out[k][q][0] += kInv2Pi * (xa[k][1] * b2 - xa[k][2] * b1);
                out[k][q][1] += kInv2Pi * (xa[k][2] * b0 - xa[k][0] * b2);
                out[k][q][2] += kInv2Pi * (xa[k][0] * b1 - xa[k][1] * b0);
              } else {
                out[k][q][0] += (double)a[k][q][0];
              }
            }
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      if (!act[k]) continue;
      const int i = i0 + threadIdx.x + k * kThreads;
#pragma unroll
      for (int q = 0; q < NR; ++q)
#pragma unroll
        for (int d = 0; d < DIM; ++d) phi[((int64_t)(r0 + q) * v.N + i) * DIM + d] = out[k][q][d];
    }
  }
}

template <int KID, int NR>
void launch_nr(const PlanView &v, const int32_t *leaves, int nleaves, const float *wsf, int ldw,
               const float *wbar, int ldr, int r0, double *phi, cudaStream_t st) {
  constexpr int NT = (NR == 1 && KID != CSFMM_KERNEL_BIOT_SAVART) ? 4 : 2;
  near32_kernel<KID, NT, NR><<<nleaves, kThreads, 0, st>>>(v, leaves, wsf, ldw, wbar, ldr, r0, phi);
}

template <int KID>
void launch_kid(const PlanView &v, const int32_t *leaves, int nleaves, const float *wsf, int ldw,
                const float *wbar, int ldr, int r0, int nr, double *phi, cudaStream_t st) {
  switch (nr) {
    case 1: launch_nr<KID, 1>(v, leaves, nleaves, wsf, ldw, wbar, ldr, r0, phi, st); break;
    case 2: launch_nr<KID, 2>(v, leaves, nleaves, wsf, ldw, wbar, ldr, r0, phi, st); break;
    case 3: launch_nr<KID, 3>(v, leaves, nleaves, wsf, ldw, wbar, ldr, r0, phi, st); break;
    default: launch_nr<KID, 4>(v, leaves, nleaves, wsf, ldw, wbar, ldr, r0, phi, st); break;
  }
}

}  // namespace

// nr right-hand sides r0 .. r0+nr-1 (nr <= 4).
void launch_near32(const PlanView &v, const int32_t *leaves, int nleaves, const float *wsf, int ldw,
                   const float *wbar, int ldr, int r0, int nr, double *phi, cudaStream_t st) {
  switch (v.kernel_id) {
    case CSFMM_KERNEL_LAPLACE: launch_kid<CSFMM_KERNEL_LAPLACE>(v, leaves, nleaves, wsf, ldw, wbar, ldr, r0, nr, phi, st); break;
    case CSFMM_KERNEL_BIOT_SAVART: launch_kid<CSFMM_KERNEL_BIOT_SAVART>(v, leaves, nleaves, wsf, ldw, wbar, ldr, r0, nr, phi, st); break;
    case CSFMM_KERNEL_NEWTON: launch_kid<CSFMM_KERNEL_NEWTON>(v, leaves, nleaves, wsf, ldw, wbar, ldr, r0, nr, phi, st); break;
    default: launch_kid<CSFMM_KERNEL_ONE>(v, leaves, nleaves, wsf, ldw, wbar, ldr, r0, nr, phi, st); break;
  }
}

}  // namespace csfmm
