// interact32.cu -- the FP32-bulk interactions.
//
// Near field: PP and PC potentials at the target
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
// centre difference of the list entry formed in FP64 and rounded once at plan
// build (PlanView::ldc), so that r = t_i - s_j is accurate to FP32 rounding of
// |x_i - c_T| + |c_T - c_S| without cancellation against |x|=1.  Sums over
// one tile are FP32; the per-target total is FP64.
// The i = j term only exists when S = T; that tile runs a variant that masks
// r = 0, every other tile runs unmasked.
#include <math.h>

#include <algorithm>

#include "csfmm_internal.cuh"
#include "fp32_math.cuh"

namespace csfmm {

namespace {

constexpr int kThreads = 64;
constexpr int kTile = 256;
// Resident blocks per SM requested from the register allocator for the
// packed near-field kernel (16 caps it at 64 registers per thread; measured
// fastest of 8, 10, 12 and 16 on the N = 6.3M Newtonian workload).
#ifndef CSFMM_NEAR_MINB
#define CSFMM_NEAR_MINB 16
#endif
// Threads per block and packed target pairs per thread of the one-RHS near
// kernel (one block per target leaf; 2 kNearNP targets per thread).
#ifndef CSFMM_NEAR_THREADS
#define CSFMM_NEAR_THREADS 64
#endif
#ifndef CSFMM_NEAR_NP
#define CSFMM_NEAR_NP 2
#endif
constexpr int kNearThreads = CSFMM_NEAR_THREADS;
constexpr int kNearNP = CSFMM_NEAR_NP;

template <int KID>
__host__ __device__ constexpr int kdim32() {
  return KID == CSFMM_KERNEL_BIOT_SAVART ? 3 : 1;
}


// One tile for NP pairs of targets (2 NP targets) and one right-hand side:
// sA[j] = (x, x, y, y), sB[j] = (z, z, w, w) of source j.
template <int KID, int NP, bool SELF>
__device__ __forceinline__ void eval_x2(const ulonglong2 *__restrict__ sA,
                                        const ulonglong2 *__restrict__ sB, int j,
                                        const f2x (&tx)[NP], const f2x (&ty)[NP],
                                        const f2x (&tz)[NP], const int (&self)[2 * NP],
                                        f2x (&acc)[NP]) {
  const ulonglong2 A = sA[j], B = sB[j];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const f2x rx = f2_sub(tx[q], A.x), ry = f2_sub(ty[q], A.y), rz = f2_sub(tz[q], B.x);
    f2x d2 = f2_mul(rx, rx);
    d2 = f2_fma(ry, ry, d2);
    d2 = f2_fma(rz, rz, d2);
    float d0, d1;
    f2_unpack(d2, d0, d1);
    float f0 = kfactor<KID>(d0), f1 = kfactor<KID>(d1);
    if constexpr (SELF) {
      f0 = (j == self[2 * q]) ? 0.0f : f0;
      f1 = (j == self[2 * q + 1]) ? 0.0f : f1;
    }
    acc[q] = f2_fma(B.y, f2_pack(f0, f1), acc[q]);
  }
}

// Columns of a chunk unrolled in the packed tile sums.  The whole 32-column
// chunk gives the scheduler the most independent kernel evaluations to
// interleave with the MUFU operations; measured at N = 6.3M, n = 12: near
// field 3.79 / 3.69 / 3.68 / 3.63 ms and far field 0.94 / 0.89 / 0.87 /
// 0.80 ms for 4 / 8 / 16 / 32 (the register caps of the launch bounds kept;
// lifting them measured slower).
#ifndef CSFMM_X2_UNROLL
#define CSFMM_X2_UNROLL 32
#endif
#define CSFMM_STR(x) #x
#define CSFMM_UNROLL(n) _Pragma(CSFMM_STR(unroll n))
template <int KID, int NP, bool SELF>
__device__ __forceinline__ void tile_sum_x2(const ulonglong2 *__restrict__ sA,
                                            const ulonglong2 *__restrict__ sB, int nj,
                                            const f2x (&tx)[NP], const f2x (&ty)[NP],
                                            const f2x (&tz)[NP], const int (&self)[2 * NP],
                                            f2x (&hi)[NP], f2x (&lo)[NP]) {
  int jc = 0;
  for (; jc + kChunk <= nj; jc += kChunk) {  // full chunks: constant trip count
    f2x acc[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) acc[q] = 0ull;
CSFMM_UNROLL(CSFMM_X2_UNROLL)
    for (int jj = 0; jj < kChunk; ++jj) eval_x2<KID, NP, SELF>(sA, sB, jc + jj, tx, ty, tz, self, acc);
#pragma unroll
    for (int q = 0; q < NP; ++q) two_sum_fold(hi[q], lo[q], acc[q]);
  }
  if (jc < nj) {
    f2x acc[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) acc[q] = 0ull;
CSFMM_UNROLL(CSFMM_X2_UNROLL)
    for (int j = jc; j < nj; ++j) eval_x2<KID, NP, SELF>(sA, sB, j, tx, ty, tz, self, acc);
#pragma unroll
    for (int q = 0; q < NP; ++q) two_sum_fold(hi[q], lo[q], acc[q]);
  }
}

template <int KID, int NT, int NR, bool SELF>
__device__ __forceinline__ void tile_sum(const float4 *__restrict__ sp, const float *__restrict__ sw,
                                         int nj, const float (&tx)[NT], const float (&ty)[NT],
                                         const float (&tz)[NT], const int (&self)[NT],
                                         float (&ahi)[NT][NR][3], float (&alo)[NT][NR][3]) {
  constexpr int D = KID == CSFMM_KERNEL_BIOT_SAVART ? 3 : 1;
  for (int jc = 0; jc < nj; jc += kChunk) {
    const int je = min(nj, jc + kChunk);
    float a[NT][NR][3];
#pragma unroll
    for (int k = 0; k < NT; ++k)
#pragma unroll
      for (int q = 0; q < NR; ++q) a[k][q][0] = a[k][q][1] = a[k][q][2] = 0.f;
#pragma unroll 4
    for (int j = jc; j < je; ++j) {
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
#pragma unroll
    for (int k = 0; k < NT; ++k)
#pragma unroll
      for (int q = 0; q < NR; ++q)
#pragma unroll
        for (int d = 0; d < D; ++d) two_sum_fold(ahi[k][q][d], alo[k][q][d], a[k][q][d]);
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
  const int c = leaves[blockIdx.x];
  if (!cell_ok(v, c)) return;
  const int b = v.cbegin[c], e = v.cend[c], P = v.P;
  for (int i0 = b; i0 < e; i0 += kThreads * NT) {
    float ox[NT], oy[NT], oz[NT];
    bool act[NT];
    // running totals over all list entries as FP32 (hi, lo) pairs: the kernel
    // sums (log kernel: sum w (log2 d2 - 1); Biot-Savart: sum w r / d2)
    float ahi[NT][NR][3], alo[NT][NR][3];
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      const int i = i0 + threadIdx.x + k * kThreads;
      act[k] = i < e;
      const float4 o = v.off32[act[k] ? i : b];
      ox[k] = o.x; oy[k] = o.y; oz[k] = o.z;
#pragma unroll
      for (int q = 0; q < NR; ++q)
#pragma unroll
        for (int d = 0; d < 3; ++d) ahi[k][q][d] = alo[k][q][d] = 0.f;
    }
    for (int pass = 0; pass < 2; ++pass) {
      const int type = pass == 0 ? CSFMM_LIST_PP : CSFMM_LIST_PC;
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
        const bool pp = type == CSFMM_LIST_PP;
        const int sb = pp ? v.cbegin[s] : 0;
        const int nsrc = pp ? v.cend[s] - sb : P;
        const bool self_tile = pp && s == c;
        if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
          // -(1/4pi) sum w ln(d2/2) = -(ln2/4pi) (sum w log2 d2 - sum w); the
          // target's own weight is not part of the sum over the self leaf
#pragma unroll
          for (int q = 0; q < NR; ++q) {
            const float2 W = weight_total(v, s, r0 + q, pp ? 0 : 1);
#pragma unroll
            for (int k = 0; k < NT; ++k) {
              fold_minus(ahi[k][q][0], alo[k][q][0], W);
              if (self_tile && act[k])
                two_sum_fold(ahi[k][q][0], alo[k][q][0],
                             wsf[(int64_t)(r0 + q) * ldw + i0 + threadIdx.x + k * kThreads]);
            }
          }
        }
        for (int j0 = 0; j0 < nsrc; j0 += kTile) {
          const int nj = min(kTile, nsrc - j0);
          __syncthreads();
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
          }
          __syncthreads();
          int self[NT];
#pragma unroll
          for (int k = 0; k < NT; ++k) self[k] = (i0 + (int)threadIdx.x + k * kThreads) - (sb + j0);
          if (self_tile)
            tile_sum<KID, NT, NR, true>(sp, sw, nj, tx, ty, tz, self, ahi, alo);
          else
            tile_sum<KID, NT, NR, false>(sp, sw, nj, tx, ty, tz, self, ahi, alo);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      if (!act[k]) continue;
      const int i = i0 + threadIdx.x + k * kThreads;
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        double o[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) o[d] = (double)ahi[k][q][d] + (double)alo[k][q][d];
        double* dst = phi + ((int64_t)(r0 + q) * v.N + i) * DIM;
        if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
          dst[0] = -(0.69314718055994530942 * kInv4Pi) * o[0];
        } else if constexpr (KID == CSFMM_KERNEL_BIHARMONIC) {
          dst[0] = kInv4Pi * o[0];
        } else if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) {
          // (1/2pi) x × sum_j w_j r_j / |r_j|^2, with the FP64 target position
          const double x0 = v.x[i], x1 = v.x[v.N + i], x2 = v.x[2 * (int64_t)v.N + i];
          dst[0] = kInv2Pi * (x1 * o[2] - x2 * o[1]);
          dst[1] = kInv2Pi * (x2 * o[0] - x0 * o[2]);
          dst[2] = kInv2Pi * (x0 * o[1] - x1 * o[0]);
        } else {
          dst[0] = o[0];
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Symmetric PP (Eq. PP) for K(x, y) = K(y, x): one block per cross pair
// (T, S), T < S, evaluates each kernel value once and produces both
//     rows:    sum_{j in S} K(x_i, y_j) w_j   for the points i of T,
//     columns: sum_{i in T} K(x_i, y_j) w_i   for the points j of S,
// written to part[off[pair] ...] (rows first, then columns) as FP32 sums
// (the log kernel stores sum w (log2 d2 - 1); the factor -ln2/4pi is applied
// with the rest of the near field).  kSymWarps warps; each lane owns
// 2 kSymQP rows of T (kSymQP packed pairs); columns of S are staged as
// (x,x,y,y)/(z,z,w,w) tiles and processed in groups of kSymGroup: every lane
// accumulates its rows' contributions to the group's columns, then a
// butterfly transpose-reduction over the warp leaves the sum of column
// g*kSymGroup + (lane mod kSymGroup) in that lane; the warps are combined in
// a fixed order, so results are deterministic.  The row sums are FP32 over
// 32 columns (two groups), then folded into (hi, lo) pairs by two-sum, the
// chunk width of the direct kernels.
//
// Per kernel evaluation the FP32 pipe does 8 lane-ops (3 differences, |r|^2,
// the row and the column FMA) plus the column reduction, about
// 2 / (2 kSymQP) lane-ops (one add to fold the packed halves, one in the
// butterfly, per column and lane), next to one MUFU operation.  Default
// shape: one warp per leaf pair with eight rows per lane (a 256-point leaf in
// one pass) and groups of 16 columns, 16 blocks per SM (measured on the
// N = 6.3M Newtonian workload: 6.98 ms against 7.16 ms for two warps with
// four rows per lane and 32-column groups; 24 warps per SM with 16-column
// groups were slower, 7.40-7.45 ms; folding the row sums every 32 columns
// instead of 16: 6.76 against 6.92 ms).  The instruction mix, not occupancy,
// bounds this kernel: the FMA pipe is busy 76% of the cycles and the MUFU
// 69% (a synthetic loop of 8 FP32 lane-ops and one MUFU op per value reaches
// 92% of 16 values per clock per SM at 8 warps per SM); 12, 20 or 24 blocks
// per SM, 8-column groups and a software-pipelined column loop measured the
// same or slower.
// ---------------------------------------------------------------------------
#ifndef CSFMM_SYM_WARPS
#define CSFMM_SYM_WARPS 1
#endif
#ifndef CSFMM_SYM_QP
#define CSFMM_SYM_QP 4
#endif
#ifndef CSFMM_SYM_GROUP
#define CSFMM_SYM_GROUP 16
#endif
#ifndef CSFMM_SYM_MINB
#define CSFMM_SYM_MINB 16
#endif
constexpr int kSymWarps = CSFMM_SYM_WARPS;
constexpr int kSymQP = CSFMM_SYM_QP;         // packed row pairs per lane
constexpr int kSymGroup = CSFMM_SYM_GROUP;   // columns per transpose-reduction
constexpr int kSymThreads = 32 * kSymWarps;
constexpr int kSymRowsPerWarp = 2 * kSymQP * 32;
constexpr int kSymRows = kSymRowsPerWarp * kSymWarps;  // rows per pass
constexpr int kSymCols = 256;                          // columns per staged tile
static_assert(kSymGroup == 8 || kSymGroup == 16 || kSymGroup == 32, "column group");
static_assert(kSymCols % kSymGroup == 0, "a tile holds whole column groups");

// v[G] held by each lane -> the sum over the warp of v[lane mod G] (every
// lane of a G-lane group first sums its group, then the groups are added).
template <int G>
__device__ __forceinline__ float transpose_reduce(float (&v)[G], int lane) {
#pragma unroll
  for (int s = G / 2; s >= 1; s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int k = 0; k < s; ++k) {
      const float send = up ? v[k] : v[k + s];
      const float keep = up ? v[k + s] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  float r = v[0];
#pragma unroll
  for (int s = G; s < 32; s <<= 1) r += __shfl_xor_sync(0xffffffffu, r, s);
  return r;
}

// CC = false: a mirrored PP leaf pair (rows: the points of T, columns: the
// points of S, particle weights wsrc = wsf, partials at part + off[pair]).
// CC = true: a mirrored CC cell pair (Sec. 5, Eq. CC: the kernel matrix
// between the proxies of T and of S serves both entries), rows and columns
// the P proxies of T and S, proxy weights wsrc = wbar [nc][ldr][P] of the
// first right-hand side, the centre difference of CC entry entry[pair], and
// partials at part + 2 P pair (P rows, then P columns).  QP packed row pairs
// per lane.
template <int KID, bool CC, int QP>
__global__ void __launch_bounds__(kSymThreads, CSFMM_SYM_MINB) sym_kernel(
    PlanView v, const int2 *pairs, const int32_t *off, const int32_t *entry, const float *wsrc,
    int ldr, float *part) {
  constexpr int G = kSymGroup;
  constexpr int kRowsPerWarp = 2 * QP * 32;
  constexpr int kRows = kRowsPerWarp * kSymWarps;  // rows per pass
  __shared__ ulonglong2 sA[kSymCols], sB[kSymCols];
  __shared__ float colacc[kSymWarps][kSymCols];
  const int2 pr = pairs[blockIdx.x];
  const int T = pr.x, S = pr.y;
  if (!cell_ok(v, T) || !cell_ok(v, S)) return;
  const int P = v.P;
  const int tb = CC ? 0 : v.cbegin[T], sb = CC ? 0 : v.cbegin[S];
  const int nT = CC ? P : v.cend[T] - tb, nS = CC ? P : v.cend[S] - sb;
  float *rowpart = part + (CC ? (int64_t)2 * P * blockIdx.x : (int64_t)off[blockIdx.x]);
  float *colpart = rowpart + nT;
  const int64_t pT = (int64_t)T * 3 * P, pS = (int64_t)S * 3 * P;
  const float *wT = CC ? wsrc + (int64_t)T * ldr * P : wsrc + tb;
  const float *wS = CC ? wsrc + (int64_t)S * ldr * P : wsrc + sb;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float dcx, dcy, dcz;
  if constexpr (CC) {
    const float4 d = v.ldc[CSFMM_LIST_CC][entry[blockIdx.x]];
    dcx = d.x; dcy = d.y; dcz = d.z;
  } else {
    dcx = (float)(v.ccentre[3 * T] - v.ccentre[3 * S]);
    dcy = (float)(v.ccentre[3 * T + 1] - v.ccentre[3 * S + 1]);
    dcz = (float)(v.ccentre[3 * T + 2] - v.ccentre[3 * S + 2]);
  }
  int lse = 0;
  float sg = 1.f;
  if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
    lse = log_scale_exp(v, T, S);
    sg = exp2i(lse);
  }
  // log kernel: weight totals of T and S (particles, or proxies for CC) for
  // -(ln2/4pi)(sum w log2 d2 - sum w)
  double WT = 0.0, WS = 0.0;
  if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
    const float2 a = weight_total(v, T, 0, CC ? 1 : 0), b2 = weight_total(v, S, 0, CC ? 1 : 0);
    WT = (double)a.x + (double)a.y;
    WS = (double)b2.x + (double)b2.y;
  }
  for (int r0 = 0; r0 < nT; r0 += kRows) {
    // rows of this lane: r0 + warp*kRowsPerWarp + lane + 32k, k = 0..2QP-1,
    // packed as pairs (2q, 2q+1)
    f2x tx[QP], ty[QP], tz[QP], wr[QP], rhi[QP], rlo[QP];
    bool act[2 * QP];
#pragma unroll
    for (int q = 0; q < QP; ++q) {
      float x[2], y[2], z[2], w[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = 2 * q + h;
        const int i = r0 + warp * kRowsPerWarp + lane + 32 * k;
        act[k] = i < nT;
        const int ii = act[k] ? i : 0;
        float ox, oy, oz;
        if constexpr (CC) {
          ox = v.proxy32[pT + ii]; oy = v.proxy32[pT + P + ii]; oz = v.proxy32[pT + 2 * P + ii];
        } else {
          const float4 o = v.off32[tb + ii];
          ox = o.x; oy = o.y; oz = o.z;
        }
        x[h] = (ox + dcx) * sg;
        y[h] = (oy + dcy) * sg;
        z[h] = (oz + dcz) * sg;
        w[h] = act[k] ? wT[ii] : 0.f;
      }
      tx[q] = f2_pack(x[0], x[1]);
      ty[q] = f2_pack(y[0], y[1]);
      tz[q] = f2_pack(z[0], z[1]);
      wr[q] = f2_pack(w[0], w[1]);
      rhi[q] = 0ull;
      rlo[q] = 0ull;
    }
    for (int c0 = 0; c0 < nS; c0 += kSymCols) {
      const int nj = min(kSymCols, nS - c0);
      __syncthreads();
      for (int t = threadIdx.x; t < kSymCols; t += kSymThreads) {
        float x = 1.0e4f, y = 1.0e4f, z = 1.0e4f, w = 0.f;  // padding: far away, no weight
        if (t < nj) {
          const int j = c0 + t;
          if constexpr (CC) {
            x = v.proxy32[pS + j] * sg; y = v.proxy32[pS + P + j] * sg;
            z = v.proxy32[pS + 2 * P + j] * sg;
          } else {
            const float4 o = v.off32[sb + j];
            x = o.x * sg; y = o.y * sg; z = o.z * sg;
          }
          w = wS[j];
        }
        sA[t] = make_ulonglong2(f2_pack(x, x), f2_pack(y, y));
        sB[t] = make_ulonglong2(f2_pack(z, z), f2_pack(w, w));
      }
      __syncthreads();
      const int ng = (nj + G - 1) / G;
      f2x racc[QP];
      for (int g = 0; g < ng; ++g) {
        f2x colv[G];
        if ((g & 1) == 0) {
#pragma unroll
          for (int q = 0; q < QP; ++q) racc[q] = 0ull;
        }
#pragma unroll
        for (int j = 0; j < G; ++j) {
          const ulonglong2 A = sA[g * G + j], B = sB[g * G + j];
          colv[j] = 0ull;
#pragma unroll
          for (int q = 0; q < QP; ++q) {
            const f2x rx = f2_sub(tx[q], A.x), ry = f2_sub(ty[q], A.y), rz = f2_sub(tz[q], B.x);
            f2x d2 = f2_mul(rx, rx);
            d2 = f2_fma(ry, ry, d2);
            d2 = f2_fma(rz, rz, d2);
            float d0, d1;
            f2_unpack(d2, d0, d1);
            const f2x f = f2_pack(kfactor<KID>(d0), kfactor<KID>(d1));
            racc[q] = f2_fma(B.y, f, racc[q]);
            colv[j] = f2_fma(f, wr[q], colv[j]);
          }
        }
        if ((g & 1) || g + 1 == ng) {
#pragma unroll
          for (int q = 0; q < QP; ++q) two_sum_fold(rhi[q], rlo[q], racc[q]);
        }
        float cv[G];
#pragma unroll
        for (int j = 0; j < G; ++j) {
          float lo, hi;
          f2_unpack(colv[j], lo, hi);
          cv[j] = lo + hi;
        }
        const float red = transpose_reduce<G>(cv, lane);
        if (lane < G) colacc[warp][g * G + lane] = red;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < nj; t += kSymThreads) {
        float val = 0.f;
#pragma unroll
        for (int u = 0; u < kSymWarps; ++u) val += colacc[u][t];
        if (r0 == 0) colpart[c0 + t] = val;
        else colpart[c0 + t] += val;
      }
    }
#pragma unroll
    for (int q = 0; q < QP; ++q) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = 2 * q + h;
        if (!act[k]) continue;
        const int i = r0 + warp * kRowsPerWarp + lane + 32 * k;
        double val = f2_total(rhi[q], rlo[q], h);
        if constexpr (KID == CSFMM_KERNEL_LAPLACE) val -= (1 + 2 * lse) * WS;
        rowpart[i] = (float)val;
      }
    }
  }
  if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
    __syncthreads();
    for (int t = threadIdx.x; t < nS; t += kSymThreads)
      colpart[t] = (float)((double)colpart[t] - (1 + 2 * lse) * WT);
  }
}

// Packed variant for one right-hand side and a scalar kernel (Laplace,
// Newtonian, K = 1): same arithmetic per pair, two targets per instruction.
// With part != nullptr the PP entries that belong to a cross pair come from the
// symmetric cross-pair partials (final potentials, added in list order); the
// self entry and entries without a mirror are evaluated here.
template <int KID, int NP>
__global__ void __launch_bounds__(kNearThreads, CSFMM_NEAR_MINB) near32x2_kernel(PlanView v, const int32_t *leaves,
                                                            const float *wsf, const float *wbar,
                                                            int ldr, int r0, double *phi,
                                                            const float *part) {
  constexpr int NT = 2 * NP;
  __shared__ ulonglong2 sA[kTile], sB[kTile];
  const int c = leaves[blockIdx.x];
  if (!cell_ok(v, c)) return;
  const int b = v.cbegin[c], e = v.cend[c], P = v.P;
  const float *wr = wsf + (int64_t)r0 * v.N;
  for (int i0 = b; i0 < e; i0 += kNearThreads * NT) {
    float ox[NT], oy[NT], oz[NT];
    // running totals of the target pairs over all list entries (and the
    // cross-pair partials) as FP32 (hi, lo) pairs; the log kernel holds
    // sum w (log2 d2 - 1) and is scaled by -ln2/4pi at the end
    f2x hi[NP], lo[NP];
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      const int i = i0 + threadIdx.x + k * kNearThreads;
      const float4 o = v.off32[i < e ? i : b];
      ox[k] = o.x; oy[k] = o.y; oz[k] = o.z;
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) hi[q] = lo[q] = 0ull;
    for (int pass = 0; pass < 2; ++pass) {
      const int type = pass == 0 ? CSFMM_LIST_PP : CSFMM_LIST_PC;
      const int e0 = v.loff[type][c], e1 = v.loff[type][c + 1];
      for (int ee = e0; ee < e1; ++ee) {
        const int s = v.lsrc[type][ee];
        if (!cell_ok(v, s)) continue;
        if (part && type == CSFMM_LIST_PP && v.sym_contrib[ee] >= 0) {
          const float *pp = part + v.sym_contrib[ee] - b;
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            const int i = i0 + threadIdx.x + 2 * q * kNearThreads, i1 = i + kNearThreads;
            two_sum_fold(hi[q], lo[q], f2_pack(i < e ? pp[i] : 0.f, i1 < e ? pp[i1] : 0.f));
          }
          continue;
        }
        const float4 dcv = v.ldc[type][ee];
        const float dcx = dcv.x, dcy = dcv.y, dcz = dcv.z;
        f2x tx[NP], ty[NP], tz[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          tx[q] = f2_pack(ox[2 * q] + dcx, ox[2 * q + 1] + dcx);
          ty[q] = f2_pack(oy[2 * q] + dcy, oy[2 * q + 1] + dcy);
          tz[q] = f2_pack(oz[2 * q] + dcz, oz[2 * q + 1] + dcz);
        }
        const bool pp = type == CSFMM_LIST_PP;
        const int sb = pp ? v.cbegin[s] : 0;
        const int nsrc = pp ? v.cend[s] - sb : P;
        const bool self_tile = pp && s == c;
        if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
          // -(1/4pi) sum w ln(d2/2) = -(ln2/4pi) (sum w log2 d2 - sum w); the
          // target's own weight is not part of the sum over the self leaf
          const float2 W = weight_total(v, s, r0, pp ? 0 : 1);
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            fold_minus(hi[q], lo[q], W);
            if (self_tile) {
              const int i = i0 + threadIdx.x + 2 * q * kNearThreads, i1 = i + kNearThreads;
              two_sum_fold(hi[q], lo[q], f2_pack(i < e ? wr[i] : 0.f, i1 < e ? wr[i1] : 0.f));
            }
          }
        }
        for (int j0 = 0; j0 < nsrc; j0 += kTile) {
          const int nj = min(kTile, nsrc - j0);
          __syncthreads();
          for (int t = threadIdx.x; t < nj; t += kNearThreads) {
            float x, y, z, w;
            if (pp) {
              const int j = sb + j0 + t;
              const float4 o = v.off32[j];
              x = o.x; y = o.y; z = o.z;
              w = wr[j];
            } else {
              const int64_t so = (int64_t)s * 3 * P;
              const int k = j0 + t;
              x = v.proxy32[so + k]; y = v.proxy32[so + P + k]; z = v.proxy32[so + 2 * P + k];
              w = wbar[((int64_t)s * ldr + r0) * P + k];
            }
            sA[t] = make_ulonglong2(f2_pack(x, x), f2_pack(y, y));
            sB[t] = make_ulonglong2(f2_pack(z, z), f2_pack(w, w));
          }
          __syncthreads();
          int self[NT];
#pragma unroll
          for (int k = 0; k < NT; ++k) self[k] = (i0 + (int)threadIdx.x + k * kNearThreads) - (sb + j0);
          if (self_tile)
            tile_sum_x2<KID, NP, true>(sA, sB, nj, tx, ty, tz, self, hi, lo);
          else
            tile_sum_x2<KID, NP, false>(sA, sB, nj, tx, ty, tz, self, hi, lo);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NP; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = i0 + threadIdx.x + (2 * q + h) * kNearThreads;
        double o = f2_total(hi[q], lo[q], h);
        if constexpr (KID == CSFMM_KERNEL_LAPLACE) o *= -(0.69314718055994530942 * kInv4Pi);
        if constexpr (KID == CSFMM_KERNEL_BIHARMONIC) o *= kInv4Pi;
        if (i < e) phi[((int64_t)r0 * v.N + i)] = o;
      }
  }
}


// ---------------------------------------------------------------------------
// Far field: CP and CC proxy potentials of every cell (Sec. 5, Eqs. CP and
// CC, accumulated as Eq. CP_CC_accumulated):
//     psi_T(t_m) = sum_{S in CP(T)} sum_{y_j in S} K(t_m, y_j) w_j
//                + sum_{S in CC(T)} sum_k K(t_m, s_k) wbar_k(S)
// One block per cell (cells without CP/CC entries write zeros), blockDim a
// multiple of 32 covering P / (2 kFarNP), 2 kFarNP target proxies m, m +
// blockDim, ... per thread.  Same pair-relative FP32 arithmetic as the near
// field; a target proxy never coincides with a source (the pair is well
// separated).
// ---------------------------------------------------------------------------
// Packed target pairs per thread of the far kernel (two targets per pair).
// Measured at N = 6.3M, n = 12 (P = 169): one pair with 96 threads 2.19 ms,
// two pairs with 64 threads 2.46 ms (a third of the lanes idle).
#ifndef CSFMM_FAR_NP
#define CSFMM_FAR_NP 1
#endif
#ifndef CSFMM_FAR_MINB
#define CSFMM_FAR_MINB 8
#endif
#ifndef CSFMM_FAR_MAXT
#define CSFMM_FAR_MAXT 160
#endif
constexpr int kFarNP = CSFMM_FAR_NP;

template <int KID>
__global__ void __launch_bounds__(CSFMM_FAR_MAXT, CSFMM_FAR_MINB) far32x2_kernel(PlanView v, const float *wsf,
                                                      const float *wbar, int ldr, int r0,
                                                      double *psi, const float *cpart) {
  constexpr int NP = kFarNP, NT = 2 * NP;
  __shared__ ulonglong2 sA[kTile], sB[kTile];
  const int c = blockIdx.x, P = v.P, nth = blockDim.x;
  const int64_t po = (int64_t)c * 3 * P;
  float ox[NT], oy[NT], oz[NT];
#pragma unroll
  for (int h = 0; h < NT; ++h) {
    const int m = threadIdx.x + h * nth;
    const int mm = m < P ? m : 0;
    ox[h] = v.proxy32[po + mm];
    oy[h] = v.proxy32[po + P + mm];
    oz[h] = v.proxy32[po + 2 * P + mm];
  }
  // running totals of the target pairs over all entries (FP32 pairs)
  f2x hi[NP], lo[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) hi[q] = lo[q] = 0ull;
  const float *wr = wsf + (int64_t)r0 * v.N;
  int self_none[NT];
#pragma unroll
  for (int h = 0; h < NT; ++h) self_none[h] = -1;
  for (int pass = 0; pass < 2; ++pass) {
    const int type = pass == 0 ? CSFMM_LIST_CP : CSFMM_LIST_CC;
    const int e0 = v.loff[type][c], e1 = v.loff[type][c + 1];
    for (int ee = e0; ee < e1; ++ee) {
      const int s = v.lsrc[type][ee];
      if (!cell_ok(v, s)) continue;
      if (cpart && type == CSFMM_LIST_CC && v.cc_contrib[ee] >= 0) {
        // a mirrored CC pair: this cell's sums come from the pair's partials
        const float *pp = cpart + v.cc_contrib[ee];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          const int m0 = threadIdx.x + 2 * q * nth, m1 = m0 + nth;
          two_sum_fold(hi[q], lo[q], f2_pack(m0 < P ? pp[m0] : 0.f, m1 < P ? pp[m1] : 0.f));
        }
        continue;
      }
      const float4 dcv = v.ldc[type][ee];
      const float dcx = dcv.x, dcy = dcv.y, dcz = dcv.z;
      f2x tx[NP], ty[NP], tz[NP];
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        tx[q] = f2_pack(ox[2 * q] + dcx, ox[2 * q + 1] + dcx);
        ty[q] = f2_pack(oy[2 * q] + dcy, oy[2 * q + 1] + dcy);
        tz[q] = f2_pack(oz[2 * q] + dcz, oz[2 * q + 1] + dcz);
      }
      const bool cp = type == CSFMM_LIST_CP;
      const int sb = cp ? v.cbegin[s] : 0;
      const int nsrc = cp ? v.cend[s] - sb : P;
      if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
        const float2 W = weight_total(v, s, r0, cp ? 0 : 1);
#pragma unroll
        for (int q = 0; q < NP; ++q) fold_minus(hi[q], lo[q], W);
      }
      for (int j0 = 0; j0 < nsrc; j0 += kTile) {
        const int nj = min(kTile, nsrc - j0);
        __syncthreads();
        for (int t = threadIdx.x; t < nj; t += nth) {
          float x, y, z, w;
          if (cp) {
            const int j = sb + j0 + t;
            const float4 o = v.off32[j];
            x = o.x; y = o.y; z = o.z;
            w = wr[j];
          } else {
            const int64_t so = (int64_t)s * 3 * P;
            const int k = j0 + t;
            x = v.proxy32[so + k]; y = v.proxy32[so + P + k]; z = v.proxy32[so + 2 * P + k];
            w = wbar[((int64_t)s * ldr + r0) * P + k];
          }
          sA[t] = make_ulonglong2(f2_pack(x, x), f2_pack(y, y));
          sB[t] = make_ulonglong2(f2_pack(z, z), f2_pack(w, w));
        }
        __syncthreads();
        tile_sum_x2<KID, NP, false>(sA, sB, nj, tx, ty, tz, self_none, hi, lo);
      }
    }
  }
#pragma unroll
  for (int h = 0; h < NT; ++h) {
    const int m = threadIdx.x + h * nth;
    double o = f2_total(hi[h / 2], lo[h / 2], h & 1);
    if constexpr (KID == CSFMM_KERNEL_LAPLACE) o *= -(0.69314718055994530942 * kInv4Pi);
    if constexpr (KID == CSFMM_KERNEL_BIHARMONIC) o *= kInv4Pi;
    if (m < P) psi[((int64_t)c * ldr + r0) * P + m] = o;
  }
}

// Scalar far field for Biot-Savart and for several right-hand sides.
template <int KID, int NR>
__global__ void __launch_bounds__(160) far32_kernel(PlanView v, const float *wsf, const float *wbar,
                                                    int ldr, int r0, double *psi) {
  constexpr int DIM = kdim32<KID>();
  constexpr int NT = 2;
  __shared__ float4 sp[kTile];
  __shared__ float sw[NR * kTile];
  const int c = blockIdx.x, P = v.P, nth = blockDim.x;
  const int64_t po = (int64_t)c * 3 * P;
  float ox[NT], oy[NT], oz[NT];
  // running totals over all entries as FP32 (hi, lo) pairs
  float ahi[NT][NR][3], alo[NT][NR][3];
#pragma unroll
  for (int h = 0; h < NT; ++h) {
    const int m = threadIdx.x + h * nth;
    const int mm = m < P ? m : 0;
    ox[h] = v.proxy32[po + mm];
    oy[h] = v.proxy32[po + P + mm];
    oz[h] = v.proxy32[po + 2 * P + mm];
#pragma unroll
    for (int q = 0; q < NR; ++q)
#pragma unroll
      for (int d = 0; d < 3; ++d) ahi[h][q][d] = alo[h][q][d] = 0.f;
  }
  const int self_none[NT] = {-1, -1};
  for (int pass = 0; pass < 2; ++pass) {
    const int type = pass == 0 ? CSFMM_LIST_CP : CSFMM_LIST_CC;
    const int e0 = v.loff[type][c], e1 = v.loff[type][c + 1];
    for (int ee = e0; ee < e1; ++ee) {
      const int s = v.lsrc[type][ee];
      if (!cell_ok(v, s)) continue;
      const float4 dcv = v.ldc[type][ee];
      const float dcx = dcv.x, dcy = dcv.y, dcz = dcv.z;
      float tx[NT], ty[NT], tz[NT];
#pragma unroll
      for (int h = 0; h < NT; ++h) {
        tx[h] = ox[h] + dcx;
        ty[h] = oy[h] + dcy;
        tz[h] = oz[h] + dcz;
      }
      const bool cp = type == CSFMM_LIST_CP;
      const int sb = cp ? v.cbegin[s] : 0;
      const int nsrc = cp ? v.cend[s] - sb : P;
      if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          const float2 W = weight_total(v, s, r0 + q, cp ? 0 : 1);
#pragma unroll
          for (int h = 0; h < NT; ++h) fold_minus(ahi[h][q][0], alo[h][q][0], W);
        }
      }
      for (int j0 = 0; j0 < nsrc; j0 += kTile) {
        const int nj = min(kTile, nsrc - j0);
        __syncthreads();
        for (int t = threadIdx.x; t < nj; t += nth) {
          float4 val;
          float wv[NR];
          if (cp) {
            const int j = sb + j0 + t;
            val = v.off32[j];
#pragma unroll
            for (int q = 0; q < NR; ++q) wv[q] = wsf[(int64_t)(r0 + q) * v.N + j];
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
        }
        __syncthreads();
        tile_sum<KID, NT, NR, false>(sp, sw, nj, tx, ty, tz, self_none, ahi, alo);
      }
    }
  }
#pragma unroll
  for (int h = 0; h < NT; ++h) {
    const int m = threadIdx.x + h * nth;
    if (m >= P) continue;
    double xa[3] = {0.0, 0.0, 0.0};
    if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) {
      xa[0] = v.proxy[po + m];
      xa[1] = v.proxy[po + P + m];
      xa[2] = v.proxy[po + 2 * P + m];
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      double o[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) o[d] = (double)ahi[h][q][d] + (double)alo[h][q][d];
      double *dst = psi + ((int64_t)c * ldr + r0 + q) * DIM * P + m;
      if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
        dst[0] = -(0.69314718055994530942 * kInv4Pi) * o[0];
      } else if constexpr (KID == CSFMM_KERNEL_BIHARMONIC) {
        dst[0] = kInv4Pi * o[0];
      } else if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) {
        dst[0] = kInv2Pi * (xa[1] * o[2] - xa[2] * o[1]);
        dst[P] = kInv2Pi * (xa[2] * o[0] - xa[0] * o[2]);
        dst[2 * P] = kInv2Pi * (xa[0] * o[1] - xa[1] * o[0]);
      } else {
        dst[0] = o[0];
      }
    }
  }
}

template <int KID>
void launch_far_kid(const PlanView &v, int ncells, const float *wsf, const float *wbar, int ldr,
                    int r0, int nr, double *psi, cudaStream_t st, const float *cpart) {
  const int nth = ((v.P + 63) / 64) * 32;  // 2 targets per thread
  if constexpr (KID != CSFMM_KERNEL_BIOT_SAVART) {
    if (nr == 1) {
      const int per = 64 * kFarNP;  // targets of one warp
      far32x2_kernel<KID><<<ncells, ((v.P + per - 1) / per) * 32, 0, st>>>(v, wsf, wbar, ldr,
                                                                            r0, psi, cpart);
      return;
    }
  }
  switch (nr) {
    case 1: far32_kernel<KID, 1><<<ncells, nth, 0, st>>>(v, wsf, wbar, ldr, r0, psi); break;
    case 2: far32_kernel<KID, 2><<<ncells, nth, 0, st>>>(v, wsf, wbar, ldr, r0, psi); break;
    case 3: far32_kernel<KID, 3><<<ncells, nth, 0, st>>>(v, wsf, wbar, ldr, r0, psi); break;
    default: far32_kernel<KID, 4><<<ncells, nth, 0, st>>>(v, wsf, wbar, ldr, r0, psi); break;
  }
}


template <int KID, int NR>
void launch_nr(const PlanView &v, const int32_t *leaves, int nleaves, const float *wsf, int ldw,
               const float *wbar, int ldr, int r0, double *phi, cudaStream_t st,
               const float *part) {
  if constexpr (NR == 1 && KID != CSFMM_KERNEL_BIOT_SAVART) {
    near32x2_kernel<KID, kNearNP><<<nleaves, kNearThreads, 0, st>>>(v, leaves, wsf, wbar, ldr, r0,
                                                                  phi, part);
  } else {
    near32_kernel<KID, 2, NR><<<nleaves, kThreads, 0, st>>>(v, leaves, wsf, ldw, wbar, ldr, r0, phi);
  }
}

template <int KID>
void launch_kid(const PlanView &v, const int32_t *leaves, int nleaves, const float *wsf, int ldw,
                const float *wbar, int ldr, int r0, int nr, double *phi, cudaStream_t st,
                const float *part) {
  switch (nr) {
    case 1: launch_nr<KID, 1>(v, leaves, nleaves, wsf, ldw, wbar, ldr, r0, phi, st, part); break;
    case 2: launch_nr<KID, 2>(v, leaves, nleaves, wsf, ldw, wbar, ldr, r0, phi, st, nullptr); break;
    case 3: launch_nr<KID, 3>(v, leaves, nleaves, wsf, ldw, wbar, ldr, r0, phi, st, nullptr); break;
    default: launch_nr<KID, 4>(v, leaves, nleaves, wsf, ldw, wbar, ldr, r0, phi, st, nullptr); break;
  }
}

}  // namespace

// nr right-hand sides r0 .. r0+nr-1 (nr <= 4); psi [nc][ldr][dim][P] FP64.
void launch_far32(const PlanView &v, int ncells, const float *wsf, const float *wbar, int ldr,
                  int r0, int nr, double *psi, cudaStream_t st, const float *cpart) {
  switch (v.kernel_id) {
    case CSFMM_KERNEL_LAPLACE: launch_far_kid<CSFMM_KERNEL_LAPLACE>(v, ncells, wsf, wbar, ldr, r0, nr, psi, st, cpart); break;
    case CSFMM_KERNEL_BIOT_SAVART: launch_far_kid<CSFMM_KERNEL_BIOT_SAVART>(v, ncells, wsf, wbar, ldr, r0, nr, psi, st, nullptr); break;
    case CSFMM_KERNEL_NEWTON: launch_far_kid<CSFMM_KERNEL_NEWTON>(v, ncells, wsf, wbar, ldr, r0, nr, psi, st, cpart); break;
    case CSFMM_KERNEL_SAL: launch_far_kid<CSFMM_KERNEL_SAL>(v, ncells, wsf, wbar, ldr, r0, nr, psi, st, cpart); break;
    case CSFMM_KERNEL_BIHARMONIC: launch_far_kid<CSFMM_KERNEL_BIHARMONIC>(v, ncells, wsf, wbar, ldr, r0, nr, psi, st, cpart); break;
    default: launch_far_kid<CSFMM_KERNEL_ONE>(v, ncells, wsf, wbar, ldr, r0, nr, psi, st, cpart); break;
  }
}

// nr right-hand sides r0 .. r0+nr-1 (nr <= 4).
void launch_near32(const PlanView &v, const int32_t *leaves, int nleaves, const float *wsf, int ldw,
                   const float *wbar, int ldr, int r0, int nr, double *phi, cudaStream_t st,
                   const float *part) {
  switch (v.kernel_id) {
    case CSFMM_KERNEL_LAPLACE: launch_kid<CSFMM_KERNEL_LAPLACE>(v, leaves, nleaves, wsf, ldw, wbar, ldr, r0, nr, phi, st, part); break;
    case CSFMM_KERNEL_BIOT_SAVART: launch_kid<CSFMM_KERNEL_BIOT_SAVART>(v, leaves, nleaves, wsf, ldw, wbar, ldr, r0, nr, phi, st, nullptr); break;
    case CSFMM_KERNEL_NEWTON: launch_kid<CSFMM_KERNEL_NEWTON>(v, leaves, nleaves, wsf, ldw, wbar, ldr, r0, nr, phi, st, part); break;
    case CSFMM_KERNEL_SAL: launch_kid<CSFMM_KERNEL_SAL>(v, leaves, nleaves, wsf, ldw, wbar, ldr, r0, nr, phi, st, part); break;
    case CSFMM_KERNEL_BIHARMONIC: launch_kid<CSFMM_KERNEL_BIHARMONIC>(v, leaves, nleaves, wsf, ldw, wbar, ldr, r0, nr, phi, st, part); break;
    default: launch_kid<CSFMM_KERNEL_ONE>(v, leaves, nleaves, wsf, ldw, wbar, ldr, r0, nr, phi, st, part); break;
  }
}

void launch_pp_sym32(const PlanView &v, const int2 *pairs, const int32_t *off, int npairs,
                     const float *wsf, float *part, cudaStream_t st) {
  if (npairs <= 0) return;
#define CSFMM_PPSYM(K) \
  sym_kernel<K, false, kSymQP><<<npairs, kSymThreads, 0, st>>>(v, pairs, off, nullptr, wsf, 0, part)
  switch (v.kernel_id) {
    case CSFMM_KERNEL_LAPLACE: CSFMM_PPSYM(CSFMM_KERNEL_LAPLACE); break;
    case CSFMM_KERNEL_NEWTON: CSFMM_PPSYM(CSFMM_KERNEL_NEWTON); break;
    case CSFMM_KERNEL_SAL: CSFMM_PPSYM(CSFMM_KERNEL_SAL); break;
    case CSFMM_KERNEL_BIHARMONIC: CSFMM_PPSYM(CSFMM_KERNEL_BIHARMONIC); break;
    default: CSFMM_PPSYM(CSFMM_KERNEL_ONE); break;
  }
#undef CSFMM_PPSYM
}

namespace {
template <int KID>
void launch_cc_sym_kid(const PlanView &v, const int2 *pairs, const int32_t *entry, int npairs,
                       const float *wbar, int ldr, float *part, cudaStream_t st) {
  // row pairs per lane: the P rows of a pass with few idle lanes
  if (v.P <= 128)
    sym_kernel<KID, true, 2><<<npairs, kSymThreads, 0, st>>>(v, pairs, nullptr, entry, wbar, ldr, part);
  else if (v.P <= 192)
    sym_kernel<KID, true, 3><<<npairs, kSymThreads, 0, st>>>(v, pairs, nullptr, entry, wbar, ldr, part);
  else
    sym_kernel<KID, true, 4><<<npairs, kSymThreads, 0, st>>>(v, pairs, nullptr, entry, wbar, ldr, part);
}
}  // namespace

void launch_cc_sym32(const PlanView &v, const int2 *pairs, const int32_t *entry, int npairs,
                     const float *wbar, int ldr, float *part, cudaStream_t st) {
  if (npairs <= 0) return;
  switch (v.kernel_id) {
    case CSFMM_KERNEL_LAPLACE: launch_cc_sym_kid<CSFMM_KERNEL_LAPLACE>(v, pairs, entry, npairs, wbar, ldr, part, st); break;
    case CSFMM_KERNEL_NEWTON: launch_cc_sym_kid<CSFMM_KERNEL_NEWTON>(v, pairs, entry, npairs, wbar, ldr, part, st); break;
    case CSFMM_KERNEL_SAL: launch_cc_sym_kid<CSFMM_KERNEL_SAL>(v, pairs, entry, npairs, wbar, ldr, part, st); break;
    case CSFMM_KERNEL_BIHARMONIC: launch_cc_sym_kid<CSFMM_KERNEL_BIHARMONIC>(v, pairs, entry, npairs, wbar, ldr, part, st); break;
    default: launch_cc_sym_kid<CSFMM_KERNEL_ONE>(v, pairs, entry, npairs, wbar, ldr, part, st); break;
  }
}

}  // namespace csfmm
