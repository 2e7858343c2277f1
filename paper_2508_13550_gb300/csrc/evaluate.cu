// evaluate.cu -- one CSFMM evaluation (Algorithm "CSFMM") on a built plan:
//   gather     weights into tree order
//   P2M        leaf proxy weights, Eq. (PC) right-hand side          (Sec. 6)
//   M2M        parent proxy weights from children, Eq. (upwardpass2) (Sec. 6)
//   far        CP and CC proxy potentials of every target cell,
//              Eqs. (CP), (CC), accumulated as Eq. (CP_CC_accumulated) (Sec. 8)
//   near       PP and PC potentials at the target particles, Eqs. (PP), (PC)
//   L2L        parent proxy potentials interpolated to child proxies,
//              Eq. (downward_2), top-down                             (Sec. 8.1)
//   L2P        leaf proxy potentials interpolated to the particles, added to
//              the near-field potentials, written in input order
//
// Two precision forms share the structure (template parameter Real):
//   double  everything in FP64;
//   float   kernel evaluations on pair-relative FP32 coordinates: the centre
//           difference c_T - c_S of a (target, source) cell pair is formed in
//           FP64 and rounded once, particles and proxies carry FP32 offsets
//           from their cell centre; sums over one source cell in FP32, sums
//           across source cells and the final per-target value in FP64.
// Every target cell or leaf is owned by one thread block, so no atomics are
// used and results are deterministic.
#include <math.h>

#include "csfmm_internal.cuh"
#include "dilog.cuh"
#include "downward_df.cuh"

namespace csfmm {

namespace {

constexpr int kRB = 4;  // right-hand sides per kernel pass

template <typename Real>
__device__ __forceinline__ const Real *La_of(const PlanView &v);
template <>
__device__ __forceinline__ const double *La_of<double>(const PlanView &v) { return v.La64; }
template <>
__device__ __forceinline__ const float *La_of<float>(const PlanView &v) { return v.La32; }
template <typename Real>
__device__ __forceinline__ const Real *Lb_of(const PlanView &v);
template <>
__device__ __forceinline__ const double *Lb_of<double>(const PlanView &v) { return v.Lb64; }
template <>
__device__ __forceinline__ const float *Lb_of<float>(const PlanView &v) { return v.Lb32; }
template <typename Real>
__device__ __forceinline__ const Real *M_of(const PlanView &v);
template <>
__device__ __forceinline__ const double *M_of<double>(const PlanView &v) { return v.m2m64; }
// Shrunk boxes: the [2][p][p] matrices from child cell c to its parent (the
// FP32-bulk form reads its double-float copies in the _df kernels).
template <typename Real>
__device__ __forceinline__ const Real *Mcell_of(const PlanView &v, int c);
template <>
__device__ __forceinline__ const double *Mcell_of<double>(const PlanView &v, int c) {
  return v.mcell64 + (int64_t)c * 2 * v.p * v.p;
}

// FP64 kernel factors of the reference form (the FP32-bulk kernels live in
// interact32.cu).
__device__ __forceinline__ double fast_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ double fast_log2(double x) { return log2(x); }
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }

// ---------------------------------------------------------------------------
// Kernel sums.  For a fixed target x and a tile of sources y_j with weights
// w_j and r_j = x - y_j (d2 = |r_j|^2), the kernel factor f_j is computed once
// per source and shared by all right-hand sides:
//   Laplace      f = log2(d2);  a += w f, sw += w;  value = -(ln 2/(4 pi)) (a - sw)
//                (since -(1/4pi) ln(d2/2) = -(ln2/4pi)(log2 d2 - 1))
//   Newtonian    f = 1/sqrt(d2);  a += w f
//   Biot-Savart  f = 1/d2;  a += w f r (3 components);  value = (1/(2 pi)) x cross a
//                (since x cross y = -x cross r and 1 - x.y = d2/2)
//   biharmonic   f = dilog(1 - d2/4);  a += w f;  value = a / (4 pi)
//   SAL          f = (1 - b0)/sqrt(d2) - (a1 - b1) ln(t + t^2), t = sqrt(d2)/2;  a += w f
//   K = 1        a += w
// ---------------------------------------------------------------------------
template <int KID, typename Real>
struct KFac {
  Real f, rx, ry, rz;
  __device__ __forceinline__ KFac(Real x, Real y, Real z) : rx(x), ry(y), rz(z) {
    Real d2 = x * x + y * y + z * z;
    if constexpr (KID == CSFMM_KERNEL_LAPLACE) f = fast_log2(d2);
    else if constexpr (KID == CSFMM_KERNEL_NEWTON) f = fast_rsqrt(d2);
    else if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) f = fast_rcp(d2);
    else if constexpr (KID == CSFMM_KERNEL_BIHARMONIC) f = (Real)dilog64(1.0 - 0.25 * (double)d2);
    else if constexpr (KID == CSFMM_KERNEL_SAL) f = sal64(d2);
    else f = 1;
  }
};

template <int KID, typename Real>
struct Acc {
  Real a0 = 0, a1 = 0, a2 = 0, sw = 0;
  __device__ __forceinline__ void add(const KFac<KID, Real> &k, Real w) {
    if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
      a0 += w * k.f;
      sw += w;
    } else if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) {
      Real q = w * k.f;
      a0 += q * k.rx;
      a1 += q * k.ry;
      a2 += q * k.rz;
    } else if constexpr (KID == CSFMM_KERNEL_NEWTON || KID == CSFMM_KERNEL_BIHARMONIC ||
                         KID == CSFMM_KERNEL_SAL) {
      a0 += w * k.f;
    } else {
      a0 += w;
    }
  }
  // Adds the tile's kernel sum into out[0..dim) (FP64); x = target position.
  __device__ __forceinline__ void flush(double *out, double x0, double x1, double x2) const {
    if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
      out[0] += -(0.69314718055994530942 * kInv4Pi) * ((double)a0 - (double)sw);
    } else if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) {
      double b0 = a0, b1 = a1, b2 = a2;
      out[0] += kInv2Pi * (x1 * b2 - x2 * b1);
      out[1] += kInv2Pi * (x2 * b0 - x0 * b2);
      out[2] += kInv2Pi * (x0 * b1 - x1 * b0);
    } else if constexpr (KID == CSFMM_KERNEL_BIHARMONIC) {
      out[0] += kInv4Pi * (double)a0;
    } else {
      out[0] += (double)a0;
    }
  }
};

template <int KID>
constexpr int kdim() {
  return KID == CSFMM_KERNEL_BIOT_SAVART ? 3 : 1;
}

// ---------------------------------------------------------------------------
// gather: ws[r][i] = w[r][perm[i]] (zero for a target-only point, perm[i] >= nsrc)
// ---------------------------------------------------------------------------
__global__ void gather_kernel(const int32_t *perm, const double *w, double *ws, float *wsf, int N,
                              int nrhs, int ld_ws, int nsrc) {
  int64_t total = (int64_t)N * nrhs;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(q / N);
    int i = (int)(q - (int64_t)r * N);
    const int j = perm[i];
    double x = j < nsrc ? w[(int64_t)r * nsrc + j] : 0.0;
    ws[(int64_t)r * ld_ws + i] = x;
    if (wsf) wsf[(int64_t)r * ld_ws + i] = (float)x;
  }
}

__device__ __forceinline__ float2 split_f32(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

// ---------------------------------------------------------------------------
// P2M: for leaf c, wbar[c][r][k1 p + k2] = sum_j La[j][k1] Lb[j][k2] w_r[j].
// One block per leaf (blockDim >= P), one thread per proxy; the Lagrange
// rows of CH points at a time are staged through shared memory (coalesced)
// and each chunk's sum is added to an FP64 total.  The FP32 form reads the
// stochastically rounded rows, so the rounding errors of the rows (and of
// their products) differ from leaf to leaf even where every leaf holds the
// same local point pattern.
// ---------------------------------------------------------------------------
template <typename Real, int NR>
__global__ void p2m_kernel(PlanView v, const int32_t *leaves, const double *ws, int ldw, int r0,
                           Real *wbar, int ldr, float2 *wtot) {
  constexpr int CH = 64;
  __shared__ Real sLa[CH * kMaxP], sLb[CH * kMaxP];
  __shared__ __align__(16) Real sw[CH * NR];  // [point][rhs]: one vector load per point
  const int c = leaves[blockIdx.x];
  if (!cell_ok(v, c)) return;
  const int b = v.cbegin[c], e = v.cend[c], p = v.p, P = v.P;
  const Real *La = La_of<Real>(v), *Lb = Lb_of<Real>(v);
  const int k = threadIdx.x;
  const int k1 = k / p, k2 = k - (k / p) * p;
  double acc[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) acc[q] = 0.0;
  for (int j0 = b; j0 < e; j0 += CH) {
    const int nj = min(CH, e - j0);
    __syncthreads();
    for (int t = threadIdx.x; t < nj * p; t += blockDim.x) {
      sLa[t] = La[(int64_t)j0 * p + t];
      sLb[t] = Lb[(int64_t)j0 * p + t];
    }
    for (int t = threadIdx.x; t < NR * CH; t += blockDim.x) {
      const int q = t / CH, j = t - q * CH;
      sw[j * NR + q] = j < nj ? (Real)ws[(int64_t)(r0 + q) * ldw + j0 + j] : (Real)0;
    }
    __syncthreads();
    if (k < P) {
      Real ch[NR];
#pragma unroll
      for (int q = 0; q < NR; ++q) ch[q] = 0;
      for (int j = 0; j < nj; ++j) {
        const Real l = sLa[j * p + k1] * sLb[j * p + k2];
#pragma unroll
        for (int q = 0; q < NR; ++q) ch[q] += l * sw[j * NR + q];
      }
#pragma unroll
      for (int q = 0; q < NR; ++q) acc[q] += (double)ch[q];
    }
  }
  if (k < P) {
#pragma unroll
    for (int q = 0; q < NR; ++q) wbar[((int64_t)c * ldr + r0 + q) * P + k] = (Real)acc[q];
  }
  if constexpr (sizeof(Real) == 4) {
    if (wtot) {
      // totals of the leaf's FP32 particle weights (u < NR) and of its FP32
      // proxy weights (u >= NR), summed in FP64 in a fixed order
      __shared__ double red[2 * NR][32];
      double a[2 * NR];
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        a[q] = 0.0;
        for (int j = b + threadIdx.x; j < e; j += blockDim.x)
          a[q] += (double)(float)ws[(int64_t)(r0 + q) * ldw + j];
        a[NR + q] = k < P ? (double)(Real)acc[q] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 2 * NR; ++u) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a[u] += __shfl_xor_sync(0xffffffffu, a[u], o);
        if ((threadIdx.x & 31) == 0) red[u][threadIdx.x >> 5] = a[u];
      }
      __syncthreads();
      if (threadIdx.x < 2 * NR) {
        const int u = threadIdx.x, q = u % NR, kind = u / NR;
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[u][w];
        wtot[((int64_t)c * ldr + r0 + q) * 2 + kind] = split_f32(t);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// M2M at one level: parent wbar = sum_c (M_qa (x) M_qb) child wbar.
// One block per cell of the level (leaves exit), threads over proxies.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void m2m_kernel(PlanView v, int cell0, int r0, int nr, Real *wbar, int ldr) {
  __shared__ Real sM[2 * kMaxP * kMaxP];
  __shared__ Real sw[kMaxP * kMaxP], st[kMaxP * kMaxP];
  const int c = cell0 + blockIdx.x;
  const int p = v.p, P = v.P;
  const int32_t *ch = v.cchild + 4 * c;
  if (ch[0] < 0 && ch[1] < 0 && ch[2] < 0 && ch[3] < 0) return;
  const Real *M = M_of<Real>(v);
  for (int t = threadIdx.x; t < 2 * p * p; t += blockDim.x) sM[t] = M[t];
  for (int r = r0; r < r0 + nr; ++r) {
    Real acc[(kMaxP * kMaxP + 127) / 128];
    const int nper = (P + blockDim.x - 1) / blockDim.x;
    for (int u = 0; u < nper; ++u) acc[u] = 0;
    for (int q = 0; q < 4; ++q) {
      int cc = ch[q];
      if (cc < 0) continue;
      int qa = q & 1, qb = q >> 1;
      __syncthreads();
      if (v.mcell64) {  // shrunk boxes: this child's own matrices
        const Real *Mc = Mcell_of<Real>(v, cc);
        for (int t = threadIdx.x; t < 2 * p * p; t += blockDim.x) sM[t] = Mc[t];
        qa = 0;
        qb = 1;
      }
      for (int t = threadIdx.x; t < P; t += blockDim.x) sw[t] = wbar[((int64_t)cc * ldr + r) * P + t];
      __syncthreads();
      // st[m1][k2] = sum_m2 M[qb][k2][m2] w[m1][m2]
      for (int t = threadIdx.x; t < P; t += blockDim.x) {
        int m1 = t / p, k2 = t - m1 * p;
        const Real *Mr = sM + (qb * p + k2) * p;
        Real s = 0;
        for (int m2 = 0; m2 < p; ++m2) s += Mr[m2] * sw[m1 * p + m2];
        st[t] = s;
      }
      __syncthreads();
      // acc[k1][k2] += sum_m1 M[qa][k1][m1] st[m1][k2]
      for (int u = 0, t = threadIdx.x; t < P; ++u, t += blockDim.x) {
        int k1 = t / p, k2 = t - k1 * p;
        const Real *Mr = sM + (qa * p + k1) * p;
        Real s = 0;
        for (int m1 = 0; m1 < p; ++m1) s += Mr[m1] * st[m1 * p + k2];
        acc[u] += s;
      }
    }
    for (int u = 0, t = threadIdx.x; t < P; ++u, t += blockDim.x)
      wbar[((int64_t)c * ldr + r) * P + t] = acc[u];
  }
}

// M2M of the FP32 form: same contraction as m2m_kernel with the matrices as
// FP32 rounding + remainder (m2m32) and every sum in double-float; proxy
// weights are stored in FP32.  The same constant matrices act on every cell
// of every level, and the proxy weights of a smooth field repeat nearly the
// same pattern from cell to cell, so rounding the contraction to FP32 biases
// all proxy weights alike (measured: a relative bias of up to 8e-8 in the
// potentials at degree 8); in double-float that bias is gone.
constexpr int kM2MThreads = 192;  // one thread per parent proxy at P <= 192
constexpr int kM2MWarps = kM2MThreads / 32;
__global__ void __launch_bounds__(kM2MThreads) m2m_df_kernel(PlanView v, int cell0, int r0, int nr,
                                                             float *wbar, int ldr, float2 *wtot) {
  // per right-hand side and warp (launched with kM2MThreads threads): partial
  // totals of the cell's proxy weights
  __shared__ double red[kMaxNrhs][kM2MWarps];
  __shared__ float sMh[2 * kMaxP * kMaxP], sMl[2 * kMaxP * kMaxP];
  __shared__ float sw[kMaxP * kMaxP], sth[kMaxP * kMaxP], stl[kMaxP * kMaxP];
  const int c = cell0 + blockIdx.x;
  const int p = v.p, P = v.P;
  const int32_t *ch = v.cchild + 4 * c;
  if (ch[0] < 0 && ch[1] < 0 && ch[2] < 0 && ch[3] < 0) return;
  for (int t = threadIdx.x; t < 2 * p * p; t += blockDim.x) {
    sMh[t] = v.m2m32[t];
    sMl[t] = v.m2m32[2 * p * p + t];
  }
  for (int r = r0; r < r0 + nr; ++r) {
    constexpr int kPer = (kMaxP * kMaxP + kM2MThreads - 1) / kM2MThreads;
    float ah[kPer], al[kPer];
    for (int u = 0; u < kPer; ++u) ah[u] = al[u] = 0.f;
    for (int q = 0; q < 4; ++q) {
      const int cc = ch[q];
      if (cc < 0) continue;
      int qa = q & 1, qb = q >> 1;
      __syncthreads();
      if (v.mcell32) {  // shrunk boxes: this child's own matrices
        const float *Mc = v.mcell32 + (int64_t)cc * 4 * p * p;
        for (int t = threadIdx.x; t < 2 * p * p; t += blockDim.x) {
          sMh[t] = Mc[t];
          sMl[t] = Mc[2 * p * p + t];
        }
        qa = 0;
        qb = 1;
      }
      for (int t = threadIdx.x; t < P; t += blockDim.x) sw[t] = wbar[((int64_t)cc * ldr + r) * P + t];
      __syncthreads();
      // st[m1][k2] = sum_m2 M[qb][k2][m2] w[m1][m2]
      for (int t = threadIdx.x; t < P; t += blockDim.x) {
        const int m1 = t / p, k2 = t - m1 * p;
        const int o = (qb * p + k2) * p;
        float sh = 0.f, sl = 0.f;
        for (int m2 = 0; m2 < p; ++m2) df_acc_prod(sh, sl, sMh[o + m2], sMl[o + m2], sw[m1 * p + m2], 0.f);
        sth[t] = sh;
        stl[t] = sl;
      }
      __syncthreads();
      // acc[k1][k2] += sum_m1 M[qa][k1][m1] st[m1][k2]
      for (int u = 0, t = threadIdx.x; t < P; ++u, t += blockDim.x) {
        const int k1 = t / p, k2 = t - k1 * p;
        const int o = (qa * p + k1) * p;
        for (int m1 = 0; m1 < p; ++m1)
          df_acc_prod(ah[u], al[u], sMh[o + m1], sMl[o + m1], sth[m1 * p + k2], stl[m1 * p + k2]);
      }
    }
    double tq = 0.0;
    for (int u = 0, t = threadIdx.x; t < P; ++u, t += blockDim.x) {
      const float o = __fadd_rn(ah[u], al[u]);
      wbar[((int64_t)c * ldr + r) * P + t] = o;
      tq += (double)o;
    }
    if (wtot) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tq += __shfl_xor_sync(0xffffffffu, tq, o);
      if ((threadIdx.x & 31) == 0) red[r - r0][threadIdx.x >> 5] = tq;
    }
  }
  if (wtot) {  // totals of the cell's FP32 proxy weights, fixed summation order
    __syncthreads();
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      double s = 0.0;
      for (int w = 0; w < kM2MWarps; ++w) s += red[r][w];
      wtot[((int64_t)c * ldr + r0 + r) * 2 + 1] = split_f32(s);
    }
  }
}

// ---------------------------------------------------------------------------
// L2L at one level: child psi += (M_qa (x) M_qb)^T parent psi.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void l2l_kernel(PlanView v, int cell0, int r0, int nr, int dim, Real *psi, int ldr) {
  __shared__ Real sM[2 * kMaxP * kMaxP];
  __shared__ Real sp[kMaxP * kMaxP], st[kMaxP * kMaxP];
  const int c = cell0 + blockIdx.x;
  const int p = v.p, P = v.P;
  const int32_t *ch = v.cchild + 4 * c;
  if (ch[0] < 0 && ch[1] < 0 && ch[2] < 0 && ch[3] < 0) return;
  const Real *M = M_of<Real>(v);
  for (int t = threadIdx.x; t < 2 * p * p; t += blockDim.x) sM[t] = M[t];
  for (int r = r0; r < r0 + nr; ++r)
    for (int d = 0; d < dim; ++d) {
      __syncthreads();
      for (int t = threadIdx.x; t < P; t += blockDim.x)
        sp[t] = psi[(((int64_t)c * ldr + r) * dim + d) * P + t];
      for (int q = 0; q < 4; ++q) {
        int cc = ch[q];
        if (cc < 0) continue;
        int qa = q & 1, qb = q >> 1;
        __syncthreads();
        if (v.mcell64) {  // shrunk boxes: this child's own matrices
          const Real *Mc = Mcell_of<Real>(v, cc);
          for (int t = threadIdx.x; t < 2 * p * p; t += blockDim.x) sM[t] = Mc[t];
          qa = 0;
          qb = 1;
          __syncthreads();
        }
        // st[m1][n2] = sum_m2 psi[m1][m2] M[qb][m2][n2]
        for (int t = threadIdx.x; t < P; t += blockDim.x) {
          int m1 = t / p, n2 = t - m1 * p;
          Real s = 0;
          for (int m2 = 0; m2 < p; ++m2) s += sp[m1 * p + m2] * sM[(qb * p + m2) * p + n2];
          st[t] = s;
        }
        __syncthreads();
        Real *dst = psi + (((int64_t)cc * ldr + r) * dim + d) * P;
        for (int t = threadIdx.x; t < P; t += blockDim.x) {
          int n1 = t / p, n2 = t - n1 * p;
          Real s = 0;
          for (int m1 = 0; m1 < p; ++m1) s += sM[(qa * p + m1) * p + n1] * st[m1 * p + n2];
          dst[t] += s;
        }
      }
    }
}

// L2L of the FP32 form (downward_df.cuh), one block per parent cell of a level.
__global__ void l2l_df_kernel(PlanView v, int cell0, int r0, int nr, int dim, double *psi,
                              int ldr) {
  __shared__ float sm[kL2LDfSmemFloats];
  l2l_df_cell(v, cell0 + blockIdx.x, r0, nr, dim, psi, ldr, sm);
}

// ---------------------------------------------------------------------------
// far: psi[c][r][d][m] = sum over CP sources (particles) and CC sources
// (proxies) of K(t_m, y) w.  One block per cell (all cells; cells without
// CP/CC entries write zeros), one thread per target proxy m.
// ---------------------------------------------------------------------------
constexpr int kFarTile = 128;

template <int KID, typename Real, int NR>
__global__ void far_kernel(PlanView v, const double *ws, int ldw, const Real *wbar, int ldr,
                           int r0, Real *psi) {
  constexpr int nr = NR;
  // psi[c][r][d][m] with rhs stride ldr
  constexpr int DIM = kdim<KID>();
  __shared__ Real sx[kFarTile], sy[kFarTile], sz[kFarTile], sw[kRB * kFarTile];
  const int c = blockIdx.x;
  const int P = v.P;
  const int m = threadIdx.x;
  const bool active = m < P;
  double out[NR][DIM];
#pragma unroll
  for (int q = 0; q < NR; ++q)
#pragma unroll
    for (int d = 0; d < DIM; ++d) out[q][d] = 0.0;
  // target proxy: absolute (FP64 form) or offset from the cell centre (FP32 form)
  const int64_t po = (int64_t)c * 3 * P;
  double tx = 0, ty = 0, tz = 0;  // absolute target position (for Biot-Savart)
  Real ox = 0, oy = 0, oz = 0;    // offset from centre
  if (active) {
    tx = v.proxy[po + m];
    ty = v.proxy[po + P + m];
    tz = v.proxy[po + 2 * P + m];
    ox = (Real)v.proxy32[po + m];
    oy = (Real)v.proxy32[po + P + m];
    oz = (Real)v.proxy32[po + 2 * P + m];
  }
  const double cTx = v.ccentre[3 * c], cTy = v.ccentre[3 * c + 1], cTz = v.ccentre[3 * c + 2];
  for (int pass = 0; pass < 2; ++pass) {
    const int type = pass == 0 ? CSFMM_LIST_CP : CSFMM_LIST_CC;
    const int e0 = v.loff[type][c], e1 = v.loff[type][c + 1];
    for (int e = e0; e < e1; ++e) {
      const int s = v.lsrc[type][e];
      // pair-relative target coordinates (FP32 form): t = offset + (c_T - c_S)
      Real rx0, ry0, rz0;
      if constexpr (sizeof(Real) == 4) {
        rx0 = ox + (Real)(cTx - v.ccentre[3 * s]);
        ry0 = oy + (Real)(cTy - v.ccentre[3 * s + 1]);
        rz0 = oz + (Real)(cTz - v.ccentre[3 * s + 2]);
      } else {
        rx0 = tx;
        ry0 = ty;
        rz0 = tz;
      }
      const int nsrc = (type == CSFMM_LIST_CP) ? v.cend[s] - v.cbegin[s] : P;
      for (int j0 = 0; j0 < nsrc; j0 += kFarTile) {
        const int nj = min(kFarTile, nsrc - j0);
        __syncthreads();
        for (int t = threadIdx.x; t < nj; t += blockDim.x) {
          if (type == CSFMM_LIST_CP) {
            const int j = v.cbegin[s] + j0 + t;
            if constexpr (sizeof(Real) == 4) {
              float4 o = v.off32[j];
              sx[t] = o.x; sy[t] = o.y; sz[t] = o.z;
            } else {
              sx[t] = v.x[j]; sy[t] = v.x[v.N + j]; sz[t] = v.x[2 * (int64_t)v.N + j];
            }
#pragma unroll
            for (int q = 0; q < NR; ++q) sw[q * kFarTile + t] = (Real)ws[(int64_t)(r0 + q) * ldw + j];
          } else {
            const int64_t so = (int64_t)s * 3 * P;
            const int k = j0 + t;
            if constexpr (sizeof(Real) == 4) {
              sx[t] = v.proxy32[so + k]; sy[t] = v.proxy32[so + P + k]; sz[t] = v.proxy32[so + 2 * P + k];
            } else {
              sx[t] = v.proxy[so + k]; sy[t] = v.proxy[so + P + k]; sz[t] = v.proxy[so + 2 * P + k];
            }
#pragma unroll
            for (int q = 0; q < NR; ++q) sw[q * kFarTile + t] = wbar[((int64_t)s * ldr + r0 + q) * P + k];
          }
        }
        __syncthreads();
        if (active) {
          Acc<KID, Real> acc[NR];
          for (int j = 0; j < nj; ++j) {
            KFac<KID, Real> kf(rx0 - sx[j], ry0 - sy[j], rz0 - sz[j]);
#pragma unroll
            for (int q = 0; q < NR; ++q) acc[q].add(kf, sw[q * kFarTile + j]);
          }
#pragma unroll
          for (int q = 0; q < NR; ++q) acc[q].flush(out[q], tx, ty, tz);
        }
      }
    }
  }
  if (active) {
    for (int q = 0; q < nr; ++q)
#pragma unroll
      for (int d = 0; d < DIM; ++d) psi[(((int64_t)c * ldr + r0 + q) * DIM + d) * P + m] = (Real)out[q][d];
  }
}

// ---------------------------------------------------------------------------
// near: phi[r][i][d] = sum over PP sources (particles, i = j omitted) and PC
// sources (proxies) of K(x_i, y) w.  One block per leaf, one thread per
// target particle (looping over chunks of the block size).
// ---------------------------------------------------------------------------
constexpr int kNearTile = 128;

template <int KID, typename Real, int NR>
__global__ void near_kernel(PlanView v, const int32_t *leaves, const double *ws, int ldw,
                            const Real *wbar, int ldr, int r0, double *phi) {
  constexpr int nr = NR;
  constexpr int DIM = kdim<KID>();
  __shared__ Real sx[kNearTile], sy[kNearTile], sz[kNearTile], sw[kRB * kNearTile];
  const int c = leaves[blockIdx.x];
  if (!cell_ok(v, c)) return;
  const int b = v.cbegin[c], e = v.cend[c];
  const int P = v.P;
  const double cTx = v.ccentre[3 * c], cTy = v.ccentre[3 * c + 1], cTz = v.ccentre[3 * c + 2];
  for (int i0 = b; i0 < e; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    const bool active = i < e;
    double out[NR][DIM];
#pragma unroll
    for (int q = 0; q < NR; ++q)
#pragma unroll
      for (int d = 0; d < DIM; ++d) out[q][d] = 0.0;
    double tx = 0, ty = 0, tz = 0;
    Real ox = 0, oy = 0, oz = 0;
    if (active) {
      tx = v.x[i];
      ty = v.x[v.N + i];
      tz = v.x[2 * (int64_t)v.N + i];
      float4 o = v.off32[i];
      ox = o.x; oy = o.y; oz = o.z;
    }
    for (int pass = 0; pass < 2; ++pass) {
      const int type = pass == 0 ? CSFMM_LIST_PP : CSFMM_LIST_PC;
      const int e0 = v.loff[type][c], e1 = v.loff[type][c + 1];
      for (int ee = e0; ee < e1; ++ee) {
        const int s = v.lsrc[type][ee];
        if (!cell_ok(v, s)) continue;
        Real rx0, ry0, rz0;
        if constexpr (sizeof(Real) == 4) {
          rx0 = ox + (Real)(cTx - v.ccentre[3 * s]);
          ry0 = oy + (Real)(cTy - v.ccentre[3 * s + 1]);
          rz0 = oz + (Real)(cTz - v.ccentre[3 * s + 2]);
        } else {
          rx0 = tx;
          ry0 = ty;
          rz0 = tz;
        }
        const bool pp = type == CSFMM_LIST_PP;
        const int sb = pp ? v.cbegin[s] : 0;
        const int nsrc = pp ? v.cend[s] - v.cbegin[s] : P;
        const int self = (pp && s == c) ? i - sb : -1;  // index of x_i among the sources
        for (int j0 = 0; j0 < nsrc; j0 += kNearTile) {
          const int nj = min(kNearTile, nsrc - j0);
          __syncthreads();
          for (int t = threadIdx.x; t < nj; t += blockDim.x) {
            if (pp) {
              const int j = sb + j0 + t;
              if constexpr (sizeof(Real) == 4) {
                float4 o = v.off32[j];
                sx[t] = o.x; sy[t] = o.y; sz[t] = o.z;
              } else {
                sx[t] = v.x[j]; sy[t] = v.x[v.N + j]; sz[t] = v.x[2 * (int64_t)v.N + j];
              }
#pragma unroll
              for (int q = 0; q < NR; ++q) sw[q * kNearTile + t] = (Real)ws[(int64_t)(r0 + q) * ldw + j];
            } else {
              const int64_t so = (int64_t)s * 3 * P;
              const int k = j0 + t;
              if constexpr (sizeof(Real) == 4) {
                sx[t] = v.proxy32[so + k]; sy[t] = v.proxy32[so + P + k]; sz[t] = v.proxy32[so + 2 * P + k];
              } else {
                sx[t] = v.proxy[so + k]; sy[t] = v.proxy[so + P + k]; sz[t] = v.proxy[so + 2 * P + k];
              }
#pragma unroll
              for (int q = 0; q < NR; ++q) sw[q * kNearTile + t] = wbar[((int64_t)s * ldr + r0 + q) * P + k];
            }
          }
          __syncthreads();
          if (active) {
            Acc<KID, Real> acc[NR];
            const int skip = self - j0;  // in [0, nj) only on the tile holding x_i
            for (int j = 0; j < nj; ++j) {
              if (j == skip) continue;
              KFac<KID, Real> kf(rx0 - sx[j], ry0 - sy[j], rz0 - sz[j]);
#pragma unroll
              for (int q = 0; q < NR; ++q) acc[q].add(kf, sw[q * kNearTile + j]);
            }
#pragma unroll
            for (int q = 0; q < NR; ++q) acc[q].flush(out[q], tx, ty, tz);
          }
        }
      }
    }
    if (active) {
      for (int q = 0; q < nr; ++q)
#pragma unroll
        for (int d = 0; d < DIM; ++d) phi[((int64_t)(r0 + q) * v.N + i) * DIM + d] = out[q][d];
    }
  }
}

// ---------------------------------------------------------------------------
// L2P + finalize: out[r][perm[i] - tbase][d] = phi[r][i][d] + sum_m psi_leaf[m] La[i][m1] Lb[i][m2]
// for the targets (perm[i] >= tbase).
// One block per leaf, one thread per point of a chunk; the chunk's Lagrange
// rows are staged through shared memory once for every (r, d).
// ---------------------------------------------------------------------------

template <typename Real>
__global__ void __launch_bounds__(kL2PThreads) l2p_kernel(PlanView v, const int32_t *leaves,
                                                          const Real *psi, int ldr, int nrhs,
                                                          int dim, const double *phi, double *out) {
  __shared__ Real sp[kMaxP * kMaxP];
  __shared__ Real sLa[kL2PThreads * kMaxP], sLb[kL2PThreads * kMaxP];
  const int c = leaves[blockIdx.x];
  if (!cell_ok(v, c)) return;
  const int b = v.cbegin[c], e = v.cend[c], p = v.p, P = v.P;
  const Real *La = La_of<Real>(v), *Lb = Lb_of<Real>(v);
  for (int i0 = b; i0 < e; i0 += kL2PThreads) {
    const int nj = min(kL2PThreads, e - i0);
    __syncthreads();
    for (int t = threadIdx.x; t < nj * p; t += kL2PThreads) {
      sLa[t] = La[(int64_t)i0 * p + t];
      sLb[t] = Lb[(int64_t)i0 * p + t];
    }
    const int t = threadIdx.x;
    const int i = i0 + t;
    for (int r = 0; r < nrhs; ++r)
      for (int d = 0; d < dim; ++d) {
        __syncthreads();
        for (int u = threadIdx.x; u < P; u += kL2PThreads)
          sp[u] = psi[(((int64_t)c * ldr + r) * dim + d) * P + u];
        __syncthreads();
        if (t < nj && v.perm[i] >= v.tbase) {
          const Real *la = sLa + t * p, *lb = sLb + t * p;
          Real acc = 0;
          for (int m1 = 0; m1 < p; ++m1) {
            Real s = 0;
            for (int m2 = 0; m2 < p; ++m2) s += sp[m1 * p + m2] * lb[m2];
            acc += la[m1] * s;
          }
          const int64_t oi = ((int64_t)r * v.N + i) * dim + d;
          out[((int64_t)r * v.ntgt + v.perm[i] - v.tbase) * dim + d] = phi[oi] + (double)acc;
        }
      }
  }
}

// L2P + finalize of the FP32-bulk form (downward_df.cuh), one block of
// kL2PThreads per leaf; shared memory sized for the compile-time degree and
// 7 resident blocks per SM requested (72 registers): at N = 6.3M, n = 12,
// 0.562 ms against 0.589 ms with kMaxP-sized shared memory (6 blocks) and
// 0.582 / 0.692 ms with 6 / 1 requested.
#ifndef CSFMM_L2P_MINB
#define CSFMM_L2P_MINB 7
#endif
template <int PC>
__global__ void __launch_bounds__(kL2PThreads, CSFMM_L2P_MINB) l2p_df_kernel(
    PlanView v, const int32_t *leaves, const double *psi, int ldr, int nrhs, int dim,
    const double *phi, double *out) {
  __shared__ __align__(16) float sm[l2p_df_smem_floats<PC>()];
  l2p_df_leaf<PC>(v, leaves[blockIdx.x], psi, ldr, nrhs, dim, phi, out, sm);
}

void launch_l2p_df(int p, int nleaves, const PlanView &v, const int32_t *leaves, const double *psi,
                   int ldr, int nrhs, int dim, const double *phi, double *out, cudaStream_t st) {
#define CSFMM_L2P(PC) \
  l2p_df_kernel<PC><<<nleaves, kL2PThreads, 0, st>>>(v, leaves, psi, ldr, nrhs, dim, phi, out)
  switch (p) {
    case 7: CSFMM_L2P(7); break;
    case 9: CSFMM_L2P(9); break;
    case 11: CSFMM_L2P(11); break;
    case 13: CSFMM_L2P(13); break;
    default: CSFMM_L2P(0); break;
  }
#undef CSFMM_L2P
}

const void *l2p_df_function(int p) {
  switch (p) {
    case 7: return (const void *)l2p_df_kernel<7>;
    case 9: return (const void *)l2p_df_kernel<9>;
    case 11: return (const void *)l2p_df_kernel<11>;
    case 13: return (const void *)l2p_df_kernel<13>;
    default: return (const void *)l2p_df_kernel<0>;
  }
}

template <int KID, typename Real>
void launch_far(const PlanView &v, Plan &pl, Workspace &W, int nr, int r0, int tb_prox,
                Real *wbar, double *psi, cudaStream_t st) {
  const int N = (int)pl.N, ldr = W.max_nrhs;
  switch (nr) {
    case 1: far_kernel<KID, Real, 1><<<pl.ncells, tb_prox, 0, st>>>(v, W.ws, N, wbar, ldr, r0, psi); break;
    case 2: far_kernel<KID, Real, 2><<<pl.ncells, tb_prox, 0, st>>>(v, W.ws, N, wbar, ldr, r0, psi); break;
    case 3: far_kernel<KID, Real, 3><<<pl.ncells, tb_prox, 0, st>>>(v, W.ws, N, wbar, ldr, r0, psi); break;
    default: far_kernel<KID, Real, 4><<<pl.ncells, tb_prox, 0, st>>>(v, W.ws, N, wbar, ldr, r0, psi); break;
  }
}

template <int KID, typename Real>
void launch_near(const PlanView &v, Plan &pl, Workspace &W, int nr, int r0, const Real *wbar,
                 cudaStream_t st) {
  const int N = (int)pl.N, ldr = W.max_nrhs;
  switch (nr) {
    case 1: near_kernel<KID, Real, 1><<<pl.nleaves, kNearTile, 0, st>>>(v, pl.leaves, W.ws, N, wbar, ldr, r0, W.phi); break;
    case 2: near_kernel<KID, Real, 2><<<pl.nleaves, kNearTile, 0, st>>>(v, pl.leaves, W.ws, N, wbar, ldr, r0, W.phi); break;
    case 3: near_kernel<KID, Real, 3><<<pl.nleaves, kNearTile, 0, st>>>(v, pl.leaves, W.ws, N, wbar, ldr, r0, W.phi); break;
    default: near_kernel<KID, Real, 4><<<pl.nleaves, kNearTile, 0, st>>>(v, pl.leaves, W.ws, N, wbar, ldr, r0, W.phi); break;
  }
}

template <int KID, typename Real>
csfmm_status run_passes(Plan &pl, Workspace &W, const double *w, int nrhs, double *out,
                        cudaStream_t st) {
  PlanView v = pl.view();
  const int N = (int)pl.N, P = pl.P, dim = pl.dim;
  const int ldr = W.max_nrhs;  // rhs stride of wbar / psi
  Real *wbar;
  if constexpr (sizeof(Real) == 4) wbar = W.wbar32; else wbar = W.wbar;
  double *psi = W.psi;  // FP64 proxy potentials in both forms
  // weight totals per cell for the log kernel's FP32 sums
  float2 *wtot = (sizeof(Real) == 4 && KID == CSFMM_KERNEL_LAPLACE) ? W.wtot : nullptr;
  v.wtot = wtot;
  v.wtot_ld = ldr;
  pl.launches = 0;
  // Two streams: after the gather the upward pass, the far field and L2L go
  // to the workspace's side stream while the symmetric and the rest of the
  // near field run on st; the near field waits for the upward pass (its PC
  // entries read proxy weights) and L2P for L2L.  The log kernel's symmetric
  // pass reads the leaves' weight totals of P2M, so there P2M stays on st
  // before the fork.  Phase timing brackets every phase with its own events
  // on the stream it runs on.
  const bool overlap = W.side != nullptr && !(pl.schedule & CSFMM_SCHED_NO_OVERLAP);
  cudaStream_t sf = overlap ? ((pl.schedule & CSFMM_SCHED_SIDE_FIRST) ? W.side_hi : W.side) : st;
  const bool p2m_first = !overlap || (sizeof(Real) == 4 && KID == CSFMM_KERNEL_LAPLACE);
#define CSFMM_BEGIN(ph, s)                           \
  do {                                               \
    csfmm_status s__ = pl.phase(ph, true, s);        \
    if (s__ != CSFMM_OK) return s__;                 \
  } while (0)
#define CSFMM_END(ph, s)                             \
  do {                                               \
    csfmm_status s__ = pl.phase(ph, false, s);       \
    if (s__ != CSFMM_OK) return s__;                 \
  } while (0)
  CSFMM_BEGIN(CSFMM_PHASE_GATHER, st);
  gather_kernel<<<grid_for((int64_t)N * nrhs, 256, sm_count() * 32), 256, 0, st>>>(
      pl.perm, w, W.ws, sizeof(Real) == 4 ? W.wsf : nullptr, N, nrhs, N, (int)pl.nsrc);
  ++pl.launches;
  CSFMM_END(CSFMM_PHASE_GATHER, st);
  const int tb_prox = ((P + 31) / 32) * 32;
  const int tb_p2m = tb_prox < 64 ? 64 : tb_prox;
  auto p2m = [&](cudaStream_t s) -> csfmm_status {
    CSFMM_BEGIN(CSFMM_PHASE_P2M, s);
    for (int r0 = 0; r0 < nrhs; r0 += (sizeof(Real) == 4 && nrhs - r0 >= 8) ? 8 : kRB) {
      int nr = min(kRB, nrhs - r0);
      if (sizeof(Real) == 4 && nrhs - r0 >= 8) nr = 8;  // FP32 form: 8 RHS per pass over the rows
      switch (nr) {
        case 8: p2m_kernel<Real, 8><<<pl.nleaves, tb_p2m, 0, s>>>(v, pl.leaves, W.ws, N, r0, wbar, ldr, wtot); break;
        case 1: p2m_kernel<Real, 1><<<pl.nleaves, tb_p2m, 0, s>>>(v, pl.leaves, W.ws, N, r0, wbar, ldr, wtot); break;
        case 2: p2m_kernel<Real, 2><<<pl.nleaves, tb_p2m, 0, s>>>(v, pl.leaves, W.ws, N, r0, wbar, ldr, wtot); break;
        case 3: p2m_kernel<Real, 3><<<pl.nleaves, tb_p2m, 0, s>>>(v, pl.leaves, W.ws, N, r0, wbar, ldr, wtot); break;
        default: p2m_kernel<Real, 4><<<pl.nleaves, tb_p2m, 0, s>>>(v, pl.leaves, W.ws, N, r0, wbar, ldr, wtot); break;
      }
      ++pl.launches;
    }
    CSFMM_END(CSFMM_PHASE_P2M, s);
    return CSFMM_OK;
  };
  csfmm_status s0;
  W.last_persistent = false;
  if constexpr (sizeof(Real) == 4 && KID != CSFMM_KERNEL_BIOT_SAVART) {
    // several right-hand sides: the upward pass, then one persistent launch
    // for the far field, the near field, L2L and L2P (persistent.cu); its
    // time is recorded as the NEAR phase
    int pchunk = 0;
    if (persistent_eligible(pl, W, nrhs, &pchunk)) {
      if ((s0 = p2m(st)) != CSFMM_OK) return s0;
      CSFMM_BEGIN(CSFMM_PHASE_M2M, st);
      for (int l = pl.nlevels - 2; l >= 0; --l) {
        const int c0 = pl.level_begin[l], nlev = pl.level_begin[l + 1] - c0;
        m2m_df_kernel<<<nlev, kM2MThreads, 0, st>>>(v, c0, 0, nrhs, wbar, ldr, wtot);
        ++pl.launches;
      }
      CSFMM_END(CSFMM_PHASE_M2M, st);
      CSFMM_BEGIN(CSFMM_PHASE_NEAR, st);
      if ((s0 = launch_persistent(v, pl, W, nrhs, pchunk, out, st, &W.last_persist_args)) !=
          CSFMM_OK)
        return s0;
      ++pl.launches;
      CSFMM_END(CSFMM_PHASE_NEAR, st);
      for (int ph : {CSFMM_PHASE_CCSYM, CSFMM_PHASE_FAR, CSFMM_PHASE_PPSYM, CSFMM_PHASE_L2L,
                     CSFMM_PHASE_L2P}) {
        CSFMM_BEGIN(ph, st);  // empty: their work is inside the persistent launch
        CSFMM_END(ph, st);
      }
      W.last_persistent = true;
      W.last_persist_view = v;
      CSFMM_CUDA(cudaGetLastError());
      pl.stats.launches_per_evaluate = pl.launches;
      return CSFMM_OK;
    }
  }
  if (p2m_first && (s0 = p2m(st)) != CSFMM_OK) return s0;
  if (overlap) {
    CSFMM_CUDA(cudaEventRecord(W.ev_fork, st));
    CSFMM_CUDA(cudaStreamWaitEvent(sf, W.ev_fork, 0));
  }
  if (!p2m_first && (s0 = p2m(sf)) != CSFMM_OK) return s0;
  CSFMM_BEGIN(CSFMM_PHASE_M2M, sf);
  for (int l = pl.nlevels - 2; l >= 0; --l) {
    int c0 = pl.level_begin[l], nlev = pl.level_begin[l + 1] - c0;
    if constexpr (sizeof(Real) == 4)
      m2m_df_kernel<<<nlev, kM2MThreads, 0, sf>>>(v, c0, 0, nrhs, wbar, ldr, wtot);
    else
      m2m_kernel<Real><<<nlev, 128, 0, sf>>>(v, c0, 0, nrhs, wbar, ldr);
    ++pl.launches;
  }
  CSFMM_END(CSFMM_PHASE_M2M, sf);
  if (overlap) CSFMM_CUDA(cudaEventRecord(W.ev_up, sf));
  // FP32 form, scalar kernels: chunks of 16 or 8 right-hand sides share every
  // kernel value; the rest goes in chunks of up to kRB
  const bool multi = sizeof(Real) == 4 && KID != CSFMM_KERNEL_BIOT_SAVART;
  auto chunk = [&](int r0) {
    const int left = nrhs - r0;
    if (multi && left >= 16 && pl.rhs_chunk >= 16) return 16;
    if (multi && left >= 8 && pl.rhs_chunk >= 8) return 8;
    return min(kRB, left);
  };
  // single right-hand side, symmetric scalar kernel: the mirrored CC pairs are
  // evaluated once for both directions, then the far field reads their sums
  const bool ccsym = sizeof(Real) == 4 && nrhs == 1 && KID != CSFMM_KERNEL_BIOT_SAVART &&
                     pl.n_cc_pairs > 0 && W.cc_part != nullptr &&
                     !(pl.schedule & CSFMM_SCHED_NO_SYMMETRIC);
  CSFMM_BEGIN(CSFMM_PHASE_CCSYM, sf);
  if constexpr (sizeof(Real) == 4) {
    if (ccsym) {
      launch_cc_sym32(v, pl.cc_pairs, pl.cc_entry, pl.n_cc_pairs, wbar, ldr, W.cc_part, sf);
      ++pl.launches;
    }
  }
  CSFMM_END(CSFMM_PHASE_CCSYM, sf);
  CSFMM_BEGIN(CSFMM_PHASE_FAR, sf);
  for (int r0 = 0; r0 < nrhs; r0 += chunk(r0)) {
    const int nr = chunk(r0);
    if constexpr (sizeof(Real) == 4) {
      if (nr > kRB)
        launch_multi32(v, true, pl.ncells, pl.leaves, W.wsf, wbar, ldr, r0, nr, W.phi, psi,
                       pl.schedule, sf);
      else
        launch_far32(v, pl.ncells, W.wsf, wbar, ldr, r0, nr, psi, sf,
                     ccsym ? W.cc_part : nullptr);
    } else {
      launch_far<KID, Real>(v, pl, W, nr, r0, tb_prox, wbar, psi, sf);
    }
    ++pl.launches;
  }
  CSFMM_END(CSFMM_PHASE_FAR, sf);
  auto l2l = [&](cudaStream_t s) -> csfmm_status {
    CSFMM_BEGIN(CSFMM_PHASE_L2L, s);
    // double-float L2L: one thread per child proxy (P = 169: 192 threads, 0.200
    // against 0.229 ms with 128 at N = 6.3M, n = 12)
    const int tb_l2l = std::max(64, ((pl.P + 31) / 32) * 32);
    for (int l = 0; l + 1 < pl.nlevels; ++l) {
      int c0 = pl.level_begin[l], nlev = pl.level_begin[l + 1] - c0;
      if constexpr (sizeof(Real) == 4)
        l2l_df_kernel<<<nlev, tb_l2l, 0, s>>>(v, c0, 0, nrhs, dim, psi, ldr);
      else
        l2l_kernel<double><<<nlev, 128, 0, s>>>(v, c0, 0, nrhs, dim, psi, ldr);
      ++pl.launches;
    }
    CSFMM_END(CSFMM_PHASE_L2L, s);
    return CSFMM_OK;
  };
  if (overlap) {
    if ((s0 = l2l(sf)) != CSFMM_OK) return s0;
    CSFMM_CUDA(cudaEventRecord(W.ev_done, sf));
  }
  // single right-hand side, symmetric scalar kernel: the cross pairs of the PP
  // lists are evaluated once for both directions first
  const bool sym = sizeof(Real) == 4 && nrhs == 1 && KID != CSFMM_KERNEL_BIOT_SAVART &&
                   pl.n_sym_pairs > 0 && W.sym_part != nullptr &&
                   !(pl.schedule & CSFMM_SCHED_NO_SYMMETRIC);
  CSFMM_BEGIN(CSFMM_PHASE_PPSYM, st);
  if (sym) {
    launch_pp_sym32(v, pl.sym_pairs, pl.sym_off, pl.n_sym_pairs, W.wsf, W.sym_part, st);
    ++pl.launches;
  }
  CSFMM_END(CSFMM_PHASE_PPSYM, st);
  if (overlap) CSFMM_CUDA(cudaStreamWaitEvent(st, W.ev_up, 0));
  CSFMM_BEGIN(CSFMM_PHASE_NEAR, st);
  for (int r0 = 0; r0 < nrhs; r0 += chunk(r0)) {
    const int nr = chunk(r0);
    if constexpr (sizeof(Real) == 4) {
      if (nr == 16 && (pl.schedule & CSFMM_SCHED_TENSOR_NEAR))
        launch_near16_tc(v, pl.nleaves, pl.leaves, W.wsf, wbar, ldr, r0, W.phi, st);
      else if (nr > kRB)
        launch_multi32(v, false, pl.nleaves, pl.leaves, W.wsf, wbar, ldr, r0, nr, W.phi, psi,
                       pl.schedule, st);
      else
        launch_near32(v, pl.leaves, pl.nleaves, W.wsf, N, wbar, ldr, r0, nr, W.phi, st,
                      sym ? W.sym_part : nullptr);
    } else {
      launch_near<KID, Real>(v, pl, W, nr, r0, wbar, st);
    }
    ++pl.launches;
  }
  CSFMM_END(CSFMM_PHASE_NEAR, st);
  if (overlap) CSFMM_CUDA(cudaStreamWaitEvent(st, W.ev_done, 0));
  else if ((s0 = l2l(st)) != CSFMM_OK) return s0;
  CSFMM_BEGIN(CSFMM_PHASE_L2P, st);
  if constexpr (sizeof(Real) == 4)
    launch_l2p_df(pl.p, pl.nleaves, v, pl.leaves, psi, ldr, nrhs, dim, W.phi, out, st);
  else
    l2p_kernel<double><<<pl.nleaves, kL2PThreads, 0, st>>>(v, pl.leaves, psi, ldr, nrhs, dim, W.phi, out);
  ++pl.launches;
  CSFMM_END(CSFMM_PHASE_L2P, st);
#undef CSFMM_BEGIN
#undef CSFMM_END
  CSFMM_CUDA(cudaGetLastError());
  pl.stats.launches_per_evaluate = pl.launches;
  return CSFMM_OK;
}

// Tree code (Algorithm "CSTC"): gather, the upward pass (P2M, M2M) of the
// plan's precision form, then the per-target walks of cstc.cu.
template <int KID, typename Real>
csfmm_status run_cstc(Plan &pl, Workspace &W, const double *w, int nrhs, double *out,
                      cudaStream_t st) {
  PlanView v = pl.view();
  const int N = (int)pl.N, P = pl.P;
  const int ldr = W.max_nrhs;
  Real *wbar;
  if constexpr (sizeof(Real) == 4) wbar = W.wbar32; else wbar = W.wbar;
  float2 *wtot = (sizeof(Real) == 4 && KID == CSFMM_KERNEL_LAPLACE) ? W.wtot : nullptr;
  v.wtot = wtot;
  v.wtot_ld = ldr;
  gather_kernel<<<grid_for((int64_t)N * nrhs, 256, sm_count() * 32), 256, 0, st>>>(
      pl.perm, w, W.ws, sizeof(Real) == 4 ? W.wsf : nullptr, N, nrhs, N, (int)pl.nsrc);
  const int tb_prox = ((P + 31) / 32) * 32;
  const int tb_p2m = tb_prox < 64 ? 64 : tb_prox;
  for (int r0 = 0; r0 < nrhs; r0 += kRB) {
    const int nr = min(kRB, nrhs - r0);
    switch (nr) {
      case 1: p2m_kernel<Real, 1><<<pl.nleaves, tb_p2m, 0, st>>>(v, pl.leaves, W.ws, N, r0, wbar, ldr, wtot); break;
      case 2: p2m_kernel<Real, 2><<<pl.nleaves, tb_p2m, 0, st>>>(v, pl.leaves, W.ws, N, r0, wbar, ldr, wtot); break;
      case 3: p2m_kernel<Real, 3><<<pl.nleaves, tb_p2m, 0, st>>>(v, pl.leaves, W.ws, N, r0, wbar, ldr, wtot); break;
      default: p2m_kernel<Real, 4><<<pl.nleaves, tb_p2m, 0, st>>>(v, pl.leaves, W.ws, N, r0, wbar, ldr, wtot); break;
    }
  }
  for (int l = pl.nlevels - 2; l >= 0; --l) {
    const int c0 = pl.level_begin[l], nlev = pl.level_begin[l + 1] - c0;
    if constexpr (sizeof(Real) == 4)
      m2m_df_kernel<<<nlev, kM2MThreads, 0, st>>>(v, c0, 0, nrhs, wbar, ldr, wtot);
    else
      m2m_kernel<Real><<<nlev, 128, 0, st>>>(v, c0, 0, nrhs, wbar, ldr);
  }
  if constexpr (sizeof(Real) == 4)
    launch_cstc(v, true, pl.theta, pl.level_begin[1], nrhs, ldr, W.ws, W.wsf, nullptr, W.wbar32,
                out, st);
  else
    launch_cstc(v, false, pl.theta, pl.level_begin[1], nrhs, ldr, W.ws, nullptr, W.wbar, nullptr,
                out, st);
  CSFMM_CUDA(cudaGetLastError());
  return CSFMM_OK;
}

template <typename Real>
csfmm_status dispatch_cstc(Plan &pl, Workspace &W, const double *w, int nrhs, double *out,
                           cudaStream_t st) {
  switch (pl.kernel_id) {
    case CSFMM_KERNEL_LAPLACE: return run_cstc<CSFMM_KERNEL_LAPLACE, Real>(pl, W, w, nrhs, out, st);
    case CSFMM_KERNEL_BIOT_SAVART: return run_cstc<CSFMM_KERNEL_BIOT_SAVART, Real>(pl, W, w, nrhs, out, st);
    case CSFMM_KERNEL_NEWTON: return run_cstc<CSFMM_KERNEL_NEWTON, Real>(pl, W, w, nrhs, out, st);
    case CSFMM_KERNEL_SAL: return run_cstc<CSFMM_KERNEL_SAL, Real>(pl, W, w, nrhs, out, st);
    case CSFMM_KERNEL_BIHARMONIC: return run_cstc<CSFMM_KERNEL_BIHARMONIC, Real>(pl, W, w, nrhs, out, st);
    case CSFMM_KERNEL_ONE: return run_cstc<CSFMM_KERNEL_ONE, Real>(pl, W, w, nrhs, out, st);
  }
  set_error("unknown kernel id %d", pl.kernel_id);
  return CSFMM_ERR_INVALID_ARG;
}

template <typename Real>
csfmm_status dispatch_kernel(Plan &pl, Workspace &W, const double *w, int nrhs, double *out,
                             cudaStream_t st) {
  switch (pl.kernel_id) {
    case CSFMM_KERNEL_LAPLACE: return run_passes<CSFMM_KERNEL_LAPLACE, Real>(pl, W, w, nrhs, out, st);
    case CSFMM_KERNEL_BIOT_SAVART: return run_passes<CSFMM_KERNEL_BIOT_SAVART, Real>(pl, W, w, nrhs, out, st);
    case CSFMM_KERNEL_NEWTON: return run_passes<CSFMM_KERNEL_NEWTON, Real>(pl, W, w, nrhs, out, st);
    case CSFMM_KERNEL_SAL: return run_passes<CSFMM_KERNEL_SAL, Real>(pl, W, w, nrhs, out, st);
    case CSFMM_KERNEL_BIHARMONIC: return run_passes<CSFMM_KERNEL_BIHARMONIC, Real>(pl, W, w, nrhs, out, st);
    case CSFMM_KERNEL_ONE: return run_passes<CSFMM_KERNEL_ONE, Real>(pl, W, w, nrhs, out, st);
  }
  set_error("unknown kernel id %d", pl.kernel_id);
  return CSFMM_ERR_INVALID_ARG;
}

}  // namespace

csfmm_status Plan::phase(int ph, bool begin, cudaStream_t st) {
  if (!timing) return CSFMM_OK;
  if (ph == 0 && begin) {
    // a new timed evaluation: a begin and an end event for every phase
    for (int k = 0; k < 2 * CSFMM_NUM_PHASES; ++k) {
      cudaEvent_t e;
      CSFMM_CUDA(cudaEventCreate(&e));
      events.push_back(e);
    }
    ++timed_calls;
  }
  cudaEvent_t e = events[events.size() - 2 * CSFMM_NUM_PHASES + 2 * ph + (begin ? 0 : 1)];
  CSFMM_CUDA(cudaEventRecord(e, st));
  return CSFMM_OK;
}

csfmm_status Workspace::create_side() {
  if (side) return CSFMM_OK;
  int prio_least = 0, prio_greatest = 0;
  cudaError_t e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  if (e == cudaSuccess)
    e = cudaStreamCreateWithPriority(&side_hi, cudaStreamNonBlocking, prio_greatest);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_up, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    release_side();
    return cuda_status(e, "workspace side stream");
  }
  return CSFMM_OK;
}

csfmm_status workspace_alloc(Plan &pl, Workspace &W, int max_nrhs) {
  W.plan = &pl;
  W.max_nrhs = max_nrhs;
  const size_t N = (size_t)pl.N, nc = (size_t)pl.ncells, P = (size_t)pl.P, R = (size_t)max_nrhs;
  csfmm_status s;
  if ((s = W.arena.alloc(&W.ws, R * N)) != CSFMM_OK) return s;
  if (pl.precision == CSFMM_FP64) {
    if ((s = W.arena.alloc(&W.wbar, nc * R * P)) != CSFMM_OK) return s;
  } else {
    if ((s = W.arena.alloc(&W.wbar32, nc * R * P)) != CSFMM_OK) return s;
    if ((s = W.arena.alloc(&W.wsf, R * N)) != CSFMM_OK) return s;
    if ((s = W.arena.alloc(&W.wtot, nc * R * 2)) != CSFMM_OK) return s;
    if (pl.kernel_id != CSFMM_KERNEL_BIOT_SAVART &&
        (s = W.arena.alloc(&W.ctr, persistent_counter_ints(pl))) != CSFMM_OK)
      return s;
    if (pl.n_sym_pairs > 0 && pl.kernel_id != CSFMM_KERNEL_BIOT_SAVART &&
        (s = W.arena.alloc(&W.sym_part, (size_t)pl.sym_part_len)) != CSFMM_OK)
      return s;
    if (pl.n_cc_pairs > 0 &&
        (s = W.arena.alloc(&W.cc_part, (size_t)2 * P * pl.n_cc_pairs)) != CSFMM_OK)
      return s;
  }
  if ((s = W.arena.alloc(&W.psi, nc * R * pl.dim * P)) != CSFMM_OK) return s;
  if ((s = W.arena.alloc(&W.phi, R * N * pl.dim)) != CSFMM_OK) return s;
  return W.create_side();
}

namespace {

csfmm_status enqueue(Plan &pl, Workspace &W, const double *w, int nrhs, double *out,
                     cudaStream_t st) {
  if (pl.precision == CSFMM_FP64) return dispatch_kernel<double>(pl, W, w, nrhs, out, st);
  return dispatch_kernel<float>(pl, W, w, nrhs, out, st);
}

// Captures one evaluation into a graph and records its gather and L2P nodes.
csfmm_status capture(Plan &pl, Workspace &W, const double *w, int nrhs, double *out,
                     cudaStream_t st, GraphEntry &g) {
  CSFMM_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  csfmm_status s = enqueue(pl, W, w, nrhs, out, st);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (s != CSFMM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
  g.graph = graph;
  size_t n = 0;
  CSFMM_CUDA(cudaGraphGetNodes(graph, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  CSFMM_CUDA(cudaGraphGetNodes(graph, nodes.data(), &n));
  const void *f_gather = (const void *)gather_kernel;
  const void *f_l2p = pl.precision == CSFMM_FP64 ? (const void *)l2p_kernel<double>
                                                 : l2p_df_function(pl.p);
  const void *f_persist =
      W.last_persistent
          ? persistent_function(pl, W.last_persist_args.nrhs / W.last_persist_args.nch)
          : nullptr;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType ty;
    CSFMM_CUDA(cudaGraphNodeGetType(nd, &ty));
    if (ty != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp{};
    CSFMM_CUDA(cudaGraphKernelNodeGetParams(nd, &kp));
    if (kp.func == f_gather) {
      g.gather = nd;
      g.gather_params = kp;
    } else if (kp.func == f_l2p) {
      g.l2p = nd;
      g.l2p_params = kp;
    } else if (f_persist && kp.func == f_persist) {
      g.persist = nd;
      g.persist_params = kp;
    }
  }
  if (!g.gather || (!g.l2p && !g.persist)) {
    set_error("graph capture: gather or output node not found");
    return CSFMM_ERR_CUDA;
  }
  if (g.persist) {
    g.persist_view = W.last_persist_view;
    g.persist_args = W.last_persist_args;
  }
  // node priorities captured from the streams (CSFMM_SCHED_SIDE_FIRST) hold in the graph
  CSFMM_CUDA(cudaGraphInstantiate(&g.exec, graph, cudaGraphInstantiateFlagUseNodePriority));
  g.nrhs = nrhs;
  g.w = w;
  g.out = out;
  g.launches = pl.launches;
  return CSFMM_OK;
}

// Points the captured gather and L2P nodes at new caller buffers; the other
// arguments are rebuilt from the plan and workspace exactly as at capture.
// The argument arrays must list every kernel parameter: the checks below tie
// their lengths to the kernels' signatures.
template <class... A>
constexpr int arity(void (*)(A...)) {
  return (int)sizeof...(A);
}
static_assert(arity(gather_kernel) == 8, "retarget: gather_kernel arguments");
static_assert(arity(l2p_kernel<double>) == 8 && arity(l2p_df_kernel<7>) == 8,
              "retarget: L2P arguments");
csfmm_status retarget(Plan &pl, Workspace &W, GraphEntry &g, const double *w, double *out) {
  const int N = (int)pl.N;
  {
    const int32_t *perm = pl.perm;
    double *ws = W.ws;
    float *wsf = pl.precision == CSFMM_FP64 ? nullptr : W.wsf;
    int nrhs = g.nrhs, ld = N, n = N, nsrc = (int)pl.nsrc;
    // one entry per parameter of gather_kernel, in order
    void *args[] = {(void *)&perm, (void *)&w, (void *)&ws, (void *)&wsf, (void *)&n,
                    (void *)&nrhs, (void *)&ld, (void *)&nsrc};
    cudaKernelNodeParams kp = g.gather_params;
    kp.kernelParams = args;
    kp.extra = nullptr;
    CSFMM_CUDA(cudaGraphExecKernelNodeSetParams(g.exec, g.gather, &kp));
  }
  if (g.persist) {
    // the persistent kernel writes the output: same arguments, new out
    PersistArgs a = g.persist_args;
    a.out = out;
    void *args[] = {(void *)&g.persist_view, (void *)&a};
    cudaKernelNodeParams kp = g.persist_params;
    kp.kernelParams = args;
    kp.extra = nullptr;
    CSFMM_CUDA(cudaGraphExecKernelNodeSetParams(g.exec, g.persist, &kp));
    g.persist_args = a;
  } else {
    PlanView v = pl.view();
    const int32_t *leaves = pl.leaves;
    const void *psi = W.psi;
    int ldr = W.max_nrhs, nrhs = g.nrhs, dim = pl.dim;
    const double *phi = W.phi;
    void *args[] = {(void *)&v, (void *)&leaves, (void *)&psi, (void *)&ldr, (void *)&nrhs,
                    (void *)&dim, (void *)&phi, (void *)&out};
    cudaKernelNodeParams kp = g.l2p_params;
    kp.kernelParams = args;
    kp.extra = nullptr;
    CSFMM_CUDA(cudaGraphExecKernelNodeSetParams(g.exec, g.l2p, &kp));
  }
  g.w = w;
  g.out = out;
  return CSFMM_OK;
}

}  // namespace

// Evaluates nrhs <= W.max_nrhs right-hand sides.  With use_graphs (and no
// phase timing, on a stream other than the legacy default stream) the launch
// sequence is captured once per right-hand-side count and replayed.
csfmm_status cstc_impl(Plan &pl, Workspace &W, const double *w, int nrhs, double *out,
                       cudaStream_t st) {
  if (nrhs > W.max_nrhs) {
    set_error("nrhs %d exceeds the workspace capacity %d", nrhs, W.max_nrhs);
    return CSFMM_ERR_INVALID_ARG;
  }
  if (pl.nlevels > 18) {
    set_error("the tree code walks trees of at most 18 levels (this plan has %d)", pl.nlevels);
    return CSFMM_ERR_UNSUPPORTED;
  }
  if (pl.precision == CSFMM_FP64) return dispatch_cstc<double>(pl, W, w, nrhs, out, st);
  return dispatch_cstc<float>(pl, W, w, nrhs, out, st);
}

csfmm_status evaluate_impl(Plan &pl, Workspace &W, const double *w, int nrhs, double *out,
                           cudaStream_t st) {
  if (nrhs > W.max_nrhs) {
    set_error("nrhs %d exceeds the workspace capacity %d", nrhs, W.max_nrhs);
    return CSFMM_ERR_INVALID_ARG;
  }
  W.last_nrhs = nrhs;
  const bool graphs = pl.use_graphs && W.graphs_ok && !pl.timing && st != nullptr &&
                      st != cudaStreamLegacy && st != cudaStreamPerThread;
  if (!graphs) return enqueue(pl, W, w, nrhs, out, st);
  GraphEntry *g = nullptr;
  for (GraphEntry &e : W.graphs)
    if (e.nrhs == nrhs) g = &e;
  if (!g) {
    GraphEntry ne;
    csfmm_status s = capture(pl, W, w, nrhs, out, st, ne);
    if (s != CSFMM_OK) {
      if (ne.exec) cudaGraphExecDestroy(ne.exec);
      if (ne.graph) cudaGraphDestroy(ne.graph);
      return s;
    }
    W.graphs.push_back(ne);
    g = &W.graphs.back();
  } else if (g->w != w || g->out != out) {
    csfmm_status s = retarget(pl, W, *g, w, out);
    if (s != CSFMM_OK) return s;
  }
  pl.stats.launches_per_evaluate = g->launches;
  CSFMM_CUDA(cudaGraphLaunch(g->exec, st));
  return CSFMM_OK;
}

}  // namespace csfmm
