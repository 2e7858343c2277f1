// direct.cu -- direct summation of Eq. (nbodysum), phi_i = sum_{j != i} K(x_i, x_j) w_j
// (Sec. 1), tiled: one thread per target, sources staged through shared memory
// in tiles of kTile points.  FP64 form: FP64 kernel values, plain sums within a
// tile and Neumaier-compensated sums across tiles.  FP32 form: the difference
// x_i - y_j is formed in FP64 and rounded once, kernel values and tile sums in
// FP32, FP64 sums across tiles.
#include <math.h>

#include "csfmm_internal.cuh"

namespace csfmm {

namespace {

constexpr int kTile = 128;
constexpr int kRBd = 4;

__device__ __forceinline__ void neumaier(double &s, double &c, double v) {
  double t = s + v;
  if (fabs(s) >= fabs(v)) c += (s - t) + v;
  else c += (v - t) + s;
  s = t;
}

template <int KID, typename Real>
__global__ void direct_kernel(const double *pts, int N, const double *w, int r0, int nr,
                              const int64_t *targets, int nt, double *out) {
  constexpr int DIM = KID == CSFMM_KERNEL_BIOT_SAVART ? 3 : 1;
  __shared__ double sx[kTile], sy[kTile], sz[kTile];
  __shared__ Real sw[kRBd * kTile];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = t < nt;
  int64_t i = -1;
  double x0 = 0, x1 = 0, x2 = 0;
  if (active) {
    i = targets ? targets[t] : t;
    x0 = pts[3 * i];
    x1 = pts[3 * i + 1];
    x2 = pts[3 * i + 2];
  }
  double s[kRBd][DIM], c[kRBd][DIM];
#pragma unroll
  for (int q = 0; q < kRBd; ++q)
#pragma unroll
    for (int d = 0; d < DIM; ++d) s[q][d] = c[q][d] = 0.0;
  for (int j0 = 0; j0 < N; j0 += kTile) {
    const int nj = min(kTile, N - j0);
    __syncthreads();
    for (int u = threadIdx.x; u < nj; u += blockDim.x) {
      const int64_t j = j0 + u;
      sx[u] = pts[3 * j];
      sy[u] = pts[3 * j + 1];
      sz[u] = pts[3 * j + 2];
#pragma unroll
      for (int q = 0; q < kRBd; ++q) sw[q * kTile + u] = q < nr ? (Real)w[(int64_t)(r0 + q) * N + j] : (Real)0;
    }
    __syncthreads();
    if (!active) continue;
    Real a[kRBd][3], sumw[kRBd];
#pragma unroll
    for (int q = 0; q < kRBd; ++q) {
      a[q][0] = a[q][1] = a[q][2] = 0;
      sumw[q] = 0;
    }
    for (int u = 0; u < nj; ++u) {
      if (j0 + u == i) continue;
      Real rx = (Real)(x0 - sx[u]), ry = (Real)(x1 - sy[u]), rz = (Real)(x2 - sz[u]);
      Real d2 = rx * rx + ry * ry + rz * rz;
      Real kv, q3 = 0;
      if constexpr (KID == CSFMM_KERNEL_LAPLACE) kv = log(d2 * (Real)0.5);
      else if constexpr (KID == CSFMM_KERNEL_NEWTON) kv = (Real)1 / sqrt(d2);
      else if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) q3 = (Real)1 / d2;
      else kv = 1;
#pragma unroll
      for (int q = 0; q < kRBd; ++q) {
        Real wq = sw[q * kTile + u];
        if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) {
          Real f = wq * q3;
          a[q][0] += f * rx;
          a[q][1] += f * ry;
          a[q][2] += f * rz;
        } else {
          a[q][0] += wq * kv;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kRBd; ++q) {
      if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
        neumaier(s[q][0], c[q][0], -kInv4Pi * (double)a[q][0]);
      } else if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) {
        double b0 = a[q][0], b1 = a[q][1], b2 = a[q][2];
        neumaier(s[q][0], c[q][0], kInv2Pi * (x1 * b2 - x2 * b1));
        neumaier(s[q][1], c[q][1], kInv2Pi * (x2 * b0 - x0 * b2));
        neumaier(s[q][2], c[q][2], kInv2Pi * (x0 * b1 - x1 * b0));
      } else {
        neumaier(s[q][0], c[q][0], (double)a[q][0]);
      }
    }
  }
  if (active) {
    for (int q = 0; q < nr; ++q)
#pragma unroll
      for (int d = 0; d < DIM; ++d) out[((int64_t)(r0 + q) * nt + t) * DIM + d] = s[q][d] + c[q][d];
  }
}

template <typename Real>
csfmm_status launch_direct(const double *pts, int N, int kid, const double *w, int nrhs,
                           const int64_t *targets, int nt, double *out, cudaStream_t st) {
  int grid = grid_for(nt, kTile);
  for (int r0 = 0; r0 < nrhs; r0 += kRBd) {
    int nr = min(kRBd, nrhs - r0);
    switch (kid) {
      case CSFMM_KERNEL_LAPLACE:
        direct_kernel<CSFMM_KERNEL_LAPLACE, Real><<<grid, kTile, 0, st>>>(pts, N, w, r0, nr, targets, nt, out);
        break;
      case CSFMM_KERNEL_BIOT_SAVART:
        direct_kernel<CSFMM_KERNEL_BIOT_SAVART, Real><<<grid, kTile, 0, st>>>(pts, N, w, r0, nr, targets, nt, out);
        break;
      case CSFMM_KERNEL_NEWTON:
        direct_kernel<CSFMM_KERNEL_NEWTON, Real><<<grid, kTile, 0, st>>>(pts, N, w, r0, nr, targets, nt, out);
        break;
      default:
        direct_kernel<CSFMM_KERNEL_ONE, Real><<<grid, kTile, 0, st>>>(pts, N, w, r0, nr, targets, nt, out);
        break;
    }
    CSFMM_CUDA(cudaGetLastError());
  }
  return CSFMM_OK;
}

}  // namespace

csfmm_status direct_impl(const double *points, int64_t N, int kernel_id, const double *w,
                         int nrhs, const int64_t *targets, int64_t ntargets, double *out,
                         int precision, cudaStream_t st) {
  int nt = targets ? (int)ntargets : (int)N;
  if (nt == 0) return CSFMM_OK;
  if (precision == CSFMM_FP64)
    return launch_direct<double>(points, (int)N, kernel_id, w, nrhs, targets, nt, out, st);
  return launch_direct<float>(points, (int)N, kernel_id, w, nrhs, targets, nt, out, st);
}

}  // namespace csfmm
