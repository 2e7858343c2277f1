// direct.cu -- direct summation of Eq. (nbodysum), phi_i = sum_{j != i} K(x_i, x_j) w_j
// (Sec. 1), tiled: one thread per target, sources staged through shared memory
// in tiles of kTile points (split across grid rows when there are few targets).
// FP64 form: FP64 kernel values, plain sums within a tile and
// Neumaier-compensated sums across tiles.  FP32 form: coordinates as
// double-float pairs (x = x_hi + x_lo), the difference formed as
// (x_hi - y_hi) + (x_lo - y_lo) (the first term is exact for nearby points, so
// d is accurate to FP32 rounding of d itself), one-instruction kernel factors,
// FP32 sums over chunks of 32 sources folded by two-sum, and FP64 sums across
// tiles -- no FP64 arithmetic per pair.
#include <math.h>

#include "csfmm_internal.cuh"
#include "dilog.cuh"
#include "fp32_math.cuh"

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

// Sources [j_lo, j_hi) of split blockIdx.y, j_lo = blockIdx.y * chunk.  With one
// split the result goes to out[r][t][d]; with several, each split writes its
// (sum, compensation) pair to part[split][r][t][d][2] for a fixed-order reduction.
template <int KID, typename Real>
__global__ void direct_kernel(const double *pts, int N, const double *w, int r0, int nr,
                              const int64_t *targets, int nt, double *out, int chunk,
                              double *part, int64_t n_out) {
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
  const int j_lo = (int)min((int64_t)blockIdx.y * chunk, (int64_t)N);
  const int j_hi = (int)min((int64_t)j_lo + chunk, (int64_t)N);
  for (int j0 = j_lo; j0 < j_hi; j0 += kTile) {
    const int nj = min(kTile, j_hi - j0);
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
      else if constexpr (KID == CSFMM_KERNEL_BIHARMONIC) kv = (Real)dilog64(1.0 - 0.25 * (double)d2);
      else if constexpr (KID == CSFMM_KERNEL_SAL) kv = (Real)sal64((double)d2);
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
      } else if constexpr (KID == CSFMM_KERNEL_BIHARMONIC) {
        neumaier(s[q][0], c[q][0], kInv4Pi * (double)a[q][0]);
      } else {
        neumaier(s[q][0], c[q][0], (double)a[q][0]);
      }
    }
  }
  if (active) {
    for (int q = 0; q < nr; ++q)
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const int64_t o = ((int64_t)(r0 + q) * nt + t) * DIM + d;
        if (part) {
          double *pp = part + 2 * ((int64_t)blockIdx.y * n_out + o);
          pp[0] = s[q][d];
          pp[1] = c[q][d];
        } else {
          out[o] = s[q][d] + c[q][d];
        }
      }
  }
}

// FP32 form.  Shared tile: A[u] = (x_hi, y_hi, z_hi, w_0), B[u] = (x_lo, y_lo,
// z_lo, -), further weights in sw.  Same output contract as direct_kernel.
template <int KID, int NR>
__global__ void direct32_kernel(const double *pts, int N, const double *w, int r0, int nr,
                                const int64_t *targets, int nt, double *out, int chunk,
                                double *part, int64_t n_out) {
  constexpr int DIM = KID == CSFMM_KERNEL_BIOT_SAVART ? 3 : 1;
  __shared__ float4 sA[kTile], sB[kTile];
  __shared__ float sw[NR * kTile];
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
  const float xh0 = (float)x0, xh1 = (float)x1, xh2 = (float)x2;
  const float xl0 = (float)(x0 - (double)xh0), xl1 = (float)(x1 - (double)xh1),
              xl2 = (float)(x2 - (double)xh2);
  double s[NR][DIM], c[NR][DIM];
#pragma unroll
  for (int q = 0; q < NR; ++q)
#pragma unroll
    for (int d = 0; d < DIM; ++d) s[q][d] = c[q][d] = 0.0;
  const int j_lo = (int)min((int64_t)blockIdx.y * chunk, (int64_t)N);
  const int j_hi = (int)min((int64_t)j_lo + chunk, (int64_t)N);
  for (int j0 = j_lo; j0 < j_hi; j0 += kTile) {
    const int nj = min(kTile, j_hi - j0);
    __syncthreads();
    for (int u = threadIdx.x; u < nj; u += blockDim.x) {
      const int64_t j = j0 + u;
      const double y0 = pts[3 * j], y1 = pts[3 * j + 1], y2 = pts[3 * j + 2];
      const float yh0 = (float)y0, yh1 = (float)y1, yh2 = (float)y2;
      sA[u] = make_float4(yh0, yh1, yh2, (float)w[(int64_t)r0 * N + j]);
      sB[u] = make_float4((float)(y0 - (double)yh0), (float)(y1 - (double)yh1),
                          (float)(y2 - (double)yh2), 0.f);
#pragma unroll
      for (int q = 1; q < NR; ++q) sw[q * kTile + u] = (float)w[(int64_t)(r0 + q) * N + j];
    }
    __syncthreads();
    if (!active) continue;
    float hi[NR][3], lo[NR][3];
#pragma unroll
    for (int q = 0; q < NR; ++q)
#pragma unroll
      for (int d = 0; d < 3; ++d) hi[q][d] = lo[q][d] = 0.f;
    for (int u0 = 0; u0 < nj; u0 += kChunk) {
      const int u1 = min(nj, u0 + kChunk);
      float a[NR][3];
#pragma unroll
      for (int q = 0; q < NR; ++q) a[q][0] = a[q][1] = a[q][2] = 0.f;
      for (int u = u0; u < u1; ++u) {
        if (j0 + u == i) continue;
        const float4 A = sA[u], B = sB[u];
        const float rx = (xh0 - A.x) + (xl0 - B.x);
        const float ry = (xh1 - A.y) + (xl1 - B.y);
        const float rz = (xh2 - A.z) + (xl2 - B.z);
        const float f = kfactor<KID>(fmaf(rz, rz, fmaf(ry, ry, rx * rx)));
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          const float wq = q == 0 ? A.w : sw[q * kTile + u];
          if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) {
            const float g = wq * f;
            a[q][0] = fmaf(g, rx, a[q][0]);
            a[q][1] = fmaf(g, ry, a[q][1]);
            a[q][2] = fmaf(g, rz, a[q][2]);
          } else if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
            a[q][0] = fmaf(wq, f - 1.0f, a[q][0]);  // log2(d2) - 1 = log2(d2 / 2)
          } else {
            a[q][0] = fmaf(wq, f, a[q][0]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < NR; ++q)
#pragma unroll
        for (int d = 0; d < DIM; ++d) two_sum_fold(hi[q][d], lo[q][d], a[q][d]);
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      double b[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) b[d] = (double)hi[q][d] + (double)lo[q][d];
      if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
        neumaier(s[q][0], c[q][0], -(0.69314718055994530942 * kInv4Pi) * b[0]);
      } else if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) {
        neumaier(s[q][0], c[q][0], kInv2Pi * (x1 * b[2] - x2 * b[1]));
        neumaier(s[q][1], c[q][1], kInv2Pi * (x2 * b[0] - x0 * b[2]));
        neumaier(s[q][2], c[q][2], kInv2Pi * (x0 * b[1] - x1 * b[0]));
      } else if constexpr (KID == CSFMM_KERNEL_BIHARMONIC) {
        neumaier(s[q][0], c[q][0], kInv4Pi * b[0]);
      } else {
        neumaier(s[q][0], c[q][0], b[0]);
      }
    }
  }
  if (active) {
#pragma unroll
    for (int q = 0; q < NR; ++q)
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const int64_t o = ((int64_t)(r0 + q) * nt + t) * DIM + d;
        if (part) {
          double *pp = part + 2 * ((int64_t)blockIdx.y * n_out + o);
          pp[0] = s[q][d];
          pp[1] = c[q][d];
        } else {
          out[o] = s[q][d] + c[q][d];
        }
      }
  }
}

// out[o] = Neumaier sum over splits of part[split][o] (o over nrhs * nt * dim).
__global__ void direct_reduce_kernel(const double *part, int nsplit, int64_t n_out, double *out) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_out;
       o += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0, c = 0.0;
    for (int k = 0; k < nsplit; ++k) {
      neumaier(s, c, part[2 * (k * n_out + o)]);
      c += part[2 * (k * n_out + o) + 1];
    }
    out[o] = s + c;
  }
}

template <int KID>
void launch_direct32(dim3 grid, cudaStream_t st, const double *pts, int N, const double *w, int r0,
                     int nr, const int64_t *targets, int nt, double *out, int chunk, double *part,
                     int64_t n_out) {
  switch (nr) {
    case 1: direct32_kernel<KID, 1><<<grid, kTile, 0, st>>>(pts, N, w, r0, nr, targets, nt, out, chunk, part, n_out); break;
    case 2: direct32_kernel<KID, 2><<<grid, kTile, 0, st>>>(pts, N, w, r0, nr, targets, nt, out, chunk, part, n_out); break;
    case 3: direct32_kernel<KID, 3><<<grid, kTile, 0, st>>>(pts, N, w, r0, nr, targets, nt, out, chunk, part, n_out); break;
    default: direct32_kernel<KID, 4><<<grid, kTile, 0, st>>>(pts, N, w, r0, nr, targets, nt, out, chunk, part, n_out); break;
  }
}

// Few target tiles cannot fill the GPU; then the sources are split into
// nsplit chunks (one grid row each) whose partial sums are reduced in a fixed
// order, so results do not depend on scheduling.
template <typename Real>
csfmm_status launch_direct(const double *pts, int N, int kid, const double *w, int nrhs,
                           const int64_t *targets, int nt, double *out, cudaStream_t st) {
  const int tiles = grid_for(nt, kTile);
  const int dim = kid == CSFMM_KERNEL_BIOT_SAVART ? 3 : 1;
  int nsplit = 1;
  const int nsm = sm_count();
  if (tiles < 4 * nsm) {
    nsplit = (4 * nsm + tiles - 1) / tiles;
    const int max_split = (N + 4 * kTile - 1) / (4 * kTile);  // at least 4 tiles per split
    if (nsplit > max_split) nsplit = max_split;
    if (nsplit > 2048) nsplit = 2048;
    if (nsplit < 1) nsplit = 1;
  }
  const int chunk = (N + nsplit - 1) / nsplit;
  const int64_t n_out = (int64_t)nrhs * nt * dim;
  double *part = nullptr;
  if (nsplit > 1) {
    CSFMM_CUDA(cudaMallocFromPoolAsync((void **)&part, sizeof(double) * 2 * (size_t)nsplit * n_out, memory_pool(), st));
  }
  dim3 grid(tiles, nsplit);
  csfmm_status result = CSFMM_OK;
  for (int r0 = 0; r0 < nrhs && result == CSFMM_OK; r0 += kRBd) {
    int nr = min(kRBd, nrhs - r0);
    if constexpr (sizeof(Real) == 4) {
      switch (kid) {
        case CSFMM_KERNEL_LAPLACE: launch_direct32<CSFMM_KERNEL_LAPLACE>(grid, st, pts, N, w, r0, nr, targets, nt, out, chunk, part, n_out); break;
        case CSFMM_KERNEL_BIOT_SAVART: launch_direct32<CSFMM_KERNEL_BIOT_SAVART>(grid, st, pts, N, w, r0, nr, targets, nt, out, chunk, part, n_out); break;
        case CSFMM_KERNEL_NEWTON: launch_direct32<CSFMM_KERNEL_NEWTON>(grid, st, pts, N, w, r0, nr, targets, nt, out, chunk, part, n_out); break;
        case CSFMM_KERNEL_BIHARMONIC: launch_direct32<CSFMM_KERNEL_BIHARMONIC>(grid, st, pts, N, w, r0, nr, targets, nt, out, chunk, part, n_out); break;
        case CSFMM_KERNEL_SAL: launch_direct32<CSFMM_KERNEL_SAL>(grid, st, pts, N, w, r0, nr, targets, nt, out, chunk, part, n_out); break;
        default: launch_direct32<CSFMM_KERNEL_ONE>(grid, st, pts, N, w, r0, nr, targets, nt, out, chunk, part, n_out); break;
      }
    } else {
      switch (kid) {
        case CSFMM_KERNEL_LAPLACE:
          direct_kernel<CSFMM_KERNEL_LAPLACE, Real><<<grid, kTile, 0, st>>>(pts, N, w, r0, nr, targets, nt, out, chunk, part, n_out);
          break;
        case CSFMM_KERNEL_BIOT_SAVART:
          direct_kernel<CSFMM_KERNEL_BIOT_SAVART, Real><<<grid, kTile, 0, st>>>(pts, N, w, r0, nr, targets, nt, out, chunk, part, n_out);
          break;
        case CSFMM_KERNEL_NEWTON:
          direct_kernel<CSFMM_KERNEL_NEWTON, Real><<<grid, kTile, 0, st>>>(pts, N, w, r0, nr, targets, nt, out, chunk, part, n_out);
          break;
        case CSFMM_KERNEL_BIHARMONIC:
          direct_kernel<CSFMM_KERNEL_BIHARMONIC, Real><<<grid, kTile, 0, st>>>(pts, N, w, r0, nr, targets, nt, out, chunk, part, n_out);
          break;
        case CSFMM_KERNEL_SAL:
          direct_kernel<CSFMM_KERNEL_SAL, Real><<<grid, kTile, 0, st>>>(pts, N, w, r0, nr, targets, nt, out, chunk, part, n_out);
          break;
        default:
          direct_kernel<CSFMM_KERNEL_ONE, Real><<<grid, kTile, 0, st>>>(pts, N, w, r0, nr, targets, nt, out, chunk, part, n_out);
          break;
      }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) result = cuda_status(e, "direct_kernel launch");
  }
  if (part) {
    if (result == CSFMM_OK) {
      direct_reduce_kernel<<<grid_for(n_out, 256, sm_count() * 8), 256, 0, st>>>(part, nsplit, n_out, out);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) result = cuda_status(e, "direct_reduce_kernel launch");
    }
    cudaError_t e = cudaFreeAsync(part, st);
    if (e != cudaSuccess && result == CSFMM_OK) result = cuda_status(e, "cudaFreeAsync");
  }
  return result;
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
