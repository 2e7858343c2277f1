// multi32.cu -- the per-phase kernels of the FP32-bulk interactions for
// several right-hand sides (multi32.cuh): one block per target leaf (near
// field) or cell (far field), with the tile shape chosen at run time from the
// plan's schedule bits (csfmm_options.schedule): threads per block of the
// near field (128 or 64), targets per thread (2 or 1) and sources per FP32
// chunk of the tile sums (32 or 16).
#include <algorithm>

#include "csfmm_internal.cuh"
#include "fp32_math.cuh"
#include "multi32.cuh"

namespace csfmm {

namespace {

template <int KID, int NR, bool FAR, int NT, int CH>
__global__ void __launch_bounds__(CSFMM_MULTI_THREADS) multi32_kernel(
    PlanView v, const int32_t *leaves, const float *wsf, const float *wbar, int ldr, int r0,
    double *phi, double *psi) {
  __shared__ float4 sp[kMultiTile];
  __shared__ ulonglong2 sw4[(NR / 4) * kMultiTile];
  const int c = FAR ? (int)blockIdx.x : leaves[blockIdx.x];
  multi32_item<KID, NR, FAR, NT, CH>(v, c, wsf, wbar, ldr, r0, phi, psi, sp, sw4, threadIdx.x,
                                     blockDim.x, 0);
}

template <int KID, int NR, int NT, int CH>
void launch_shape(const PlanView &v, bool far, int ngrid, const int32_t *leaves, const float *wsf,
                  const float *wbar, int ldr, int r0, double *phi, double *psi, int near_threads,
                  cudaStream_t st) {
  if (far) {
    const int per = 32 * NT;  // targets covered by one warp
    const int nth = std::min(CSFMM_MULTI_THREADS, std::max(32, ((v.P + per - 1) / per) * 32));
    multi32_kernel<KID, NR, true, NT, CH><<<ngrid, nth, 0, st>>>(v, leaves, wsf, wbar, ldr, r0,
                                                                  phi, psi);
  } else {
    multi32_kernel<KID, NR, false, NT, CH><<<ngrid, near_threads, 0, st>>>(v, leaves, wsf, wbar,
                                                                           ldr, r0, phi, psi);
  }
}

template <int KID, int NR>
void launch_nr(const PlanView &v, bool far, int ngrid, const int32_t *leaves, const float *wsf,
               const float *wbar, int ldr, int r0, double *phi, double *psi, int schedule,
               cudaStream_t st) {
  const int nth = (schedule & CSFMM_SCHED_NEAR_64_THREADS) ? 64 : CSFMM_MULTI_THREADS;
  const bool one = (schedule & CSFMM_SCHED_ONE_TARGET) != 0;
  const bool c16 = (schedule & CSFMM_SCHED_CHUNK_16) != 0;
  if (one) {
    if (c16) launch_shape<KID, NR, 1, 16>(v, far, ngrid, leaves, wsf, wbar, ldr, r0, phi, psi, nth, st);
    else launch_shape<KID, NR, 1, 32>(v, far, ngrid, leaves, wsf, wbar, ldr, r0, phi, psi, nth, st);
  } else {
    if (c16) launch_shape<KID, NR, 2, 16>(v, far, ngrid, leaves, wsf, wbar, ldr, r0, phi, psi, nth, st);
    else launch_shape<KID, NR, 2, 32>(v, far, ngrid, leaves, wsf, wbar, ldr, r0, phi, psi, nth, st);
  }
}

template <int KID>
void launch_kid(const PlanView &v, bool far, int ngrid, const int32_t *leaves, const float *wsf,
                const float *wbar, int ldr, int r0, int nr, double *phi, double *psi,
                int schedule, cudaStream_t st) {
  if (nr == 16) launch_nr<KID, 16>(v, far, ngrid, leaves, wsf, wbar, ldr, r0, phi, psi, schedule, st);
  else launch_nr<KID, 8>(v, far, ngrid, leaves, wsf, wbar, ldr, r0, phi, psi, schedule, st);
}

}  // namespace

// Right-hand sides r0 .. r0+nr-1 with nr = 8 or 16 for the scalar kernels:
// near field (far = false, one block per leaf) or far field (far = true).
void launch_multi32(const PlanView &v, bool far, int ngrid, const int32_t *leaves,
                    const float *wsf, const float *wbar, int ldr, int r0, int nr, double *phi,
                    double *psi, int schedule, cudaStream_t st) {
  switch (v.kernel_id) {
    case CSFMM_KERNEL_LAPLACE: launch_kid<CSFMM_KERNEL_LAPLACE>(v, far, ngrid, leaves, wsf, wbar, ldr, r0, nr, phi, psi, schedule, st); break;
    case CSFMM_KERNEL_NEWTON: launch_kid<CSFMM_KERNEL_NEWTON>(v, far, ngrid, leaves, wsf, wbar, ldr, r0, nr, phi, psi, schedule, st); break;
    case CSFMM_KERNEL_SAL: launch_kid<CSFMM_KERNEL_SAL>(v, far, ngrid, leaves, wsf, wbar, ldr, r0, nr, phi, psi, schedule, st); break;
    case CSFMM_KERNEL_BIHARMONIC: launch_kid<CSFMM_KERNEL_BIHARMONIC>(v, far, ngrid, leaves, wsf, wbar, ldr, r0, nr, phi, psi, schedule, st); break;
    default: launch_kid<CSFMM_KERNEL_ONE>(v, far, ngrid, leaves, wsf, wbar, ldr, r0, nr, phi, psi, schedule, st); break;
  }
}

}  // namespace csfmm
