// bve.cu -- one fourth-order Runge-Kutta step of the barotropic vorticity
// equation on a rotating sphere by the vortex method of Sec. 2.3
// (Eq. BVE_ODEs): particles x_i with relative vorticity zeta_i and fixed areas
// A_i move with the velocity of the Biot-Savart N-body sum,
//     dx_i/dt = sum_j K_BS(x_i, x_j) zeta_j A_j,    dzeta_i/dt = -2 Omega dz_i/dt,
// the velocity computed by the CSFMM (a plan built at every stage's positions)
// or by direct summation.  Stage positions are projected back onto the
// sphere (the kernel is defined there).  The paper's remeshing is not part of
// the step.
#include <math.h>

#include <cuda_runtime.h>

#include "csfmm_internal.cuh"

namespace csfmm {

namespace {

// w = zeta * A
__global__ void bve_weights_kernel(const double *zeta, const double *area, int64_t N, double *w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    w[i] = zeta[i] * area[i];
}

// Stage update from the stage velocity u [N][3] (b = the stage's weight in
// the RK4 combination, the running sum ksum initialised by the first stage):
//   ksum += b u;  xs = P(x + a u), zs = zeta - 2 Omega a u_z   (next stage)
// and on the last stage the step result
//   xs = P(x + c ksum), zs = zeta - 2 Omega c ksum_z           (c = dt/6),
// P the projection onto the unit sphere.
__global__ void bve_stage_kernel(const double *x, const double *zeta, const double *u, int64_t N,
                                 int first, int last, double a, double b, double c,
                                 double two_omega, double *ksum, double *xs, double *zs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double k[3];
    for (int d = 0; d < 3; ++d) {
      k[d] = (first ? 0.0 : ksum[3 * i + d]) + b * u[3 * i + d];
      ksum[3 * i + d] = k[d];
    }
    const double s = last ? c : a;
    double v[3];
    for (int d = 0; d < 3; ++d) v[d] = last ? k[d] : u[3 * i + d];
    double y[3], nrm = 0.0;
    for (int d = 0; d < 3; ++d) {
      y[d] = x[3 * i + d] + s * v[d];
      nrm += y[d] * y[d];
    }
    nrm = sqrt(nrm);
    for (int d = 0; d < 3; ++d) xs[3 * i + d] = y[d] / nrm;
    zs[i] = zeta[i] - two_omega * s * v[2];
  }
}

}  // namespace

// One RK4 step from (x, zeta); stage 0 evaluates on first_plan when it is not
// NULL (a Biot-Savart plan built at x), every other stage on a plan built at
// its positions (or by the direct sum when degree == 0).
csfmm_status bve_rk4(const double *x, const double *zeta, const double *area, int64_t N,
                     double dt, double omega, int degree, double theta, int max_leaf,
                     int precision, csfmm_plan first_plan, double *x_out, double *zeta_out,
                     cudaStream_t st) {
  // scratch: stage positions and vorticity, weights, velocity, running sum
  double *buf = nullptr;
  const size_t n3 = (size_t)3 * N;
  CSFMM_CUDA(cudaMallocFromPoolAsync((void **)&buf, sizeof(double) * (3 * n3 + 2 * (size_t)N), memory_pool(), st));
  double *xs = buf, *u = buf + n3, *ksum = buf + 2 * n3, *zs = buf + 3 * n3,
         *w = buf + 3 * n3 + N;
  const int grid = grid_for(N, 256, sm_count() * 8);
  const double two_omega = 2.0 * omega;
  // RK4: stage s evaluates the velocity at (xs, zs); a = offset of the next
  // stage, b = weight of this stage in the combination (1, 2, 2, 1)
  const double a_next[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};
  const double b_w[4] = {1.0, 2.0, 2.0, 1.0};
  csfmm_status s = CSFMM_OK;
  const double *xcur = x, *zcur = zeta;
  csfmm_options opt{};
  opt.precision = precision;
  opt.max_nrhs = 1;
  void *stream = (void *)st;
  for (int stage = 0; stage < 4 && s == CSFMM_OK; ++stage) {
    bve_weights_kernel<<<grid, 256, 0, st>>>(zcur, area, N, w);
    if (stage == 0 && first_plan) {
      s = csfmm_evaluate(first_plan, w, 1, u, stream);
      if (s == CSFMM_OK) s = csfmm_plan_sync(first_plan, stream);
    } else if (degree > 0) {
      csfmm_plan plan = nullptr;
      s = csfmm_plan_create(xcur, N, CSFMM_KERNEL_BIOT_SAVART, degree, theta, max_leaf, &opt,
                            stream, &plan);
      if (s == CSFMM_OK) s = csfmm_evaluate(plan, w, 1, u, stream);
      if (s == CSFMM_OK) s = csfmm_plan_sync(plan, stream);
      csfmm_plan_destroy(plan);
    } else {
      s = csfmm_direct(xcur, N, CSFMM_KERNEL_BIOT_SAVART, w, 1, u, precision, stream);
    }
    if (s != CSFMM_OK) break;
    const bool last = stage == 3;
    bve_stage_kernel<<<grid, 256, 0, st>>>(x, zeta, u, N, stage == 0, last, a_next[stage],
                                           b_w[stage], dt / 6.0, two_omega, ksum,
                                           last ? x_out : xs, last ? zeta_out : zs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_status(e, "bve_stage_kernel launch");
    xcur = xs;
    zcur = zs;
  }
  cudaError_t e = cudaFreeAsync(buf, st);
  if (e != cudaSuccess && s == CSFMM_OK) s = cuda_status(e, "cudaFreeAsync");
  return s;
}

}  // namespace csfmm

using namespace csfmm;

static bool bve_args_ok(int64_t N, double dt, int degree, const char *who) {
  if (N < 1 || !(dt > 0.0) || degree < 0) {
    set_error("%s: N >= 1, dt > 0 and degree >= 0 required", who);
    return false;
  }
  return true;
}

extern "C" csfmm_status csfmm_bve_step(const double *x, const double *zeta, const double *area,
                                       int64_t N, double dt, double omega, int degree,
                                       double theta, int max_leaf, int precision, double *x_out,
                                       double *zeta_out, void *stream) {
  if (!x || !zeta || !area || !x_out || !zeta_out) {
    set_error("csfmm_bve_step: NULL array");
    return CSFMM_ERR_INVALID_ARG;
  }
  if (!bve_args_ok(N, dt, degree, "csfmm_bve_step")) return CSFMM_ERR_INVALID_ARG;
  return bve_rk4(x, zeta, area, N, dt, omega, degree, theta, max_leaf, precision, nullptr, x_out,
                 zeta_out, (cudaStream_t)stream);
}

extern "C" csfmm_status csfmm_bve_step_remeshed(csfmm_remesh_grid grid, csfmm_plan grid_plan,
                                                const double *zeta, const double *tracer,
                                                const double *area, double dt, double omega,
                                                int degree, double theta, int max_leaf,
                                                int precision, double *zeta_out,
                                                double *tracer_out, void *stream) {
  if (!grid || !zeta || !area || !zeta_out || (!tracer) != (!tracer_out)) {
    set_error("csfmm_bve_step_remeshed: NULL argument (tracer and tracer_out go together)");
    return CSFMM_ERR_INVALID_ARG;
  }
  const int64_t M = remesh_grid_size(grid);
  if (!bve_args_ok(M, dt, degree, "csfmm_bve_step_remeshed")) return CSFMM_ERR_INVALID_ARG;
  if (grid_plan && (grid_plan->impl.N != M ||
                    grid_plan->impl.kernel_id != CSFMM_KERNEL_BIOT_SAVART)) {
    set_error("csfmm_bve_step_remeshed: grid_plan must be a Biot-Savart plan of the grid's %lld "
              "points", (long long)M);
    return CSFMM_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int nf = tracer ? 2 : 1;
  double *buf = nullptr;
  CSFMM_CUDA(cudaMallocFromPoolAsync((void **)&buf, sizeof(double) * (3 + 2 * nf) * (size_t)M, memory_pool(), st));
  // moved positions; moved fields [nf][M] (vorticity, tracer); remeshed fields
  double *xm = buf, *fm = buf + 3 * (size_t)M, *fo = fm + nf * (size_t)M;
  csfmm_status s = bve_rk4(remesh_grid_points(grid), zeta, area, M, dt, omega, degree, theta,
                           max_leaf, precision, grid_plan, xm, fm, st);
  // the tracer is carried unchanged by the particles (dq/dt = 0 along paths)
  if (s == CSFMM_OK && tracer) {
    cudaError_t e = cudaMemcpyAsync(fm + M, tracer, sizeof(double) * M, cudaMemcpyDeviceToDevice,
                                    st);
    if (e != cudaSuccess) s = cuda_status(e, "cudaMemcpyAsync");
  }
  if (s == CSFMM_OK) s = remesh_impl(grid, xm, fm, nf, fo, st);
  if (s == CSFMM_OK) {
    cudaError_t e = cudaMemcpyAsync(zeta_out, fo, sizeof(double) * M, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && tracer)
      e = cudaMemcpyAsync(tracer_out, fo + M, sizeof(double) * M, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) s = cuda_status(e, "cudaMemcpyAsync");
  }
  cudaError_t e = cudaFreeAsync(buf, st);
  if (e != cudaSuccess && s == CSFMM_OK) s = cuda_status(e, "cudaFreeAsync");
  return s;
}
