// static_scratch.cu -- csfmm_evaluate_static: an evaluation that allocates
// no device memory.  The per-evaluation scratch (weights in tree order, proxy
// weights, proxy potentials, near-field potentials) is carved from one
// file-scope __device__ array of CSFMM_STATIC_SCRATCH_BYTES, so a caller that
// must not call cudaMalloc on its request path can still evaluate a plan
// built earlier, even while the plan's own workspace is in use elsewhere.
//
// The array lives in every device that loads the library until the process
// exits.  Host code cannot use the array's name as a device address, so the
// address is looked up once per device with cudaGetSymbolAddress (with that
// device current) the first time this entry point runs on it.
#include <mutex>

#include "csfmm_internal.cuh"

namespace {

__device__ __align__(256) unsigned char g_static_scratch[CSFMM_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void *g_addr[kMaxDevices] = {};

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

csfmm_status scratch_address(int device, unsigned char **out) {
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      csfmm::set_error("cudaGetSymbolAddress of the static scratch failed: %s",
                       cudaGetErrorString(e));
      return CSFMM_ERR_CUDA;
    }
    g_addr[device] = p;
  }
  *out = (unsigned char *)g_addr[device];
  return CSFMM_OK;
}

// Device memory of `device` (or managed memory): the kernels read and write
// it directly, so memory of another GPU is refused.
bool is_device_memory(const void *p, int device) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace

extern "C" csfmm_status csfmm_evaluate_static(csfmm_plan plan, const double *weights, int nrhs,
                                              double *out, void *stream) {
  using namespace csfmm;
  if (!plan) {
    set_error("plan is NULL");
    return CSFMM_ERR_INVALID_ARG;
  }
  Plan &pl = plan->impl;
  if (nrhs < 1 || nrhs > 64) {
    set_error("nrhs must be in [1, 64] (got %d)", nrhs);
    return CSFMM_ERR_INVALID_ARG;
  }
  int device = -1;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  if (device != pl.device || device < 0 || device >= kMaxDevices) {
    set_error("the current device %d is not the plan's device %d", device, pl.device);
    return CSFMM_ERR_INVALID_ARG;
  }
  if (!is_device_memory(weights, device) || !is_device_memory(out, device)) {
    set_error("weights and out must be device memory of the plan's device %d", device);
    return CSFMM_ERR_INVALID_ARG;
  }
  const size_t N = (size_t)pl.N, nc = (size_t)pl.ncells, P = (size_t)pl.P, R = (size_t)nrhs;
  const size_t dim = (size_t)pl.dim;
  const size_t real = pl.precision == CSFMM_FP64 ? sizeof(double) : sizeof(float);
  const size_t b_ws = round256(R * N * sizeof(double));
  const size_t b_wbar = round256(nc * R * P * real);
  const size_t b_psi = round256(nc * R * dim * P * sizeof(double));
  const size_t b_phi = round256(R * N * dim * sizeof(double));
  const size_t b_wsf = pl.precision == CSFMM_FP64 ? 0 : round256(R * N * sizeof(float));
  const size_t b_wtot = pl.precision == CSFMM_FP64 ? 0 : round256(nc * R * 2 * sizeof(float2));
  // FP32 bulk, one right-hand side, symmetric kernel: the partial sums of the
  // mirrored PP leaf pairs and CC cell pairs, so that the same symmetric
  // passes run as in csfmm_evaluate
  const bool sym = pl.precision != CSFMM_FP64 && nrhs == 1 && pl.n_sym_pairs > 0 &&
                   pl.kernel_id != CSFMM_KERNEL_BIOT_SAVART;
  const size_t b_sym = sym ? round256((size_t)pl.sym_part_len * sizeof(float)) : 0;
  const size_t b_cc =
      pl.precision != CSFMM_FP64 && nrhs == 1 && pl.n_cc_pairs > 0
          ? round256((size_t)2 * P * pl.n_cc_pairs * sizeof(float))
          : 0;
  // FP32 bulk, scalar kernels: the work and dependency counters of the
  // persistent launch (several right-hand sides)
  const size_t b_ctr = pl.precision != CSFMM_FP64 && pl.kernel_id != CSFMM_KERNEL_BIOT_SAVART
                           ? round256(persistent_counter_ints(pl) * sizeof(int))
                           : 0;
  const size_t need = b_ws + b_wbar + b_psi + b_phi + b_wsf + b_wtot + b_sym + b_ctr + b_cc;
  if (need > (size_t)CSFMM_STATIC_SCRATCH_BYTES) {
    set_error("this evaluation needs %zu bytes of scratch; the static scratch holds %zu bytes "
              "(use csfmm_evaluate, or fewer right-hand sides)",
              need, (size_t)CSFMM_STATIC_SCRATCH_BYTES);
    return CSFMM_ERR_INVALID_ARG;
  }
  unsigned char *base = nullptr;
  csfmm_status s = scratch_address(device, &base);
  if (s != CSFMM_OK) return s;
  // Every scratch buffer is fully written before it is read (gather, P2M/M2M,
  // far, the symmetric pass, near; the persistent launch clears its counters
  // itself), so nothing needs clearing between calls.
  // W has no side stream: the passes run in order on `stream`.
  Workspace W;
  W.graphs_ok = false;  // W lives only for this call
  W.plan = &pl;
  W.max_nrhs = nrhs;
  W.ws = reinterpret_cast<double *>(base);
  if (pl.precision == CSFMM_FP64) W.wbar = reinterpret_cast<double *>(base + b_ws);
  else W.wbar32 = reinterpret_cast<float *>(base + b_ws);
  W.psi = reinterpret_cast<double *>(base + b_ws + b_wbar);
  W.phi = reinterpret_cast<double *>(base + b_ws + b_wbar + b_psi);
  if (b_wsf) W.wsf = reinterpret_cast<float *>(base + b_ws + b_wbar + b_psi + b_phi);
  if (b_wtot) W.wtot = reinterpret_cast<float2 *>(base + b_ws + b_wbar + b_psi + b_phi + b_wsf);
  if (b_sym)
    W.sym_part = reinterpret_cast<float *>(base + b_ws + b_wbar + b_psi + b_phi + b_wsf + b_wtot);
  if (b_ctr)
    W.ctr = reinterpret_cast<int *>(base + b_ws + b_wbar + b_psi + b_phi + b_wsf + b_wtot + b_sym);
  if (b_cc)
    W.cc_part = reinterpret_cast<float *>(base + b_ws + b_wbar + b_psi + b_phi + b_wsf + b_wtot +
                                          b_sym + b_ctr);
  return evaluate_impl(pl, W, weights, nrhs, out, (cudaStream_t)stream);
}
