// api.cu -- the extern "C" entry points declared in include/csfmm.h: argument
// checks on the host, plan and workspace lifetime, export of plan structures.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <new>
#include <vector>

#include "csfmm_internal.cuh"


namespace csfmm {

static thread_local char g_err[512] = "no error";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

csfmm_status cuda_status(cudaError_t e, const char *what) {
  set_error("%s failed: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return CSFMM_ERR_OUT_OF_MEMORY;
  }
  return CSFMM_ERR_CUDA;
}

}  // namespace csfmm

using namespace csfmm;

namespace {

bool kernel_ok(int k) {
  return k == CSFMM_KERNEL_LAPLACE || k == CSFMM_KERNEL_BIOT_SAVART || k == CSFMM_KERNEL_NEWTON ||
         k == CSFMM_KERNEL_BIHARMONIC || k == CSFMM_KERNEL_SAL || k == CSFMM_KERNEL_ONE;
}

int kernel_dim(int k) { return k == CSFMM_KERNEL_BIOT_SAVART ? 3 : 1; }

csfmm_status check_device_pointer(const void *p, const char *name) {
  if (!p) {
    set_error("%s is NULL", name);
    return CSFMM_ERR_INVALID_ARG;
  }
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("%s: cannot query pointer attributes (%s)", name, cudaGetErrorString(e));
    return CSFMM_ERR_INVALID_ARG;
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) {
    set_error("%s is not device memory", name);
    return CSFMM_ERR_INVALID_ARG;
  }
  return CSFMM_OK;
}

csfmm_status evaluate_chunks(Plan &pl, Workspace &W, const double *w, int nrhs, double *out,
                             cudaStream_t st) {
  for (int r0 = 0; r0 < nrhs; r0 += W.max_nrhs) {
    int nr = nrhs - r0 < W.max_nrhs ? nrhs - r0 : W.max_nrhs;
    csfmm_status s = evaluate_impl(pl, W, w + (size_t)r0 * pl.nsrc, nr,
                                   out + (size_t)r0 * pl.ntgt * pl.dim, st);
    if (s != CSFMM_OK) return s;
  }
  return CSFMM_OK;
}

csfmm_status check_eval_args(csfmm_plan plan, const double *weights, int nrhs, const double *out) {
  if (!plan) {
    set_error("plan is NULL");
    return CSFMM_ERR_INVALID_ARG;
  }
  if (nrhs < 1) {
    set_error("nrhs must be >= 1 (got %d)", nrhs);
    return CSFMM_ERR_INVALID_ARG;
  }
  csfmm_status s;
  if ((s = check_device_pointer(weights, "weights")) != CSFMM_OK) return s;
  if ((s = check_device_pointer(out, "out")) != CSFMM_OK) return s;
  return CSFMM_OK;
}

}  // namespace

extern "C" {

const char *csfmm_last_error(void) { return g_err; }

const char *csfmm_version(void) { return "csfmm-gb300 0.1 (sm_103a)"; }

csfmm_status csfmm_plan_create(const double *points, int64_t N, int kernel_id, int degree,
                               double theta, int max_leaf, const csfmm_options *opt,
                               void *stream, csfmm_plan *out) {
  auto t0 = std::chrono::steady_clock::now();
  if (!out) {
    set_error("out is NULL");
    return CSFMM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (N < 1 || N >= ((int64_t)1 << 31)) {
    set_error("N must be in [1, 2^31) (got %lld)", (long long)N);
    return CSFMM_ERR_INVALID_ARG;
  }
  if (!kernel_ok(kernel_id)) {
    set_error("unknown kernel id %d", kernel_id);
    return CSFMM_ERR_INVALID_ARG;
  }
  if (degree < 1 || degree > kMaxDegree) {
    set_error("degree must be in [1, %d] (got %d)", kMaxDegree, degree);
    return CSFMM_ERR_INVALID_ARG;
  }
  if (!(theta > 0.0 && theta < 1.0)) {
    set_error("theta must be in (0, 1) (got %g)", theta);
    return CSFMM_ERR_INVALID_ARG;
  }
  if (max_leaf < 1) {
    set_error("max_leaf must be >= 1 (got %d)", max_leaf);
    return CSFMM_ERR_INVALID_ARG;
  }
  csfmm_options o{};
  o.precision = CSFMM_FP64;
  o.max_nrhs = 16;
  if (opt) o = *opt;
  if (o.precision != CSFMM_FP64 && o.precision != CSFMM_FP32_BULK) {
    set_error("unknown precision %d", o.precision);
    return CSFMM_ERR_INVALID_ARG;
  }
  if (o.max_nrhs < 1) o.max_nrhs = 16;
  if (o.max_nrhs > csfmm::kMaxNrhs) {
    set_error("max_nrhs must be <= %d (got %d)", csfmm::kMaxNrhs, o.max_nrhs);
    return CSFMM_ERR_INVALID_ARG;
  }
  csfmm_status s = check_device_pointer(points, "points");
  if (s != CSFMM_OK) return s;

  csfmm_plan h = new (std::nothrow) csfmm_plan_s;
  if (!h) {
    set_error("host allocation failed");
    return CSFMM_ERR_OUT_OF_MEMORY;
  }
  Plan &pl = h->impl;
  cudaGetDevice(&pl.device);
  pl.N = N;
  pl.nsrc = N;
  pl.ntgt = N;
  pl.tbase = 0;
  pl.kernel_id = kernel_id;
  pl.n = degree;
  pl.p = degree + 1;
  pl.P = pl.p * pl.p;
  pl.N0 = max_leaf;
  pl.theta = theta;
  pl.precision = o.precision;
  pl.dim = kernel_dim(kernel_id);
  pl.max_nrhs = o.max_nrhs;
  pl.use_graphs = o.use_graphs;
  pl.shrink = o.shrink != 0;
  pl.no_persistent = o.no_persistent != 0;
  if (o.schedule < 0 || o.schedule > 127) {
    set_error("schedule must be an OR of CSFMM_SCHED_* bits (got %d)", o.schedule);
    delete h;
    return CSFMM_ERR_INVALID_ARG;
  }
  pl.schedule = o.schedule;
  pl.rhs_chunk = o.rhs_chunk == 0 ? 16 : o.rhs_chunk;
  if (pl.rhs_chunk != 16 && pl.rhs_chunk != 8 && pl.rhs_chunk != 4) {
    set_error("rhs_chunk must be 0, 4, 8 or 16 (got %d)", o.rhs_chunk);
    delete h;
    return CSFMM_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  s = build_tree(pl, points, st);
  if (s == CSFMM_OK) {
    pl.ws = new (std::nothrow) Workspace;
    if (!pl.ws) {
      set_error("host allocation failed");
      s = CSFMM_ERR_OUT_OF_MEMORY;
    } else {
      pl.ws->arena.stream = st;
      s = workspace_alloc(pl, *pl.ws, pl.max_nrhs);
    }
  }
  if (s != CSFMM_OK) {
    cudaStreamSynchronize(st);
    if (pl.ws) {
      pl.ws->arena.release();
      delete pl.ws;
    }
    pl.arena.release();
    delete h;
    return s;
  }
  csfmm_stats &S = pl.stats;
  S.N = N;
  S.kernel_id = kernel_id;
  S.degree = degree;
  S.max_leaf = max_leaf;
  S.precision = pl.precision;
  S.theta = theta;
  S.nlevels = pl.nlevels;
  S.ncells = pl.ncells;
  S.nleaves = pl.nleaves;
  S.device_bytes = pl.arena.bytes + pl.ws->arena.bytes;
  S.build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = h;
  return CSFMM_OK;
}

csfmm_status csfmm_plan_create_targets(const double *sources, int64_t Ns, const double *targets,
                                       int64_t Nt, int kernel_id, int degree, double theta,
                                       int max_leaf, const csfmm_options *opt, void *stream,
                                       csfmm_plan *out) {
  if (!out || !sources || !targets || Ns < 1 || Nt < 1 || Ns + Nt >= ((int64_t)1 << 31)) {
    set_error("csfmm_plan_create_targets: non-NULL arrays, Ns, Nt >= 1 and Ns + Nt < 2^31 "
              "required");
    if (out) *out = nullptr;
    return CSFMM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  double *u = nullptr;
  CSFMM_CUDA(cudaMallocFromPoolAsync((void **)&u, sizeof(double) * 3 * (size_t)(Ns + Nt), memory_pool(), st));
  cudaError_t e = cudaMemcpyAsync(u, sources, sizeof(double) * 3 * (size_t)Ns,
                                  cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(u + 3 * (size_t)Ns, targets, sizeof(double) * 3 * (size_t)Nt,
                        cudaMemcpyDeviceToDevice, st);
  csfmm_status s = e == cudaSuccess ? CSFMM_OK : cuda_status(e, "cudaMemcpyAsync");
  // one tree over sources then targets; the build synchronises the stream
  if (s == CSFMM_OK)
    s = csfmm_plan_create(u, Ns + Nt, kernel_id, degree, theta, max_leaf, opt, stream, out);
  e = cudaFreeAsync(u, st);
  if (s == CSFMM_OK && e != cudaSuccess) s = cuda_status(e, "cudaFreeAsync");
  if (s != CSFMM_OK) {
    if (*out) csfmm_plan_destroy(*out);
    *out = nullptr;
    return s;
  }
  Plan &pl = (*out)->impl;
  pl.nsrc = Ns;
  pl.ntgt = Nt;
  pl.tbase = Ns;
  return CSFMM_OK;
}

csfmm_status csfmm_evaluate(csfmm_plan plan, const double *weights, int nrhs, double *out,
                            void *stream) {
  csfmm_status s = check_eval_args(plan, weights, nrhs, out);
  if (s != CSFMM_OK) return s;
  return evaluate_chunks(plan->impl, *plan->impl.ws, weights, nrhs, out, (cudaStream_t)stream);
}

csfmm_status csfmm_evaluate_cstc(csfmm_plan plan, const double *weights, int nrhs, double *out,
                                 void *stream) {
  csfmm_status s = check_eval_args(plan, weights, nrhs, out);
  if (s != CSFMM_OK) return s;
  Plan &pl = plan->impl;
  Workspace &W = *pl.ws;
  for (int r0 = 0; r0 < nrhs; r0 += W.max_nrhs) {
    const int nr = nrhs - r0 < W.max_nrhs ? nrhs - r0 : W.max_nrhs;
    s = cstc_impl(pl, W, weights + (size_t)r0 * pl.nsrc, nr, out + (size_t)r0 * pl.ntgt * pl.dim,
                  (cudaStream_t)stream);
    if (s != CSFMM_OK) return s;
  }
  return CSFMM_OK;
}

csfmm_status csfmm_evaluate_host(csfmm_plan plan, const double *weights, int nrhs, double *out,
                                 void *stream) {
  if (!plan || !weights || !out || nrhs < 1) {
    set_error("plan, weights and out must be non-NULL and nrhs >= 1");
    return CSFMM_ERR_INVALID_ARG;
  }
  Plan &pl = plan->impl;
  Workspace &W = *pl.ws;
  cudaStream_t st = (cudaStream_t)stream;
  if (!W.stage_w) {
    W.arena.stream = st;
    csfmm_status s = W.arena.alloc(&W.stage_w, (size_t)W.max_nrhs * pl.nsrc);
    if (s != CSFMM_OK) return s;
    s = W.arena.alloc(&W.stage_out, (size_t)W.max_nrhs * pl.ntgt * pl.dim);
    if (s != CSFMM_OK) return s;
    pl.stats.device_bytes = pl.arena.bytes + W.arena.bytes;
  }
  for (int r0 = 0; r0 < nrhs; r0 += W.max_nrhs) {
    int nr = nrhs - r0 < W.max_nrhs ? nrhs - r0 : W.max_nrhs;
    CSFMM_CUDA(cudaMemcpyAsync(W.stage_w, weights + (size_t)r0 * pl.nsrc,
                               sizeof(double) * (size_t)nr * pl.nsrc, cudaMemcpyHostToDevice, st));
    csfmm_status s = evaluate_impl(pl, W, W.stage_w, nr, W.stage_out, st);
    if (s != CSFMM_OK) return s;
    CSFMM_CUDA(cudaMemcpyAsync(out + (size_t)r0 * pl.ntgt * pl.dim, W.stage_out,
                               sizeof(double) * (size_t)nr * pl.ntgt * pl.dim, cudaMemcpyDeviceToHost,
                               st));
  }
  CSFMM_CUDA(cudaStreamSynchronize(st));
  return CSFMM_OK;
}

csfmm_status csfmm_workspace_create(csfmm_plan plan, int max_nrhs, csfmm_workspace *out) {
  if (!plan || !out || max_nrhs < 1 || max_nrhs > csfmm::kMaxNrhs) {
    set_error("plan and out must be non-NULL and 1 <= max_nrhs <= 64");
    return CSFMM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  csfmm_workspace w = new (std::nothrow) csfmm_workspace_s;
  if (!w) {
    set_error("host allocation failed");
    return CSFMM_ERR_OUT_OF_MEMORY;
  }
  w->impl.arena.stream = release_stream();
  csfmm_status s = workspace_alloc(plan->impl, w->impl, max_nrhs);
  // the buffers are used on the caller's streams: wait for the allocations
  cudaError_t e = cudaStreamSynchronize(w->impl.arena.stream);
  if (s == CSFMM_OK && e != cudaSuccess) s = cuda_status(e, "cudaStreamSynchronize");
  if (s != CSFMM_OK) {
    w->impl.arena.release();
    delete w;
    return s;
  }
  *out = w;
  return CSFMM_OK;
}

csfmm_status csfmm_workspace_destroy(csfmm_workspace ws) {
  if (!ws) return CSFMM_OK;
  ws->impl.release_graphs();
  ws->impl.arena.release();
  delete ws;
  return CSFMM_OK;
}

csfmm_status csfmm_evaluate_ws(csfmm_plan plan, csfmm_workspace ws, const double *weights, int nrhs,
                               double *out, void *stream) {
  csfmm_status s = check_eval_args(plan, weights, nrhs, out);
  if (s != CSFMM_OK) return s;
  if (!ws || ws->impl.plan != &plan->impl) {
    set_error("workspace is NULL or belongs to another plan");
    return CSFMM_ERR_INVALID_ARG;
  }
  return evaluate_chunks(plan->impl, ws->impl, weights, nrhs, out, (cudaStream_t)stream);
}

csfmm_status csfmm_direct(const double *points, int64_t N, int kernel_id, const double *weights,
                          int nrhs, double *out, int precision, void *stream) {
  return csfmm_direct_targets(points, N, kernel_id, weights, nrhs, nullptr, 0, out, precision,
                              stream);
}

csfmm_status csfmm_direct_targets(const double *points, int64_t N, int kernel_id,
                                  const double *weights, int nrhs, const int64_t *targets,
                                  int64_t ntargets, double *out, int precision, void *stream) {
  if (N < 1 || N >= ((int64_t)1 << 31) || nrhs < 1 || !kernel_ok(kernel_id) ||
      (precision != CSFMM_FP64 && precision != CSFMM_FP32_BULK) ||
      (targets && (ntargets < 0 || ntargets >= ((int64_t)1 << 31)))) {
    set_error("invalid N, nrhs, kernel id, precision or target count");
    return CSFMM_ERR_INVALID_ARG;
  }
  csfmm_status s;
  if ((s = check_device_pointer(points, "points")) != CSFMM_OK) return s;
  if ((s = check_device_pointer(weights, "weights")) != CSFMM_OK) return s;
  if ((s = check_device_pointer(out, "out")) != CSFMM_OK) return s;
  if (targets && (s = check_device_pointer(targets, "targets")) != CSFMM_OK) return s;
  return direct_impl(points, N, kernel_id, weights, nrhs, targets, ntargets, out, precision,
                     (cudaStream_t)stream);
}

csfmm_status csfmm_plan_stats(csfmm_plan plan, csfmm_stats *stats) {
  if (!plan || !stats) {
    set_error("plan and stats must be non-NULL");
    return CSFMM_ERR_INVALID_ARG;
  }
  *stats = plan->impl.stats;
  return CSFMM_OK;
}

csfmm_status csfmm_plan_export_cells(csfmm_plan plan, int32_t *face, int32_t *level, int64_t *ia,
                                     int64_t *ib, int64_t *begin, int64_t *end, int32_t *parent,
                                     int32_t *child, double *centre, double *radius) {
  if (!plan) {
    set_error("plan is NULL");
    return CSFMM_ERR_INVALID_ARG;
  }
  Plan &pl = plan->impl;
  const size_t nc = (size_t)pl.ncells;
  if (face) CSFMM_CUDA(cudaMemcpy(face, pl.cface, 4 * nc, cudaMemcpyDeviceToHost));
  if (level) CSFMM_CUDA(cudaMemcpy(level, pl.clevel, 4 * nc, cudaMemcpyDeviceToHost));
  if (ia) CSFMM_CUDA(cudaMemcpy(ia, pl.cia, 8 * nc, cudaMemcpyDeviceToHost));
  if (ib) CSFMM_CUDA(cudaMemcpy(ib, pl.cib, 8 * nc, cudaMemcpyDeviceToHost));
  if (parent) CSFMM_CUDA(cudaMemcpy(parent, pl.cparent, 4 * nc, cudaMemcpyDeviceToHost));
  if (child) CSFMM_CUDA(cudaMemcpy(child, pl.cchild, 16 * nc, cudaMemcpyDeviceToHost));
  if (centre) CSFMM_CUDA(cudaMemcpy(centre, pl.ccentre, 24 * nc, cudaMemcpyDeviceToHost));
  if (radius) CSFMM_CUDA(cudaMemcpy(radius, pl.cradius, 8 * nc, cudaMemcpyDeviceToHost));
  if (begin || end) {
    std::vector<int32_t> tmp(nc);
    if (begin) {
      CSFMM_CUDA(cudaMemcpy(tmp.data(), pl.cbegin, 4 * nc, cudaMemcpyDeviceToHost));
      for (size_t c = 0; c < nc; ++c) begin[c] = tmp[c];
    }
    if (end) {
      CSFMM_CUDA(cudaMemcpy(tmp.data(), pl.cend, 4 * nc, cudaMemcpyDeviceToHost));
      for (size_t c = 0; c < nc; ++c) end[c] = tmp[c];
    }
  }
  return CSFMM_OK;
}

csfmm_status csfmm_plan_export_list(csfmm_plan plan, int list_type, int32_t *t, int32_t *s) {
  if (!plan || list_type < 0 || list_type > 3 || !t || !s) {
    set_error("invalid plan, list type or output pointer");
    return CSFMM_ERR_INVALID_ARG;
  }
  Plan &pl = plan->impl;
  const size_t nc = (size_t)pl.ncells;
  std::vector<int32_t> off(nc + 1);
  CSFMM_CUDA(cudaMemcpy(off.data(), pl.loff[list_type], 4 * (nc + 1), cudaMemcpyDeviceToHost));
  const int64_t n = pl.nlist[list_type];
  if (n > 0) CSFMM_CUDA(cudaMemcpy(s, pl.lsrc[list_type], 4 * (size_t)n, cudaMemcpyDeviceToHost));
  for (size_t c = 0; c < nc; ++c)
    for (int32_t e = off[c]; e < off[c + 1]; ++e) t[e] = (int32_t)c;
  return CSFMM_OK;
}

csfmm_status csfmm_plan_export_order(csfmm_plan plan, int64_t *order) {
  if (!plan || !order) {
    set_error("plan and order must be non-NULL");
    return CSFMM_ERR_INVALID_ARG;
  }
  Plan &pl = plan->impl;
  std::vector<int32_t> tmp((size_t)pl.N);
  CSFMM_CUDA(cudaMemcpy(tmp.data(), pl.perm, 4 * (size_t)pl.N, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < pl.N; ++i) order[i] = tmp[(size_t)i];
  return CSFMM_OK;
}

csfmm_status csfmm_plan_export_proxies(csfmm_plan plan, double *proxies) {
  if (!plan || !proxies) {
    set_error("plan and proxies must be non-NULL");
    return CSFMM_ERR_INVALID_ARG;
  }
  Plan &pl = plan->impl;
  const size_t nc = (size_t)pl.ncells, P = (size_t)pl.P;
  std::vector<double> tmp(nc * 3 * P);
  CSFMM_CUDA(cudaMemcpy(tmp.data(), pl.proxy, 8 * tmp.size(), cudaMemcpyDeviceToHost));
  for (size_t c = 0; c < nc; ++c)
    for (size_t k = 0; k < P; ++k)
      for (int d = 0; d < 3; ++d) proxies[(c * P + k) * 3 + d] = tmp[(c * 3 + d) * P + k];
  return CSFMM_OK;
}

csfmm_status csfmm_plan_export_proxy_weights(csfmm_plan plan, int nrhs, double *wbar) {
  if (!plan || !wbar || nrhs < 1) {
    set_error("invalid plan, nrhs or output pointer");
    return CSFMM_ERR_INVALID_ARG;
  }
  Plan &pl = plan->impl;
  Workspace &W = *pl.ws;
  if (nrhs > W.last_nrhs) {
    set_error("nrhs %d exceeds the last evaluation's %d", nrhs, W.last_nrhs);
    return CSFMM_ERR_INVALID_ARG;
  }
  CSFMM_CUDA(cudaDeviceSynchronize());
  const size_t nc = (size_t)pl.ncells, P = (size_t)pl.P, R = (size_t)W.max_nrhs;
  std::vector<double> tmp(nc * R * P);
  if (pl.precision == CSFMM_FP64) {
    CSFMM_CUDA(cudaMemcpy(tmp.data(), W.wbar, 8 * tmp.size(), cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> t32(nc * R * P);
    CSFMM_CUDA(cudaMemcpy(t32.data(), W.wbar32, 4 * t32.size(), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < t32.size(); ++i) tmp[i] = t32[i];
  }
  for (size_t c = 0; c < nc; ++c)
    for (int r = 0; r < nrhs; ++r)
      memcpy(wbar + (c * nrhs + r) * P, tmp.data() + (c * R + r) * P, 8 * P);
  return CSFMM_OK;
}

csfmm_status csfmm_plan_sync(csfmm_plan plan, void *stream) {
  if (!plan) {
    set_error("plan is NULL");
    return CSFMM_ERR_INVALID_ARG;
  }
  Plan &pl = plan->impl;
  CSFMM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  int st = 0;
  CSFMM_CUDA(cudaMemcpy(&st, pl.status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st & kStatusTimeout) {
    // a timeout is reported once: the word is cleared so that the plan can
    // be evaluated again
    const int zero = 0;
    CSFMM_CUDA(cudaMemcpy(pl.status, &zero, sizeof(int), cudaMemcpyHostToDevice));
    set_error("a bounded device-side wait timed out (status 0x%x)", st);
    return CSFMM_ERR_TIMEOUT;
  }
  if (st) {
    set_error("device status word 0x%x", st);
    return CSFMM_ERR_DEVICE;
  }
  return CSFMM_OK;
}

csfmm_status csfmm_plan_test_wait(csfmm_plan plan, int never_ready, double limit_ms) {
  if (!plan || !(limit_ms > 0.0) || limit_ms > 60000.0) {
    set_error("plan must be non-NULL and 0 < limit_ms <= 60000");
    return CSFMM_ERR_INVALID_ARG;
  }
  plan->impl.wait_never_ready = never_ready != 0;
  plan->impl.wait_limit_ms = limit_ms;
  return CSFMM_OK;
}

csfmm_status csfmm_plan_enable_timing(csfmm_plan plan, int on) {
  if (!plan) {
    set_error("plan is NULL");
    return CSFMM_ERR_INVALID_ARG;
  }
  plan->impl.timing = on != 0;
  return CSFMM_OK;
}

csfmm_status csfmm_plan_phase_times(csfmm_plan plan, double *ms, int64_t *calls) {
  if (!plan || !ms) {
    set_error("plan and ms must be non-NULL");
    return CSFMM_ERR_INVALID_ARG;
  }
  Plan &pl = plan->impl;
  for (int k = 0; k < CSFMM_NUM_PHASES; ++k) ms[k] = 0.0;
  const size_t per = 2 * CSFMM_NUM_PHASES;
  csfmm_status st = CSFMM_OK;
  for (size_t c = 0; c + per <= pl.events.size(); c += per) {
    for (int k = 0; k < CSFMM_NUM_PHASES; ++k) {
      float t = 0.f;
      cudaError_t e = cudaEventSynchronize(pl.events[c + 2 * k + 1]);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, pl.events[c + 2 * k], pl.events[c + 2 * k + 1]);
      if (e != cudaSuccess && st == CSFMM_OK) st = cuda_status(e, "cudaEventElapsedTime");
      ms[k] += t;
    }
  }
  if (calls) *calls = pl.timed_calls;
  for (cudaEvent_t e : pl.events) cudaEventDestroy(e);
  pl.events.clear();
  pl.timed_calls = 0;
  return st;
}

csfmm_status csfmm_plan_destroy(csfmm_plan plan) {
  if (!plan) return CSFMM_OK;
  Plan &pl = plan->impl;
  for (cudaEvent_t e : pl.events) cudaEventDestroy(e);
  pl.events.clear();
  if (pl.ws) {
    pl.ws->release_graphs();
    pl.ws->arena.release();
    delete pl.ws;
    pl.ws = nullptr;
  }
  pl.arena.release();
  delete plan;
  return CSFMM_OK;
}

}  // extern "C"
