// autotune.cu -- csfmm_autotune: picks the maximum leaf size N0, then the
// launch schedule and tile shapes (persistent or per-phase launches,
// right-hand-side chunk, threads and targets per thread of the multi-right-
// hand-side kernels, FP32 chunk width, symmetric pass, side-stream overlap),
// by timing real evaluations of the caller's point set.
//
// The leaf size changes the tree and hence the approximation, and the FP32
// chunk width the rounding, so a candidate is accepted only if its error
// against an FP64 direct sum on fixed sampled targets stays within
// err_factor of the error of the paper's default N0 = 4 n^2 with default
// options; the other choices change only the work layout.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "csfmm_internal.cuh"

namespace {

std::mutex g_cache_mutex;

std::string cache_key(int device, int kid, int degree, double theta, int prec, int nrhs,
                      int64_t N) {
  cudaDeviceProp prop;
  char name[256] = "unknown";
  if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) snprintf(name, sizeof name, "%s", prop.name);
  for (char *c = name; *c; ++c)
    if (*c == ' ' || *c == '|') *c = '_';
  char buf[512];
  snprintf(buf, sizeof buf, "%s|k%d|n%d|t%.9g|p%d|r%d|N%lld", name, kid, degree, theta, prec,
           nrhs, (long long)N);
  return buf;
}

bool finite_nonneg(double x) { return isfinite(x) && x >= 0.0; }

// One cache line of the current format, validated; false for anything else.
bool parse_line(const char *line, std::string *key, csfmm_tune_result *r) {
  char tag[8], k[512], extra[8];
  csfmm_tune_result t{};
  const int n = sscanf(line, "%7s %511s %d %d %d %d %lf %lf %lf %lf %7s", tag, k, &t.max_leaf,
                       &t.rhs_chunk, &t.no_persistent, &t.schedule, &t.ms_per_eval, &t.rel_err,
                       &t.default_ms, &t.default_rel_err, extra);
  if (n != 10 || strcmp(tag, "v2") != 0) return false;  // stale format, cut short or trailing text
  if (t.max_leaf < 1 || (t.rhs_chunk != 0 && t.rhs_chunk != 4 && t.rhs_chunk != 8 &&
                         t.rhs_chunk != 16) ||
      (t.no_persistent != 0 && t.no_persistent != 1) || t.schedule < 0 || t.schedule > 127 ||
      !finite_nonneg(t.ms_per_eval) || !finite_nonneg(t.rel_err) ||
      !finite_nonneg(t.default_ms) || !finite_nonneg(t.default_rel_err))
    return false;
  *key = k;
  *r = t;
  return true;
}

bool cache_lookup(const char *path, const std::string &key, csfmm_tune_result *out) {
  std::lock_guard<std::mutex> lk(g_cache_mutex);
  FILE *f = fopen(path, "r");
  if (!f) return false;
  char *line = nullptr;
  size_t cap = 0;
  ssize_t n;
  bool found = false;
  while ((n = getline(&line, &cap, f)) >= 0) {
    // longer than any valid line, or holding a NUL byte: not a cache line
    if (n > 1000 || memchr(line, 0, (size_t)n)) continue;
    std::string k;
    csfmm_tune_result r{};
    if (parse_line(line, &k, &r) && k == key) {
      *out = r;  // the last valid matching line wins
      found = true;
    }
  }
  free(line);
  fclose(f);
  return found;
}

void cache_store(const char *path, const std::string &key, const csfmm_tune_result &r) {
  std::lock_guard<std::mutex> lk(g_cache_mutex);
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "v2 %s %d %d %d %d %.9g %.9g %.9g %.9g\n", key.c_str(), r.max_leaf, r.rhs_chunk,
          r.no_persistent, r.schedule, r.ms_per_eval, r.rel_err, r.default_ms,
          r.default_rel_err);
  fclose(f);
}

__global__ void sample_targets_kernel(int64_t *t, int n, int64_t N) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) t[i] = (int64_t)(((uint64_t)i * 2654435761ull + 12345ull) % (uint64_t)N);
}

__global__ void pick_kernel(const double *out, const int64_t *t, int n, int dim, double *dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n * dim) dst[i] = out[t[i / dim] * dim + i % dim];
}

struct Scratch {
  std::vector<void *> p;
  ~Scratch() {
    for (void *q : p) cudaFree(q);
  }
  template <class T>
  csfmm_status alloc(T **x, size_t n) {
    if (cudaMalloc((void **)x, n * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      csfmm::set_error("autotune: cudaMalloc of %zu bytes failed", n * sizeof(T));
      return CSFMM_ERR_OUT_OF_MEMORY;
    }
    p.push_back(*x);
    return CSFMM_OK;
  }
};

}  // namespace

using namespace csfmm;

extern "C" csfmm_status csfmm_autotune(const double *points, int64_t N, int kernel_id, int degree,
                                       double theta, const double *weights, int nrhs,
                                       int precision, const char *cache_path, double err_factor,
                                       csfmm_tune_result *out) {
  if (!points || !weights || !out || N < 1 || nrhs < 1 || nrhs > 64 || degree < 1 ||
      degree > kMaxDegree || !(err_factor >= 1.0)) {
    set_error("autotune: invalid arguments");
    return CSFMM_ERR_INVALID_ARG;
  }
  *out = csfmm_tune_result{};
  int device = 0;
  cudaGetDevice(&device);
  const std::string key = cache_key(device, kernel_id, degree, theta, precision, nrhs, N);
  if (cache_path && cache_lookup(cache_path, key, out)) {
    out->from_cache = 1;
    return CSFMM_OK;
  }
  const int dim = kernel_id == CSFMM_KERNEL_BIOT_SAVART ? 3 : 1;
  const int ns = (int)(N < 256 ? N : 256);
  Scratch sc;
  int64_t *tg;
  double *ref, *got, *outbuf;
  csfmm_status s;
  if ((s = sc.alloc(&tg, ns)) != CSFMM_OK) return s;
  if ((s = sc.alloc(&ref, (size_t)ns * dim)) != CSFMM_OK) return s;
  if ((s = sc.alloc(&got, (size_t)ns * dim)) != CSFMM_OK) return s;
  if ((s = sc.alloc(&outbuf, (size_t)nrhs * N * dim)) != CSFMM_OK) return s;
  cudaStream_t st;
  CSFMM_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
  };
  sample_targets_kernel<<<(ns + 127) / 128, 128, 0, st>>>(tg, ns, N);
  s = csfmm_direct_targets(points, N, kernel_id, weights, 1, tg, ns, ref, CSFMM_FP64, st);
  if (s != CSFMM_OK) {
    cleanup();
    return s;
  }
  std::vector<double> href((size_t)ns * dim), hgot((size_t)ns * dim);
  cudaMemcpyAsync(href.data(), ref, sizeof(double) * href.size(), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  double rnorm = 0.0;
  for (double v : href) rnorm += v * v;
  rnorm = sqrt(rnorm);

  struct Cand {
    int leaf, chunk, nop, sched;
    double ms, err;
  };
  std::vector<Cand> cands;
  // times one configuration of an existing plan and records it
  auto measure = [&](csfmm_plan plan, int leaf, int chunk, int nop, int sched) -> csfmm_status {
    plan->impl.rhs_chunk = chunk == 0 ? 16 : chunk;
    plan->impl.no_persistent = nop;
    plan->impl.schedule = sched;
    csfmm_status r = csfmm_evaluate(plan, weights, nrhs, outbuf, st);  // warm-up
    cudaEventRecord(e0, st);
    for (int k = 0; k < 3 && r == CSFMM_OK; ++k) r = csfmm_evaluate(plan, weights, nrhs, outbuf, st);
    cudaEventRecord(e1, st);
    if (r == CSFMM_OK) r = csfmm_plan_sync(plan, st);
    if (r != CSFMM_OK) return r;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    pick_kernel<<<(ns * dim + 127) / 128, 128, 0, st>>>(outbuf, tg, ns, dim, got);
    cudaMemcpyAsync(hgot.data(), got, sizeof(double) * hgot.size(), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    double dn = 0.0;
    for (size_t i = 0; i < hgot.size(); ++i) dn += (hgot[i] - href[i]) * (hgot[i] - href[i]);
    cands.push_back({leaf, chunk, nop, sched, ms / 3.0, rnorm > 0 ? sqrt(dn) / rnorm : sqrt(dn)});
    return CSFMM_OK;
  };
  auto build = [&](int leaf, csfmm_plan *plan) {
    csfmm_options opt{};
    opt.precision = precision;
    opt.max_nrhs = nrhs;
    return csfmm_plan_create(points, N, kernel_id, degree, theta, leaf, &opt, st, plan);
  };
  auto accepted = [&](const Cand &c) { return c.err <= err_factor * cands[0].err + 1e-300; };

  // stage 1: the leaf size, default options (the paper's N0 = 4 n^2 first)
  const int n2 = degree * degree;
  const int mult[] = {4, 1, 2, 3, 6, 8};
  std::vector<int> leaves;
  for (int mlt : mult) {
    const int leaf = mlt * n2 < 8 ? 8 : mlt * n2;
    bool dup = false;
    for (int l : leaves) dup |= l == leaf;
    if (!dup) leaves.push_back(leaf);
  }
  for (int leaf : leaves) {
    csfmm_plan plan = nullptr;
    s = build(leaf, &plan);
    if (s == CSFMM_OK) s = measure(plan, leaf, 0, 0, 0);
    if (plan) csfmm_plan_destroy(plan);
    if (s != CSFMM_OK) {
      cleanup();
      return s;
    }
  }
  const Cand *b1 = &cands[0];
  for (const Cand &c : cands)
    if (accepted(c) && c.ms < b1->ms) b1 = &c;
  const int best_leaf = b1->leaf;

  // stage 2: launch schedule and tile shapes at that leaf size
  std::vector<Cand> sched;  // (chunk, nop, schedule) to try
  const bool scalar = kernel_id != CSFMM_KERNEL_BIOT_SAVART;
  if (precision == CSFMM_FP32_BULK && scalar && nrhs >= 8) {
    if (nrhs % 8 == 0) sched.push_back({0, 8, 0, 0, 0, 0});        // persistent, chunks of 8
    for (int ch : {0, 8, 4})
      for (int shape = 0; shape < 8; ++shape) sched.push_back({0, ch, 1, shape, 0, 0});
  } else {
    if (precision == CSFMM_FP32_BULK && scalar && nrhs == 1)
      sched.push_back({0, 0, 0, CSFMM_SCHED_NO_SYMMETRIC, 0, 0});
    sched.push_back({0, 0, 0, CSFMM_SCHED_NO_OVERLAP, 0, 0});
    sched.push_back({0, 0, 0, CSFMM_SCHED_SIDE_FIRST, 0, 0});
  }
  {
    csfmm_plan plan = nullptr;
    s = build(best_leaf, &plan);
    for (size_t k = 0; k < sched.size() && s == CSFMM_OK; ++k)
      s = measure(plan, best_leaf, sched[k].chunk, sched[k].nop, sched[k].sched);
    if (plan) csfmm_plan_destroy(plan);
    if (s != CSFMM_OK) {
      cleanup();
      return s;
    }
  }
  cleanup();
  const Cand &def = cands[0];
  const Cand *best = &def;
  for (const Cand &c : cands)
    if (accepted(c) && c.ms < best->ms) best = &c;
  out->max_leaf = best->leaf;
  out->rhs_chunk = best->chunk;
  out->no_persistent = best->nop;
  out->schedule = best->sched;
  out->ms_per_eval = best->ms;
  out->rel_err = best->err;
  out->default_ms = def.ms;
  out->default_rel_err = def.err;
  out->candidates = (int)cands.size();
  out->from_cache = 0;
  if (cache_path) cache_store(cache_path, key, *out);
  return CSFMM_OK;
}

extern "C" csfmm_status csfmm_tune_cache_read(const char *path, const char *key,
                                              csfmm_tune_result *out) {
  if (!path || !key || !out) {
    set_error("path, key and out must be non-NULL");
    return CSFMM_ERR_INVALID_ARG;
  }
  csfmm_tune_result r{};
  if (!cache_lookup(path, key, &r)) {
    set_error("not found: no valid line for this key in %s", path);
    return CSFMM_ERR_INVALID_ARG;
  }
  r.from_cache = 1;
  r.candidates = 0;
  *out = r;
  return CSFMM_OK;
}
