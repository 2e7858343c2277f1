// autotune.cu -- csfmm_autotune: picks the maximum leaf size N0 and, for the
// FP32-bulk multi-right-hand-side kernels, the right-hand-side chunk width,
// by timing real evaluations of the caller's point set.
//
// The leaf size changes the tree and hence the approximation, so a candidate
// is accepted only if its error against an FP64 direct sum on fixed sampled
// targets stays within err_factor of the error of the paper's default
// N0 = 4 n^2; the chunk width changes only the order of FP32 sums.
#include <math.h>
#include <stdio.h>
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

bool cache_lookup(const char *path, const std::string &key, csfmm_tune_result *out) {
  std::lock_guard<std::mutex> lk(g_cache_mutex);
  FILE *f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    char k[512];
    csfmm_tune_result r{};
    if (sscanf(line, "%511s %d %d %lf %lf %lf %lf", k, &r.max_leaf, &r.rhs_chunk, &r.ms_per_eval,
               &r.rel_err, &r.default_ms, &r.default_rel_err) == 7 &&
        key == k && r.max_leaf >= 1) {
      *out = r;  // the last matching line wins
      found = true;
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char *path, const std::string &key, const csfmm_tune_result &r) {
  std::lock_guard<std::mutex> lk(g_cache_mutex);
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %.6g %.6g %.6g %.6g\n", key.c_str(), r.max_leaf, r.rhs_chunk,
          r.ms_per_eval, r.rel_err, r.default_ms, r.default_rel_err);
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

  const int n2 = degree * degree;
  const int mult[] = {4, 1, 2, 3, 6, 8};  // the default first
  std::vector<int> chunks = {0};
  if (precision == CSFMM_FP32_BULK && nrhs >= 8 && kernel_id != CSFMM_KERNEL_BIOT_SAVART)
    chunks = {0, 8, 4};
  struct Cand { int leaf, chunk; double ms, err; };
  std::vector<Cand> cands;
  for (int mlt : mult) {
    const int leaf = mlt * n2 < 8 ? 8 : mlt * n2;
    bool dup = false;
    for (const Cand &c : cands) dup |= c.leaf == leaf;
    if (dup) continue;
    csfmm_options opt{};
    opt.precision = precision;
    opt.max_nrhs = nrhs;
    csfmm_plan plan = nullptr;
    s = csfmm_plan_create(points, N, kernel_id, degree, theta, leaf, &opt, st, &plan);
    if (s != CSFMM_OK) {
      cleanup();
      return s;
    }
    for (int ch : chunks) {
      plan->impl.rhs_chunk = ch == 0 ? 16 : ch;
      s = csfmm_evaluate(plan, weights, nrhs, outbuf, st);  // warm-up
      cudaEventRecord(e0, st);
      for (int k = 0; k < 3 && s == CSFMM_OK; ++k) s = csfmm_evaluate(plan, weights, nrhs, outbuf, st);
      cudaEventRecord(e1, st);
      if (s == CSFMM_OK) s = csfmm_plan_sync(plan, st);
      if (s != CSFMM_OK) {
        csfmm_plan_destroy(plan);
        cleanup();
        return s;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      pick_kernel<<<(ns * dim + 127) / 128, 128, 0, st>>>(outbuf, tg, ns, dim, got);
      cudaMemcpyAsync(hgot.data(), got, sizeof(double) * hgot.size(), cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
      double dn = 0.0;
      for (size_t i = 0; i < hgot.size(); ++i) dn += (hgot[i] - href[i]) * (hgot[i] - href[i]);
      cands.push_back({leaf, ch, ms / 3.0, rnorm > 0 ? sqrt(dn) / rnorm : sqrt(dn)});
    }
    csfmm_plan_destroy(plan);
  }
  cleanup();
  const Cand &def = cands[0];
  const Cand *best = &def;
  for (const Cand &c : cands)
    if (c.err <= err_factor * def.err + 1e-300 && c.ms < best->ms) best = &c;
  out->max_leaf = best->leaf;
  out->rhs_chunk = best->chunk;
  out->ms_per_eval = best->ms;
  out->rel_err = best->err;
  out->default_ms = def.ms;
  out->default_rel_err = def.err;
  out->candidates = (int)cands.size();
  out->from_cache = 0;
  if (cache_path) cache_store(cache_path, key, *out);
  return CSFMM_OK;
}
