// tree.cu -- device construction of the cubed-sphere quadtree (Sec. 3), the
// cell geometry and Chebyshev proxies (Sec. 4) and the PP/PC/CP/CC lists of
// the dual tree traversal (Sec. 8, Algorithm "CSFMM").
//
// Steps (all device kernels; the host only drives the per-level loops and
// reads back per-level totals):
//   1. key_points: face of each point, face-plane coordinates (a, b), integer
//      cell coordinates by binary search in the tangent table, 39-bit key
//      (3 face bits + 18 Morton-interleaved bit pairs).
//   2. radix sort of (key, index): project-written stable LSD sort, 4-bit digits.
//   3. level-synchronous node build: a cell with more than N0 points splits into
//      its non-empty quadrants; child key ranges by binary search.
//   4. geometry: centre, radius (largest chord to the four corners), angles;
//      proxies; per-point Lagrange values and FP32 offsets.
//   5. traversal: frontier of (target, source) cell pairs, starting from all
//      ordered pairs of roots; each pair is either accepted into a list or
//      replaced by the pairs with the children of the cluster that splits.
//   6. lists sorted by (type, target, source) and grouped by target (CSR).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "csfmm_internal.cuh"

namespace csfmm {

// ---------------------------------------------------------------------------
// Host tangent table, identical for every plan of the process.
// ---------------------------------------------------------------------------
static std::once_flag g_tan_once;
static std::vector<double> g_tan;

const double *host_tan_table() {
  std::call_once(g_tan_once, [] {
    const int64_t M = (int64_t)1 << kD;
    const double kHalfPi = 1.57079632679489661923;
    const double kQuarterPi = 0.78539816339744830962;
    volatile double H = ldexp(kHalfPi, -kD);
    g_tan.resize((size_t)M + 1);
    for (int64_t k = 0; k <= M; ++k) {
      volatile double prod = (double)k * H;  // rounded product, no contraction
      g_tan[(size_t)k] = tan(prod - kQuarterPi);
    }
  });
  return g_tan.data();
}

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxPoolDevices] = {};
cudaStream_t g_release[kMaxPoolDevices] = {};
const double *g_dev_tan[kMaxPoolDevices] = {};
int g_sms[kMaxPoolDevices] = {};

int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxPoolDevices) {
    cudaGetLastError();
    d = 0;
  }
  return d;
}
}  // namespace

cudaMemPool_t memory_pool() {
  const int d = current_device();
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[d]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = d;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      cudaDeviceGetDefaultMemPool(&pool, d);  // still stream-ordered
    } else {
      uint64_t keep = kPoolKeepBytes;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    g_pool[d] = pool;
  }
  return g_pool[d];
}

cudaStream_t release_stream() {
  const int d = current_device();
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_release[d]) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      s = nullptr;  // the legacy default stream
    }
    g_release[d] = s;
  }
  return g_release[d];
}

const double *device_tan_table() {
  const int d = current_device();
  const double *Th = host_tan_table();
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_dev_tan[d]) {
    const size_t bytes = sizeof(double) * (((size_t)1 << kD) + 1);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(p, Th, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (p) cudaFree(p);
      set_error("uploading the tangent table failed: %s", cudaGetErrorString(e));
      return nullptr;
    }
    g_dev_tan[d] = (const double *)p;
  }
  return g_dev_tan[d];
}

int sm_count() {
  const int d = current_device();
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_sms[d]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = 1;
    }
    g_sms[d] = n;
  }
  return g_sms[d];
}

int grid_for(int64_t n, int block, int max_blocks) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return (int)g;
}

// ---------------------------------------------------------------------------
// Exclusive scan of int32 (1024 items per block, recursive over block sums).
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_sums, int *total) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
    int s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) warp_sums[lane] = s;
  }
  __syncthreads();
  int base = warp ? warp_sums[warp - 1] : 0;
  if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
  return base + x - v;
}

__global__ void scan_blocks_kernel(const int32_t *in, int32_t *out, int32_t *block_sums, int n) {
  __shared__ int warp_sums[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int v[kScanItems];
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int total;
  int pre = block_exclusive_scan(s, warp_sums, &total);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = pre;
    pre += v[k];
  }
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void add_block_offsets_kernel(int32_t *out, const int32_t *offs, int n) {
  int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  int add = offs[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k, i += kScanThreads)
    if (i < n) out[i] += add;
}

size_t scan_tmp_elems(int n) {
  size_t t = 0;
  int64_t m = n;
  while (true) {
    int64_t nb = (m + kScanTile - 1) / kScanTile;
    if (nb < 1) nb = 1;
    t += (size_t)nb + 1;
    if (nb == 1) break;
    m = nb;
  }
  return t + 2;
}

static void scan_rec(const int32_t *in, int32_t *out, int n, int32_t *tmp, cudaStream_t st) {
  int nb = (n + kScanTile - 1) / kScanTile;
  if (nb < 1) nb = 1;
  int32_t *sums = tmp;
  scan_blocks_kernel<<<nb, kScanThreads, 0, st>>>(in, out, sums, n);
  if (nb == 1) return;
  int32_t *sums_scanned = tmp + nb;  // in place is fine: each block reads before writing
  scan_rec(sums, sums, nb, sums_scanned, st);
  add_block_offsets_kernel<<<nb, kScanThreads, 0, st>>>(out, sums, n);
}

// total = last input + last exclusive prefix, for one or two scans, gathered
// on the device so that a single read (one host synchronisation) returns them.
__global__ void scan_totals_kernel(const int32_t *in1, const int32_t *out1, const int32_t *in2,
                                   const int32_t *out2, int n, int32_t *dst) {
  dst[0] = in1[n - 1] + out1[n - 1];
  if (in2) dst[1] = in2[n - 1] + out2[n - 1];
}

// tmp[0..1] (kept free by scan_tmp_elems) receive the totals.
csfmm_status exclusive_scan_i32(const int32_t *in, int32_t *out, int n, int32_t *total_host,
                                int32_t *tmp, cudaStream_t st) {
  // in may alias out only if total_host == nullptr (the last input is needed).
  if (n <= 0) {
    if (total_host) *total_host = 0;
    return CSFMM_OK;
  }
  scan_rec(in, out, n, tmp + 2, st);
  CSFMM_CUDA(cudaGetLastError());
  if (total_host) {
    scan_totals_kernel<<<1, 1, 0, st>>>(in, out, nullptr, nullptr, n, tmp);
    CSFMM_CUDA(cudaGetLastError());
    CSFMM_CUDA(cudaMemcpyAsync(total_host, tmp, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CSFMM_CUDA(cudaStreamSynchronize(st));
  }
  return CSFMM_OK;
}

// Two exclusive scans of length n (no aliasing of in and out) and one host read
// of both totals.
static csfmm_status exclusive_scan2_i32(const int32_t *in1, int32_t *out1, const int32_t *in2,
                                        int32_t *out2, int n, int32_t *total1, int32_t *total2,
                                        int32_t *tmp, cudaStream_t st) {
  *total1 = *total2 = 0;
  if (n <= 0) return CSFMM_OK;
  scan_rec(in1, out1, n, tmp + 2, st);
  scan_rec(in2, out2, n, tmp + 2, st);
  CSFMM_CUDA(cudaGetLastError());
  scan_totals_kernel<<<1, 1, 0, st>>>(in1, out1, in2, out2, n, tmp);
  CSFMM_CUDA(cudaGetLastError());
  int32_t t[2] = {0, 0};
  CSFMM_CUDA(cudaMemcpyAsync(t, tmp, sizeof(t), cudaMemcpyDeviceToHost, st));
  CSFMM_CUDA(cudaStreamSynchronize(st));
  *total1 = t[0];
  *total2 = t[1];
  return CSFMM_OK;
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (u64 key, i32 value), 4-bit digits.
// ---------------------------------------------------------------------------
// A block sorts a tile of kSortThreads x ITEMS keys; ITEMS shrinks with n so
// that a pass has at least about two blocks per SM (a 164k-key sort with
// 4096-key tiles ran 40 blocks on a GB300).
constexpr int kSortThreads = 256;
constexpr int kSortMinItems = 2;

static int sort_items(int n) {
  const int64_t kBlocks = 2 * (int64_t)sm_count();
  if (n >= kBlocks * kSortThreads * 16) return 16;
  if (n >= kBlocks * kSortThreads * 8) return 8;
  if (n >= kBlocks * kSortThreads * 4) return 4;
  return kSortMinItems;
}

// Sized for the smallest tile, so that it never decreases with n.
size_t radix_tmp_elems(int n) {
  const int tile = kSortThreads * kSortMinItems;
  int nb = (n + tile - 1) / tile;
  if (nb < 1) nb = 1;
  return (size_t)16 * nb + scan_tmp_elems(16 * nb) + 16;
}

template <int ITEMS>
__global__ void radix_hist_kernel(const uint64_t *keys, int n, int shift, int32_t *hist, int nb) {
  constexpr int kSortTile = kSortThreads * ITEMS;
  __shared__ int cnt[16];
  if (threadIdx.x < 16) cnt[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int k = threadIdx.x; k < kSortTile; k += kSortThreads) {
    int64_t i = base + k;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 15u], 1);
  }
  __syncthreads();
  if (threadIdx.x < 16) hist[threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

template <int kSortItems>
__global__ void radix_scatter_kernel(const uint64_t *keys, const int32_t *vals, uint64_t *okeys,
                                     int32_t *ovals, int n, int shift, const int32_t *offs, int nb) {
  constexpr int kSortTile = kSortThreads * kSortItems;
  __shared__ int tcount[16][kSortThreads + 1];
  int t = threadIdx.x;
  int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)t * kSortItems;
  uint64_t k[kSortItems];
  int32_t v[kSortItems];
  int c[16];
#pragma unroll
  for (int d = 0; d < 16; ++d) c[d] = 0;
#pragma unroll
  for (int q = 0; q < kSortItems; ++q) {
    int64_t i = base + q;
    if (i < n) {
      k[q] = keys[i];
      v[q] = vals[i];
      int d = (int)((k[q] >> shift) & 15u);
#pragma unroll
      for (int e = 0; e < 16; ++e) c[e] += (e == d);
    }
  }
#pragma unroll
  for (int d = 0; d < 16; ++d) tcount[d][t] = c[d];
  __syncthreads();
  // exclusive scan of tcount[d][0..256) for every digit d: warp w takes digits 2w, 2w+1
  {
    int lane = t & 31, w = t >> 5;
    for (int d = 2 * w; d < 2 * w + 2 && d < 16; ++d) {
      int loc[8];
      int s = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        loc[j] = tcount[d][lane * 8 + j];
        s += loc[j];
      }
      int x = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      int pre = x - s;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        tcount[d][lane * 8 + j] = pre;
        pre += loc[j];
      }
    }
  }
  __syncthreads();
  int run[16];
#pragma unroll
  for (int d = 0; d < 16; ++d) run[d] = offs[d * nb + blockIdx.x] + tcount[d][t];
#pragma unroll
  for (int q = 0; q < kSortItems; ++q) {
    int64_t i = base + q;
    if (i < n) {
      int d = (int)((k[q] >> shift) & 15u);
      int pos = 0;
#pragma unroll
      for (int e = 0; e < 16; ++e)
        if (e == d) pos = run[e]++;
      okeys[pos] = k[q];
      ovals[pos] = v[q];
    }
  }
}

csfmm_status radix_sort_u64(uint64_t *keys, int32_t *vals, uint64_t *keys_alt, int32_t *vals_alt,
                            int n, int begin_bit, int end_bit, int32_t *tmp, size_t tmp_elems,
                            cudaStream_t st, bool *result_in_alt) {
  *result_in_alt = false;
  if (n <= 1) return CSFMM_OK;
  const int items = sort_items(n);
  const int nb = (n + kSortThreads * items - 1) / (kSortThreads * items);
  if (tmp_elems < radix_tmp_elems(n)) {
    set_error("radix sort: temporary buffer too small");
    return CSFMM_ERR_INVALID_ARG;
  }
  int32_t *hist = tmp;
  int32_t *scan_tmp = tmp + 16 * (size_t)nb;
  uint64_t *ka = keys, *kb = keys_alt;
  int32_t *va = vals, *vb = vals_alt;
  bool alt = false;
  for (int shift = begin_bit; shift < end_bit; shift += 4) {
    switch (items) {
      case 16: radix_hist_kernel<16><<<nb, kSortThreads, 0, st>>>(ka, n, shift, hist, nb); break;
      case 8: radix_hist_kernel<8><<<nb, kSortThreads, 0, st>>>(ka, n, shift, hist, nb); break;
      case 4: radix_hist_kernel<4><<<nb, kSortThreads, 0, st>>>(ka, n, shift, hist, nb); break;
      default: radix_hist_kernel<2><<<nb, kSortThreads, 0, st>>>(ka, n, shift, hist, nb); break;
    }
    csfmm_status s = exclusive_scan_i32(hist, hist, 16 * nb, nullptr, scan_tmp, st);
    if (s != CSFMM_OK) return s;
    switch (items) {
      case 16:
        radix_scatter_kernel<16><<<nb, kSortThreads, 0, st>>>(ka, va, kb, vb, n, shift, hist, nb);
        break;
      case 8:
        radix_scatter_kernel<8><<<nb, kSortThreads, 0, st>>>(ka, va, kb, vb, n, shift, hist, nb);
        break;
      case 4:
        radix_scatter_kernel<4><<<nb, kSortThreads, 0, st>>>(ka, va, kb, vb, n, shift, hist, nb);
        break;
      default:
        radix_scatter_kernel<2><<<nb, kSortThreads, 0, st>>>(ka, va, kb, vb, n, shift, hist, nb);
        break;
    }
    CSFMM_CUDA(cudaGetLastError());
    std::swap(ka, kb);
    std::swap(va, vb);
    alt = !alt;
  }
  *result_in_alt = alt;
  return CSFMM_OK;
}

// ---------------------------------------------------------------------------
// Step 1: keys.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread18(uint64_t x) {
  uint64_t r = 0;
#pragma unroll
  for (int i = 0; i < kD; ++i) r |= ((x >> i) & 1ull) << (2 * i);
  return r;
}

// Largest k < 2^kD with k == 0 or T[k] <= a.
__device__ __forceinline__ int fine_coord(const double *T, double a) {
  int lo = 0, hi = (1 << kD) - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (T[mid] <= a) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void face_coords_dev(const double *x, int *face, double *a, double *b) {
  int ax = 0;
  double m = fabs(x[0]);
  if (fabs(x[1]) > m) { ax = 1; m = fabs(x[1]); }
  if (fabs(x[2]) > m) { ax = 2; m = fabs(x[2]); }
  int u = ax + 1 == 3 ? 0 : ax + 1;
  int v = u + 1 == 3 ? 0 : u + 1;
  *face = 2 * ax + (x[ax] < 0.0 ? 1 : 0);
  *a = __ddiv_rn(x[u], m);
  *b = __ddiv_rn(x[v], m);
}

__global__ void key_points_kernel(const double *pts, int N, const double *T, uint64_t *keys,
                                  int32_t *idx, int *status) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double x[3] = {pts[3 * (int64_t)i], pts[3 * (int64_t)i + 1], pts[3 * (int64_t)i + 2]};
    double n2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    if (!(fabs(n2 - 1.0) <= 1e-12)) {
      atomicOr(status, kStatusNotOnSphere);
      keys[i] = 0;
      idx[i] = i;
      continue;
    }
    int f;
    double a, b;
    face_coords_dev(x, &f, &a, &b);
    uint64_t qa = (uint64_t)fine_coord(T, a), qb = (uint64_t)fine_coord(T, b);
    keys[i] = ((uint64_t)f << (2 * kD)) | spread18(qa) | (spread18(qb) << 1);
    idx[i] = i;
  }
}

__global__ void permute_points_kernel(const double *pts, const int32_t *perm, double *x, int N) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    int64_t j = perm[i];
    x[i] = pts[3 * j];
    x[N + (int64_t)i] = pts[3 * j + 1];
    x[2 * (int64_t)N + i] = pts[3 * j + 2];
  }
}

// ---------------------------------------------------------------------------
// Step 3: level-synchronous node build.
// ---------------------------------------------------------------------------
struct LevelArrays {
  int32_t *begin = nullptr, *end = nullptr, *face = nullptr, *parent = nullptr;
  int64_t *ia = nullptr, *ib = nullptr;
  int32_t *nchild = nullptr, *first_child = nullptr;  // first_child: scan of nchild
  int32_t *crange = nullptr;                          // [n][4][2] child ranges
  int n = 0;
};

__device__ __forceinline__ int lower_bound_key(const uint64_t *keys, int lo, int hi, uint64_t k) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (keys[mid] < k) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void count_children_kernel(const uint64_t *keys, LevelArrays L, int level, int N0,
                                      int can_split) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  int b = L.begin[c], e = L.end[c];
  int cnt = 0;
  if (can_split && e - b > N0) {
    // key prefix of the cell: face bits, then 2*level Morton bits
    int shift = 2 * (kD - level - 1);  // bit position of the child quadrant digit
    uint64_t prefix = keys[b] >> (shift + 2);
    int pos = b;
    for (int q = 0; q < 4; ++q) {
      uint64_t hi_key = ((prefix << 2) | (uint64_t)(q + 1)) << shift;
      int qend = (q == 3) ? e : lower_bound_key(keys, pos, e, hi_key);
      L.crange[8 * c + 2 * q] = pos;
      L.crange[8 * c + 2 * q + 1] = qend;
      if (qend > pos) ++cnt;
      pos = qend;
    }
  } else {
    for (int q = 0; q < 4; ++q) {
      L.crange[8 * c + 2 * q] = 0;
      L.crange[8 * c + 2 * q + 1] = 0;
    }
  }
  L.nchild[c] = cnt;
}

__global__ void emit_children_kernel(LevelArrays L, LevelArrays C, int parent_base) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  int j = L.first_child[c];
  for (int q = 0; q < 4; ++q) {
    int b = L.crange[8 * c + 2 * q], e = L.crange[8 * c + 2 * q + 1];
    if (e <= b) continue;
    C.begin[j] = b;
    C.end[j] = e;
    C.face[j] = L.face[c];
    C.ia[j] = 2 * L.ia[c] + (q & 1);
    C.ib[j] = 2 * L.ib[c] + (q >> 1);
    C.parent[j] = parent_base + c;
    ++j;
  }
}

// Copies one level into the plan's cell arrays and fills child[4].
__global__ void finalize_level_kernel(LevelArrays L, int base, int child_base, int level,
                                      int32_t *cface, int32_t *clevel, int32_t *cbegin,
                                      int32_t *cend, int32_t *cparent, int32_t *cchild,
                                      int64_t *cia, int64_t *cib) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  int g = base + c;
  cface[g] = L.face[c];
  clevel[g] = level;
  cbegin[g] = L.begin[c];
  cend[g] = L.end[c];
  cparent[g] = L.parent[c];
  cia[g] = L.ia[c];
  cib[g] = L.ib[c];
  int j = child_base + L.first_child[c];
  for (int q = 0; q < 4; ++q) {
    int b = L.crange[8 * c + 2 * q], e = L.crange[8 * c + 2 * q + 1];
    if (L.nchild[c] > 0 && e > b) cchild[4 * g + q] = j++;
    else cchild[4 * g + q] = -1;
  }
}

// ---------------------------------------------------------------------------
// Step 4: geometry, proxies, per-point interpolation data.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t compact18(uint64_t x) {
  uint64_t r = 0;
#pragma unroll
  for (int i = 0; i < kD; ++i) r |= ((x >> (2 * i)) & 1ull) << i;
  return r;
}

// Box of every cell in fine face coordinates, box[c] = (alo, ahi, blo, bhi):
// the dyadic square of (level, ia, ib), or with shrinking the fine cells of
// its points (from the sorted keys) with each edge moved out to an even
// coordinate, so that the midpoint is a tangent-table entry.  One block per
// cell.
__global__ void cell_box_kernel(PlanView v, const uint64_t *keys, const int64_t *cia,
                                const int64_t *cib, int shrink, int64_t *box) {
  const int c = blockIdx.x;
  const int sh = kD - v.clevel[c];
  if (!shrink) {
    if (threadIdx.x == 0) {
      box[4 * c] = cia[c] << sh;
      box[4 * c + 1] = (cia[c] + 1) << sh;
      box[4 * c + 2] = cib[c] << sh;
      box[4 * c + 3] = (cib[c] + 1) << sh;
    }
    return;
  }
  __shared__ int64_t red[4][32];
  int64_t amin = INT64_MAX, amax = -1, bmin = INT64_MAX, bmax = -1;
  const uint64_t mask = (1ull << (2 * kD)) - 1;
  for (int i = v.cbegin[c] + threadIdx.x; i < v.cend[c]; i += blockDim.x) {
    const uint64_t k = keys[i] & mask;
    const int64_t qa = (int64_t)compact18(k), qb = (int64_t)compact18(k >> 1);
    amin = qa < amin ? qa : amin;
    amax = qa > amax ? qa : amax;
    bmin = qb < bmin ? qb : bmin;
    bmax = qb > bmax ? qb : bmax;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    int64_t t;
    t = __shfl_xor_sync(0xffffffffu, amin, o); amin = t < amin ? t : amin;
    t = __shfl_xor_sync(0xffffffffu, amax, o); amax = t > amax ? t : amax;
    t = __shfl_xor_sync(0xffffffffu, bmin, o); bmin = t < bmin ? t : bmin;
    t = __shfl_xor_sync(0xffffffffu, bmax, o); bmax = t > bmax ? t : bmax;
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = amin; red[1][w] = amax; red[2][w] = bmin; red[3][w] = bmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int j = 1; j < nw; ++j) {
      amin = red[0][j] < amin ? red[0][j] : amin;
      amax = red[1][j] > amax ? red[1][j] : amax;
      bmin = red[2][j] < bmin ? red[2][j] : bmin;
      bmax = red[3][j] > bmax ? red[3][j] : bmax;
    }
    box[4 * c] = amin & ~(int64_t)1;
    box[4 * c + 1] = (amax + 2) & ~(int64_t)1;
    box[4 * c + 2] = bmin & ~(int64_t)1;
    box[4 * c + 3] = (bmax + 2) & ~(int64_t)1;
  }
}

// Centre = sphere image of the box midpoint, radius = largest chord to the four
// corners (all tangent-table entries), midpoint angles and half-widths.
__global__ void cell_geometry_kernel(PlanView v, const double *T, double *ccentre, double *cradius,
                                     double *cxmid, double *cymid, double *chalf, double *chy,
                                     const int64_t *box) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= v.ncells) return;
  const double kHalfPi = 1.57079632679489661923;
  const double kQuarterPi = 0.78539816339744830962;
  const int f = v.cface[c];
  const int64_t alo = box[4 * c], ahi = box[4 * c + 1], blo = box[4 * c + 2], bhi = box[4 * c + 3];
  const int64_t amid = (alo + ahi) / 2, bmid = (blo + bhi) / 2;
  double cc[3], corner[3];
  face_point_rn(f, T[amid], T[bmid], cc);
  double r = 0.0, d;
  face_point_rn(f, T[alo], T[blo], corner); d = chord_rn(corner, cc); r = d > r ? d : r;
  face_point_rn(f, T[ahi], T[blo], corner); d = chord_rn(corner, cc); r = d > r ? d : r;
  face_point_rn(f, T[alo], T[bhi], corner); d = chord_rn(corner, cc); r = d > r ? d : r;
  face_point_rn(f, T[ahi], T[bhi], corner); d = chord_rn(corner, cc); r = d > r ? d : r;
  ccentre[3 * c] = cc[0];
  ccentre[3 * c + 1] = cc[1];
  ccentre[3 * c + 2] = cc[2];
  cradius[c] = r;
  const double H = scalbn(kHalfPi, -kD), H2 = scalbn(kHalfPi, -(kD + 1));
  chalf[c] = __dmul_rn((double)(ahi - alo), H2);
  chy[c] = __dmul_rn((double)(bhi - blo), H2);
  cxmid[c] = __dsub_rn(__dmul_rn((double)amid, H), kQuarterPi);
  cymid[c] = __dsub_rn(__dmul_rn((double)bmid, H), kQuarterPi);
}

// Shrunk boxes: for every cell with a parent, parent Lagrange polynomial k at
// the child's node m along each axis, M[c][axis][k][m] = L_k(t_m) with
// t_m = (2 (mid_c - mid_p) + w_c s_m) / w_p from the integer box edges.
__global__ void cell_matrix_kernel(PlanView v, const int64_t *box, double *m64, float *m32) {
  const int c = blockIdx.x;
  const int pa = v.cparent[c];
  if (pa < 0) return;
  const int p = v.p, pp = p * p;
  __shared__ double s[kMaxP];
  if (threadIdx.x < p) s[threadIdx.x] = v.cheb[threadIdx.x];
  __syncthreads();
  for (int t = threadIdx.x; t < 2 * p; t += blockDim.x) {
    const int axis = t / p, m = t - axis * p;
    const int64_t clo = box[4 * c + 2 * axis], chi = box[4 * c + 2 * axis + 1];
    const int64_t plo = box[4 * pa + 2 * axis], phi = box[4 * pa + 2 * axis + 1];
    const double dm = (double)((clo + chi) - (plo + phi));
    const double tm = __ddiv_rn(__dadd_rn(dm, __dmul_rn((double)(chi - clo), s[m])),
                                (double)(phi - plo));
    double L[kMaxP];
    lagrange_dev(v.n, s, tm, L);
    for (int k = 0; k < p; ++k) {
      const int64_t o = (int64_t)c * 2 * pp + axis * pp + k * p + m;
      m64[o] = L[k];
      const float hi = __double2float_rn(L[k]);
      m32[(int64_t)c * 4 * pp + axis * pp + k * p + m] = hi;
      m32[(int64_t)c * 4 * pp + 2 * pp + axis * pp + k * p + m] = __double2float_rn(L[k] - (double)hi);
    }
  }
}

__global__ void proxies_kernel(PlanView v, double *proxy, float *proxy32) {
  int c = blockIdx.x;
  const int P = v.P, p = v.p;
  double cx = v.ccentre[3 * c], cy = v.ccentre[3 * c + 1], cz = v.ccentre[3 * c + 2];
  // the p tangents of each face coordinate, shared by the P = p^2 proxies
  // (blockDim >= 2 p)
  __shared__ double ta[kMaxP], tb[kMaxP];
  if (threadIdx.x < p) ta[threadIdx.x] = tan(v.cxmid[c] + v.chalf[c] * v.cheb[threadIdx.x]);
  else if (threadIdx.x < 2 * p)
    tb[threadIdx.x - p] = tan(v.cymid[c] + v.chy[c] * v.cheb[threadIdx.x - p]);
  __syncthreads();
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    int k1 = k / p, k2 = k - k1 * p;
    const double a = ta[k1], b = tb[k2];
    double x[3];
    face_point_rn(v.cface[c], a, b, x);
    int64_t o = (int64_t)c * 3 * P;
    proxy[o + k] = x[0];
    proxy[o + P + k] = x[1];
    proxy[o + 2 * P + k] = x[2];
    proxy32[o + k] = (float)(x[0] - cx);
    proxy32[o + P + k] = (float)(x[1] - cy);
    proxy32[o + 2 * P + k] = (float)(x[2] - cz);
  }
}

// L_k(u), k = 0..n, at the Chebyshev nodes s (Sec. 4, Eq. barycentric) with
// one division: with d_k = u - s_k and l_k = prod_{j != k} d_j (prefix and
// suffix products), L_k = w_k l_k / sum_j w_j l_j, which equals the
// barycentric form (w_k / d_k) / sum_j (w_j / d_j).  A node u == s_k makes
// every l_j with j != k zero, so L = delta exactly.
__device__ __forceinline__ void lagrange_prod(int n, const double *s, double u, double *L) {
  double d[kMaxP], pre[kMaxP];
  double acc = 1.0;
  for (int k = 0; k <= n; ++k) {
    d[k] = u - s[k];
    pre[k] = acc;
    acc *= d[k];
  }
  double suf = 1.0, den = 0.0;
  for (int k = n; k >= 0; --k) {
    L[k] = bary_w(k, n) * pre[k] * suf;
    suf *= d[k];
    den += L[k];
  }
  const double inv = 1.0 / den;
  for (int k = 0; k <= n; ++k) L[k] *= inv;
}

// FP32 centre difference c_T - c_S of every entry of one list type (one
// thread per target cell T), formed in FP64 and rounded once.  With
// `stochastic` (far-field entries of the 1/|x - y| kernels, Newtonian and SAL)
// it is rounded stochastically with a hash of (T, S, axis): on a uniform grid
// the same cell offsets recur along a face, and rounding them all to nearest
// shifted every far-field interaction of an offset the same way (measured at
// N = 6.3M, n = 12, land-mask weights: a signed bias of -1.8e-8 in the
// Newtonian potential and E = 1.96e-8; -1.1e-8 and 1.4e-8 with stochastic
// rounding).  Stochastic rounding doubles the variance of the rounding error,
// and where that error is random rather than systematic it costs accuracy
// (log and dilogarithm kernels: E of the Poisson Y43 field 1.48e-7 -> 1.86e-7
// at n = 12, of the biharmonic test field 6.4e-8 -> 8.6e-8), so the other
// kernels and the near field keep round-to-nearest.
__global__ void list_centre_diff_kernel(const double *centre, const int32_t *loff,
                                        const int32_t *lsrc, int nc, bool stochastic,
                                        float4 *out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc) return;
  for (int e = loff[t]; e < loff[t + 1]; ++e) {
    const int s = lsrc[e];
    const double dx = centre[3 * t] - centre[3 * s], dy = centre[3 * t + 1] - centre[3 * s + 1],
                 dz = centre[3 * t + 2] - centre[3 * s + 2];
    if (stochastic) {
      const uint32_t h = hash32(((uint32_t)t * 0x9e3779b1u) ^ hash32((uint32_t)s + 0x7f4a7c15u));
      out[e] = make_float4(round_stochastic(dx, hash32(h)), round_stochastic(dy, hash32(h + 1u)),
                           round_stochastic(dz, hash32(h + 2u)), 0.f);
    } else {
      out[e] = make_float4((float)dx, (float)dy, (float)dz, 0.f);
    }
  }
}

// ---------------------------------------------------------------------------
// Double-float arithmetic (value = h + l, |l| <= ulp(h)/2) for the FP32 form's
// Lagrange rows: Knuth's two-sum and FMA-exact products, about 2^-46 relative
// per operation, on the FP32 pipe (GB300's FP64 pipe runs 1/64 of its rate).
// ---------------------------------------------------------------------------
struct DF {
  float h, l;
};
__device__ __forceinline__ DF df_norm(float s, float e) {  // |s| >= |e|
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ DF df_of(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ DF df_sub(DF a, DF b) {
  const float s = __fsub_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fadd_rn(-b.h, -bb));
  e = __fadd_rn(e, __fsub_rn(a.l, b.l));
  return df_norm(s, e);
}
__device__ __forceinline__ DF df_add(DF a, DF b) { return df_sub(a, DF{-b.h, -b.l}); }
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  return df_norm(p, e);
}
__device__ __forceinline__ DF df_scale(DF a, float w) {  // w a power of two times +-1
  return {a.h * w, a.l * w};
}
// 1 / b: FP32 quotient refined by one Newton step on the double-float residual
__device__ __forceinline__ DF df_recip(DF b) {
  const float q = __frcp_rn(b.h);
  const DF r = df_sub(DF{1.f, 0.f}, df_mul(DF{q, 0.f}, b));  // 1 - q b, small
  return df_norm(q, __fmul_rn(r.h, q));
}

// Lagrange rows of the FP32 form in double-float: the product form of
// lagrange_prod with d_k = u - s_k, prefix and suffix products and one
// reciprocal (the weights w_k are +-1 and +-1/2, exact scalings).  The
// FP32 row value is then rounded stochastically from (h, l): away from h
// toward h + l's side with probability |l| / gap, decided by the hash, so the
// expected value is h + l; the remainder is (h - chosen) + l.
__device__ __forceinline__ void lagrange_rows_df(int n, const DF *sd, double u, uint32_t hbase,
                                                 uint32_t hstep, float *hi_out, float *lo_out) {
  DF d[kMaxP], pre[kMaxP];
  const DF ud = df_of(u);
  DF acc{1.f, 0.f};
  for (int k = 0; k <= n; ++k) {
    d[k] = df_sub(ud, sd[k]);
    pre[k] = acc;
    acc = df_mul(acc, d[k]);
  }
  DF L[kMaxP];
  DF suf{1.f, 0.f}, den{0.f, 0.f};
  for (int k = n; k >= 0; --k) {
    const float w = ((k & 1) ? -1.f : 1.f) * ((k == 0 || k == n) ? 0.5f : 1.f);
    L[k] = df_scale(df_mul(pre[k], suf), w);
    suf = df_mul(suf, d[k]);
    den = df_add(den, L[k]);
  }
  const DF inv = df_recip(den);
  for (int k = 0; k <= n; ++k) {
    const DF x = df_mul(L[k], inv);
    float hi = x.h;
    if (x.l != 0.f) {
      const uint32_t hb = (uint32_t)__float_as_int(x.h);
      // the neighbour of h on the side of h + l
      const bool away = (x.l > 0.f) == (x.h > 0.f);
      const float nb = __int_as_float((int)(away ? hb + 1u : hb - 1u));
      const float gap = fabsf(__fsub_rn(nb, x.h));
      const float prob = __fdiv_rn(fabsf(x.l), gap);
      const uint32_t hh = hash32(hbase + hstep * (uint32_t)k);
      if (((float)(hh >> 8) + 0.5f) * 5.9604644775390625e-8f < prob) hi = nb;
    }
    hi_out[k] = hi;
    lo_out[k] = __fadd_rn(__fsub_rn(x.h, hi), x.l);
  }
}

// One block per leaf: leaf id of each point, FP32 offset from the leaf centre and
// the Lagrange values in the leaf's local coordinates (FP64 rows for the FP64
// form; stochastically rounded FP32 rows plus their FP32 remainders for the
// FP32 form, formed in double-float).
__global__ void leaf_points_kernel(PlanView v, const int32_t *leaves, int32_t *leaf_of,
                                   float4 *off32, double *La64, double *Lb64, float *La32,
                                   float *Lb32, float *La32lo, float *Lb32lo) {
  int c = leaves[blockIdx.x];
  int b = v.cbegin[c], e = v.cend[c];
  const int p = v.p, n = v.n;
  __shared__ double s[kMaxP];
  __shared__ DF sd[kMaxP];
  if (threadIdx.x < p) {
    s[threadIdx.x] = v.cheb[threadIdx.x];
    sd[threadIdx.x] = df_of(v.cheb[threadIdx.x]);
  }
  __syncthreads();
  double cx = v.ccentre[3 * c], cy = v.ccentre[3 * c + 1], cz = v.ccentre[3 * c + 2];
  double xm = v.cxmid[c], ym = v.cymid[c], h = v.chalf[c], hy = v.chy[c];
  for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
    double x[3] = {v.x[i], v.x[v.N + i], v.x[2 * v.N + i]};
    leaf_of[i] = c;
    off32[i] = make_float4((float)(x[0] - cx), (float)(x[1] - cy), (float)(x[2] - cz), 0.f);
    double a, bb;
    // the point lies on the leaf's face (same face convention as the keys)
    {
      int ax = 0;
      double m = fabs(x[0]);
      if (fabs(x[1]) > m) { ax = 1; m = fabs(x[1]); }
      if (fabs(x[2]) > m) { ax = 2; m = fabs(x[2]); }
      int uu = ax + 1 == 3 ? 0 : ax + 1;
      int vv = uu + 1 == 3 ? 0 : uu + 1;
      a = x[uu] / m;
      bb = x[vv] / m;
    }
    double u = (atan(a) - xm) / h;
    double w = (atan(bb) - ym) / hy;
    if (La64) {
      double L[kMaxP];
      lagrange_prod(n, s, u, L);
      for (int k = 0; k < p; ++k) La64[(int64_t)i * p + k] = L[k];
      lagrange_prod(n, s, w, L);
      for (int k = 0; k < p; ++k) Lb64[(int64_t)i * p + k] = L[k];
    }
    if (La32) {
      // hashes of (point, axis, node): 2 o and 2 o + 1 for row entry o = i p + k
      const int64_t o0 = (int64_t)i * p;
      lagrange_rows_df(n, sd, u, (uint32_t)(2 * o0), 2u, La32 + o0, La32lo + o0);
      lagrange_rows_df(n, sd, w, (uint32_t)(2 * o0 + 1), 2u, Lb32 + o0, Lb32lo + o0);
    }
  }
}

// M[q][k][m] = L_k((s_m + 2q - 1)/2): parent Lagrange polynomial k at child node m.
__global__ void m2m_matrix_kernel(int n, const double *s, double *m64, float *m32) {
  int p = n + 1;
  int t = threadIdx.x;
  if (t >= 2 * p) return;
  int q = t / p, m = t - q * p;
  double L[kMaxP];
  lagrange_dev(n, s, 0.5 * (s[m] + (double)(2 * q - 1)), L);
  for (int k = 0; k < p; ++k) {
    const float hi = (float)L[k];
    m64[(q * p + k) * p + m] = L[k];
    m32[(q * p + k) * p + m] = hi;                          // FP32 rounding ...
    m32[2 * p * p + (q * p + k) * p + m] = (float)(L[k] - (double)hi);  // ... and remainder
  }
}

// ---------------------------------------------------------------------------
// Step 5: dual traversal.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void atomic_min_pos_double(unsigned long long *addr, double v) {
  // positive doubles order like their bit patterns
  atomicMin(addr, (unsigned long long)__double_as_longlong(v));
}

// outcome: 0..3 list type, 4 split target, 5 split source
__global__ void traverse_step_kernel(PlanView v, double theta, const int2 *frontier, int nf,
                                     int32_t *is_list, int32_t *nkids, int8_t *outcome,
                                     unsigned long long *margin_bits) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf) return;
  int t = frontier[i].x, s = frontier[i].y;
  const double *ct = v.ccentre + 3 * t, *cs = v.ccentre + 3 * s;
  double R = chord_rn(ct, cs);
  double lhs = __dadd_rn(v.cradius[t], v.cradius[s]);
  double rhs = __dmul_rn(theta, R);
  bool sep = lhs < rhs;
  if (R > 0.0) atomic_min_pos_double(margin_bits, fabs(lhs - rhs) / rhs);
  int nct = 0, ncs = 0;
  for (int q = 0; q < 4; ++q) {
    nct += v.cchild[4 * t + q] >= 0;
    ncs += v.cchild[4 * s + q] >= 0;
  }
  bool bigT = nct > 0, bigS = ncs > 0;
  int oc, nk = 0;
  if (sep && (bigT || bigS)) {
    oc = (!bigT && bigS) ? CSFMM_LIST_PC : (bigT && !bigS) ? CSFMM_LIST_CP : CSFMM_LIST_CC;
  } else if (bigT || bigS) {
    bool split_t = (bigT && bigS) ? (v.clevel[t] <= v.clevel[s]) : bigT;
    oc = split_t ? 4 : 5;
    nk = split_t ? nct : ncs;
  } else {
    oc = CSFMM_LIST_PP;
  }
  outcome[i] = (int8_t)oc;
  is_list[i] = oc < 4;
  nkids[i] = nk;
}

__global__ void traverse_emit_kernel(PlanView v, const int2 *frontier, int nf, const int8_t *outcome,
                                     const int32_t *list_off, const int32_t *kid_off, int2 *next,
                                     int3 *accepted, int acc_base) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf) return;
  int t = frontier[i].x, s = frontier[i].y;
  int oc = outcome[i];
  if (oc < 4) {
    accepted[acc_base + list_off[i]] = make_int3(t, s, oc);
  } else {
    int j = kid_off[i];
    for (int q = 0; q < 4; ++q) {
      if (oc == 4) {
        int c = v.cchild[4 * t + q];
        if (c >= 0) next[j++] = make_int2(c, s);
      } else {
        int c = v.cchild[4 * s + q];
        if (c >= 0) next[j++] = make_int2(t, c);
      }
    }
  }
}

__global__ void list_keys_kernel(const int3 *acc, int n, int bits, uint64_t *keys, int32_t *vals) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int3 a = acc[i];
  keys[i] = ((uint64_t)a.z << (2 * bits)) | ((uint64_t)a.x << bits) | (uint64_t)a.y;
  vals[i] = i;
}

// CSR offsets of one list type: off[c] = first entry with target >= c.
__global__ void list_offsets_kernel(const uint64_t *keys, int lo, int hi, int type, int bits,
                                    int ncells, int32_t *off, int32_t *src) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > ncells) return;
  {
    uint64_t k = ((uint64_t)type << (2 * bits)) | ((uint64_t)c << bits);
    int a = lo, b = hi;
    while (a < b) {
      int mid = (a + b) >> 1;
      if (keys[mid] < k) a = mid + 1;
      else b = mid;
    }
    off[c] = a - lo;
  }
  for (int e = lo + c; e < hi; e += (ncells + 1)) {
    src[e - lo] = (int32_t)(keys[e] & ((1ull << bits) - 1));
  }
}

__global__ void collect_leaves_kernel(const int32_t *cchild, int ncells, const int32_t *leaf_rank,
                                      int32_t *leaves) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  bool leaf = cchild[4 * c] < 0 && cchild[4 * c + 1] < 0 && cchild[4 * c + 2] < 0 &&
              cchild[4 * c + 3] < 0;
  if (leaf) leaves[leaf_rank[c]] = c;
}

__global__ void leaf_flags_kernel(const int32_t *cchild, int ncells, int32_t *flag) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  flag[c] = cchild[4 * c] < 0 && cchild[4 * c + 1] < 0 && cchild[4 * c + 2] < 0 &&
            cchild[4 * c + 3] < 0;
}

// ---------------------------------------------------------------------------
// Cross pairs of the symmetric near field.
// ---------------------------------------------------------------------------
// Index of the PP entry (s, c) in s's row (sources sorted), or -1.
__device__ __forceinline__ int mirror_entry(const int32_t *off, const int32_t *src, int s, int c) {
  int lo = off[s], hi = off[s + 1];
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (src[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  return (lo < off[s + 1] && src[lo] == c) ? lo : -1;
}

// The lists are not mirror-symmetric in general (the two traversal orders can
// resolve a region at different levels), so a PP entry (c, s), s > c, is a
// cross pair only if (s, c) is also a PP entry.
__global__ void sym_flag_kernel(const int32_t *off, const int32_t *src, int ncells, int32_t *flag) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  for (int q = off[c]; q < off[c + 1]; ++q) {
    const int s = src[q];
    flag[q] = s > c && mirror_entry(off, src, s, c) >= 0;
  }
}

__global__ void sym_emit_kernel(const int32_t *off, const int32_t *src, int ncells,
                                const int32_t *flag, const int32_t *pidx, const int32_t *cbegin,
                                const int32_t *cend, int2 *pairs, int32_t *sizes) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  for (int q = off[c]; q < off[c + 1]; ++q) {
    if (!flag[q]) continue;
    const int s = src[q];
    pairs[pidx[q]] = make_int2(c, s);
    sizes[pidx[q]] = (cend[c] - cbegin[c]) + (cend[s] - cbegin[s]);
  }
}

// contrib[q] for PP entry q = (c, s): where leaf c's partial sums of this
// interaction start in the partial buffer (rows of pair (c, s) if s > c,
// columns of pair (s, c) if s < c), -1 for the self entry.
__global__ void sym_contrib_kernel(const int32_t *off, const int32_t *src, int ncells,
                                   const int32_t *flag, const int32_t *pidx,
                                   const int32_t *sym_off, const int32_t *cbegin,
                                   const int32_t *cend, int32_t *contrib) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  for (int q = off[c]; q < off[c + 1]; ++q) {
    const int s = src[q];
    int val = -1;  // evaluated directly by the near-field kernel
    if (s > c) {
      if (flag[q]) val = sym_off[pidx[q]];
    } else if (s < c) {
      const int m = mirror_entry(off, src, s, c);
      if (m >= 0 && flag[m]) val = sym_off[pidx[m]] + (cend[s] - cbegin[s]);
    }
    contrib[q] = val;
  }
}

// Mirrored CC pairs (T, S), T < S: the pair and the index of its CC entry.
__global__ void cc_pair_emit_kernel(const int32_t *off, const int32_t *src, int ncells,
                                    const int32_t *flag, const int32_t *pidx, int2 *pairs,
                                    int32_t *entry) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  for (int q = off[c]; q < off[c + 1]; ++q) {
    if (!flag[q]) continue;
    pairs[pidx[q]] = make_int2(c, src[q]);
    entry[pidx[q]] = q;
  }
}

// contrib[q] for CC entry q = (c, s): where cell c's proxy sums of this entry
// start in the pair partials (2 P per pair: the rows, i.e. the proxies of
// the lower cell, then the columns), -1 if the entry has no mirror.
__global__ void cc_contrib_kernel(const int32_t *off, const int32_t *src, int ncells,
                                  const int32_t *flag, const int32_t *pidx, int P,
                                  int32_t *contrib) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  for (int q = off[c]; q < off[c + 1]; ++q) {
    const int s = src[q];
    int val = -1;
    if (s > c) {
      if (flag[q]) val = 2 * P * pidx[q];
    } else {
      const int m = mirror_entry(off, src, s, c);
      if (m >= 0 && flag[m]) val = 2 * P * pidx[m] + P;
    }
    contrib[q] = val;
  }
}

// ---------------------------------------------------------------------------
// Host driver.
// ---------------------------------------------------------------------------
namespace {

// Temporary device buffers of the build, freed in stream order on every
// return path.
struct TempArena {
  std::vector<void *> ptrs;
  cudaStream_t stream;
  explicit TempArena(cudaStream_t s) : stream(s) {}
  ~TempArena() {
    for (void *p : ptrs) cudaFreeAsync(p, stream);
  }
  template <class T>
  csfmm_status alloc(T **p, size_t count) {
    if (count == 0) count = 1;
    void *q = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&q, count * sizeof(T), memory_pool(), stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("device allocation of %zu bytes failed during plan build", count * sizeof(T));
      return CSFMM_ERR_OUT_OF_MEMORY;
    }
    ptrs.push_back(q);
    *p = (T *)q;
    return CSFMM_OK;
  }
};

#define CSFMM_TRY(expr)                      \
  do {                                       \
    csfmm_status s__ = (expr);               \
    if (s__ != CSFMM_OK) return s__;         \
  } while (0)

csfmm_status alloc_level(TempArena &tmp, LevelArrays &L, int n) {
  L.n = n;
  CSFMM_TRY(tmp.alloc(&L.begin, n));
  CSFMM_TRY(tmp.alloc(&L.end, n));
  CSFMM_TRY(tmp.alloc(&L.face, n));
  CSFMM_TRY(tmp.alloc(&L.parent, n));
  CSFMM_TRY(tmp.alloc(&L.ia, n));
  CSFMM_TRY(tmp.alloc(&L.ib, n));
  CSFMM_TRY(tmp.alloc(&L.nchild, n));
  CSFMM_TRY(tmp.alloc(&L.first_child, n));
  CSFMM_TRY(tmp.alloc(&L.crange, (size_t)8 * n));
  return CSFMM_OK;
}

}  // namespace

PlanView Plan::view() const {
  PlanView v{};
  v.N = (int)N; v.n = n; v.p = p; v.P = P; v.N0 = N0; v.ncells = ncells; v.dim = dim;
  v.kernel_id = kernel_id;
  v.nsrc = (int)nsrc; v.ntgt = (int)ntgt; v.tbase = (int)tbase;
  v.x = x; v.perm = perm; v.La64 = La64; v.Lb64 = Lb64; v.La32 = La32; v.Lb32 = Lb32;
  v.La32lo = La32lo; v.Lb32lo = Lb32lo;
  v.off32 = off32;
  v.cbegin = cbegin; v.cend = cend; v.clevel = clevel; v.cface = cface; v.cparent = cparent;
  v.cchild = cchild; v.ccentre = ccentre; v.cradius = cradius; v.cxmid = cxmid; v.cymid = cymid;
  v.chalf = chalf; v.chy = chy; v.proxy = proxy; v.proxy32 = proxy32;
  v.mcell64 = mcell64; v.mcell32 = mcell32;
  for (int t = 0; t < 4; ++t) { v.loff[t] = loff[t]; v.lsrc[t] = lsrc[t]; v.ldc[t] = ldc[t]; }
  v.sym_contrib = sym_contrib;
  v.cc_contrib = cc_contrib;
  v.m2m64 = m2m64; v.m2m32 = m2m32; v.cheb = cheb; v.status = status;
  v.wtot = nullptr; v.wtot_ld = 0;
  return v;
}

// First index of each of nb boundary keys in the sorted keys[0..n):
// out[b] = lower_bound(keys, bound_b), bound_b = b << shift.  One thread per
// boundary (a handful of binary searches instead of copying the keys back).
__global__ void key_bounds_kernel(const uint64_t *keys, int n, int nb, int shift, int32_t *out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const uint64_t k = (uint64_t)b << shift;
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (keys[mid] < k) lo = mid + 1;
    else hi = mid;
  }
  out[b] = lo;
}

// Plan statistics from the sorted list keys (type, target, source): kernel
// evaluations per list type and the number of (target, source) point pairs
// covered; 64-bit integer atomics, so the totals do not depend on the order.
__global__ void list_stats_kernel(const uint64_t *lk, int n, int bits, const int32_t *cbegin,
                                  const int32_t *cend, int P, unsigned long long *acc) {
  unsigned long long ev[4] = {0, 0, 0, 0}, cov = 0;
  const uint64_t mask = (1ull << bits) - 1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const uint64_t k = lk[e];
    const int ty = (int)(k >> (2 * bits));
    const int t = (int)((k >> bits) & mask), s = (int)(k & mask);
    const unsigned long long nt = (unsigned long long)(cend[t] - cbegin[t]);
    const unsigned long long ns = (unsigned long long)(cend[s] - cbegin[s]);
    cov += nt * ns;
    if (ty == CSFMM_LIST_PP) ev[0] += nt * ns - (t == s ? nt : 0);
    else if (ty == CSFMM_LIST_PC) ev[1] += nt * (unsigned long long)P;
    else if (ty == CSFMM_LIST_CP) ev[2] += (unsigned long long)P * ns;
    else ev[3] += (unsigned long long)P * (unsigned long long)P;
  }
  for (int q = 0; q < 4; ++q)
    if (ev[q]) atomicAdd(&acc[q], ev[q]);
  if (cov) atomicAdd(&acc[4], cov);
}

// Kernel evaluations of the symmetric near field's cross pairs.
__global__ void sym_stats_kernel(const int2 *pairs, int n, const int32_t *cbegin,
                                 const int32_t *cend, unsigned long long *acc) {
  unsigned long long se = 0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int2 q = pairs[e];
    se += (unsigned long long)(cend[q.x] - cbegin[q.x]) * (unsigned long long)(cend[q.y] - cbegin[q.y]);
  }
  if (se) atomicAdd(acc, se);
}

csfmm_status build_tree(Plan &pl, const double *points, cudaStream_t st) {
  const int N = (int)pl.N;
  TempArena tmp(st);
  DeviceArena &A = pl.arena;
  A.stream = st;

  // tangent table (resident on the device) and Chebyshev nodes
  const double *T = device_tan_table();
  if (!T) return CSFMM_ERR_CUDA;
  std::vector<double> cheb_h(pl.p);
  for (int k = 0; k <= pl.n; ++k) cheb_h[k] = cos((double)k * 3.14159265358979323846 / pl.n);
  CSFMM_TRY(A.alloc(&pl.cheb, pl.p));
  CSFMM_CUDA(cudaMemcpyAsync(pl.cheb, cheb_h.data(), sizeof(double) * pl.p, cudaMemcpyHostToDevice, st));
  CSFMM_TRY(A.alloc(&pl.status, 4));
  CSFMM_CUDA(cudaMemsetAsync(pl.status, 0, 4 * sizeof(int), st));

  // 1-2. keys and sort
  uint64_t *keys, *keys2;
  int32_t *idx, *idx2;
  CSFMM_TRY(tmp.alloc(&keys, N));
  CSFMM_TRY(tmp.alloc(&keys2, N));
  CSFMM_TRY(tmp.alloc(&idx, N));
  CSFMM_TRY(tmp.alloc(&idx2, N));
  size_t rtmp_n = radix_tmp_elems(N);
  int32_t *rtmp;
  CSFMM_TRY(tmp.alloc(&rtmp, rtmp_n));
  key_points_kernel<<<grid_for(N, 256, sm_count() * 64), 256, 0, st>>>(points, N, T, keys, idx, pl.status);
  CSFMM_CUDA(cudaGetLastError());
  // (the status word is read with the face bounds below: a point off the sphere
  // has key 0 and sorts like any other)
  bool in_alt = false;
  CSFMM_TRY(radix_sort_u64(keys, idx, keys2, idx2, N, 0, 2 * kD + 4, rtmp, rtmp_n, st, &in_alt));
  if (in_alt) {
    std::swap(keys, keys2);
    std::swap(idx, idx2);
  }
  CSFMM_TRY(A.alloc(&pl.perm, N));
  CSFMM_CUDA(cudaMemcpyAsync(pl.perm, idx, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, st));
  CSFMM_TRY(A.alloc(&pl.x, (size_t)3 * N));
  permute_points_kernel<<<grid_for(N, 256, sm_count() * 64), 256, 0, st>>>(points, pl.perm, pl.x, N);
  CSFMM_CUDA(cudaGetLastError());

  // 3. roots: non-empty faces, found from the sorted keys on the host side
  std::vector<int> root_begin, root_end, root_face;
  {
    // face boundaries: binary searches of the sorted keys on the device
    int32_t *fb;
    CSFMM_TRY(tmp.alloc(&fb, 8));
    key_bounds_kernel<<<1, 32, 0, st>>>(keys, N, 7, 2 * kD, fb);
    CSFMM_CUDA(cudaGetLastError());
    CSFMM_CUDA(cudaMemcpyAsync(fb + 7, pl.status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    int32_t hb7[8];
    CSFMM_CUDA(cudaMemcpyAsync(hb7, fb, sizeof(hb7), cudaMemcpyDeviceToHost, st));
    CSFMM_CUDA(cudaStreamSynchronize(st));
    if (hb7[7] & kStatusNotOnSphere) {
      set_error("a point is not on the unit sphere (| |x|^2 - 1 | > 1e-12) or is not finite");
      return CSFMM_ERR_NOT_ON_SPHERE;
    }
    for (int f = 0; f < 6; ++f) {
      const int b = hb7[f], e = hb7[f + 1];
      if (e > b) {
        root_begin.push_back(b);
        root_end.push_back(e);
        root_face.push_back(f);
      }
    }
  }
  std::vector<LevelArrays> levels;
  std::vector<int> level_base;
  {
    LevelArrays L0;
    int n0 = (int)root_begin.size();
    CSFMM_TRY(alloc_level(tmp, L0, n0));
    std::vector<int32_t> par(n0, -1);
    std::vector<int64_t> zero(n0, 0);
    CSFMM_CUDA(cudaMemcpyAsync(L0.begin, root_begin.data(), 4 * n0, cudaMemcpyHostToDevice, st));
    CSFMM_CUDA(cudaMemcpyAsync(L0.end, root_end.data(), 4 * n0, cudaMemcpyHostToDevice, st));
    CSFMM_CUDA(cudaMemcpyAsync(L0.face, root_face.data(), 4 * n0, cudaMemcpyHostToDevice, st));
    CSFMM_CUDA(cudaMemcpyAsync(L0.parent, par.data(), 4 * n0, cudaMemcpyHostToDevice, st));
    CSFMM_CUDA(cudaMemcpyAsync(L0.ia, zero.data(), 8 * n0, cudaMemcpyHostToDevice, st));
    CSFMM_CUDA(cudaMemcpyAsync(L0.ib, zero.data(), 8 * n0, cudaMemcpyHostToDevice, st));
    CSFMM_CUDA(cudaStreamSynchronize(st));  // host vectors above go out of scope
    levels.push_back(L0);
    level_base.push_back(0);
  }
  int total_cells = levels[0].n;
  int32_t *scan_tmp = nullptr;
  size_t scan_tmp_cap = 0;
  for (int l = 0;; ++l) {
    LevelArrays &L = levels[l];
    count_children_kernel<<<grid_for(L.n, 128), 128, 0, st>>>(keys, L, l, pl.N0, l < kLMax);
    CSFMM_CUDA(cudaGetLastError());
    size_t need = scan_tmp_elems(L.n);
    if (need > scan_tmp_cap) {
      CSFMM_TRY(tmp.alloc(&scan_tmp, need));
      scan_tmp_cap = need;
    }
    int32_t nnext = 0;
    CSFMM_TRY(exclusive_scan_i32(L.nchild, L.first_child, L.n, &nnext, scan_tmp, st));
    if (nnext == 0) break;
    LevelArrays C;
    CSFMM_TRY(alloc_level(tmp, C, nnext));
    emit_children_kernel<<<grid_for(L.n, 128), 128, 0, st>>>(L, C, level_base[l]);
    CSFMM_CUDA(cudaGetLastError());
    level_base.push_back(total_cells);
    total_cells += nnext;
    levels.push_back(C);
  }
  pl.nlevels = (int)levels.size();
  pl.ncells = total_cells;
  pl.level_begin.assign(level_base.begin(), level_base.end());
  pl.level_begin.push_back(total_cells);
  const int nc = total_cells;
  CSFMM_TRY(A.alloc(&pl.cface, nc));
  CSFMM_TRY(A.alloc(&pl.clevel, nc));
  CSFMM_TRY(A.alloc(&pl.cbegin, nc));
  CSFMM_TRY(A.alloc(&pl.cend, nc));
  CSFMM_TRY(A.alloc(&pl.cparent, nc));
  CSFMM_TRY(A.alloc(&pl.cchild, (size_t)4 * nc));
  CSFMM_TRY(A.alloc(&pl.cia, nc));
  CSFMM_TRY(A.alloc(&pl.cib, nc));
  for (int l = 0; l < pl.nlevels; ++l) {
    int child_base = l + 1 < pl.nlevels ? level_base[l + 1] : 0;
    finalize_level_kernel<<<grid_for(levels[l].n, 128), 128, 0, st>>>(
        levels[l], level_base[l], child_base, l, pl.cface, pl.clevel, pl.cbegin, pl.cend,
        pl.cparent, pl.cchild, pl.cia, pl.cib);
    CSFMM_CUDA(cudaGetLastError());
  }

  // leaves in cell order
  int32_t *flag, *rank;
  CSFMM_TRY(tmp.alloc(&flag, nc));
  CSFMM_TRY(tmp.alloc(&rank, nc));
  leaf_flags_kernel<<<grid_for(nc, 128), 128, 0, st>>>(pl.cchild, nc, flag);
  size_t need = scan_tmp_elems(nc);
  if (need > scan_tmp_cap) {
    CSFMM_TRY(tmp.alloc(&scan_tmp, need));
    scan_tmp_cap = need;
  }
  int32_t nleaves = 0;
  CSFMM_TRY(exclusive_scan_i32(flag, rank, nc, &nleaves, scan_tmp, st));
  pl.nleaves = nleaves;
  CSFMM_TRY(A.alloc(&pl.leaves, nleaves));
  collect_leaves_kernel<<<grid_for(nc, 128), 128, 0, st>>>(pl.cchild, nc, rank, pl.leaves);
  CSFMM_CUDA(cudaGetLastError());

  // 4. geometry, proxies, interpolation data
  CSFMM_TRY(A.alloc(&pl.ccentre, (size_t)3 * nc));
  CSFMM_TRY(A.alloc(&pl.cradius, nc));
  CSFMM_TRY(A.alloc(&pl.cxmid, nc));
  CSFMM_TRY(A.alloc(&pl.cymid, nc));
  CSFMM_TRY(A.alloc(&pl.chalf, nc));
  CSFMM_TRY(A.alloc(&pl.chy, nc));
  int64_t *cbox;
  CSFMM_TRY(tmp.alloc(&cbox, (size_t)4 * nc));
  {
    PlanView v = pl.view();
    cell_box_kernel<<<nc, 256, 0, st>>>(v, keys, pl.cia, pl.cib, pl.shrink, cbox);
    CSFMM_CUDA(cudaGetLastError());
    cell_geometry_kernel<<<grid_for(nc, 128), 128, 0, st>>>(v, T, pl.ccentre, pl.cradius, pl.cxmid,
                                                            pl.cymid, pl.chalf, pl.chy, cbox);
    CSFMM_CUDA(cudaGetLastError());
  }
  CSFMM_TRY(A.alloc(&pl.proxy, (size_t)3 * nc * pl.P));
  CSFMM_TRY(A.alloc(&pl.proxy32, (size_t)3 * nc * pl.P));
  CSFMM_TRY(A.alloc(&pl.leaf_of, N));
  CSFMM_TRY(A.alloc(&pl.off32, N));
  if (pl.precision == CSFMM_FP64) {
    CSFMM_TRY(A.alloc(&pl.La64, (size_t)N * pl.p));
    CSFMM_TRY(A.alloc(&pl.Lb64, (size_t)N * pl.p));
  } else {
    CSFMM_TRY(A.alloc(&pl.La32, (size_t)N * pl.p));
    CSFMM_TRY(A.alloc(&pl.Lb32, (size_t)N * pl.p));
    CSFMM_TRY(A.alloc(&pl.La32lo, (size_t)N * pl.p));
    CSFMM_TRY(A.alloc(&pl.Lb32lo, (size_t)N * pl.p));
  }
  CSFMM_TRY(A.alloc(&pl.m2m64, (size_t)2 * pl.p * pl.p));
  CSFMM_TRY(A.alloc(&pl.m2m32, (size_t)4 * pl.p * pl.p));
  {
    PlanView v = pl.view();
    proxies_kernel<<<nc, 128, 0, st>>>(v, pl.proxy, pl.proxy32);
    CSFMM_CUDA(cudaGetLastError());
    leaf_points_kernel<<<nleaves, 128, 0, st>>>(v, pl.leaves, pl.leaf_of, pl.off32, pl.La64,
                                                pl.Lb64, pl.La32, pl.Lb32, pl.La32lo, pl.Lb32lo);
    CSFMM_CUDA(cudaGetLastError());
    m2m_matrix_kernel<<<1, 64, 0, st>>>(pl.n, pl.cheb, pl.m2m64, pl.m2m32);
    CSFMM_CUDA(cudaGetLastError());
  }
  if (pl.shrink) {
    CSFMM_TRY(A.alloc(&pl.mcell64, (size_t)2 * nc * pl.p * pl.p));
    CSFMM_TRY(A.alloc(&pl.mcell32, (size_t)4 * nc * pl.p * pl.p));
    PlanView v = pl.view();
    cell_matrix_kernel<<<nc, 64, 0, st>>>(v, cbox, pl.mcell64, pl.mcell32);
    CSFMM_CUDA(cudaGetLastError());
  }

  // 5. traversal
  unsigned long long *margin_bits;
  CSFMM_TRY(tmp.alloc(&margin_bits, 1));
  {
    unsigned long long inf_bits = 0x7ff0000000000000ull;
    CSFMM_CUDA(cudaMemcpyAsync(margin_bits, &inf_bits, 8, cudaMemcpyHostToDevice, st));
  }
  int nroots = levels[0].n;
  int nf = nroots * nroots;
  int2 *frontier;
  int fcap = std::max(nf, 1024);
  CSFMM_TRY(tmp.alloc(&frontier, fcap));
  {
    std::vector<int2> f0;
    for (int t = 0; t < nroots; ++t)
      for (int s = 0; s < nroots; ++s) f0.push_back(make_int2(t, s));
    CSFMM_CUDA(cudaMemcpyAsync(frontier, f0.data(), sizeof(int2) * nf, cudaMemcpyHostToDevice, st));
    CSFMM_CUDA(cudaStreamSynchronize(st));
  }
  int3 *accepted = nullptr;
  int acc_n = 0, acc_cap = 0;
  PlanView v = pl.view();
  while (nf > 0) {
    int32_t *is_list, *nkids, *loffs, *koffs;
    int8_t *outcome;
    int2 *next;
    CSFMM_TRY(tmp.alloc(&is_list, nf));
    CSFMM_TRY(tmp.alloc(&nkids, nf));
    CSFMM_TRY(tmp.alloc(&loffs, nf));
    CSFMM_TRY(tmp.alloc(&koffs, nf));
    CSFMM_TRY(tmp.alloc(&outcome, nf));
    traverse_step_kernel<<<grid_for(nf, 256), 256, 0, st>>>(v, pl.theta, frontier, nf, is_list,
                                                            nkids, outcome, margin_bits);
    CSFMM_CUDA(cudaGetLastError());
    need = scan_tmp_elems(nf);
    if (need > scan_tmp_cap) {
      CSFMM_TRY(tmp.alloc(&scan_tmp, need));
      scan_tmp_cap = need;
    }
    int32_t nacc = 0, nnext = 0;
    CSFMM_TRY(exclusive_scan2_i32(is_list, loffs, nkids, koffs, nf, &nacc, &nnext, scan_tmp, st));
    if (acc_n + nacc > acc_cap) {
      int ncap = std::max(2 * acc_cap, acc_n + nacc + 1024);
      int3 *na;
      CSFMM_TRY(tmp.alloc(&na, ncap));
      if (acc_n) CSFMM_CUDA(cudaMemcpyAsync(na, accepted, sizeof(int3) * acc_n, cudaMemcpyDeviceToDevice, st));
      accepted = na;
      acc_cap = ncap;
    }
    CSFMM_TRY(tmp.alloc(&next, std::max(nnext, 1)));
    traverse_emit_kernel<<<grid_for(nf, 256), 256, 0, st>>>(v, frontier, nf, outcome, loffs, koffs,
                                                            next, accepted, acc_n);
    CSFMM_CUDA(cudaGetLastError());
    acc_n += nacc;
    frontier = next;
    nf = nnext;
  }

  // 6. lists: sort by (type, target, source), CSR per type
  int bits = 1;
  while ((1 << bits) <= nc) ++bits;
  uint64_t *lk, *lk2;
  int32_t *lv, *lv2;
  int nacc_all = std::max(acc_n, 1);
  CSFMM_TRY(tmp.alloc(&lk, nacc_all));
  CSFMM_TRY(tmp.alloc(&lk2, nacc_all));
  CSFMM_TRY(tmp.alloc(&lv, nacc_all));
  CSFMM_TRY(tmp.alloc(&lv2, nacc_all));
  if (acc_n > 0) {
    list_keys_kernel<<<grid_for(acc_n, 256), 256, 0, st>>>(accepted, acc_n, bits, lk, lv);
    CSFMM_CUDA(cudaGetLastError());
    size_t rt = radix_tmp_elems(acc_n);
    int32_t *rt_buf;
    CSFMM_TRY(tmp.alloc(&rt_buf, rt));
    int endbit = 2 * bits + 2;
    endbit = (endbit + 3) & ~3;
    CSFMM_TRY(radix_sort_u64(lk, lv, lk2, lv2, acc_n, 0, endbit, rt_buf, rt, st, &in_alt));
    if (in_alt) {
      std::swap(lk, lk2);
      std::swap(lv, lv2);
    }
  }
  int type_lo[5] = {0, 0, 0, 0, 0};
  {
    // first entry of each list type (binary searches on the device) and the
    // traversal's MAC margin, in one read: tb[0..5) and the 8 bytes at tb + 6
    int32_t *tb;
    CSFMM_TRY(tmp.alloc(&tb, 8));
    CSFMM_CUDA(cudaMemsetAsync(tb, 0, 5 * sizeof(int32_t), st));
    if (acc_n) {
      key_bounds_kernel<<<1, 32, 0, st>>>(lk, acc_n, 5, 2 * bits, tb);
      CSFMM_CUDA(cudaGetLastError());
    }
    CSFMM_CUDA(cudaMemcpyAsync(tb + 6, margin_bits, 8, cudaMemcpyDeviceToDevice, st));
    int32_t h8[8];
    CSFMM_CUDA(cudaMemcpyAsync(h8, tb, sizeof(h8), cudaMemcpyDeviceToHost, st));
    CSFMM_CUDA(cudaStreamSynchronize(st));
    for (int t = 0; t < 5; ++t) type_lo[t] = h8[t];
    double m;
    memcpy(&m, h8 + 6, 8);
    pl.stats.mac_margin = m;
  }
  for (int ty = 0; ty < 4; ++ty) {
    int lo = type_lo[ty], hi = type_lo[ty + 1];
    pl.nlist[ty] = hi - lo;
    CSFMM_TRY(A.alloc(&pl.loff[ty], (size_t)nc + 1));
    CSFMM_TRY(A.alloc(&pl.lsrc[ty], (size_t)std::max(hi - lo, 1)));
    list_offsets_kernel<<<grid_for(nc + 1, 128), 128, 0, st>>>(lk, lo, hi, ty, bits, nc,
                                                                pl.loff[ty], pl.lsrc[ty]);
    CSFMM_CUDA(cudaGetLastError());
  }

  // FP32 form: the centre difference of every list entry, rounded once
  if (pl.precision == CSFMM_FP32_BULK) {
    for (int ty = 0; ty < 4; ++ty) {
      CSFMM_TRY(A.alloc(&pl.ldc[ty], (size_t)std::max<int64_t>(pl.nlist[ty], 1)));
      list_centre_diff_kernel<<<grid_for(nc, 128), 128, 0, st>>>(
          pl.ccentre, pl.loff[ty], pl.lsrc[ty], nc,
          (ty == CSFMM_LIST_CP || ty == CSFMM_LIST_CC) &&
              (pl.kernel_id == CSFMM_KERNEL_NEWTON || pl.kernel_id == CSFMM_KERNEL_SAL),
          pl.ldc[ty]);
      CSFMM_CUDA(cudaGetLastError());
    }
  }

  // symmetric near field: cross pairs of the PP lists (FP32 form)
  if (pl.precision == CSFMM_FP32_BULK && pl.nlist[CSFMM_LIST_PP] > 0) {
    const int npp = (int)pl.nlist[CSFMM_LIST_PP];
    int32_t *flag, *pidx, *sizes;
    CSFMM_TRY(tmp.alloc(&flag, npp));
    CSFMM_TRY(tmp.alloc(&pidx, npp));
    sym_flag_kernel<<<grid_for(nc, 128), 128, 0, st>>>(pl.loff[CSFMM_LIST_PP],
                                                        pl.lsrc[CSFMM_LIST_PP], nc, flag);
    CSFMM_CUDA(cudaGetLastError());
    need = scan_tmp_elems(npp);
    if (need > scan_tmp_cap) {
      CSFMM_TRY(tmp.alloc(&scan_tmp, need));
      scan_tmp_cap = need;
    }
    int32_t npairs = 0;
    CSFMM_TRY(exclusive_scan_i32(flag, pidx, npp, &npairs, scan_tmp, st));
    if (npairs > 0) {
      CSFMM_TRY(A.alloc(&pl.sym_pairs, npairs));
      CSFMM_TRY(A.alloc(&pl.sym_off, npairs));
      CSFMM_TRY(tmp.alloc(&sizes, npairs));
      sym_emit_kernel<<<grid_for(nc, 128), 128, 0, st>>>(pl.loff[CSFMM_LIST_PP],
                                                          pl.lsrc[CSFMM_LIST_PP], nc, flag, pidx,
                                                          pl.cbegin, pl.cend, pl.sym_pairs, sizes);
      CSFMM_CUDA(cudaGetLastError());
      need = scan_tmp_elems(npairs);
      if (need > scan_tmp_cap) {
        CSFMM_TRY(tmp.alloc(&scan_tmp, need));
        scan_tmp_cap = need;
      }
      // sizes sum to < 2^31 floats: each point appears once per PP partner
      int32_t part_len = 0;
      CSFMM_TRY(exclusive_scan_i32(sizes, pl.sym_off, npairs, &part_len, scan_tmp, st));
      CSFMM_TRY(A.alloc(&pl.sym_contrib, npp));
      sym_contrib_kernel<<<grid_for(nc, 128), 128, 0, st>>>(pl.loff[CSFMM_LIST_PP],
                                                             pl.lsrc[CSFMM_LIST_PP], nc, flag,
                                                             pidx, pl.sym_off, pl.cbegin, pl.cend,
                                                             pl.sym_contrib);
      CSFMM_CUDA(cudaGetLastError());
      pl.n_sym_pairs = npairs;
      pl.sym_part_len = part_len;
    }
  }

  // symmetric far field: mirrored CC pairs (FP32 form, scalar kernels); the
  // partial offsets are int32, so a plan with 2 P npairs >= 2^31 keeps the
  // direct evaluation
  if (pl.precision == CSFMM_FP32_BULK && pl.kernel_id != CSFMM_KERNEL_BIOT_SAVART &&
      pl.nlist[CSFMM_LIST_CC] > 0) {
    const int ncc = (int)pl.nlist[CSFMM_LIST_CC];
    int32_t *flag, *pidx;
    CSFMM_TRY(tmp.alloc(&flag, ncc));
    CSFMM_TRY(tmp.alloc(&pidx, ncc));
    sym_flag_kernel<<<grid_for(nc, 128), 128, 0, st>>>(pl.loff[CSFMM_LIST_CC],
                                                        pl.lsrc[CSFMM_LIST_CC], nc, flag);
    CSFMM_CUDA(cudaGetLastError());
    need = scan_tmp_elems(ncc);
    if (need > scan_tmp_cap) {
      CSFMM_TRY(tmp.alloc(&scan_tmp, need));
      scan_tmp_cap = need;
    }
    int32_t npairs = 0;
    CSFMM_TRY(exclusive_scan_i32(flag, pidx, ncc, &npairs, scan_tmp, st));
    if (npairs > 0 && (int64_t)2 * pl.P * npairs < ((int64_t)1 << 31)) {
      CSFMM_TRY(A.alloc(&pl.cc_pairs, npairs));
      CSFMM_TRY(A.alloc(&pl.cc_entry, npairs));
      CSFMM_TRY(A.alloc(&pl.cc_contrib, ncc));
      cc_pair_emit_kernel<<<grid_for(nc, 128), 128, 0, st>>>(pl.loff[CSFMM_LIST_CC],
                                                              pl.lsrc[CSFMM_LIST_CC], nc, flag,
                                                              pidx, pl.cc_pairs, pl.cc_entry);
      CSFMM_CUDA(cudaGetLastError());
      cc_contrib_kernel<<<grid_for(nc, 128), 128, 0, st>>>(pl.loff[CSFMM_LIST_CC],
                                                            pl.lsrc[CSFMM_LIST_CC], nc, flag,
                                                            pidx, pl.P, pl.cc_contrib);
      CSFMM_CUDA(cudaGetLastError());
      pl.n_cc_pairs = npairs;
      pl.stats.cc_sym_pairs = npairs;
    }
  }

  // statistics: reductions over the lists and symmetric pairs on the device
  {
    unsigned long long *acc;
    CSFMM_TRY(tmp.alloc(&acc, 6));
    CSFMM_CUDA(cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 6, st));
    if (acc_n > 0) {
      list_stats_kernel<<<grid_for(acc_n, 256, sm_count() * 8), 256, 0, st>>>(lk, acc_n, bits, pl.cbegin,
                                                                      pl.cend, pl.P, acc);
      CSFMM_CUDA(cudaGetLastError());
    }
    if (pl.n_sym_pairs > 0) {
      sym_stats_kernel<<<grid_for(pl.n_sym_pairs, 256, sm_count() * 8), 256, 0, st>>>(
          pl.sym_pairs, (int)pl.n_sym_pairs, pl.cbegin, pl.cend, acc + 5);
      CSFMM_CUDA(cudaGetLastError());
    }
    unsigned long long h[6];
    CSFMM_CUDA(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st));
    CSFMM_CUDA(cudaStreamSynchronize(st));
    for (int t = 0; t < 4; ++t) {
      pl.stats.evals[t] = (int64_t)h[t];
      pl.stats.n_list[t] = pl.nlist[t];
    }
    pl.stats.pairs_covered = (int64_t)h[4];
    if (pl.n_sym_pairs > 0) {
      pl.stats.sym_pairs = pl.n_sym_pairs;
      pl.stats.sym_evals = (int64_t)h[5];
    }
  }
  CSFMM_CUDA(cudaStreamSynchronize(st));
  return CSFMM_OK;
}

}  // namespace csfmm
