// remesh.cu -- remeshing of the vortex method for the barotropic vorticity
// equation onto a fixed grid (Sec. 12 remeshes at every time step by local
// interpolation), and the remeshed RK4 step.
//
// After a step the particles return to the grid points g_k, which keep their
// areas, and the value at g_k of each carried field is that of a local
// quadratic fitted to the moved particles near g_k.  With h_k the chord from
// g_k to its nearest neighbour, e1, e2 orthonormal and orthogonal to g_k, and
// a particle x with x.g_k > 0 in scaled gnomonic coordinates
//     (u, v) = (x.e1, x.e2) / ((x.g_k) h_k),   s^2 = u^2 + v^2,
// the data are the particles with s < kSc = 2.2, weighted by
// (1 - s^2/kSc^2)^4, and c0 + c1 u + c2 v + c3 u^2 + c4 u v + c5 v^2 is fitted
// by weighted least squares; the value is c0.  The weights vanish smoothly at
// the edge of the data disc, so the result depends continuously on the
// particle positions.
//
// Finding the data: every particle is put in the Voronoi cell of its nearest
// grid point by a greedy walk on the grid's triangulation from the grid point
// it started at (on a Delaunay triangulation a vertex that is not the nearest
// always has a strictly nearer neighbour), and the particles are counting-
// sorted by cell (buckets sorted by particle index, so every sum runs in a
// fixed order).  A particle in the cell of grid point c is at least
// |g_c - g_k|/2 from g_k (c is its nearest grid point), and the grid point
// nearest to g_k outside the ring-R neighbourhood of g_k lies on ring R+1 (the
// cells met by the segment from g_k to any outer grid point are no farther
// from g_k).  So the cells of the smallest ring R whose next ring stays at
// least twice the data-disc chord from g_k hold every datum of g_k.  Of these,
// the cells whose grid point is farther from g_k than the data chord plus the
// cell's own radius (its farthest Voronoi vertex) hold none and are dropped;
// the stencil is fixed per grid point when the grid is made.
//
// Work per remeshing: one walk per particle, the counting sort, and four
// lanes per grid point that filter the stencil's particles, accumulate the
// 21 + 6 weighted normal-equation sums in FP64 and solve by an unrolled 6x6
// Cholesky (the scaled coordinates keep its condition number near 1e2).
#include <math.h>

#include <cuda_runtime.h>

#include "csfmm_internal.cuh"

struct csfmm_remesh_grid_s {
  int M = 0, max_ring = 0;
  int64_t nadj = 0;
  csfmm::DeviceArena arena;
  double *g = nullptr;        // [M][3] grid points
  double *h = nullptr;        // [M] chord to the nearest neighbour
  int32_t *aoff = nullptr;    // [M+1] triangulation neighbours (CSR)
  int32_t *adj = nullptr;     // [nadj]
  double *rho = nullptr;      // [M] largest chord from a grid point to its Voronoi cell
  int32_t *soff = nullptr;    // [M+1] stencils (CSR)
  int32_t *sten = nullptr;    // [soff[M]]
  // per-remeshing scratch
  int32_t *cell = nullptr;    // [M] cell of each particle
  int32_t *cnt = nullptr;     // [M+1] particles per cell
  int32_t *boff = nullptr;    // [M+1] bucket offsets
  int32_t *cursor = nullptr;  // [M]
  int32_t *bucket = nullptr;  // [M] particles by cell
  int32_t *scan_tmp = nullptr;
  int *status = nullptr;
};

namespace csfmm {

namespace {

constexpr double kSc = 2.2;        // radius of the data disc in units of h_k
constexpr int kRemeshMaxRing = 8;    // rings searched for a stencil
constexpr int kRemeshMaxStencil = 384;  // grid points in one stencil search
constexpr int kRemeshMaxWalk = 1 << 16;  // greedy steps of one particle (M < 2^31 vertices,
                                         // but a step of the remeshed method moves a few cells)
constexpr int kRemeshMaxBucketSort = 4096;

// Bits of the remeshing status word.
constexpr int kRmAdjacency = 1;  // a neighbour index out of range or a vertex without neighbours
constexpr int kRmStencil = 2;    // no stencil within kRemeshMaxRing rings / kRemeshMaxStencil points
constexpr int kRmWalk = 4;       // a walk that did not end within kRemeshMaxWalk steps
constexpr int kRmBucket = 8;     // a cell holding more than kRemeshMaxBucketSort particles
constexpr int kRmFit = 16;       // a stencil with fewer than 6 particles or a singular fit
constexpr int kRmNotOnSphere = 32;

// Squared chord ((d0 d0 + d1 d1) + d2 d2), rounded after every operation, so
// that a particle on a cell boundary (symmetric inputs put some exactly there)
// is assigned by the same comparison on every platform.
__device__ __forceinline__ double dist2(const double *a, const double *b) {
  const double d0 = a[0] - b[0], d1 = a[1] - b[1], d2 = a[2] - b[2];
  return __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
}

__global__ void adj_convert_kernel(const int64_t *off, const int64_t *adj, int M, int64_t nadj,
                                   const double *g, int32_t *aoff, int32_t *adj32, double *h,
                                   int *status) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= M; k += gridDim.x * blockDim.x) {
    const int64_t b = off[k];
    if (b < 0 || b > nadj) {
      atomicOr(status, kRmAdjacency);
      aoff[k] = 0;
      continue;
    }
    aoff[k] = (int32_t)b;
    if (k == M) continue;
    const int64_t e = off[k + 1];
    const double *gk = g + 3 * (size_t)k;
    const double r2 = gk[0] * gk[0] + gk[1] * gk[1] + gk[2] * gk[2];
    if (!(fabs(r2 - 1.0) <= 1e-12)) atomicOr(status, kRmNotOnSphere);
    if (e <= b || e > nadj) {
      atomicOr(status, kRmAdjacency);
      h[k] = 1.0;
      continue;
    }
    double best = 1e300;
    for (int64_t i = b; i < e; ++i) {
      const int64_t j = adj[i];
      if (j < 0 || j >= M || j == k) {
        atomicOr(status, kRmAdjacency);
        adj32[i] = k;
        continue;
      }
      adj32[i] = (int32_t)j;
      best = fmin(best, dist2(gk, g + 3 * (size_t)j));
    }
    h[k] = best < 1e300 ? sqrt(best) : 1.0;
  }
}

// Chord of the data disc's edge at g_k: s = kSc is the angle atan(kSc h_k)
// from g_k; slightly enlarged so that rounding cannot drop a datum.
__device__ __forceinline__ double data_chord(double hk) {
  return 2.0 * sin(0.5 * atan(kSc * hk)) * (1.0 + 1e-9);
}

// rho_c: the largest chord from grid point c to a vertex of its Voronoi cell,
// which bounds the chord from g_c to any particle in its cell (the cell is
// convex and inside the hemisphere about g_c, so its farthest point is a
// vertex).  The vertices are the circumcentres of the triangles (c, a, b) at c,
// taken as the pairs of neighbours of c joined by an edge: three mutually
// joined points that are not a face only add a candidate to the maximum.  A
// degenerate triangle, or none at all, gives rho = 2 (the whole sphere).
__global__ void cell_radius_kernel(const double *g, const int32_t *aoff, const int32_t *adj,
                                   int M, double *rho) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < M; c += gridDim.x * blockDim.x) {
    const double *gc = g + 3 * (size_t)c;
    double best = 0.0;
    bool any = false;
    for (int e = aoff[c]; e < aoff[c + 1]; ++e) {
      const int a = adj[e];
      const double *ga = g + 3 * (size_t)a;
      for (int f = aoff[a]; f < aoff[a + 1]; ++f) {
        const int b = adj[f];
        if (b <= a) continue;  // each pair once
        bool joined = false;
        for (int t = aoff[c]; t < aoff[c + 1] && !joined; ++t) joined = adj[t] == b;
        if (!joined) continue;
        const double *gb = g + 3 * (size_t)b;
        const double d1[3] = {ga[0] - gc[0], ga[1] - gc[1], ga[2] - gc[2]};
        const double d2[3] = {gb[0] - gc[0], gb[1] - gc[1], gb[2] - gc[2]};
        double q[3] = {d1[1] * d2[2] - d1[2] * d2[1], d1[2] * d2[0] - d1[0] * d2[2],
                       d1[0] * d2[1] - d1[1] * d2[0]};
        const double nn = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
        any = true;
        if (!(nn > 0.0)) {
          best = 2.0;
          continue;
        }
        double sc = rsqrt(nn);
        if (q[0] * gc[0] + q[1] * gc[1] + q[2] * gc[2] < 0.0) sc = -sc;
        q[0] *= sc;
        q[1] *= sc;
        q[2] *= sc;
        best = fmax(best, sqrt(dist2(q, gc)));
      }
    }
    rho[c] = any ? fmin(best, 2.0) : 2.0;
  }
}

// Breadth-first rings around k, one warp per grid point, in S (shared memory,
// S[0] = k): stops after the smallest ring R whose next ring lies at least
// twice the data chord away.  Returns n (the stencil size: S[0..n) holds rings
// 0..R, in no particular order) and R, or -1 when no ring up to
// kRemeshMaxRing qualifies within kRemeshMaxStencil points.  The lanes take
// the vertices of a ring 32 at a time and step through their neighbour lists
// together; a neighbour of ring r lies in ring r - 1, r or r + 1, so it is new
// unless it is in S from the start of ring r - 1 on, and of equal new
// neighbours met in one step the lowest lane's is kept.  Of rings 0..R only
// the cells that can hold a datum are kept: a particle in the cell of c is
// within rho_c of g_c, so by the triangle inequality for chords the cell holds
// none when |g_c - g_k| > data chord + rho_c (about 28 of 91 cells stay on the
// icosahedral grids).  Warp-uniform result.
__device__ int stencil_set(int k, const double *g, const double *h, const double *rho,
                           const int32_t *aoff, const int32_t *adj, int *S, int *ring_out) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned below = (1u << lane) - 1u;
  const double need = 2.0 * data_chord(h[k]);
  const double *gk = g + 3 * (size_t)k;
  if (lane == 0) S[0] = k;
  __syncwarp();
  int n = 1, lo = 0, plo = 0;
  for (int r = 0; r <= kRemeshMaxRing; ++r) {
    // grow ring r + 1 from ring r = S[lo..hi)
    const int hi = n;
    double dmin = 1e300;
    for (int base = lo; base < hi; base += 32) {
      const int i = base + (int)lane;
      const int v = i < hi ? S[i] : 0;
      const int eb = i < hi ? aoff[v] : 0;
      const int deg = i < hi ? aoff[v + 1] - eb : 0;
      int maxdeg = deg;
      for (int o = 16; o; o >>= 1) maxdeg = max(maxdeg, __shfl_xor_sync(~0u, maxdeg, o));
      for (int j = 0; j < maxdeg; ++j) {
        const int w = j < deg ? adj[eb + j] : -1;
        bool fresh = j < deg;
        for (int t = plo; t < n && fresh; ++t) fresh = S[t] != w;
        const unsigned same = __match_any_sync(~0u, w);
        if (same & below) fresh = false;
        const unsigned add = __ballot_sync(~0u, fresh);
        if (n + __popc(add) > kRemeshMaxStencil) return -1;
        if (fresh) {
          S[n + __popc(add & below)] = w;
          dmin = fmin(dmin, sqrt(dist2(gk, g + 3 * (size_t)w)));
        }
        n += __popc(add);
        __syncwarp();
      }
    }
    for (int o = 16; o; o >>= 1) dmin = fmin(dmin, __shfl_xor_sync(~0u, dmin, o));
    if (dmin >= need) {
      *ring_out = r;  // rings 0..r qualify: S[0..hi) holds every datum
      const double chord = data_chord(h[k]);
      int m = 0;  // compact in place: a write lands below the chunk being read
      for (int base = 0; base < hi; base += 32) {
        const int i = base + (int)lane;
        const int c = i < hi ? S[i] : 0;
        const bool keep =
            i < hi && sqrt(dist2(gk, g + 3 * (size_t)c)) <= chord + rho[c] * (1.0 + 1e-9);
        const unsigned kb = __ballot_sync(~0u, keep);
        __syncwarp();  // every lane has read its S[i]
        if (keep) S[m + __popc(kb & below)] = c;
        m += __popc(kb);
        __syncwarp();
      }
      return m;
    }
    plo = lo;
    lo = hi;  // (a ring with no new grid point has dmin = 1e300: the whole grid)
  }
  return -1;
}

constexpr int kStencilWarps = 8;  // warps (grid points at a time) per block

__global__ void __launch_bounds__(32 * kStencilWarps)
stencil_count_kernel(const double *g, const double *h, const double *rho, const int32_t *aoff,
                     const int32_t *adj, int M, int32_t *cnt, int *max_ring, int *status) {
  __shared__ int Ss[kStencilWarps][kRemeshMaxStencil];
  const int wid = threadIdx.x >> 5;
  int *S = Ss[wid];
  for (int k = blockIdx.x * kStencilWarps + wid; k < M; k += gridDim.x * kStencilWarps) {
    int r = 0;
    const int n = stencil_set(k, g, h, rho, aoff, adj, S, &r);
    if ((threadIdx.x & 31) == 0) {
      if (n < 0) atomicOr(status, kRmStencil);
      else atomicMax(max_ring, r);
      cnt[k] = n < 0 ? 0 : n;
    }
    __syncwarp();
  }
}

// The stencil of k in ascending order: each element goes to its rank (the
// grid points are distinct).
__global__ void __launch_bounds__(32 * kStencilWarps)
stencil_fill_kernel(const double *g, const double *h, const double *rho, const int32_t *aoff,
                    const int32_t *adj, int M, const int32_t *soff, int32_t *sten, int *status) {
  __shared__ int Ss[kStencilWarps][kRemeshMaxStencil];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int *S = Ss[wid];
  for (int k = blockIdx.x * kStencilWarps + wid; k < M; k += gridDim.x * kStencilWarps) {
    int r = 0;
    const int n = stencil_set(k, g, h, rho, aoff, adj, S, &r);
    if (n >= 0 && soff[k + 1] - soff[k] == n) {
      for (int i = lane; i < n; i += 32) {
        const int v = S[i];
        int rank = 0;
        for (int t = 0; t < n; ++t) rank += S[t] < v;
        sten[soff[k] + rank] = v;
      }
    } else {
      // the count pass found another size (the search is deterministic, so
      // this does not happen): valid indices, and the grid is refused
      for (int i = soff[k] + lane; i < soff[k + 1]; i += 32) sten[i] = k;
      if (lane == 0) atomicOr(status, kRmStencil);
    }
    __syncwarp();
  }
}

// Nearest grid point of particle p by a greedy walk from grid point p, in the
// order (squared chord, index) so that the walk is deterministic; which of two
// equally near grid points a particle gets does not change any result (both
// are nearest, which is all the stencil bound uses).
__global__ void walk_kernel(const double *x, const double *g, const int32_t *aoff,
                            const int32_t *adj, int M, int32_t *cell, int32_t *cnt, int *status) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < M; p += gridDim.x * blockDim.x) {
    const double xp[3] = {x[3 * (size_t)p], x[3 * (size_t)p + 1], x[3 * (size_t)p + 2]};
    int v = p;
    double d = dist2(xp, g + 3 * (size_t)v);
    int it = 0;
    for (; it < kRemeshMaxWalk; ++it) {
      int best = v;
      double bd = d;
      for (int e = aoff[v]; e < aoff[v + 1]; ++e) {
        const int w = adj[e];
        const double dw = dist2(xp, g + 3 * (size_t)w);
        if (dw < bd || (dw == bd && w < best)) {
          bd = dw;
          best = w;
        }
      }
      if (best == v) break;
      v = best;
      d = bd;
    }
    if (it == kRemeshMaxWalk) atomicOr(status, kRmWalk);
    cell[p] = v;
    atomicAdd(&cnt[v], 1);
  }
}

__global__ void bucket_fill_kernel(const int32_t *cell, int M, const int32_t *boff,
                                   int32_t *cursor, int32_t *bucket) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < M; p += gridDim.x * blockDim.x) {
    const int c = cell[p];
    bucket[boff[c] + atomicAdd(&cursor[c], 1)] = p;
  }
}

__global__ void bucket_sort_kernel(const int32_t *boff, int M, int32_t *bucket, int *status) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < M; c += gridDim.x * blockDim.x) {
    const int b = boff[c], e = boff[c + 1];
    if (e - b > kRemeshMaxBucketSort) {
      atomicOr(status, kRmBucket);
      continue;
    }
    for (int i = b + 1; i < e; ++i) {
      const int v = bucket[i];
      int j = i - 1;
      while (j >= b && bucket[j] > v) {
        bucket[j + 1] = bucket[j];
        --j;
      }
      bucket[j + 1] = v;
    }
  }
}

// Step 3: weighted quadratic least squares at every grid point.
// NF fields f[0..NF) (stride M) share the normal matrix; each gets its own
// right-hand side and solve.  kFitLanes lanes serve one grid point: lane l
// takes stencil cells l, l + kFitLanes, ... and the partial sums are added
// across the lanes by a butterfly (every lane ends with the same bits, as
// IEEE addition commutes), so the result does not depend on scheduling.  A
// candidate is tested against the disc without division,
// (x.e1)^2 + (x.e2)^2 < kSc^2 (x.g_k h_k)^2, and a datum costs one reciprocal.
constexpr int kFitLanes = 4;

template <int NF>
__global__ void __launch_bounds__(128) fit_kernel(const double *x, const double *f,
                                                  const double *g, const double *h,
                                                  const int32_t *soff, const int32_t *sten,
                                                  const int32_t *boff, const int32_t *bucket,
                                                  int M, double *out, int *status) {
  const int sub = threadIdx.x % kFitLanes;
  const unsigned group = ((1u << kFitLanes) - 1u) << ((threadIdx.x & 31) & ~(kFitLanes - 1));
  for (int k = (blockIdx.x * blockDim.x + threadIdx.x) / kFitLanes; k < M;
       k += gridDim.x * blockDim.x / kFitLanes) {
    const double gk[3] = {g[3 * (size_t)k], g[3 * (size_t)k + 1], g[3 * (size_t)k + 2]};
    // e1 = a x g / |a x g| with a = e_z, or e_x near the poles; e2 = g x e1
    double e1[3];
    if (fabs(gk[2]) < 0.9) {
      e1[0] = -gk[1];
      e1[1] = gk[0];
      e1[2] = 0.0;
    } else {
      e1[0] = 0.0;
      e1[1] = -gk[2];
      e1[2] = gk[1];
    }
    const double in = rsqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    e1[0] *= in;
    e1[1] *= in;
    e1[2] *= in;
    const double e2[3] = {gk[1] * e1[2] - gk[2] * e1[1], gk[2] * e1[0] - gk[0] * e1[2],
                          gk[0] * e1[1] - gk[1] * e1[0]};
    const double hk = h[k];
    constexpr double kSc2 = kSc * kSc;
    double A[21], b[NF][6];  // packed lower triangle of sum w phi phi^T, sum w phi f
#pragma unroll
    for (int i = 0; i < 21; ++i) A[i] = 0.0;
#pragma unroll
    for (int q = 0; q < NF; ++q)
#pragma unroll
      for (int i = 0; i < 6; ++i) b[q][i] = 0.0;
    int n = 0;
    for (int s = soff[k] + sub; s < soff[k + 1]; s += kFitLanes) {
      const int c = sten[s];
      for (int q = boff[c]; q < boff[c + 1]; ++q) {
        const int p = bucket[q];
        const double *xp = x + 3 * (size_t)p;
        const double x0 = xp[0], x1 = xp[1], x2 = xp[2];
        const double dot = x0 * gk[0] + x1 * gk[1] + x2 * gk[2];
        const double den = dot * hk;
        const double a1 = x0 * e1[0] + x1 * e1[1] + x2 * e1[2];
        const double a2 = x0 * e2[0] + x1 * e2[1] + x2 * e2[2];
        if (!(dot > 0.0) || !(a1 * a1 + a2 * a2 < kSc2 * (den * den))) continue;
        const double r = 1.0 / den;
        const double u = a1 * r, v = a2 * r;
        const double om = fmax(1.0 - (u * u + v * v) * (1.0 / kSc2), 0.0);
        const double om2 = om * om;
        const double w = om2 * om2;
        const double phi[6] = {1.0, u, v, u * u, u * v, v * v};
        int t = 0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          const double wi = w * phi[i];
#pragma unroll
          for (int j = 0; j <= i; ++j) A[t++] += wi * phi[j];
        }
#pragma unroll
        for (int q = 0; q < NF; ++q) {
          const double wf = w * f[(size_t)q * M + p];
#pragma unroll
          for (int i = 0; i < 6; ++i) b[q][i] += wf * phi[i];
        }
        ++n;
      }
    }
#pragma unroll
    for (int o = 1; o < kFitLanes; o <<= 1) {
#pragma unroll
      for (int i = 0; i < 21; ++i) A[i] += __shfl_xor_sync(group, A[i], o);
#pragma unroll
      for (int q = 0; q < NF; ++q)
#pragma unroll
        for (int i = 0; i < 6; ++i) b[q][i] += __shfl_xor_sync(group, b[q][i], o);
      n += __shfl_xor_sync(group, n, o);
    }
    if (n < 6) {
      if (sub == 0) {
        atomicOr(status, kRmFit);
#pragma unroll
        for (int q = 0; q < NF; ++q) out[(size_t)q * M + k] = 0.0;
      }
      continue;
    }
    // Cholesky A = L L^T in place (packed lower triangle), then L y = b, L^T c = y,
    // with the reciprocals of the diagonal from rsqrt (no division).
    double amax = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) amax = fmax(amax, A[i * (i + 1) / 2 + i]);
    bool ok = true;
    double rl[6];
    // (constant trip counts with guards, so that every loop unrolls and A stays
    // in registers)
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      double d = A[j * (j + 1) / 2 + j];
#pragma unroll
      for (int m = 0; m < 6; ++m)
        if (m < j) d -= A[j * (j + 1) / 2 + m] * A[j * (j + 1) / 2 + m];
      if (!(d > 1e-13 * amax)) ok = false;
      rl[j] = rsqrt(fmax(d, 1e-300));
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        if (i <= j) continue;
        double s = A[i * (i + 1) / 2 + j];
#pragma unroll
        for (int m = 0; m < 6; ++m)
          if (m < j) s -= A[i * (i + 1) / 2 + m] * A[j * (j + 1) / 2 + m];
        A[i * (i + 1) / 2 + j] = s * rl[j];
      }
    }
    if (!ok) {
      if (sub == 0) {
        atomicOr(status, kRmFit);
#pragma unroll
        for (int q = 0; q < NF; ++q) out[(size_t)q * M + k] = 0.0;
      }
      continue;
    }
#pragma unroll
    for (int q = 0; q < NF; ++q) {
      double y[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        double s = b[q][i];
#pragma unroll
        for (int m = 0; m < i; ++m) s -= A[i * (i + 1) / 2 + m] * y[m];
        y[i] = s * rl[i];
      }
      double c[6];
#pragma unroll
      for (int i = 5; i >= 0; --i) {
        double s = y[i];
#pragma unroll
        for (int m = i + 1; m < 6; ++m) s -= A[m * (m + 1) / 2 + i] * c[m];
        c[i] = s * rl[i];
      }
      if (sub == 0) out[(size_t)q * M + k] = c[0];
    }
  }
}

csfmm_status remesh_status(int st) {
  if (st == 0) return CSFMM_OK;
  set_error("remeshing failed (status 0x%x:%s%s%s%s%s%s)", st,
            st & kRmAdjacency ? " bad neighbour lists" : "",
            st & kRmStencil ? " no stencil holds the data disc (grid too irregular or too small)" : "",
            st & kRmWalk ? " nearest-point walk did not end" : "",
            st & kRmBucket ? " too many particles in one cell" : "",
            st & kRmFit ? " fewer than 6 particles or a singular fit in a data disc" : "",
            st & kRmNotOnSphere ? " grid point off the unit sphere" : "");
  return (st & kRmNotOnSphere) ? CSFMM_ERR_NOT_ON_SPHERE
         : (st & (kRmAdjacency | kRmStencil)) ? CSFMM_ERR_INVALID_ARG
                                               : CSFMM_ERR_DEVICE;
}

}  // namespace

// Remeshing of moved particles x (particle p started at grid point p) carrying
// f onto the grid; enqueued on st, then the status word is read (synchronous).
csfmm_status remesh_impl(csfmm_remesh_grid G, const double *x, const double *f, int nfield,
                         double *f_out, cudaStream_t st) {
  const int M = G->M;
  const int grid = grid_for(M, 256, sm_count() * 8);
  CSFMM_CUDA(cudaMemsetAsync(G->status, 0, sizeof(int), st));
  CSFMM_CUDA(cudaMemsetAsync(G->cnt, 0, sizeof(int32_t) * (M + 1), st));
  CSFMM_CUDA(cudaMemsetAsync(G->cursor, 0, sizeof(int32_t) * M, st));
  walk_kernel<<<grid, 256, 0, st>>>(x, G->g, G->aoff, G->adj, M, G->cell, G->cnt, G->status);
  CSFMM_CUDA(cudaGetLastError());
  csfmm_status s = exclusive_scan_i32(G->cnt, G->boff, M + 1, nullptr, G->scan_tmp, st);
  if (s != CSFMM_OK) return s;
  bucket_fill_kernel<<<grid, 256, 0, st>>>(G->cell, M, G->boff, G->cursor, G->bucket);
  bucket_sort_kernel<<<grid, 256, 0, st>>>(G->boff, M, G->bucket, G->status);
  // fields in pairs (the second pair re-reads the stencil; the walk and sort are shared)
  const int fg = grid_for((int64_t)M * kFitLanes, 128, sm_count() * 16);
  for (int q = 0; q < nfield; q += 2) {
    const double *fq = f + (size_t)q * M;
    double *oq = f_out + (size_t)q * M;
    if (nfield - q >= 2)
      fit_kernel<2><<<fg, 128, 0, st>>>(x, fq, G->g, G->h, G->soff, G->sten, G->boff, G->bucket,
                                        M, oq, G->status);
    else
      fit_kernel<1><<<fg, 128, 0, st>>>(x, fq, G->g, G->h, G->soff, G->sten, G->boff, G->bucket,
                                        M, oq, G->status);
  }
  CSFMM_CUDA(cudaGetLastError());
  int hs = 0;
  CSFMM_CUDA(cudaMemcpyAsync(&hs, G->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CSFMM_CUDA(cudaStreamSynchronize(st));
  return remesh_status(hs);
}

int64_t remesh_grid_size(csfmm_remesh_grid G) { return G->M; }
const double *remesh_grid_points(csfmm_remesh_grid G) { return G->g; }

}  // namespace csfmm

using namespace csfmm;

extern "C" csfmm_status csfmm_remesh_grid_create(const double *grid, int64_t M,
                                                 const int64_t *adj_offsets, const int64_t *adj,
                                                 void *stream, csfmm_remesh_grid *out) {
  if (!out) {
    set_error("out is NULL");
    return CSFMM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (!grid || !adj_offsets || !adj || M < 7 || M >= ((int64_t)1 << 30)) {
    set_error("csfmm_remesh_grid_create: device arrays and 7 <= M < 2^30 required");
    return CSFMM_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int64_t nadj = 0;
  CSFMM_CUDA(cudaMemcpyAsync(&nadj, adj_offsets + M, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CSFMM_CUDA(cudaStreamSynchronize(st));
  if (nadj < M || nadj >= ((int64_t)1 << 31)) {
    set_error("csfmm_remesh_grid_create: adj_offsets[M] = %lld is not a neighbour count in "
              "[M, 2^31)", (long long)nadj);
    return CSFMM_ERR_INVALID_ARG;
  }
  auto *G = new csfmm_remesh_grid_s();
  G->arena.stream = st;
  G->M = (int)M;
  G->nadj = nadj;
  csfmm_status s = CSFMM_OK;
  auto A = [&](auto **p, size_t n) {
    if (s == CSFMM_OK) s = G->arena.alloc(p, n);
  };
  A(&G->g, 3 * (size_t)M);
  A(&G->h, (size_t)M);
  A(&G->aoff, (size_t)M + 1);
  A(&G->adj, (size_t)nadj);
  A(&G->rho, (size_t)M);
  A(&G->soff, (size_t)M + 1);
  A(&G->cell, (size_t)M);
  A(&G->cnt, (size_t)M + 1);
  A(&G->boff, (size_t)M + 1);
  A(&G->cursor, (size_t)M);
  A(&G->bucket, (size_t)M);
  A(&G->scan_tmp, scan_tmp_elems((int)M + 1));
  A(&G->status, 1);
  auto fail = [&](csfmm_status e) {
    cudaStreamSynchronize(st);
    G->arena.release();
    delete G;
    return e;
  };
  if (s != CSFMM_OK) return fail(s);
  const int gr = grid_for(M + 1, 256, sm_count() * 8);
  cudaError_t e = cudaMemcpyAsync(G->g, grid, sizeof(double) * 3 * (size_t)M,
                                  cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(G->status, 0, sizeof(int), st);
  if (e != cudaSuccess) return fail(cuda_status(e, "csfmm_remesh_grid_create copy"));
  adj_convert_kernel<<<gr, 256, 0, st>>>(adj_offsets, adj, (int)M, nadj, G->g, G->aoff, G->adj,
                                         G->h, G->status);
  int hs = 0;
  e = cudaMemcpyAsync(&hs, G->status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(cuda_status(e, "adj_convert_kernel"));
  if (hs) return fail(remesh_status(hs));
  // offsets must increase: checked above per vertex (e > b) together with the range
  // the scan of the stencil sizes reuses cnt; cursor[0] receives the largest ring
  e = cudaMemsetAsync(G->cursor, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMemsetAsync"));
  const int grs = grid_for(M, kStencilWarps, sm_count() * 16);
  cell_radius_kernel<<<gr, 256, 0, st>>>(G->g, G->aoff, G->adj, (int)M, G->rho);
  stencil_count_kernel<<<grs, 32 * kStencilWarps, 0, st>>>(G->g, G->h, G->rho, G->aoff, G->adj,
                                                            (int)M, G->cnt, G->cursor, G->status);
  int32_t total = 0;
  e = cudaMemsetAsync(G->cnt + M, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMemsetAsync"));
  s = exclusive_scan_i32(G->cnt, G->soff, (int)M + 1, &total, G->scan_tmp, st);
  if (s != CSFMM_OK) return fail(s);
  e = cudaMemcpyAsync(&hs, G->status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(cuda_status(e, "stencil_count_kernel"));
  if (hs) return fail(remesh_status(hs));
  A(&G->sten, (size_t)total);
  if (s != CSFMM_OK) return fail(s);
  e = cudaMemcpyAsync(&G->max_ring, G->cursor, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMemcpyAsync"));
  stencil_fill_kernel<<<grs, 32 * kStencilWarps, 0, st>>>(G->g, G->h, G->rho, G->aoff, G->adj,
                                                           (int)M, G->soff, G->sten, G->status);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&hs, G->status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(cuda_status(e, "stencil_fill_kernel"));
  if (hs) return fail(remesh_status(hs));
  *out = G;
  return CSFMM_OK;
}

extern "C" csfmm_status csfmm_remesh(csfmm_remesh_grid G, const double *x, const double *f,
                                     int nfield, double *f_out, void *stream) {
  if (!G || !x || !f || !f_out || nfield < 1 || nfield > 64) {
    set_error("csfmm_remesh: non-NULL arguments and 1 <= nfield <= 64 required");
    return CSFMM_ERR_INVALID_ARG;
  }
  const size_t bytes = sizeof(double) * (size_t)nfield * G->M;
  const char *a = (const char *)f, *b = (const char *)f_out;
  if (a < b + bytes && b < a + bytes) {
    set_error("csfmm_remesh: f_out overlaps f (every output reads many inputs)");
    return CSFMM_ERR_INVALID_ARG;
  }
  return remesh_impl(G, x, f, nfield, f_out, (cudaStream_t)stream);
}

extern "C" csfmm_status csfmm_remesh_grid_destroy(csfmm_remesh_grid G) {
  if (!G) return CSFMM_OK;
  cudaDeviceSynchronize();
  G->arena.release();
  delete G;
  return CSFMM_OK;
}
