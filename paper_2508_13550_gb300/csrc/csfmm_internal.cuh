// csfmm_internal.cuh -- shared definitions of the CUDA library behind csfmm.h.
//
// Layout of a plan in HBM (tree order = points sorted by face and Morton key
// of their (xi, eta) cell coordinates, Sec. 3):
//   x[3][N]            FP64 sorted points (SoA)
//   perm[N]            tree position -> input index
//   La[N][p], Lb[N][p] barycentric Lagrange values L_k(u_i), L_k(v_i) of every
//                      point in its leaf (Sec. 4, Eq. barycentric); FP64 for
//                      the FP64 form, an FP32 hi + lo pair for the FP32-bulk
//                      form (P2M uses hi, the double-float L2P both)
//   off32[N]           float4 offset of each point from its leaf centre
//   cells (SoA)        face, level, ia, ib, begin, end, parent, child[4],
//                      centre[3], radius, xi_mid, eta_mid, half
//   proxy[nc][3][P]    FP64 proxy points; proxy32[nc][3][P] FP32 offsets from
//                      the cell centre
//   lists              CSR by target cell for PP, PC, CP, CC
//   m2m[2][p][p]       the two 1-D child-to-parent interpolation matrices
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/csfmm.h"

namespace csfmm {

constexpr int kD = 18;          // tangent table resolution: 2^kD intervals per face
constexpr int kLMax = 17;       // deepest cell level
constexpr int kMaxDegree = 16;  // n <= 16, p <= 17, P <= 289
constexpr int kMaxP = kMaxDegree + 1;

// Bits of the plan's device status word.
constexpr int kStatusNotOnSphere = 1;
constexpr int kStatusOverflow = 2;
constexpr int kStatusInternal = 4;
constexpr int kStatusTimeout = 8;

void set_error(const char *fmt, ...);
csfmm_status cuda_status(cudaError_t e, const char *what);

#define CSFMM_CUDA(call)                                               \
  do {                                                                 \
    cudaError_t e__ = (call);                                          \
    if (e__ != cudaSuccess) return csfmm::cuda_status(e__, #call);     \
  } while (0)

struct Workspace;

// Device memory of plans, workspaces, build scratch and remeshing grids comes
// from one stream-ordered pool per device (cudaMallocFromPoolAsync) that keeps
// up to kPoolKeepBytes of freed memory for the next allocations instead of
// handing it back to the CUDA driver, so that a plan build costs some eighty
// allocations of reused memory rather than eighty cudaMalloc calls and a
// device-wide synchronisation in every cudaFree.
constexpr uint64_t kPoolKeepBytes = 4ull << 30;
constexpr int kMaxPoolDevices = 64;
cudaMemPool_t memory_pool();    // the current device's pool
cudaStream_t release_stream();  // the current device's stream for freeing idle memory
// Tangent table T[k] = tan(k (pi/2)/2^kD - pi/4) on the current device,
// uploaded once (nullptr after an error, with the message set).
const double *device_tan_table();

// Device buffers are tracked so that a failed build frees everything.
// Allocations are ordered on `stream`; release() frees on the release stream
// and may only be called when no work uses the buffers any more.
struct DeviceArena {
  std::vector<void *> ptrs;
  int64_t bytes = 0;
  cudaStream_t stream = nullptr;
  template <class T>
  csfmm_status alloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    void *q = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&q, count * sizeof(T), memory_pool(), stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("device allocation of %zu bytes failed: %s", count * sizeof(T),
                cudaGetErrorString(e));
      return CSFMM_ERR_OUT_OF_MEMORY;
    }
    ptrs.push_back(q);
    bytes += (int64_t)(count * sizeof(T));
    *p = (T *)q;
    return CSFMM_OK;
  }
  void release() {
    cudaStream_t rs = release_stream();
    for (void *p : ptrs) cudaFreeAsync(p, rs);
    ptrs.clear();
    bytes = 0;
  }
};

// Largest number of right-hand sides of one evaluation (checked by the API).
constexpr int kMaxNrhs = 64;

// Read-only view of a plan passed to kernels by value.
struct PlanView {
  int N, n, p, P, N0, ncells, dim, kernel_id;
  int nsrc, ntgt, tbase;  // weights [nrhs][nsrc]; out [nrhs][ntgt][dim] at input index - tbase
  const double *x;       // [3][N]
  const int32_t *perm;   // [N]
  const double *La64, *Lb64;  // [N][p]
  const float *La32, *Lb32;   // [N][p] stochastic FP32 rounding of the rows ...
  const float *La32lo, *Lb32lo;  // ... and of the remainders
  const float4 *off32;   // [N]
  const int32_t *cbegin, *cend, *clevel, *cface, *cparent, *cchild;
  const double *ccentre; // [nc][3]
  const double *cradius;
  const double *cxmid, *cymid, *chalf, *chy;  // box midpoints, half-widths (xi, eta)
  const double *mcell64;  // shrunk boxes: [cell][2][p][p] matrices to the parent, else null
  const float *mcell32;   // [cell][2 (rounding, remainder)][2][p][p]
  const double *proxy;   // [nc][3][P]
  const float *proxy32;  // [nc][3][P]
  const int32_t *loff[4], *lsrc[4];
  // FP32 form: centre difference c_T - c_S of every list entry as FP32 (x, y, z, 0),
  // rounded once from FP64 (stochastically for the far-field types CP, CC of the
  // 1/|x - y| kernels)
  const float4 *ldc[4];
  const int32_t *sym_contrib;
  const int32_t *cc_contrib;  // [nCC] partial-buffer offset of a mirrored CC entry, or -1
  const double *m2m64;   // [2][p][p]: M[q][k][m] = L_k((s_m + 2q - 1)/2)
  const float *m2m32;    // [2][2][p][p]: FP32 rounding of m2m64, then the remainders
  const double *cheb;    // [p]
  int *status;
  // Per evaluation (FP32 form, log kernel): weight totals of every cell as
  // unevaluated FP32 pairs, [nc][wtot_ld][2] = (particle weights of a leaf,
  // proxy weights of a cell), each summed in FP64 from the FP32 weights.
  const float2 *wtot;
  int wtot_ld;
};

// Arguments of the persistent multi-right-hand-side kernel (persistent.cu):
// one launch evaluates the far field, the near field, L2L and L2P of every
// chunk of NR right-hand sides, drawing items from a device work counter.
struct PersistArgs {
  const int32_t *leaves;
  int nleaves, ncells;
  int nl2l;                 // cells of levels 0 .. nlevels-2 (L2L items)
  int nch, nrhs, ldr;       // nch chunks of NR right-hand sides; rhs stride of wbar / psi
  int far_pair;             // 1: a far item holds two cells, one per half block
  int nfar, nnear, total;   // items: far, then near with the L2L levels inserted, then L2P
  int nlev;                 // L2L levels (nlevels - 1)
  int lvl_begin[kLMax + 2]; // cells of level l: [lvl_begin[l], lvl_begin[l+1])
  int ins[kLMax + 1];       // L2L level l follows near item ins[l] (nondecreasing)
  const float *wsf, *wbar;
  double *phi, *psi, *out;
  int *ctr;                 // [0] queue head, [1] abort flag, then far_done, l2l_done and
                            // near_done counters, ncells each
  int extra;                // test hook: completions every wait needs beyond the real count
  long long limit_ns;       // bound of every dependency wait
};

struct Plan {
  int device = 0;
  int64_t N = 0;
  // Separate targets (csfmm_plan_create_targets): the tree holds the sources
  // (input indices [0, nsrc)) and then the targets ([tbase, tbase + ntgt));
  // weights are given for the sources, results returned for the targets.  A
  // plan of one point set has nsrc = ntgt = N, tbase = 0.
  int64_t nsrc = 0, ntgt = 0, tbase = 0;
  int kernel_id = 0, n = 0, p = 0, P = 0, N0 = 0, precision = 0, dim = 1, max_nrhs = 16;
  int use_graphs = 0;
  int rhs_chunk = 16;   // FP32 bulk, scalar kernels: 16, 8 or 4
  int shrink = 0;       // cell boxes shrunk to their points
  int no_persistent = 0; // 1: several right-hand sides always take the per-phase launches
  int schedule = 0;      // CSFMM_SCHED_* bits (FP32 bulk tile shapes and launch schedule)
  // dependency waits of the persistent kernel: bound, and a test hook that
  // makes every wait need one completion more than will ever happen
  double wait_limit_ms = 2000.0;
  int wait_never_ready = 0;
  double theta = 0.7;
  int ncells = 0, nleaves = 0, nlevels = 0;
  std::vector<int> level_begin;  // cells of level l: [level_begin[l], level_begin[l+1])
  DeviceArena arena;
  double *x = nullptr;
  int32_t *perm = nullptr;
  double *La64 = nullptr, *Lb64 = nullptr;
  float *La32 = nullptr, *Lb32 = nullptr, *La32lo = nullptr, *Lb32lo = nullptr;
  float4 *off32 = nullptr;
  int32_t *leaf_of = nullptr;
  int32_t *cface = nullptr, *clevel = nullptr, *cbegin = nullptr, *cend = nullptr,
          *cparent = nullptr, *cchild = nullptr;
  int64_t *cia = nullptr, *cib = nullptr;
  double *ccentre = nullptr, *cradius = nullptr, *cxmid = nullptr, *cymid = nullptr,
         *chalf = nullptr, *chy = nullptr;  // box midpoint angles, half-widths along xi, eta
  // shrunk boxes: per-child interpolation matrices [cell][2 axes][p][p]
  // (parent L_k at the child's nodes), FP64 and FP32 rounding + remainder
  double *mcell64 = nullptr;
  float *mcell32 = nullptr;
  double *proxy = nullptr;
  float *proxy32 = nullptr;
  int32_t *loff[4] = {nullptr, nullptr, nullptr, nullptr};
  int32_t *lsrc[4] = {nullptr, nullptr, nullptr, nullptr};
  float4 *ldc[4] = {nullptr, nullptr, nullptr, nullptr};  // FP32 form: per-entry centre differences
  int64_t nlist[4] = {0, 0, 0, 0};
  // target cells that own at least one entry of a list group, for launches
  int32_t *near_targets = nullptr;  // leaves with PP or PC entries
  int n_near_targets = 0;
  int32_t *far_targets = nullptr;   // cells with CP or CC entries
  int n_far_targets = 0;
  int32_t *leaves = nullptr;        // all leaf cells
  // Symmetric near field (FP32 bulk, single right-hand side, K(x,y) = K(y,x)):
  // every PP entry (T, S) with S > T whose mirror (S, T) is also a PP entry is
  // one "cross pair" evaluated once for both directions; its partial sums
  // (rows: T's points, then columns: S's points) live at sym_off[pair] of the
  // workspace's partial buffer.
  int2 *sym_pairs = nullptr;        // [n_sym_pairs] (T, S), T < S
  int32_t *sym_off = nullptr;       // [n_sym_pairs] partial-buffer offset of the pair
  int32_t *sym_contrib = nullptr;   // [nPP] offset of the target leaf's partials of this
                                    // PP entry (-1: evaluated directly)
  int n_sym_pairs = 0;
  int64_t sym_part_len = 0;         // floats in one partial buffer
  // Symmetric far field (FP32 bulk, one right-hand side, K(x,y) = K(y,x)):
  // every CC entry (T, S), S > T, whose mirror (S, T) is also a CC entry is
  // one pair whose P x P kernel matrix serves both; its partial sums (T's
  // proxies, then S's) live at 2 P pair in the workspace's CC partial buffer.
  int2 *cc_pairs = nullptr;         // [n_cc_pairs] (T, S), T < S
  int32_t *cc_entry = nullptr;      // [n_cc_pairs] CC entry index of (T, S)
  int32_t *cc_contrib = nullptr;    // [nCC] offset of the target cell's partials of this entry
                                    // (-1: evaluated directly)
  int n_cc_pairs = 0;
  double *m2m64 = nullptr;
  float *m2m32 = nullptr;
  double *cheb = nullptr;
  int *status = nullptr;
  Workspace *ws = nullptr;          // default workspace
  csfmm_stats stats{};
  // phase timing: a begin and an end event per phase and timed evaluation,
  // recorded on the stream the phase runs on
  bool timing = false;
  std::vector<cudaEvent_t> events;
  int timed_calls = 0;
  int launches = 0;                 // kernels launched by the current evaluation
  csfmm_status phase(int ph, bool begin, cudaStream_t st);

  PlanView view() const;
};

// A captured evaluation of one right-hand-side count, replayed with
// cudaGraphLaunch; only the gather node (reads the caller's weights) and the
// L2P node (writes the caller's output) change between calls.
struct GraphEntry {
  int nrhs = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t gather = nullptr, l2p = nullptr;
  cudaKernelNodeParams gather_params{}, l2p_params{};
  // persistent launch (several right-hand sides): its node takes the output
  cudaGraphNode_t persist = nullptr;
  cudaKernelNodeParams persist_params{};
  PlanView persist_view{};
  PersistArgs persist_args{};
  const double *w = nullptr;
  double *out = nullptr;
  int launches = 0;
};

struct Workspace {
  Workspace() = default;
  Workspace(const Workspace &) = delete;
  Workspace &operator=(const Workspace &) = delete;
  ~Workspace() { release_side(); }
  Plan *plan = nullptr;
  int max_nrhs = 0;
  bool graphs_ok = true;            // false for short-lived workspaces
  std::vector<GraphEntry> graphs;   // captured evaluations (use_graphs)
  void release_graphs() {
    for (GraphEntry &g : graphs) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.graph) cudaGraphDestroy(g.graph);
    }
    graphs.clear();
  }
  DeviceArena arena;
  double *ws = nullptr;     // [max_nrhs][N] weights in tree order
  float *wsf = nullptr;     // [max_nrhs][N] the same in FP32 (FP32 form only)
  double *wbar = nullptr;   // [nc][max_nrhs][P] proxy weights (FP64 form)
  float *wbar32 = nullptr;  // [nc][max_nrhs][P] proxy weights (FP32 form)
  double *psi = nullptr;    // [nc][max_nrhs][dim][P] proxy potentials (FP64 in both forms)
  double *phi = nullptr;    // [max_nrhs][N][dim] near-field potentials, tree order
  float *sym_part = nullptr;     // [plan.sym_part_len] cross-pair partial sums (FP32 form)
  float *cc_part = nullptr;      // [2 P plan.n_cc_pairs] mirrored CC pair partial sums (FP32 form)
  float2 *wtot = nullptr;        // [nc][max_nrhs][2] weight totals (FP32 form)
  int *ctr = nullptr;            // [2 + 3 nc] work counter and dependency counters of the
                                 // persistent kernel (FP32 form, scalar kernels)
  double *stage_w = nullptr;    // device staging for host-buffer evaluations [max_nrhs][N]
  double *stage_out = nullptr;  // [max_nrhs][N][dim]
  int last_nrhs = 0;
  // the last evaluation took the persistent launch with these arguments
  bool last_persistent = false;
  PlanView last_persist_view{};
  PersistArgs last_persist_args{};
  // Second stream of an evaluation: the upward pass, far field and L2L run on
  // it while the near field runs on the caller's stream, joined by events
  // (null for short-lived workspaces, which run every pass in order).
  // side_hi: the same at the device's greatest stream priority
  // (CSFMM_SCHED_SIDE_FIRST).
  cudaStream_t side = nullptr, side_hi = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_up = nullptr, ev_done = nullptr;
  csfmm_status create_side();
  void release_side() {
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_up) cudaEventDestroy(ev_up);
    if (ev_done) cudaEventDestroy(ev_done);
    if (side) cudaStreamDestroy(side);
    if (side_hi) cudaStreamDestroy(side_hi);
    side = side_hi = nullptr;
    ev_fork = ev_up = ev_done = nullptr;
  }
};

}  // namespace csfmm

// The opaque handles of include/csfmm.h wrap one Plan / one Workspace.
struct csfmm_plan_s {
  csfmm::Plan impl;
};
struct csfmm_workspace_s {
  csfmm::Workspace impl;
};

namespace csfmm {

// Tree and list construction (tree.cu).
csfmm_status build_tree(Plan &pl, const double *points, cudaStream_t st);
// Evaluation passes (evaluate.cu).
csfmm_status evaluate_impl(Plan &pl, Workspace &ws, const double *w, int nrhs, double *out,
                           cudaStream_t st);
csfmm_status workspace_alloc(Plan &pl, Workspace &ws, int max_nrhs);
// Tree code (Algorithm "CSTC") on the plan's tree: upward pass, then one
// tree walk per target (evaluate.cu, cstc.cu).
csfmm_status cstc_impl(Plan &pl, Workspace &ws, const double *w, int nrhs, double *out,
                       cudaStream_t st);
void launch_cstc(const PlanView &v, bool f32, double theta, int nroots, int nrhs, int ldr,
                 const double *ws, const float *wsf, const double *wbar, const float *wbar32,
                 double *out, cudaStream_t st);
// FP32-bulk near (far = false) or far (far = true) field for nr = 8 or 16
// right-hand sides from r0, scalar kernels only.
// schedule: the plan's CSFMM_SCHED_* bits (tile shape) (multi32.cu).
void launch_multi32(const PlanView &v, bool far, int ngrid, const int32_t *leaves,
                    const float *wsf, const float *wbar, int ldr, int r0, int nr, double *phi,
                    double *psi, int schedule, cudaStream_t st);
// FP32-bulk far field (interact32.cu): nr <= 4 right-hand sides from r0.
// With cpart != nullptr (one right-hand side) the CC entries that belong to a
// mirrored pair are read from the pairs' partials instead of being evaluated.
void launch_far32(const PlanView &v, int ncells, const float *wsf, const float *wbar, int ldr,
                  int r0, int nr, double *psi, cudaStream_t st, const float *cpart = nullptr);
// Near field of right-hand sides r0 .. r0+15 with the kernel-matrix products
// on the tensor cores (multi_tc.cu; CSFMM_SCHED_TENSOR_NEAR).
void launch_near16_tc(const PlanView &v, int nleaves, const int32_t *leaves, const float *wsf,
                      const float *wbar, int ldr, int r0, double *phi, cudaStream_t st);
// Symmetric CC evaluation of the mirrored far-field pairs (interact32.cu), one
// right-hand side, scalar kernels: proxy weights wbar [nc][ldr][P] in, the
// pairs' partial sums out.
void launch_cc_sym32(const PlanView &v, const int2 *pairs, const int32_t *entry, int npairs,
                     const float *wbar, int ldr, float *part, cudaStream_t st);
// Symmetric PP evaluation of the cross pairs (interact32.cu), one right-hand
// side, scalar kernels; writes the pairs' partial sums into part.
void launch_pp_sym32(const PlanView &v, const int2 *pairs, const int32_t *off, int npairs,
                     const float *wsf, float *part, cudaStream_t st);
// FP32-bulk near field (interact32.cu): nr <= 4 right-hand sides from r0.  With
// part != nullptr (one right-hand side) the PP entries other than the self
// entry are read from the cross-pair partials instead of being evaluated.
void launch_near32(const PlanView &v, const int32_t *leaves, int nleaves, const float *wsf, int ldw,
                   const float *wbar, int ldr, int r0, int nr, double *phi, cudaStream_t st,
                   const float *part = nullptr);
// Persistent multi-right-hand-side launch (persistent.cu).  Eligible: FP32
// bulk, a scalar kernel, nrhs a multiple of the chunk (16 or 8) and a
// workspace with counters; *chunk receives the chunk.
bool persistent_eligible(const Plan &pl, const Workspace &W, int nrhs, int *chunk);
size_t persistent_counter_ints(const Plan &pl);
// Clears the counters and launches the kernel on st (far, near, L2L, L2P of
// all nrhs right-hand sides into out); *used receives its arguments.
csfmm_status launch_persistent(const PlanView &v, const Plan &pl, Workspace &W, int nrhs,
                               int chunk, double *out, cudaStream_t st, PersistArgs *used);
// The kernel function of a plan's persistent launch (graph node lookup).
const void *persistent_function(const Plan &pl, int chunk);
// Direct sum (direct.cu).
csfmm_status direct_impl(const double *points, int64_t N, int kernel_id, const double *w,
                         int nrhs, const int64_t *targets, int64_t ntargets, double *out,
                         int precision, cudaStream_t st);

// Remeshing (remesh.cu): synchronous remeshing of particles x (particle p
// started at grid point p) carrying nfield fields f [nfield][M] onto the grid,
// and the grid's size and points ([M][3], device).
csfmm_status remesh_impl(csfmm_remesh_grid G, const double *x, const double *f, int nfield,
                         double *f_out, cudaStream_t st);
int64_t remesh_grid_size(csfmm_remesh_grid G);
const double *remesh_grid_points(csfmm_remesh_grid G);

// Host helpers shared by the library's own files.
const double *host_tan_table();  // T[k] = tan(k (pi/2)/2^kD - pi/4), k = 0..2^kD
int grid_for(int64_t n, int block, int max_blocks = 1 << 30);
int sm_count();  // streaming multiprocessors of the current device (read once per device)
csfmm_status exclusive_scan_i32(const int32_t *in, int32_t *out, int n, int32_t *total_host,
                                int32_t *tmp, cudaStream_t st);
size_t scan_tmp_elems(int n);
csfmm_status radix_sort_u64(uint64_t *keys, int32_t *vals, uint64_t *keys_alt, int32_t *vals_alt,
                            int n, int begin_bit, int end_bit, int32_t *tmp, size_t tmp_elems,
                            cudaStream_t st, bool *result_in_alt);
size_t radix_tmp_elems(int n);

// SAL kernel in FP64, the bracket of Eq. G_SAL_approx with the Love number fit
// a1 = -2.7, b0 = -6.21196, b1 = 6.1: (1 - b0)/g - (a1 - b1) ln(g/2 + g^2/4),
// g = |x - y| = sqrt(d2).
__device__ __forceinline__ double sal64(double d2) {
  const double g = sqrt(d2), t = 0.5 * g;
  return 7.21196 / g + 8.8 * log(t + t * t);
}

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

// Sphere point of face-plane coordinates (a, b) on face f: q = sqrt((1 + a*a) + b*b),
// x_axis = +-1/q, x_u = a/q, x_v = b/q with u = (axis+1) mod 3, v = (axis+2) mod 3.
// Evaluated with explicit round-to-nearest operations (no fused multiply-add), so the
// result is the same as a host evaluation of the same expression.
__device__ __forceinline__ void face_point_rn(int f, double a, double b, double *x) {
  int ax = f >> 1;
  double sg = (f & 1) ? -1.0 : 1.0;
  int u = ax + 1 == 3 ? 0 : ax + 1;
  int v = u + 1 == 3 ? 0 : u + 1;
  double q = __dsqrt_rn(__dadd_rn(__dadd_rn(1.0, __dmul_rn(a, a)), __dmul_rn(b, b)));
  x[ax] = __ddiv_rn(sg, q);
  x[u] = __ddiv_rn(a, q);
  x[v] = __ddiv_rn(b, q);
}

__device__ __forceinline__ double chord_rn(const double *x, const double *y) {
  double dx = __dsub_rn(x[0], y[0]), dy = __dsub_rn(x[1], y[1]), dz = __dsub_rn(x[2], y[2]);
  return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

// Barycentric weights of the Chebyshev points s_k = cos(k pi/n) (Sec. 4).
__device__ __forceinline__ double bary_w(int k, int n) {
  double w = (k & 1) ? -1.0 : 1.0;
  return (k == 0 || k == n) ? 0.5 * w : w;
}

// L_k(u), k = 0..n, at nodes s (Eq. barycentric); L = delta if u is a node.
__device__ __forceinline__ void lagrange_dev(int n, const double *s, double u, double *L) {
  int hit = -1;
  for (int k = 0; k <= n; ++k)
    if (u == s[k]) hit = k;
  if (hit >= 0) {
    for (int k = 0; k <= n; ++k) L[k] = (k == hit) ? 1.0 : 0.0;
    return;
  }
  double den = 0.0;
  for (int k = 0; k <= n; ++k) {
    L[k] = bary_w(k, n) / (u - s[k]);
    den += L[k];
  }
  double inv = 1.0 / den;
  for (int k = 0; k <= n; ++k) L[k] *= inv;
}

// Unbiased stochastic rounding of x to FP32: the representable neighbour on
// the far side of x is chosen with probability |x - RN(x)| / gap, decided by
// the 24 high bits of the hash h, so the expected value is x.  The FP32
// Lagrange rows use it with a hash of (point, axis, node) and the FP32 centre
// differences of far-field list entries with a hash of (target cell, source
// cell, axis): a uniform grid repeats the same local coordinates in every leaf
// and the same cell offsets along a face, and round-to-nearest would give them
// all the same rounding errors, which then add up instead of averaging out.
__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  // integer finaliser "lowbias32" (C. Wellons, hash-prospector)
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}
// For x in the normal FP32 range the 29 low mantissa bits of the double are
// the part below the FP32 rounding toward zero, as a fraction of its gap, so
// the decision is integer work: round away from zero when 29 bits of the hash
// fall below them.  Other values (zero, FP32 subnormals, overflow) round to
// nearest.
__device__ __forceinline__ float round_stochastic(double x, uint32_t h) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;  // unbiased binary exponent
  if (e < -126 || e > 127) return __double2float_rn(x);
  const uint32_t below = (uint32_t)(b & ((1u << 29) - 1));
  const float t = __double2float_rz(x);
  if ((h >> 3) >= below) return t;
  const uint32_t tb = (uint32_t)__float_as_int(t);
  return __int_as_float((int)(tb + 1u));  // the next FP32 value away from zero
}

// Checked builds (compiled with -DCSFMM_CHECKED, the stand-in for a memory
// checker on this pool): every cell index a kernel takes from a list, a leaf
// table or a child slot is validated before use; a bad one sets the plan's
// status word (CSFMM_ERR_DEVICE from csfmm_plan_sync) and the entry is
// skipped instead of read.  Unchecked builds compile the test away.
#ifdef CSFMM_CHECKED
__device__ __forceinline__ bool cell_ok(const PlanView &v, int c) {
  const bool ok = c >= 0 && c < v.ncells && v.cbegin[c] >= 0 && v.cbegin[c] <= v.cend[c] &&
                  v.cend[c] <= v.N;
  if (!ok) atomicOr(v.status, kStatusInternal);
  return ok;
}
#else
__device__ __forceinline__ bool cell_ok(const PlanView &, int) { return true; }
#endif

constexpr double kInv4Pi = 0.079577471545947667884;  // 1/(4 pi)
constexpr double kInv2Pi = 0.15915494309189533577;   // 1/(2 pi)

}  // namespace csfmm
