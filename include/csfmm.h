/*
 * csfmm.h -- C ABI of the GB300 cubed-sphere fast multipole method (CSFMM).
 *
 * The library evaluates the spherical N-body sum of the midpoint rule
 *     phi(x_i) = sum_{j != i} K(x_i, x_j) w_j ,    i = 1..N          (Sec. 1, Eq. nbodysum)
 * for points x_j on the unit sphere, either directly (csfmm_direct) or with
 * the CSFMM of Chen & Krasny (arXiv 2508.13550): a quadtree of equiangular
 * gnomonic cubed-sphere cells (Sec. 3), barycentric Lagrange interpolation on
 * (n+1)^2 Chebyshev proxy points per cell (Sec. 4), PP/PC/CP/CC interactions
 * chosen by a dual tree traversal with the MAC (r_t + r_s)/R < theta (Sec. 5,
 * Sec. 8, Algorithm "CSFMM"), an upward pass (Sec. 6) and a downward pass
 * (Sec. 8.1).  All work runs in CUDA kernels on one GPU.
 *
 * Conventions for every entry point
 *   - Status: every function returns a csfmm_status and never throws.  The
 *     text of the last error of the calling thread is csfmm_last_error().
 *     Argument errors are detected on the host before any launch.
 *   - Memory: "device" pointers are CUDA global memory of the current
 *     device, owned by the caller; "host" pointers are host memory owned by
 *     the caller.  A plan owns every device buffer it allocates and frees it
 *     in csfmm_plan_destroy.  The library's buffers (plans, workspaces,
 *     remeshing grids, build and step scratch) come from one stream-ordered
 *     memory pool per device that keeps up to 4 GiB of freed memory for
 *     reuse, so repeated plan builds do not go back to the CUDA driver.
 *   - Streams: a stream argument is a cudaStream_t passed as void* (NULL =
 *     the legacy default stream).  Calls marked "asynchronous" only enqueue
 *     work; their inputs and outputs must stay valid until the stream reaches
 *     the end of the call.
 *   - Layout: points are [N][3] row-major FP64 unit vectors.  Weights are
 *     [nrhs][N] FP64 (weight vector r starts at weights + r*N).  Outputs are
 *     [nrhs][N][dim] FP64 in the input order of the points, dim = 3 for the
 *     Biot-Savart kernel, 1 otherwise.
 */
#ifndef CSFMM_H
#define CSFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CSFMM_OK = 0,
  CSFMM_ERR_INVALID_ARG = 1,   /* bad pointer, size, kernel id, degree, theta or leaf size */
  CSFMM_ERR_NOT_ON_SPHERE = 2, /* a point with | |x|^2 - 1 | > 1e-12 (the method assumes x on S^2, Sec. 1) */
  CSFMM_ERR_OUT_OF_MEMORY = 3, /* a device allocation failed; nothing was leaked */
  CSFMM_ERR_CUDA = 4,          /* a CUDA runtime call failed (message in csfmm_last_error) */
  CSFMM_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
  CSFMM_ERR_UNSUPPORTED = 6,   /* valid request outside what this library implements */
  CSFMM_ERR_BUSY = 7,          /* serving: no slot or memory free right now */
  CSFMM_ERR_DEVICE = 8         /* a kernel reported an internal error in the plan's status word */
} csfmm_status;

/* Kernels K(x, y) on the unit sphere (Sec. 2); 1 - x.y is evaluated as
 * |x - y|^2 / 2. */
enum {
  CSFMM_KERNEL_LAPLACE = 0,     /* G_L = -(1/4pi) ln(1 - x.y), Eq. G_L; dim 1 */
  CSFMM_KERNEL_BIOT_SAVART = 1, /* K_BS = -(1/4pi) (x cross y)/(1 - x.y), Eq. K_BS; dim 3 */
  CSFMM_KERNEL_NEWTON = 2,      /* 1/sqrt(2(1 - x.y)) = 1/|x - y|, leading term of Eq. G_SAL_approx; dim 1 */
  CSFMM_KERNEL_BIHARMONIC = 3,  /* G_B = (1/4pi) dilog((1 + x.y)/2), Eq. G_B; dim 1 */
  CSFMM_KERNEL_SAL = 4,         /* (1 - b0)/g - (a1 - b1) ln(g/2 + g^2/4), g = sqrt(2(1 - x.y)):
                                   the bracket of Eq. G_SAL_approx with the paper's Love number
                                   fit a1 = -2.7, b0 = -6.21196, b1 = 6.1; multiply the result by
                                   3 rho_w / (4 pi rho_e) for the SAL potential; dim 1 */
  CSFMM_KERNEL_ONE = 100        /* K = 1, a test kernel (every interpolation is exact) */
};

/* Precision forms. */
enum {
  CSFMM_FP64 = 0,      /* every step in FP64 */
  CSFMM_FP32_BULK = 1  /* kernel evaluations, tile sums and the upward pass in FP32 on
                          pair-relative coordinates; geometry, interpolation weights,
                          proxy potentials, the downward pass (FP64 L2L, double-float
                          L2P) and the final per-target accumulation in FP64 */
};

/* Interaction list types (Sec. 5). */
enum { CSFMM_LIST_PP = 0, CSFMM_LIST_PC = 1, CSFMM_LIST_CP = 2, CSFMM_LIST_CC = 3 };

typedef struct {
  int precision;  /* CSFMM_FP64 (default) or CSFMM_FP32_BULK */
  int max_nrhs;   /* right-hand sides processed per pass; larger nrhs is split (default 16) */
  int use_graphs; /* 1: the first evaluation of each right-hand-side count on a stream other
                     than the legacy default stream is captured into a CUDA graph that later
                     evaluations replay (only the weight and output pointers are updated);
                     evaluations with phase timing enabled are launched directly (default 0) */
  int rhs_chunk;  /* FP32 bulk, scalar kernels: right-hand sides sharing one kernel evaluation
                     in the interaction kernels, 16, 8 or 4 (0 = 16) */
  int shrink;     /* 1: every cell's interpolation box is shrunk to bound its points (Sec. 3;
                     fewer direct pairs on clustered points); 0: the cell's own square
                     (default) */
  int no_persistent; /* FP32 bulk, scalar kernels, nrhs a multiple of 8: 0 (default) evaluates
                     the far field, near field, L2L and L2P of all right-hand sides in one
                     persistent launch whose blocks draw work from a device counter and wait
                     (bounded in time) only for the downward pass's dependencies; the result
                     equals the per-phase launches bit for bit.  1: per-phase launches */
  int schedule;   /* FP32 bulk: OR of CSFMM_SCHED_* bits choosing tile shapes and launch
                     schedule (0 = the defaults); csfmm_autotune searches them */
  int reserved[1];
} csfmm_options;

/* Bits of csfmm_options.schedule (FP32 bulk).  The first three set the tile
 * shape of the per-phase multi-right-hand-side kernels (nrhs of 8 or more
 * without the persistent launch); CHUNK_16 changes the order of the FP32
 * sums and hence the rounding, the others only the work layout. */
enum {
  CSFMM_SCHED_NEAR_64_THREADS = 1,  /* near field: 64 threads per leaf instead of 128 */
  CSFMM_SCHED_ONE_TARGET = 2,       /* one target per thread instead of two */
  CSFMM_SCHED_CHUNK_16 = 4,         /* tile sums in FP32 chunks of 16 sources instead of 32 */
  CSFMM_SCHED_NO_SYMMETRIC = 8,     /* one right-hand side: evaluate every PP entry directly
                                       instead of mirrored leaf pairs once for both directions */
  CSFMM_SCHED_NO_OVERLAP = 16,      /* run every pass in order on the caller's stream instead
                                       of the upward pass, far field and L2L on a side stream */
  CSFMM_SCHED_SIDE_FIRST = 32       /* the side stream at the device's greatest stream priority:
                                       its passes take SMs ahead of the near field's mirrored
                                       pairs, which then absorb them (one RHS at N = 6.3M:
                                       13.08 against 13.17 ms per evaluation; the per-phase
                                       event times then overlap) */,
  CSFMM_SCHED_TENSOR_NEAR = 64      /* 16 right-hand sides at a time, scalar kernel: the near
                                       field's kernel-matrix x weight products on the tensor
                                       cores (warp-level TF32 mma, three products per term) in
                                       per-phase launches instead of the persistent launch.
                                       Measured on 16 RHS, N = 1.57M Poisson: near field 15.8
                                       against 16.9 ms (FP32 pipe, per-phase), error 2.2e-7
                                       against 5.1e-8; not chosen by default or by the tuner */
};

typedef struct csfmm_plan_s *csfmm_plan;

typedef struct {
  int64_t N;
  int kernel_id, degree, max_leaf, precision;
  double theta;
  int32_t nlevels, ncells, nleaves;
  int64_t n_list[4];       /* entries of the PP, PC, CP, CC lists */
  int64_t evals[4];        /* kernel evaluations per evaluate and RHS: PP (self excluded), PC, CP, CC */
  int64_t pairs_covered;   /* sum over list entries of |C_t| |C_s|; equals N^2 */
  double mac_margin;       /* min |(r_t + r_s) - theta R| / (theta R) over MAC tests with R > 0 */
  int64_t device_bytes;    /* device memory held by the plan (including its workspace) */
  double build_ms;         /* wall time of csfmm_plan_create */
  int64_t launches_per_evaluate; /* kernels launched by the last evaluation */
  int64_t sym_pairs;       /* FP32 bulk: PP leaf pairs evaluated once for both directions */
  int64_t sym_evals;       /* kernel evaluations of those pairs (each serves two interactions) */
  int64_t cc_sym_pairs;    /* FP32 bulk, scalar kernel: mirrored CC cell pairs evaluated once
                              for both directions (P^2 kernel values each) */
} csfmm_stats;

/* Evaluation phases timed by csfmm_plan_phase_times.  With the persistent
 * launch (csfmm_options.no_persistent) the NEAR phase covers that whole
 * launch (far field, near field, L2L, L2P) and CCSYM, FAR, PPSYM, L2L, L2P
 * are empty. */
enum {
  CSFMM_PHASE_GATHER = 0, CSFMM_PHASE_P2M = 1, CSFMM_PHASE_M2M = 2, CSFMM_PHASE_FAR = 3,
  CSFMM_PHASE_PPSYM = 4, /* FP32 bulk, one RHS: mirrored PP pairs (empty otherwise) */
  CSFMM_PHASE_NEAR = 5, CSFMM_PHASE_L2L = 6, CSFMM_PHASE_L2P = 7,
  CSFMM_PHASE_CCSYM = 8, /* FP32 bulk, one RHS: mirrored CC pairs, before FAR (empty otherwise) */
  CSFMM_NUM_PHASES = 9
};

/* Builds a plan on the current device: sorts the points into cubed-sphere
 * quadtree order (Sec. 3; a cell with more than max_leaf points splits into
 * its non-empty quadrants), computes cell centres, radii and Chebyshev proxy
 * points (Sec. 4), and the PP/PC/CP/CC lists of the dual tree traversal
 * (Sec. 8, Algorithm "CSFMM").
 *   points    device, [N][3] FP64 unit vectors; copied, may be freed after return
 *   N         >= 1 (< 2^31)
 *   kernel_id a CSFMM_KERNEL_* value
 *   degree    n, 1..16: (n+1)^2 proxies per cell
 *   theta     MAC parameter, 0 < theta < 1 (the paper uses 0.5..0.9)
 *   max_leaf  N0 >= 1
 *   opt       NULL for defaults
 *   stream    work is enqueued on it; the call synchronises it before returning
 *   out       receives the plan handle (NULL on error)
 * Errors: INVALID_ARG, NOT_ON_SPHERE, OUT_OF_MEMORY, CUDA. */
csfmm_status csfmm_plan_create(const double *points, int64_t N, int kernel_id, int degree,
                               double theta, int max_leaf, const csfmm_options *opt,
                               void *stream, csfmm_plan *out);

/* Builds a plan for target points that are not the sources (Sec. 1: the
 * scheme accommodates separate target and source sets): evaluations of it
 * compute phi(y_t) = sum_j K(y_t, x_j) w_j at every target y_t.  One cubed-
 * sphere tree holds the sources and the targets (a cell splits while it holds
 * more than max_leaf points, sources and targets together); the sources carry the
 * weights and the targets weight zero, so the dual traversal, upward pass,
 * interactions and downward pass are those of csfmm_plan_create on the
 * union, and the results are returned at the targets only.  The targets must
 * be distinct from the sources and from each other (a coincident pair makes
 * a singular kernel infinite, as in Eq. nbodysum).
 *   sources device [Ns][3], targets device [Nt][3] FP64 unit vectors (copied)
 *   other arguments as csfmm_plan_create
 * Evaluations of the plan (csfmm_evaluate, _ws, _static, _host, _cstc) take
 * weights [nrhs][Ns] and write out [nrhs][Nt][dim].
 * Errors: those of csfmm_plan_create. */
csfmm_status csfmm_plan_create_targets(const double *sources, int64_t Ns, const double *targets,
                                       int64_t Nt, int kernel_id, int degree, double theta,
                                       int max_leaf, const csfmm_options *opt, void *stream,
                                       csfmm_plan *out);

/* Evaluates phi for nrhs weight vectors with the plan's tree (Algorithm
 * "CSFMM": upward pass, PP/PC/CP/CC interactions, downward pass).
 * Asynchronous on stream.
 *   weights device, [nrhs][N] FP64 in input order
 *   out     device, [nrhs][N][dim] FP64 in input order (fully overwritten)
 * Calls on one plan must not overlap in time (they share its workspace):
 * serialise them on one stream or use csfmm_workspace + csfmm_evaluate_ws.
 * Errors: INVALID_ARG, CUDA, DEVICE (a deferred device status). */
csfmm_status csfmm_evaluate(csfmm_plan plan, const double *weights, int nrhs, double *out,
                            void *stream);

/* Evaluates phi with the cubed sphere tree code instead (Sec. 7, Algorithm
 * "CSTC") on the plan's tree, degree, MAC and precision form: the upward pass
 * (P2M, M2M), then every target particle x_i walks the source tree from the
 * root cells; a cluster C_s with r_s < MAC |x_i - c_s| contributes through
 * its proxies (Eq. PC) if it has children and directly (Eq. PP) otherwise,
 * one that is not well separated passes x_i to its children, and a leaf that
 * is not well separated contributes directly.  O(N log N) work against the
 * CSFMM's O(N); same arguments, layout and asynchrony as csfmm_evaluate, and
 * the same rule against overlapping calls on one plan.
 * Errors: INVALID_ARG, UNSUPPORTED (a tree of more than 18 levels), CUDA,
 * DEVICE. */
csfmm_status csfmm_evaluate_cstc(csfmm_plan plan, const double *weights, int nrhs, double *out,
                                 void *stream);

/* Same as csfmm_evaluate with HOST weights and output: copies the weights
 * to the device, evaluates, copies phi back and synchronises the stream.
 * Pinned host memory makes the copies asynchronous DMA.
 *   weights host, [nrhs][N]; out host, [nrhs][N][dim]. */
csfmm_status csfmm_evaluate_host(csfmm_plan plan, const double *weights, int nrhs, double *out,
                                 void *stream);

/* A workspace holds the per-evaluation buffers (sorted weights, proxy
 * weights, proxy potentials, near-field potentials) for up to max_nrhs
 * right-hand sides, so that evaluations of one plan can run concurrently on
 * different streams.  It must be used with the plan it was made for. */
typedef struct csfmm_workspace_s *csfmm_workspace;
csfmm_status csfmm_workspace_create(csfmm_plan plan, int max_nrhs, csfmm_workspace *out);
csfmm_status csfmm_workspace_destroy(csfmm_workspace ws);
csfmm_status csfmm_evaluate_ws(csfmm_plan plan, csfmm_workspace ws, const double *weights,
                               int nrhs, double *out, void *stream);

/* Evaluation that allocates no device memory.  The paper has no counterpart:
 * this entry point exists for callers that must not call cudaMalloc when they
 * evaluate -- a serving loop whose free device memory is all promised to its
 * admission budget, or a host application whose device memory belongs to its
 * own allocator -- and that need a second evaluation of a plan while the
 * plan's workspace is busy.  It runs the same kernels as csfmm_evaluate on
 * the same data (including the mirrored-pair pass of the FP32-bulk form with
 * one right-hand side) and gives the same result bit for bit; it runs every
 * pass in order on `stream` (csfmm_evaluate overlaps the upward pass and far
 * field with the near field on a second stream).  Its scratch (weights in
 * tree order, proxy weights, proxy potentials, near-field potentials) comes
 * from one static device array of CSFMM_STATIC_SCRATCH_BYTES that every GPU
 * loading the library keeps until the process exits.
 *   plan    a plan of the current device (built earlier, e.g. at start-up)
 *   weights device [nrhs][N]; out device [nrhs][N][dim], both memory of the
 *           plan's device (or managed memory); 1 <= nrhs <= 64
 * Scratch needed, each term rounded up to a multiple of 256 bytes:
 *     8 N nrhs                      weights in tree order
 *   + s ncells nrhs P               proxy weights (s = 8 for CSFMM_FP64, 4 for
 *                                   CSFMM_FP32_BULK)
 *   + 8 ncells nrhs dim P           proxy potentials
 *   + 8 N nrhs dim                  near-field potentials
 * and for CSFMM_FP32_BULK also
 *   + 4 N nrhs                      FP32 weights
 *   + 16 ncells nrhs                per-cell weight totals
 *   + 4 L (nrhs = 1, kernels other than Biot-Savart; L = floats of the
 *          mirrored-pair partial sums, about 2 N times the PP leaf pairs per
 *          leaf that have a mirror)
 *   + 8 P C (nrhs = 1, kernels other than Biot-Savart; C = the mirrored CC
 *          cell pairs, csfmm_stats.cc_sym_pairs)
 *   + 4 (2 + 3 ncells) (kernels other than Biot-Savart: work counters)
 * with N the points of the plan (sources and targets), P = (n+1)^2.  Larger
 * requests fail with CSFMM_ERR_INVALID_ARG and a message that states the
 * size.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress with that device current) and keeps it for the life
 * of the process; make that first call before any stream capture.  A
 * cudaDeviceReset invalidates the kept address as it invalidates plans: do
 * not call this entry point after a reset of the device.  Every call shares
 * the one array, which keeps the last call's contents: calls that overlap on
 * the GPU (other streams, other threads, other plans) race, so serialise
 * them.  Nothing in the array needs clearing between calls (every part is
 * written before it is read).  Asynchronous on stream.
 * Errors: INVALID_ARG (NULL plan, nrhs outside [1, 64], weights or out not
 * memory of the plan's device, a current device other than the plan's, or
 * more scratch than the array holds), CUDA. */
#define CSFMM_STATIC_SCRATCH_BYTES (64u << 20)
csfmm_status csfmm_evaluate_static(csfmm_plan plan, const double *weights, int nrhs, double *out,
                                   void *stream);

/* Direct sum of Eq. (nbodysum) with the i = j term omitted.  Asynchronous.
 *   points  device [N][3]; weights device [nrhs][N]; out device [nrhs][N][dim]
 *   precision CSFMM_FP64 (per-target compensated FP64 sums) or CSFMM_FP32_BULK
 *             (FP32 kernel values on FP64-differenced coordinates, FP64
 *             accumulation across 128-source tiles)
 * When there are few targets the sources are split across thread blocks; the
 * partial sums then live in temporary device memory allocated and freed in
 * stream order (from the library's memory pool) and are reduced in a fixed
 * order, so results are deterministic.
 * Errors: INVALID_ARG, CUDA, OUT_OF_MEMORY. */
csfmm_status csfmm_direct(const double *points, int64_t N, int kernel_id, const double *weights,
                          int nrhs, double *out, int precision, void *stream);

/* Direct sum at a subset of targets: out[r][t][dim] = phi(points[targets[t]]).
 *   targets device int64 [ntargets], each in [0, N). */
csfmm_status csfmm_direct_targets(const double *points, int64_t N, int kernel_id,
                                  const double *weights, int nrhs, const int64_t *targets,
                                  int64_t ntargets, double *out, int precision, void *stream);

/* Autotuner (no counterpart in the paper).  Times real evaluations of the
 * caller's point set (three each after a warm-up, CUDA events) and measures
 * the relative l2 error of the first right-hand side against an FP64 direct
 * sum on up to 256 fixed sampled targets.  Stage 1: maximum leaf sizes N0 in
 * {n^2, 2n^2, 3n^2, 4n^2, 6n^2, 8n^2} (at least 8) with the default schedule.
 * Stage 2, at the best N0 of stage 1: the launch schedule and tile shapes --
 * for the FP32-bulk form with 8 or more right-hand sides (scalar kernels) the
 * persistent launch with right-hand-side chunks of 16 and 8, and the
 * per-phase launches with chunks of 16, 8 and 4 and every tile shape of
 * CSFMM_SCHED_NEAR_64_THREADS | CSFMM_SCHED_ONE_TARGET | CSFMM_SCHED_CHUNK_16;
 * otherwise CSFMM_SCHED_NO_SYMMETRIC (FP32 bulk, one right-hand side) and
 * CSFMM_SCHED_NO_OVERLAP.  It returns the fastest candidate whose error is
 * at most err_factor times the error of the default (N0 = 4 n^2, Sec. 10,
 * and default options).  With a cache path the choice is read from /
 * appended to that text file, keyed by device name, kernel, degree, theta,
 * precision, nrhs and N (csfmm_tune_cache_read).
 *   points device [N][3]; weights device [nrhs][N] (1 <= nrhs <= 64)
 * Synchronous.  Errors: INVALID_ARG, OUT_OF_MEMORY, CUDA. */
typedef struct {
  int max_leaf;          /* chosen N0 */
  int rhs_chunk;         /* chosen csfmm_options.rhs_chunk */
  double ms_per_eval;    /* its evaluation time */
  double rel_err;        /* its error against the FP64 direct sum on the samples */
  double default_ms;     /* the same for N0 = 4 n^2 and default options */
  double default_rel_err;
  int candidates;        /* candidates timed (0 when read from the cache) */
  int from_cache;
  int no_persistent;     /* chosen csfmm_options.no_persistent */
  int schedule;          /* chosen csfmm_options.schedule */
} csfmm_tune_result;
csfmm_status csfmm_autotune(const double *points, int64_t N, int kernel_id, int degree,
                            double theta, const double *weights, int nrhs, int precision,
                            const char *cache_path, double err_factor, csfmm_tune_result *out);

/* Reads a choice from an autotuner cache file (host only, no device work):
 * the last valid line for `key`.  A line is
 *   v2 <key> <max_leaf> <rhs_chunk> <no_persistent> <schedule> <ms_per_eval>
 *      <rel_err> <default_ms> <default_rel_err>
 * with key "<device name>|k<kernel>|n<degree>|t<theta>|p<precision>|r<nrhs>|N<N>"
 * (spaces in the device name replaced by '_').  Lines of another format
 * (stale caches of earlier versions), with values out of range (leaf < 1,
 * chunk not 0/4/8/16, flags not 0/1, schedule bits outside 0..127, times or
 * errors negative or not finite) or cut short are ignored.
 * Returns OK with *out filled (from_cache = 1), or INVALID_ARG (NULL
 * argument; no valid line for key, message "not found"). */
csfmm_status csfmm_tune_cache_read(const char *path, const char *key, csfmm_tune_result *out);

/* Plan statistics (host struct). */
csfmm_status csfmm_plan_stats(csfmm_plan plan, csfmm_stats *stats);

/* Copies plan structures to HOST arrays sized from csfmm_plan_stats, for
 * tests and tools.  Cells are exported in the plan's order:
 *   face, level (int32 [ncells]); ia, ib (int64, integer (xi, eta) cell
 *   coordinates at its level); begin, end (int64, range in tree order);
 *   parent (int32, -1 for roots); child (int32 [ncells][4] by quadrant
 *   2*bit_eta + bit_xi, -1 if empty); centre (FP64 [ncells][3]); radius.
 * Any pointer may be NULL to skip that array. */
csfmm_status csfmm_plan_export_cells(csfmm_plan plan, int32_t *face, int32_t *level, int64_t *ia,
                                     int64_t *ib, int64_t *begin, int64_t *end, int32_t *parent,
                                     int32_t *child, double *centre, double *radius);
/* List entries of one type, grouped by target cell: t[e], s[e] (int32). */
csfmm_status csfmm_plan_export_list(csfmm_plan plan, int list_type, int32_t *t, int32_t *s);
/* Tree order: order[i] = input index of the i-th point in tree order. */
csfmm_status csfmm_plan_export_order(csfmm_plan plan, int64_t *order);
/* Proxy points FP64 [ncells][(n+1)^2][3], proxy index k1*(n+1) + k2. */
csfmm_status csfmm_plan_export_proxies(csfmm_plan plan, double *proxies);
/* Proxy weights after the upward pass of the last evaluation, HOST FP64
 * [ncells][nrhs][(n+1)^2] (first nrhs vectors of that call, nrhs <= its count). */
csfmm_status csfmm_plan_export_proxy_weights(csfmm_plan plan, int nrhs, double *wbar);

/* Phase timing.  While enabled, every evaluation of the plan records a CUDA
 * event before and after each phase on the stream the phase runs on (no
 * synchronisation).  An evaluation runs the upward pass, the far field and
 * L2L on a second stream of its workspace, concurrently with the near field
 * on the caller's stream, so the phase times may add up to more than the
 * evaluation's.  csfmm_plan_phase_times synchronises those events, writes the
 * summed milliseconds per phase into ms[CSFMM_NUM_PHASES] (host), the number
 * of timed evaluations into *calls (calls may be NULL), and clears the
 * record.  For the FAR and NEAR phases the sum covers every launch of the
 * phase in the evaluation.
 * Errors: INVALID_ARG (NULL plan, or NULL ms for csfmm_plan_phase_times), CUDA
 * (an event that failed; the record is cleared all the same). */
csfmm_status csfmm_plan_enable_timing(csfmm_plan plan, int on);
csfmm_status csfmm_plan_phase_times(csfmm_plan plan, double *ms, int64_t *calls);

/* ------------------------------------------------------------------------
 * Serving (continuous batching).  No counterpart in the paper: a request
 * loop that keeps plans resident on the device, admits requests as slots and
 * device memory free up, and runs admitted evaluations concurrently on
 * separate streams.
 *
 * A request names a point set by the caller's key (plan_key, e.g. the grid
 * size) plus its method parameters; plans are cached by (plan_key, kernel_id,
 * degree, theta, max_leaf, precision) and built from `points` the first time.
 * A request starts when a slot is free and the memory it needs (its plan if
 * not cached, plus a workspace for up to CSFMM_SERVER_MAX_NRHS right-hand
 * sides if none is idle) fits in hbm_budget_bytes next to what is held; idle
 * cached plans are evicted (least recently used) to make room.  Which pending
 * request starts next is set by csfmm_server_set_policy.  Plans are built
 * with use_graphs = 1.
 * ------------------------------------------------------------------------ */
#define CSFMM_SERVER_MAX_NRHS 8
typedef struct csfmm_server_s *csfmm_server;

typedef struct {
  const double *points;  /* device [N][3]; read only when the plan is built */
  int64_t N;
  uint64_t plan_key;     /* caller's identity of the point set */
  int kernel_id, degree, max_leaf, precision;
  double theta;
  const double *weights; /* device [nrhs][N], valid until the request completes */
  int nrhs;              /* 1 .. CSFMM_SERVER_MAX_NRHS */
  double *out;           /* device [nrhs][N][dim], written by the request */
} csfmm_request;

typedef struct {
  int status;            /* csfmm_status of the request */
  double submit_ms;      /* host clock (ms since the server was created) at submit */
  double admit_ms;       /* ... when its evaluation was enqueued */
  double done_ms;        /* ... when the scheduler saw its completion event */
  double gpu_ms;         /* CUDA-event time of the evaluation on its slot stream */
  int slot;              /* slot (stream) that ran it */
  int built_plan;        /* 1 if the request built its plan */
} csfmm_request_timing;

typedef struct {
  int64_t submitted, completed, failed, plans_built, plans_evicted;
  int64_t bytes_held, peak_bytes_held, budget_bytes;
  int slots, max_in_flight;
} csfmm_server_stats;

/* Creates a server on the current device with `slots` concurrent evaluation
 * slots (1..64) and a device-memory budget for plans and workspaces.
 * Errors: INVALID_ARG, CUDA. */
csfmm_status csfmm_server_create(int64_t hbm_budget_bytes, int slots, csfmm_server *out);
/* Admission order.  CSFMM_SERVE_FIFO: first come first served (the oldest
 * pending request starts, or nothing does while it does not fit).
 * CSFMM_SERVE_CHEAPEST_FIRST (the default): the pending request with the
 * smallest estimated cost N (4 + nrhs) (n+1)^2 starts first, except that a
 * request pending for more than age_ms milliseconds (default 250) goes
 * first whatever its cost, and requests of at least 2^20 points occupy at
 * most half of the slots (at least one); a smaller request runs on a
 * high-priority stream of its slot with all its passes on that stream (its
 * plan is built with CSFMM_SCHED_NO_OVERLAP), so its kernels are scheduled
 * ahead of waiting blocks of large requests.  Results do not depend on the
 * policy.  Errors: INVALID_ARG (NULL server, unknown policy, age_ms <= 0). */
enum { CSFMM_SERVE_FIFO = 0, CSFMM_SERVE_CHEAPEST_FIRST = 1 };
csfmm_status csfmm_server_set_policy(csfmm_server s, int policy, double age_ms);
/* Queues a request (copied; the buffers it points to must stay valid until
 * it completes) and returns its id.  Never blocks.  Errors: INVALID_ARG;
 * OUT_OF_MEMORY if the request alone can never fit the budget. */
csfmm_status csfmm_server_submit(csfmm_server s, const csfmm_request *req, int64_t *id);
/* *done = 1 and *timing filled when request id has completed (or failed). */
csfmm_status csfmm_server_poll(csfmm_server s, int64_t id, int *done, csfmm_request_timing *timing);
/* Blocks until request id completes; returns its status. */
csfmm_status csfmm_server_wait(csfmm_server s, int64_t id, csfmm_request_timing *timing);
/* Blocks until every submitted request has completed. */
csfmm_status csfmm_server_drain(csfmm_server s);
csfmm_status csfmm_server_stats_get(csfmm_server s, csfmm_server_stats *stats);
/* Drains, then frees every plan, workspace and stream of the server. */
csfmm_status csfmm_server_destroy(csfmm_server s);

/* One fourth-order Runge-Kutta step of the barotropic vorticity equation on
 * a sphere rotating at angular frequency omega about the z axis, by the
 * vortex method of Sec. 2.3 (Eq. BVE_ODEs): particle i at x_i with relative
 * vorticity zeta_i and fixed area A_i moves with
 *     dx_i/dt = sum_j K_BS(x_i, x_j) zeta_j A_j   (Eq. K_BS, j != i)
 * and dzeta_i/dt = -2 omega dz_i/dt, so that zeta + 2 omega z is carried by
 * each particle (Eq. BVE).  Every one of the four stages evaluates the
 * velocity at that stage's positions: with degree > 0 a CSFMM plan is built
 * there (csfmm_plan_create with the given degree, theta, max_leaf and
 * precision form) and evaluated once; with degree == 0 the velocity is the
 * direct sum (csfmm_direct in the given precision form).  The stage
 * positions and the result are projected back onto the unit sphere, on
 * which K_BS is defined.  The remeshing that the paper applies after each
 * step is not part of this call.
 *   x, zeta, area  device FP64 [N][3] unit vectors, [N], [N]
 *   dt             time step (> 0), in the time unit of 1/omega
 *   x_out, zeta_out device [N][3], [N]: the state at t + dt, in input order;
 *                  may be x and zeta themselves (an in-place step)
 * Stage scratch (9 N doubles) is allocated and freed in stream order (from
 * the library's memory pool).  Each plan build synchronises the
 * stream, so the call returns after its last plan evaluation; the final
 * update is still enqueued on stream when it returns.
 * Errors: INVALID_ARG, NOT_ON_SPHERE, OUT_OF_MEMORY, CUDA, DEVICE, TIMEOUT. */
csfmm_status csfmm_bve_step(const double *x, const double *zeta, const double *area, int64_t N,
                            double dt, double omega, int degree, double theta, int max_leaf,
                            int precision, double *x_out, double *zeta_out, void *stream);

/* Remeshing onto a fixed grid (Sec. 12 remeshes the vortex method at every
 * time step by local interpolation).  A remeshing grid holds M grid points g_k
 * (the particles' home positions, e.g. icosahedral cell centres) and the
 * neighbour lists of their triangulation, which must be the Delaunay
 * triangulation of the points (the convex hull; the refined icosahedron is
 * one).  csfmm_remesh maps M moved particles, particle p having started at
 * g_p, carrying values f_p, to values at the grid points: with h_k the chord
 * from g_k to its nearest neighbour and (u, v) the gnomonic coordinates of a
 * particle x (x.g_k > 0) in the tangent plane at g_k divided by h_k,
 * s^2 = u^2 + v^2, the particles with s < 2.2 are fitted with weights
 * (1 - s^2/2.2^2)^4 by c0 + c1 u + c2 v + c3 u^2 + c4 uv + c5 v^2 (least
 * squares) and f_out[k] = c0.  The fit reproduces quadratics in (u, v)
 * exactly, is third-order accurate for smooth data and depends continuously
 * on the particle positions.  The particles are found through their nearest
 * grid points (a greedy walk on the triangulation from g_p) and per-point
 * stencils made when the grid is made: the triangulation rings about g_k that
 * hold its data disc, less the cells whose grid point is farther from g_k
 * than the disc's chord plus the cell's own radius (the chord to its farthest
 * Voronoi vertex, a circumcentre of the triangles at the cell's point).
 *   grid         device [M][3] FP64 unit vectors (copied), 7 <= M < 2^30
 *   adj_offsets  device int64 [M+1], adj device int64 [adj_offsets[M]]: the
 *                neighbours of g_k are adj[adj_offsets[k] .. adj_offsets[k+1])
 *                (read during the call only)
 * create is synchronous.  Errors: INVALID_ARG (bad neighbour lists, a grid so
 * irregular that 8 rings do not hold a data disc), NOT_ON_SPHERE,
 * OUT_OF_MEMORY, CUDA. */
typedef struct csfmm_remesh_grid_s *csfmm_remesh_grid;
csfmm_status csfmm_remesh_grid_create(const double *grid, int64_t M, const int64_t *adj_offsets,
                                      const int64_t *adj, void *stream, csfmm_remesh_grid *out);
/*   x device [M][3] moved particles; f device [nfield][M] values carried by
 *   them (1 <= nfield <= 64, e.g. vorticity and tracers; all fields share the
 *   cells, stencils and fit matrix); f_out device [nfield][M], not
 *   overlapping f (INVALID_ARG).
 * Allocates nothing; synchronises the stream before returning (it reads the
 * grid's status word).  Calls on one grid must not overlap.
 * Errors: INVALID_ARG, CUDA, DEVICE (a walk that did not end, a cell holding
 * more than 4096 particles, a data disc with fewer than 6 particles or a
 * singular fit). */
csfmm_status csfmm_remesh(csfmm_remesh_grid grid, const double *x, const double *f, int nfield,
                          double *f_out, void *stream);
csfmm_status csfmm_remesh_grid_destroy(csfmm_remesh_grid grid);

/* One remeshed step of the vortex method (Sec. 12): csfmm_bve_step from the
 * grid points with vorticity zeta, then csfmm_remesh of the moved particles
 * onto the grid.  A passive tracer q (Sec. 12, dq/dt = 0 along particle
 * paths) rides on the same particles and is remeshed with the vorticity.
 * grid_plan, if not NULL, is a Biot-Savart plan built on the grid's points
 * (the first RK4 stage always starts there, so one plan serves every step;
 * that stage then uses the plan's own degree, MAC, leaf size and precision);
 * NULL builds one per step like the other stages.
 *   zeta, area device [M]; zeta_out device [M] (may be zeta)
 *   tracer, tracer_out device [M] (may be the same array), or both NULL
 * Synchronous.  Errors: those of csfmm_bve_step and csfmm_remesh. */
csfmm_status csfmm_bve_step_remeshed(csfmm_remesh_grid grid, csfmm_plan grid_plan,
                                     const double *zeta, const double *tracer, const double *area,
                                     double dt, double omega, int degree, double theta,
                                     int max_leaf, int precision, double *zeta_out,
                                     double *tracer_out, void *stream);

/* Waits for the plan's work on stream and returns a deferred device status
 * (CSFMM_ERR_DEVICE / CSFMM_ERR_TIMEOUT) if a kernel reported one.  A
 * timeout is reported once (the status is cleared, the plan stays usable);
 * the outputs of the evaluation that timed out are incomplete. */
csfmm_status csfmm_plan_sync(csfmm_plan plan, void *stream);

/* Dependency waits of the persistent launch (see csfmm_options.no_persistent):
 * every wait gives up after limit_ms milliseconds of wall time (default
 * 2000), sets the plan's status word and makes the other waits of the launch
 * give up at once, so that the kernel returns and csfmm_plan_sync reports
 * CSFMM_ERR_TIMEOUT.  never_ready = 1 is a test hook: every wait then needs
 * one completion more than will ever happen, so that a test can check the
 * timeout path without a fault; evaluations of such a plan are incomplete.
 * The setting applies to evaluations launched afterwards (not to a CUDA graph
 * captured earlier).
 * Errors: INVALID_ARG (NULL plan, limit_ms outside (0, 60000]). */
csfmm_status csfmm_plan_test_wait(csfmm_plan plan, int never_ready, double limit_ms);

/* Frees every device buffer of the plan.  The caller must make sure no work
 * of the plan is still running. */
csfmm_status csfmm_plan_destroy(csfmm_plan plan);

/* Thread-local text of the last error (never NULL). */
const char *csfmm_last_error(void);

/* Library version string. */
const char *csfmm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CSFMM_H */
