// persistent.cu -- one persistent launch for the interactions and the
// downward pass of a multi-right-hand-side FP32-bulk evaluation.
//
// After the gather and the upward pass (P2M, M2M: every proxy weight is then
// final), a single kernel evaluates every remaining piece of Algorithm
// "CSFMM" for all nrhs = nch x NR right-hand sides.  Its blocks stay resident
// and draw items from one device work counter, in this order:
//   far   (cell, chunk): CP and CC proxy potentials (Sec. 5, Eqs. CP, CC);
//         with P <= 128 one item holds two cells, one per half block
//   near  (leaf, chunk): PP and PC potentials at the particles (Eqs. PP, PC)
//   L2L   (cell): proxy potentials passed to the children (Sec. 8.1, Eq.
//         downward_2), all right-hand sides; the cells of level l follow the
//         first (l + 1)/(2 L) of the near items (L = L2L levels), so that
//         their parents' items finished long before and the downward chain
//         runs while other blocks work on the near field
//   L2P   (leaf): interpolation to the particles plus the near field, output
//         in input order (Algorithm "CSFMM", downward pass), after all
// Every piece of work is independent in the paper's sense (Sec. 11.3: each
// interaction is its own direct sum); the only dependencies are those of the
// downward pass, tracked by per-cell counters that an item raises (release)
// when its results are written and that later items wait for (acquire):
//   L2L(c)  waits for far(c), far(children of c) and L2L(parent of c);
//   L2P(l)  waits for near(l), far(l) and L2L(parent of l).
// An item only waits for items earlier in the queue, which were taken by
// blocks that are running, so the launch cannot deadlock whatever the number
// of resident blocks.  Every wait is bounded in time: a wait that runs out
// sets the plan's status word (timeout) and an abort flag, after which every
// other wait gives up at once and the kernel returns; the host reports
// CSFMM_ERR_TIMEOUT from csfmm_plan_sync.  Data written by another block in
// the same launch (proxy potentials, near-field potentials) is read with
// L2-coherent loads in downward_df.cuh.
//
// The item functions are those of the per-phase kernels (multi32.cuh,
// downward_df.cuh) with the same per-target operation order, so a persistent
// evaluation equals the per-phase launches bit for bit.
#include <algorithm>
#include <mutex>

#include "csfmm_internal.cuh"
#include "downward_df.cuh"
#include "fp32_math.cuh"
#include "multi32.cuh"

namespace csfmm {

namespace {

constexpr int kPersistThreads = CSFMM_MULTI_THREADS;
static_assert(kPersistThreads == kL2PThreads, "L2P items need kL2PThreads threads");
static_assert(kPersistThreads % 64 == 0, "far items may split the block into two halves");

// Shared memory of one multi-right-hand-side group (staged sources).
template <int NR>
constexpr int group_bytes() {
  return kMultiTile * (int)sizeof(float4) + (NR / 4) * kMultiTile * (int)sizeof(ulonglong2);
}
template <int NR>
constexpr int persist_smem_bytes() {
  return std::max(std::max(2 * group_bytes<NR>(), kL2PDfSmemFloats * 4), kL2LDfSmemFloats * 4);
}

__device__ __forceinline__ long long globaltimer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int load_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void add_release(int *p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One thread waits until *flag >= target.  Returns false if the wait ran
// out (then the status word and the abort flag are set) or if another wait
// had already run out.
__device__ bool wait_at_least(const PersistArgs &a, int *status, const int *flag, int target) {
  if (load_acquire(flag) >= target) return true;
  const long long t0 = globaltimer_ns();
  const volatile int *abort_flag = a.ctr + 1;
  while (true) {
    if (*abort_flag) return false;
    __nanosleep(256);
    if (load_acquire(flag) >= target) return true;
    if (globaltimer_ns() - t0 > a.limit_ns) {
      atomicExch(a.ctr + 1, 1);
      atomicOr(status, kStatusTimeout);
      return false;
    }
  }
}

// Item of queue position it: (kind, index) with kind 0 far, 1 near, 2 L2L
// (index = cell), 3 L2P (index into the leaf list).
__device__ __forceinline__ int2 decode_item(const PersistArgs &a, int it) {
  if (it < a.nfar) return make_int2(0, it);
  int pos = it - a.nfar, prev = 0;
  for (int l = 0; l < a.nlev; ++l) {
    const int span = a.ins[l] - prev;
    if (pos < span) return make_int2(1, prev + pos);
    pos -= span;
    const int nl = a.lvl_begin[l + 1] - a.lvl_begin[l];
    if (pos < nl) return make_int2(2, a.lvl_begin[l] + pos);
    pos -= nl;
    prev = a.ins[l];
  }
  if (pos < a.nnear - prev) return make_int2(1, prev + pos);
  return make_int2(3, pos - (a.nnear - prev));
}

// Raises a counter once every thread of the group (barrier bar, nth threads)
// has written its results.
__device__ __forceinline__ void signal_done(int *flag, int tid, int bar, int nth) {
  group_sync(bar, nth);
  if (tid == 0) {
    __threadfence();
    add_release(flag, 1);
  }
}

template <int KID, int NR, int PC>
__global__ void __launch_bounds__(kPersistThreads, 3) persistent_kernel(PlanView v, PersistArgs a) {
  __shared__ __align__(16) unsigned char smem[persist_smem_bytes<NR>()];
  __shared__ int s_item, s_ok;
  int *far_done = a.ctr + 2;
  int *l2l_done = far_done + a.ncells;
  int *near_done = l2l_done + a.ncells;
  const int x = a.extra;
  while (true) {
    __syncthreads();  // the previous item no longer reads shared memory or s_item
    if (threadIdx.x == 0) s_item = atomicAdd(a.ctr, 1);
    __syncthreads();
    if (s_item >= a.total) return;
    const int2 item = decode_item(a, s_item);
    const int it = item.y;
    if (item.x == 0) {  // far field of one cell (or two) and one chunk
      const int r0 = (it % a.nch) * NR;
      const int half = a.far_pair ? (int)(threadIdx.x >> 6) : 0;
      const int c = a.far_pair ? 2 * (it / a.nch) + half : it / a.nch;
      const int tid = a.far_pair ? (int)(threadIdx.x & 63) : (int)threadIdx.x;
      const int nth = a.far_pair ? 64 : kPersistThreads;
      const int bar = a.far_pair ? 1 + half : 0;
      unsigned char *g = smem + half * group_bytes<NR>();
      if (c < a.ncells) {
        multi32_item<KID, NR, true>(v, c, a.wsf, a.wbar, a.ldr, r0, a.phi, a.psi,
                                    reinterpret_cast<float4 *>(g),
                                    reinterpret_cast<ulonglong2 *>(g + kMultiTile * sizeof(float4)),
                                    tid, nth, bar);
        signal_done(far_done + c, tid, bar, nth);
      }
      continue;
    }
    if (item.x == 1) {  // near field of one leaf and one chunk
      const int leaf = a.leaves[it / a.nch], r0 = (it % a.nch) * NR;
      multi32_item<KID, NR, false>(v, leaf, a.wsf, a.wbar, a.ldr, r0, a.phi, a.psi,
                                   reinterpret_cast<float4 *>(smem),
                                   reinterpret_cast<ulonglong2 *>(smem + kMultiTile * sizeof(float4)),
                                   threadIdx.x, kPersistThreads, 0);
      signal_done(near_done + leaf, threadIdx.x, 0, kPersistThreads);
      continue;
    }
    if (item.x == 2) {  // L2L from cell c to its children, all right-hand sides
      const int c = it;
      const int32_t *ch = v.cchild + 4 * c;
      if (ch[0] < 0 && ch[1] < 0 && ch[2] < 0 && ch[3] < 0) continue;  // a leaf
      if (threadIdx.x == 0) {
        bool ok = wait_at_least(a, v.status, far_done + c, a.nch + x);
        const int par = v.cparent[c];
        if (ok && par >= 0) ok = wait_at_least(a, v.status, l2l_done + par, 1 + x);
        for (int q = 0; q < 4; ++q)
          if (ok && ch[q] >= 0) ok = wait_at_least(a, v.status, far_done + ch[q], a.nch + x);
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok) continue;
      l2l_df_cell(v, c, 0, a.nrhs, 1, a.psi, a.ldr, reinterpret_cast<float *>(smem));
      signal_done(l2l_done + c, threadIdx.x, 0, kPersistThreads);
      continue;
    }
    {  // L2P of one leaf, all right-hand sides
      const int leaf = a.leaves[it];
      if (threadIdx.x == 0) {
        bool ok = wait_at_least(a, v.status, near_done + leaf, a.nch + x);
        if (ok) ok = wait_at_least(a, v.status, far_done + leaf, a.nch + x);
        const int par = v.cparent[leaf];
        if (ok && par >= 0) ok = wait_at_least(a, v.status, l2l_done + par, 1 + x);
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok) continue;
      l2p_df_leaf<PC>(v, leaf, a.psi, a.ldr, a.nrhs, 1, a.phi, a.out,
                      reinterpret_cast<float *>(smem));
    }
  }
}

template <int KID, int NR>
const void *pick_pc(int p) {
  switch (p) {
    case 11: return (const void *)persistent_kernel<KID, NR, 11>;
    case 13: return (const void *)persistent_kernel<KID, NR, 13>;
    default: return (const void *)persistent_kernel<KID, NR, 0>;
  }
}

template <int KID>
const void *pick_nr(int nr, int p) {
  return nr == 16 ? pick_pc<KID, 16>(p) : pick_pc<KID, 8>(p);
}

// Resident blocks per SM of a kernel function, computed once per function.
int blocks_per_sm(const void *f) {
  static std::mutex mu;
  static const void *fn[64] = {};
  static int occ[64] = {};
  std::lock_guard<std::mutex> lk(mu);
  int k = 0;
  for (; k < 64 && fn[k]; ++k)
    if (fn[k] == f) return occ[k];
  int o = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, f, kPersistThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (k < 64) {
    fn[k] = f;
    occ[k] = o;
  }
  return o;
}

}  // namespace

bool persistent_eligible(const Plan &pl, const Workspace &W, int nrhs, int *chunk) {
  if (pl.precision == CSFMM_FP64 || pl.kernel_id == CSFMM_KERNEL_BIOT_SAVART ||
      pl.no_persistent || (pl.schedule & CSFMM_SCHED_TENSOR_NEAR) || !W.ctr ||
      W.wsf == nullptr || W.wbar32 == nullptr)
    return false;
  if (nrhs % 16 == 0 && pl.rhs_chunk >= 16) *chunk = 16;
  else if (nrhs % 8 == 0 && pl.rhs_chunk >= 8) *chunk = 8;
  else return false;
  return nrhs >= *chunk;
}

size_t persistent_counter_ints(const Plan &pl) { return 2 + 3 * (size_t)pl.ncells; }

const void *persistent_function(const Plan &pl, int chunk) {
  switch (pl.kernel_id) {
    case CSFMM_KERNEL_LAPLACE: return pick_nr<CSFMM_KERNEL_LAPLACE>(chunk, pl.p);
    case CSFMM_KERNEL_NEWTON: return pick_nr<CSFMM_KERNEL_NEWTON>(chunk, pl.p);
    case CSFMM_KERNEL_SAL: return pick_nr<CSFMM_KERNEL_SAL>(chunk, pl.p);
    case CSFMM_KERNEL_BIHARMONIC: return pick_nr<CSFMM_KERNEL_BIHARMONIC>(chunk, pl.p);
    case CSFMM_KERNEL_ONE: return pick_nr<CSFMM_KERNEL_ONE>(chunk, pl.p);
  }
  return nullptr;
}

csfmm_status launch_persistent(const PlanView &v, const Plan &pl, Workspace &W, int nrhs,
                               int chunk, double *out, cudaStream_t st, PersistArgs *used) {
  const void *f = persistent_function(pl, chunk);
  if (!f) {
    set_error("no persistent kernel for kernel id %d", pl.kernel_id);
    return CSFMM_ERR_INVALID_ARG;
  }
  PersistArgs a{};
  a.leaves = pl.leaves;
  a.nleaves = pl.nleaves;
  a.ncells = pl.ncells;
  a.nl2l = pl.nlevels >= 2 ? pl.level_begin[pl.nlevels - 1] : 0;
  a.nlev = pl.nlevels >= 2 ? pl.nlevels - 1 : 0;
  for (int l = 0; l <= a.nlev; ++l) a.lvl_begin[l] = pl.level_begin[l];
  a.nch = nrhs / chunk;
  a.nrhs = nrhs;
  a.ldr = W.max_nrhs;
  a.far_pair = pl.P <= 64 * CSFMM_MULTI_NT ? 1 : 0;
  a.nfar = (a.far_pair ? (pl.ncells + 1) / 2 : pl.ncells) * a.nch;
  a.nnear = pl.nleaves * a.nch;
  a.total = a.nfar + a.nnear + a.nl2l + pl.nleaves;
  for (int l = 0; l < a.nlev; ++l)
    a.ins[l] = (int)((int64_t)a.nnear * (l + 1) / (2 * a.nlev));
  a.wsf = W.wsf;
  a.wbar = W.wbar32;
  a.phi = W.phi;
  a.psi = W.psi;
  a.out = out;
  a.ctr = W.ctr;
  a.extra = pl.wait_never_ready ? 1 : 0;
  a.limit_ns = (long long)(pl.wait_limit_ms * 1e6);
  const int occ = blocks_per_sm(f);
  if (occ < 1) {
    set_error("the persistent kernel cannot be resident on this device");
    return CSFMM_ERR_CUDA;
  }
  const int grid = std::min(a.total, sm_count() * occ);
  CSFMM_CUDA(cudaMemsetAsync(W.ctr, 0, sizeof(int) * persistent_counter_ints(pl), st));
  PlanView vv = v;
  void *args[] = {(void *)&vv, (void *)&a};
  CSFMM_CUDA(cudaLaunchKernel(f, dim3(grid), dim3(kPersistThreads), args, 0, st));
  if (used) *used = a;
  return CSFMM_OK;
}

}  // namespace csfmm
