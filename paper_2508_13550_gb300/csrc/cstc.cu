// cstc.cu -- the cubed sphere tree code (Sec. 7, Algorithm "CSTC") on a built
// plan: after the upward pass of the evaluation (gather, P2M, M2M; Sec. 6),
// every target particle x_i walks the source tree from the root cells.  A
// cluster C_s that is well separated from x_i (r_s < MAC R, R the chord from
// x_i to the centre of C_s) contributes through its proxies by Eq. (PC) if it
// has children (more than N0 particles) and directly by Eq. (PP) otherwise; a
// cluster that is not well separated passes x_i on to its children, and a
// leaf that is not well separated contributes directly.
//
// GPU layout: one warp per 32 consecutive targets in tree order (neighbours,
// so their walks mostly coincide).  The warp walks the tree together with a
// shared stack of (cell, lane mask) entries; each lane takes its own decision
// for every cell in its mask with the same FP64 arithmetic (no FMA) as the
// oracle, so the interactions of each target are exactly the algorithm's.
// Lanes that need the children of a cell push them with their mask; lanes
// that chose PC or PP evaluate the cell while the others idle.
//
// Two precision forms: FP64 throughout, and FP32 kernel evaluations on
// pair-relative coordinates (x_i - c_s formed in FP64 and rounded once; proxy
// and particle offsets from the cell centre in FP32) with per-lane FP32
// (hi, lo) two-sum totals, like the FP32-bulk CSFMM kernels.
#include <math.h>

#include "csfmm_internal.cuh"
#include "dilog.cuh"
#include "fp32_math.cuh"

namespace csfmm {

namespace {

constexpr int kCstcWarps = 4;
constexpr int kCstcThreads = 32 * kCstcWarps;
// Depth-first stack bound: the roots, then at most 3 more entries per level
// (a popped cell pushes up to 4 children) over kMaxLevels levels.
constexpr int kMaxLevels = 18;
constexpr int kCstcStack = 64;
static_assert(6 + 3 * kMaxLevels + 4 <= kCstcStack, "tree walk stack");

__device__ __forceinline__ double chord_rn(double x0, double x1, double x2, const double *c) {
  const double dx = __dsub_rn(x0, c[0]), dy = __dsub_rn(x1, c[1]), dz = __dsub_rn(x2, c[2]);
  return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

// FP64 kernel term added to acc: Laplace -(1/4pi) ln(d2/2) w, Newtonian
// w / d, biharmonic dilog(1 - d2/4) w (times 1/4pi at the end), K = 1: w;
// Biot-Savart accumulates w r / d2 (r = x - y), crossed with x at the end
// (x cross y = -x cross r for unit vectors).
template <int KID>
__device__ __forceinline__ void term64(double rx, double ry, double rz, double w,
                                       double (&acc)[3]) {
  const double d2 = rx * rx + ry * ry + rz * rz;
  if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
    acc[0] += -kInv4Pi * log(0.5 * d2) * w;
  } else if constexpr (KID == CSFMM_KERNEL_NEWTON) {
    acc[0] += rsqrt(d2) * w;
  } else if constexpr (KID == CSFMM_KERNEL_BIHARMONIC) {
    acc[0] += dilog64(1.0 - 0.25 * d2) * w;  // (1/4pi) applied at the end
  } else if constexpr (KID == CSFMM_KERNEL_SAL) {
    acc[0] += sal64(d2) * w;
  } else if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) {
    const double g = w / d2;
    acc[0] += g * rx;
    acc[1] += g * ry;
    acc[2] += g * rz;
  } else {
    acc[0] += w;
  }
}

// FP32 kernel term: the sum of w f(d2) over a chunk of sources, with
// f = log2 d2 (Laplace), 1/d (Newtonian), dilog(1 - d2/4) (biharmonic),
// 1/d2 times r (Biot-Savart), 1.
template <int KID>
__device__ __forceinline__ void term32(float rx, float ry, float rz, float w, float (&acc)[3]) {
  const float d2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
  const float f = kfactor<KID>(d2);
  if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) {
    const float g = w * f;
    acc[0] = fmaf(g, rx, acc[0]);
    acc[1] = fmaf(g, ry, acc[1]);
    acc[2] = fmaf(g, rz, acc[2]);
  } else {
    acc[0] = fmaf(w, f, acc[0]);
  }
}

template <int KID, bool F32>
__global__ void __launch_bounds__(kCstcThreads) cstc_kernel(PlanView v, double theta, int nroots,
                                                            int r, int ldr, const double *ws,
                                                            const float *wsf, const double *wbar,
                                                            const float *wbar32, double *out) {
  constexpr int D = KID == CSFMM_KERNEL_BIOT_SAVART ? 3 : 1;
  __shared__ int2 stack[kCstcWarps][kCstcStack];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t N = v.N;
  const int64_t i = ((int64_t)blockIdx.x * kCstcWarps + wid) * 32 + lane;
  const bool act = i < N;
  const unsigned amask = __ballot_sync(0xffffffffu, act);
  if (amask == 0) return;  // the whole warp is past the last target
  const int64_t ii = act ? i : N - 1;
  const double x0 = v.x[ii], x1 = v.x[N + ii], x2 = v.x[2 * N + ii];
  const int P = v.P;
  int2 *stk = stack[wid];
  double acc64[3] = {0.0, 0.0, 0.0};
  float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
  int sp = 0;
  for (int c = nroots - 1; c >= 0; --c, ++sp)
    if (lane == 0) stk[sp] = make_int2(c, (int)amask);
  __syncwarp();
  while (sp > 0) {
    --sp;
    const int2 top = stk[sp];
    __syncwarp();  // every lane has read the entry before it is overwritten
    const int c = top.x;
    const bool in = ((unsigned)top.y >> lane) & 1u;
    const double *cc = v.ccentre + 3 * (int64_t)c;
    const double R = chord_rn(x0, x1, x2, cc);
    const bool sep = v.cradius[c] < __dmul_rn(theta, R);
    const int32_t *ch = v.cchild + 4 * (int64_t)c;
    const bool internal = ch[0] >= 0 || ch[1] >= 0 || ch[2] >= 0 || ch[3] >= 0;
    const unsigned rec = __ballot_sync(0xffffffffu, in && internal && !sep);
    const bool pc = in && internal && sep;
    const bool pp = in && !internal;
    if (rec) {
      if (sp + 4 > kCstcStack) {  // cannot happen for trees of <= kMaxLevels levels
        if (lane == 0) atomicOr(v.status, kStatusOverflow);
        break;
      }
      for (int q = 3; q >= 0; --q)
        if (ch[q] >= 0) {
          if (lane == 0) stk[sp] = make_int2(ch[q], (int)rec);
          ++sp;
        }
      __syncwarp();
    }
    if (__ballot_sync(0xffffffffu, pc | pp) == 0) continue;
    // the cell's sources: its proxies (PC) or its particles (PP); a lane
    // evaluates only the kind it chose for this cell
    const bool any_pc = __ballot_sync(0xffffffffu, pc) != 0;
    const int ns = any_pc ? P : v.cend[c] - v.cbegin[c];
    const int sb = any_pc ? 0 : v.cbegin[c];
    const bool mine = pc || pp;
    if constexpr (!F32) {
      double a[3] = {0.0, 0.0, 0.0};
      for (int k = 0; k < ns; ++k) {
        double y0, y1, y2, w;
        if (any_pc) {
          const int64_t po = (int64_t)c * 3 * P;
          y0 = v.proxy[po + k]; y1 = v.proxy[po + P + k]; y2 = v.proxy[po + 2 * P + k];
          w = wbar[((int64_t)c * ldr + r) * P + k];
        } else {
          const int64_t j = sb + k;
          y0 = v.x[j]; y1 = v.x[N + j]; y2 = v.x[2 * N + j];
          w = ws[(int64_t)r * N + j];
          if (j == i) continue;  // i = j omitted (Eq. PP)
        }
        if (mine) term64<KID>(x0 - y0, x1 - y1, x2 - y2, w, a);
      }
#pragma unroll
      for (int d = 0; d < D; ++d) acc64[d] += a[d];
    } else {
      const float tx = (float)(x0 - cc[0]), ty = (float)(x1 - cc[1]), tz = (float)(x2 - cc[2]);
      for (int k0 = 0; k0 < ns; k0 += kChunk) {
        const int k1 = min(ns, k0 + kChunk);
        float a[3] = {0.f, 0.f, 0.f};
        for (int k = k0; k < k1; ++k) {
          float sx, sy, sz, w;
          if (any_pc) {
            const int64_t po = (int64_t)c * 3 * P;
            sx = v.proxy32[po + k]; sy = v.proxy32[po + P + k]; sz = v.proxy32[po + 2 * P + k];
            w = wbar32[((int64_t)c * ldr + r) * P + k];
          } else {
            const int64_t j = sb + k;
            const float4 o = v.off32[j];
            sx = o.x; sy = o.y; sz = o.z;
            w = wsf[(int64_t)r * N + j];
            if (j == i) continue;  // i = j omitted (Eq. PP)
          }
          if (mine) term32<KID>(tx - sx, ty - sy, tz - sz, w, a);
        }
#pragma unroll
        for (int d = 0; d < D; ++d) two_sum_fold(hi[d], lo[d], a[d]);
      }
      if constexpr (KID == CSFMM_KERNEL_LAPLACE) {
        // -(1/4pi) sum w ln(d2/2) = -(ln2/4pi) (sum w log2 d2 - sum w): the
        // cell's weight total, without the target's own weight in its leaf
        if (mine) {
          fold_minus(hi[0], lo[0], weight_total(v, c, r, any_pc ? 1 : 0));
          if (pp && i >= sb && i < sb + ns) two_sum_fold(hi[0], lo[0], wsf[(int64_t)r * N + i]);
        }
      }
    }
  }
  if (!act || v.perm[i] < v.tbase) return;
  double o[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) o[d] = F32 ? (double)hi[d] + (double)lo[d] : acc64[d];
  double *dst = out + ((int64_t)r * v.ntgt + v.perm[i] - v.tbase) * D;
  if constexpr (KID == CSFMM_KERNEL_BIOT_SAVART) {
    dst[0] = kInv2Pi * (x1 * o[2] - x2 * o[1]);
    dst[1] = kInv2Pi * (x2 * o[0] - x0 * o[2]);
    dst[2] = kInv2Pi * (x0 * o[1] - x1 * o[0]);
  } else if constexpr (KID == CSFMM_KERNEL_LAPLACE && F32) {
    dst[0] = -(0.69314718055994530942 * kInv4Pi) * o[0];
  } else if constexpr (KID == CSFMM_KERNEL_BIHARMONIC) {
    dst[0] = kInv4Pi * o[0];
  } else {
    dst[0] = o[0];
  }
}

template <int KID>
void launch_cstc_kid(const PlanView &v, bool f32, double theta, int nroots, int nrhs, int ldr,
                     const double *ws, const float *wsf, const double *wbar, const float *wbar32,
                     double *out, cudaStream_t st) {
  const int64_t warps = (v.N + 31) / 32;
  const int grid = (int)((warps + kCstcWarps - 1) / kCstcWarps);
  for (int r = 0; r < nrhs; ++r) {
    if (f32)
      cstc_kernel<KID, true><<<grid, kCstcThreads, 0, st>>>(v, theta, nroots, r, ldr, ws, wsf,
                                                            wbar, wbar32, out);
    else
      cstc_kernel<KID, false><<<grid, kCstcThreads, 0, st>>>(v, theta, nroots, r, ldr, ws, wsf,
                                                             wbar, wbar32, out);
  }
}

}  // namespace

void launch_cstc(const PlanView &v, bool f32, double theta, int nroots, int nrhs, int ldr,
                 const double *ws, const float *wsf, const double *wbar, const float *wbar32,
                 double *out, cudaStream_t st) {
  switch (v.kernel_id) {
    case CSFMM_KERNEL_LAPLACE:
      launch_cstc_kid<CSFMM_KERNEL_LAPLACE>(v, f32, theta, nroots, nrhs, ldr, ws, wsf, wbar, wbar32, out, st);
      break;
    case CSFMM_KERNEL_BIOT_SAVART:
      launch_cstc_kid<CSFMM_KERNEL_BIOT_SAVART>(v, f32, theta, nroots, nrhs, ldr, ws, wsf, wbar, wbar32, out, st);
      break;
    case CSFMM_KERNEL_NEWTON:
      launch_cstc_kid<CSFMM_KERNEL_NEWTON>(v, f32, theta, nroots, nrhs, ldr, ws, wsf, wbar, wbar32, out, st);
      break;
    case CSFMM_KERNEL_BIHARMONIC:
      launch_cstc_kid<CSFMM_KERNEL_BIHARMONIC>(v, f32, theta, nroots, nrhs, ldr, ws, wsf, wbar, wbar32, out, st);
      break;
    case CSFMM_KERNEL_SAL:
      launch_cstc_kid<CSFMM_KERNEL_SAL>(v, f32, theta, nroots, nrhs, ldr, ws, wsf, wbar, wbar32, out, st);
      break;
    default:
      launch_cstc_kid<CSFMM_KERNEL_ONE>(v, f32, theta, nroots, nrhs, ldr, ws, wsf, wbar, wbar32, out, st);
      break;
  }
}

}  // namespace csfmm
