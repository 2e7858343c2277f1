// downward_df.cuh -- the downward pass of the FP32-bulk form in double-float
// arithmetic on the FP32 pipes (Sec. 8.1, Eq. downward_2), as block-level
// device functions shared by the per-level / per-leaf kernels of evaluate.cu
// and by the persistent multi-right-hand-side kernel of persistent.cu:
//   l2l_df_cell   child proxy potentials += (M_qa (x) M_qb)^T parent's
//   l2p_df_leaf   potential at a leaf's particles = near field + the leaf's
//                 proxy potentials interpolated to the particle, in input order
// Proxy potentials and near-field potentials that another thread block may
// have written during the same launch are read with L2-coherent loads
// (ld.global.cg), so that a block never sees a stale line of its own L1.
#pragma once

#include "csfmm_internal.cuh"

namespace csfmm {

// ---------------------------------------------------------------------------
// Double-float arithmetic on the FP32 pipes for the FP32-form passes: a value
// is an unevaluated pair (h, l), products carry their exact FP32 rounding
// error (FMA) and sums use Knuth's two-sum.  The rounded intrinsics keep the
// compiler from contracting a product into the following sum.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void df_acc_prod(float &sh, float &sl, float ah, float al, float bh,
                                            float bl) {
  const float ph = __fmul_rn(ah, bh);
  float pe = fmaf(ah, bh, -ph);
  pe = fmaf(ah, bl, pe);
  pe = fmaf(al, bh, pe);
  const float s = __fadd_rn(sh, ph);
  const float bb = __fadd_rn(s, -sh);
  const float e = __fadd_rn(__fadd_rn(sh, -__fadd_rn(s, -bb)), __fadd_rn(ph, -bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(e, pe));
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (S, C) += (ah + al) (bh + bl)
__device__ __forceinline__ void df_fma(float &S, float &C, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, fmaf(al, bh, e));
  float q;
  two_sum(S, p, S, q);
  C = __fadd_rn(C, __fadd_rn(q, e));
}

// Shared memory (floats) of l2l_df_cell: matrices (rounding, remainder) and
// the parent's potentials and one intermediate product as double-float pairs.
constexpr int kL2LDfSmemFloats = 4 * kMaxP * kMaxP + 4 * kMaxP * kMaxP;

// L2L of the FP32 form for parent cell c (any block size): the contraction of
// the FP64 L2L in double-float (FP64 proxy potentials split into FP32 pairs on
// load, matrices as FP32 rounding + remainder), each child value added to its
// FP64 slot.  Returns at once for a leaf.
__device__ __forceinline__ void l2l_df_cell(const PlanView &v, int c, int r0, int nr, int dim,
                                            double *psi, int ldr, float *sm) {
  float *sMh = sm, *sMl = sm + 2 * kMaxP * kMaxP;
  float *sph = sm + 4 * kMaxP * kMaxP, *spl = sph + kMaxP * kMaxP;
  float *sth = spl + kMaxP * kMaxP, *stl = sth + kMaxP * kMaxP;
  const int p = v.p, P = v.P;
  const int32_t *ch = v.cchild + 4 * c;
  if (ch[0] < 0 && ch[1] < 0 && ch[2] < 0 && ch[3] < 0) return;
  __syncthreads();  // the shared buffer may still be read by the block's previous work
  for (int t = threadIdx.x; t < 2 * p * p; t += blockDim.x) {
    sMh[t] = v.m2m32[t];
    sMl[t] = v.m2m32[2 * p * p + t];
  }
  for (int r = r0; r < r0 + nr; ++r)
    for (int d = 0; d < dim; ++d) {
      __syncthreads();
      for (int t = threadIdx.x; t < P; t += blockDim.x) {
        const double x = __ldcg(psi + (((int64_t)c * ldr + r) * dim + d) * P + t);
        const float h = __double2float_rn(x);
        sph[t] = h;
        spl[t] = __double2float_rn(x - (double)h);
      }
      for (int q = 0; q < 4; ++q) {
        const int cc = ch[q];
        if (cc < 0 || !cell_ok(v, cc)) continue;
        int qa = q & 1, qb = q >> 1;
        __syncthreads();
        if (v.mcell32) {  // shrunk boxes: this child's own matrices
          const float *Mc = v.mcell32 + (int64_t)cc * 4 * p * p;
          for (int t = threadIdx.x; t < 2 * p * p; t += blockDim.x) {
            sMh[t] = Mc[t];
            sMl[t] = Mc[2 * p * p + t];
          }
          qa = 0;
          qb = 1;
          __syncthreads();
        }
        // st[m1][n2] = sum_m2 psi[m1][m2] M[qb][m2][n2]
        for (int t = threadIdx.x; t < P; t += blockDim.x) {
          const int m1 = t / p, n2 = t - m1 * p;
          float sh = 0.f, sl = 0.f;
          for (int m2 = 0; m2 < p; ++m2) {
            const int o = (qb * p + m2) * p + n2;
            df_acc_prod(sh, sl, sph[m1 * p + m2], spl[m1 * p + m2], sMh[o], sMl[o]);
          }
          sth[t] = sh;
          stl[t] = sl;
        }
        __syncthreads();
        double *dst = psi + (((int64_t)cc * ldr + r) * dim + d) * P;
        for (int t = threadIdx.x; t < P; t += blockDim.x) {
          const int n1 = t / p, n2 = t - n1 * p;
          float sh = 0.f, sl = 0.f;
          for (int m1 = 0; m1 < p; ++m1) {
            const int o = (qa * p + m1) * p + n1;
            df_acc_prod(sh, sl, sMh[o], sMl[o], sth[m1 * p + n2], stl[m1 * p + n2]);
          }
          dst[t] = __ldcg(dst + t) + ((double)sh + (double)sl);
        }
      }
    }
}

// L2P + finalize of the FP32-bulk form in double-float arithmetic: the proxy
// potentials (FP64) and the Lagrange rows (FP32 hi + lo pairs) enter as
// pairs of FP32 numbers; each product is formed exactly with an FMA and the
// sums are compensated (two-sum), so the interpolation adds no FP32-level
// rounding to the per-target value (a chain of FP32 contractions through
// every tree level would otherwise dominate the bulk form's error).
//   out[r][perm[i] - tbase][d] = phi[r][i][d] + sum_m psi_leaf[m] La[i][m1] Lb[i][m2]
// for the targets of leaf c (perm[i] >= tbase).  Needs blockDim.x ==
// kL2PThreads: one thread per point of a chunk.  PC = p as a compile-time
// constant (0: runtime p) keeps each point's rows in registers and unrolls
// the contractions.
constexpr int kL2PThreads = 128;
// Shared floats of l2p_df_leaf<PC>: the proxy potentials' (hi, lo) pairs and the
// staged rows, with stride PC (kMaxP for a runtime p).
template <int PC>
constexpr int l2p_df_smem_floats() {
  return 2 * (PC > 0 ? PC : kMaxP) * (PC > 0 ? PC : kMaxP) + 4 * kL2PThreads * (PC > 0 ? PC : kMaxP);
}
constexpr int kL2PDfSmemFloats = l2p_df_smem_floats<0>();

template <int PC>
__device__ __forceinline__ void l2p_df_leaf(const PlanView &v, int c, const double *psi, int ldr,
                                            int nrhs, int dim, const double *phi, double *out,
                                            float *sm) {
  // proxy potentials as (hi, lo) pairs: one 8-byte shared load per term
  constexpr int PS = PC > 0 ? PC : kMaxP;
  float2 *sps = reinterpret_cast<float2 *>(sm);
  float *sLa = sm + 2 * PS * PS, *sLal = sLa + kL2PThreads * PS;
  float *sLb = sLal + kL2PThreads * PS, *sLbl = sLb + kL2PThreads * PS;
  if (!cell_ok(v, c)) return;
  const int b = v.cbegin[c], e = v.cend[c];
  const int p = PC > 0 ? PC : v.p, P = p * p;
  for (int i0 = b; i0 < e; i0 += kL2PThreads) {
    const int nj = min(kL2PThreads, e - i0);
    __syncthreads();
    for (int t = threadIdx.x; t < nj * p; t += kL2PThreads) {
      const int64_t o = (int64_t)i0 * p + t;
      sLa[t] = v.La32[o];
      sLal[t] = v.La32lo[o];
      sLb[t] = v.Lb32[o];
      sLbl[t] = v.Lb32lo[o];
    }
    const int t = threadIdx.x;
    const int i = i0 + t;
    for (int r = 0; r < nrhs; ++r)
      for (int d = 0; d < dim; ++d) {
        __syncthreads();
        for (int u = threadIdx.x; u < P; u += kL2PThreads) {
          const double x = __ldcg(psi + (((int64_t)c * ldr + r) * dim + d) * P + u);
          const float hi = (float)x;
          sps[u] = make_float2(hi, (float)(x - (double)hi));
        }
        __syncthreads();
        if (t < nj && v.perm[i] >= v.tbase) {
          const float *lah = sLa + t * p, *lal = sLal + t * p;
          const float *lbh = sLb + t * p, *lbl = sLbl + t * p;
          float S = 0.f, C = 0.f;
          if constexpr (PC > 0) {
            float bh[PC], bl[PC];
#pragma unroll
            for (int m2 = 0; m2 < PC; ++m2) {
              bh[m2] = lbh[m2];
              bl[m2] = lbl[m2];
            }
#pragma unroll
            for (int m1 = 0; m1 < PC; ++m1) {
              float sh = 0.f, sl = 0.f;
#pragma unroll
              for (int m2 = 0; m2 < PC; ++m2) {
                const float2 ps = sps[m1 * PC + m2];
                df_fma(sh, sl, ps.x, ps.y, bh[m2], bl[m2]);
              }
              df_fma(S, C, lah[m1], lal[m1], sh, sl);
            }
          } else {
            for (int m1 = 0; m1 < p; ++m1) {
              float sh = 0.f, sl = 0.f;
              for (int m2 = 0; m2 < p; ++m2) {
                const float2 ps = sps[m1 * p + m2];
                df_fma(sh, sl, ps.x, ps.y, lbh[m2], lbl[m2]);
              }
              df_fma(S, C, lah[m1], lal[m1], sh, sl);
            }
          }
          const int64_t oi = ((int64_t)r * v.N + i) * dim + d;
          out[((int64_t)r * v.ntgt + v.perm[i] - v.tbase) * dim + d] =
              __ldcg(phi + oi) + ((double)S + (double)C);
        }
      }
  }
}

}  // namespace csfmm
