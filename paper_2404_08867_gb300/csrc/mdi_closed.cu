// mdi_closed.cu -- MDI-LR with the closed level state (MDI_STATE_CLOSED) for the
// exponential families EXP (phi_j = exp(c_j x)) and OSC (phi_j = exp(i c_j x)),
// and its adjoint.
//
// With phi_k(x) = exp(c~_k x) (c~ = c or i c) the level recursion of Algorithm 1,
//     G_k(x) = (1/r_k) sum_{q<r_k} phi_k(u) G_{k-1}(u),   u = (q + x) / r_k,
// keeps the form G_k(x) = K_k exp(beta_k x):
//     gamma_k = beta_{k-1} + c~_k,   beta_k = gamma_k / r_k,
//     K_k = K_{k-1} S_k,  S_k = (1/r_k) sum_{q<r_k} exp(gamma_k q / r_k),
// and the rule is front * K_d (front = exp(2 pi i u) for OSC).  The cluster
// evaluation of level k is the sum S_k over its r_k points.
//
// GB300 mapping.  beta is an affine recurrence (beta_k = beta_{k-1}/a + c_k/a;
// for OSC the same real recurrence gives the imaginary part), so instead of
// walking the d levels one after the other on one SM:
//   1. the recurrence is solved as a scan of affine maps (gamma_k, all k): for
//      d <= 32 by one warp of every CTA of step 2 (shuffles), otherwise by one CTA
//      in a launch of its own;
//   2. the cluster sums of all levels run at once across the GPU: every level's
//      r_k points are cut into chunks of up to 1024, one warp per chunk;
//   3. the chunk sums of each level are added in chunk order (S_k), and
//   4. the S_k multiplied in level order by a fixed tree: when the chunk sums
//      number at most 2048, both by one CTA in one launch, otherwise a launch each.
// So d <= 32 takes two launches whatever a (the small workload's time to 1e-6),
// and the launch count never depends on d or on a beyond that.  Each launch
// waits on no other CTA, so the workspace needs no initial contents.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "mdi_common.cuh"
#include "mdi_exp2_table.inc"
#include "mdi_fp64.cuh"
#include "mdi_internal.h"
#include "mdi_nodes.cuh"

namespace mdi {

constexpr int kScanThreads = 1024;
constexpr int kChunkThreads = 256;
constexpr int64_t kChunkQ = 1024;  // most cluster points per warp chunk
constexpr int kWarpScanMaxD = 32;  // gamma by one warp of each chunk CTA up to this d
constexpr int kFinishMaxChunks = 2048;  // per-level sums and product in one CTA up to this many chunks
constexpr int kAnchor = 16;             // FP64 cluster terms: a fresh exp every 16 points of a lane

// gamma_k, k < d <= 32, by one warp: lane k holds the map beta -> (beta + c_k)/a
// of level k (k < d - 1); an inclusive Hillis-Steele scan over shuffles composes
// the maps of levels 0..k (earlier map first), which applied to beta_0 = 0 gives
// beta_k, and gamma_k = beta_{k-1} + c_k.  Valid in lanes k < d.
// ck: c_k of lane k (0 in lanes k >= d), loaded by the caller.
__device__ __forceinline__ double warp_gamma(int d, double inva, double ck) {
  const int lane = threadIdx.x & (kWarp - 1);
  double A = 1.0, B = 0.0;
  if (lane < d - 1) {
    A = inva;
    B = ck * inva;
  }
  // Lanes k >= d hold identity maps, so rounds with off >= d change no lane below d.
  for (int off = 1; off < d; off <<= 1) {
    const double pA = __shfl_up_sync(0xffffffffu, A, off), pB = __shfl_up_sync(0xffffffffu, B, off);
    if (lane >= off) {
      B = fma(A, pB, B);
      A *= pA;
    }
  }
  const double bprev = __shfl_up_sync(0xffffffffu, B, 1);
  return (lane == 0 ? 0.0 : bprev) + ck;
}

// gamma_k (real: the exponent rate, or its imaginary part for OSC) for k = 1..d.
__global__ void __launch_bounds__(kScanThreads) closed_scan_kernel(int d, double inva,
                                                                   const double *__restrict__ params,
                                                                   double *__restrict__ gamma) {
  __shared__ double sA[kScanThreads], sB[kScanThreads];
  const int per = (d + blockDim.x - 1) / blockDim.x;
  const int lo = threadIdx.x * per, hi = min(d - 1, lo + per);  // maps for levels lo+1..hi (k < d)
  // Composite of beta_k = beta_{k-1}/a + c_k/a over this thread's levels.
  double A = 1.0, B = 0.0;
  for (int k = lo; k < hi; ++k) {  // 0-based level k <-> paper's level k+1
    A *= inva;
    B = (B + params[k]) * inva;
  }
  sA[threadIdx.x] = A;
  sB[threadIdx.x] = B;
  __syncthreads();
  // Inclusive Hillis-Steele scan of affine maps (earlier map applied first).
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    double pA = 1.0, pB = 0.0;
    if ((int)threadIdx.x >= off) {
      pA = sA[threadIdx.x - off];
      pB = sB[threadIdx.x - off];
    }
    __syncthreads();
    if ((int)threadIdx.x >= off) {
      const double cA = sA[threadIdx.x], cB = sB[threadIdx.x];
      sA[threadIdx.x] = cA * pA;
      sB[threadIdx.x] = cA * pB + cB;
    }
    __syncthreads();
  }
  double beta = threadIdx.x == 0 ? 0.0 : sB[threadIdx.x - 1];  // beta at the start of the chunk
  for (int k = lo; k < min(d, lo + per); ++k) {
    const double g = beta + params[k];
    gamma[k] = g;
    beta = g * inva;
  }
}

// Chunks: levels k < d-1 have a points, cut into cpl chunks of q points; the last
// level has n_last points in cpl_last chunks.  q (a multiple of 32, at most 1024)
// is chosen so that about 8 warps per SM (two per sub-partition) get a chunk: a
// warp instruction occupies GB300's FP64 unit about as long as a dependent FP64
// result takes, so two warps per sub-partition keep it busy, and larger chunks
// spread each warp's set-up over more points.
// The reciprocals 1/a and 1/n_last of the two cluster radices are formed once on
// the host (correctly rounded, the same double the device's division gives) and
// also as float pairs: an FP64 division per chunk would cost GB300's FP64 pipe
// about as much as the chunk's own sum.
struct Chunks {
  int cpl, cpl_last, total;
  int64_t q;
  double inv_a, inv_nl;
  float2 inv_a_df, inv_nl_df;
};
static int64_t chunk_q(int d, int64_t a, int64_t n_last) {
  const double points = (double)(d - 1) * (double)a + (double)n_last;
  const double target = (double)sm_count() * 8.0;
  int64_t q = (int64_t)std::ceil(points / target);
  q = (q + 31) / 32 * 32;
  return std::max<int64_t>(32, std::min<int64_t>(kChunkQ, q));
}
static float2 split_df(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}
static Chunks make_chunks(int d, int64_t a, int64_t n_last) {
  Chunks c;
  c.inv_a = 1.0 / (double)a;
  c.inv_nl = 1.0 / (double)n_last;
  c.inv_a_df = split_df(c.inv_a);
  c.inv_nl_df = split_df(c.inv_nl);
  c.q = chunk_q(d, a, n_last);
  c.cpl = (int)((a + c.q - 1) / c.q);
  c.cpl_last = (int)((n_last + c.q - 1) / c.q);
  c.total = (d - 1) * c.cpl + c.cpl_last;
  return c;
}
__device__ __forceinline__ int chunk_base(int k, int d, int cpl) { return k < d - 1 ? k * cpl : (d - 1) * cpl; }

// Sum of exp(iota gamma_k q / r_k) (and of (q/r_k) times it, WITH_T) over one chunk
// of one level's cluster, per warp.  DF64 (exponential family): x = q (1/r) and
// gamma x as double-float pairs, the double-float exp (table copied from the
// generated constants into shared memory), Dot2 accumulation -- for levels with
// |gamma| <= 64, whose terms e^(gamma x) lie in [e^-64, e^64] and whose chunk sums
// (at most 1024 terms) stay inside the float range with normal low parts; other
// levels are summed in FP64.
// gamma: the levels' rates in global memory, or NULL for d <= kWarpScanMaxD, where
// the CTA's first warp computes them (params, 1/a) into shared memory.  FP64 terms
// of the exponential family use the table-driven exp of mdi_fp64.cuh.
template <int FAM, int PREC, bool WITH_T>
__global__ void __launch_bounds__(kChunkThreads) closed_chunk_kernel(int d, int64_t a, int64_t n_last, Chunks ch,
                                                                     const double *__restrict__ gamma_g,
                                                                     const double *__restrict__ params,
                                                                     double2 *__restrict__ partS,
                                                                     double2 *__restrict__ partT) {
  constexpr bool DFE = (PREC == MDI_PREC_DF64) && (FAM != MDI_FAM_OSC);
  constexpr bool TANG = (PREC == MDI_PREC_FP64 || PREC == MDI_PREC_DF64) && (FAM != MDI_FAM_OSC);
  __shared__ float2 s_exp2[DFE ? kExpTable : 1];
  __shared__ double s_exp2d[TANG ? kExpTable : 1];
  constexpr bool STEP = (PREC == MDI_PREC_FP64 || PREC == MDI_PREC_DF64);  // FP64 terms stepped by R
  __shared__ double s_gamma[kWarpScanMaxD];
  __shared__ double2 s_step[STEP ? kWarpScanMaxD : 1];
  // The first warp's c_k load is issued before the table copy, so the two overlap.
  const double ck = (!gamma_g && threadIdx.x < d && threadIdx.x < kWarp) ? params[threadIdx.x] : 0.0;
  if constexpr (DFE)
    for (int j = threadIdx.x; j < kExpTable; j += blockDim.x) s_exp2[j] = kExp2TableGen[j];
  if constexpr (TANG)
    for (int j = threadIdx.x; j < kExpTable; j += blockDim.x) s_exp2d[j] = kExp2TableD[j];
  __syncthreads();  // the exp table is read below
  if (!gamma_g && threadIdx.x < kWarp) {
    // gamma_k for every level, and (FP64 terms) each level's step R_k = e^{32 gamma_k / r_k}
    const int k = threadIdx.x;
    const double g = warp_gamma(d, ch.inv_a, ck);
    if (k < d) {
      s_gamma[k] = g;
      if constexpr (STEP) {
        const double arg = 32.0 * (g * ((k + 1 < d) ? ch.inv_a : ch.inv_nl));
        if constexpr (FAM == MDI_FAM_OSC) {
          double rs, rc;
          sincos(arg, &rs, &rc);
          s_step[k] = make_double2(rc, rs);
        } else {
          s_step[k] = make_double2(exp_tang64(arg, s_exp2d), 0.0);
        }
      }
    }
  }
  __syncthreads();
  const double *gamma = gamma_g ? gamma_g : s_gamma;
  const int lane = threadIdx.x & (kWarp - 1);
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
  const int nwarps = gridDim.x * blockDim.x / kWarp;
  for (int c = warp_global; c < ch.total; c += nwarps) {
    int k, j;
    if (c < (d - 1) * ch.cpl) {
      k = c / ch.cpl;
      j = c % ch.cpl;
    } else {
      k = d - 1;
      j = c - (d - 1) * ch.cpl;
    }
    const int64_t r = (k + 1 < d) ? a : n_last;
    const int64_t q0 = (int64_t)j * ch.q, q1 = min(r, q0 + ch.q);
    const double g = gamma[k], invr = (k + 1 < d) ? ch.inv_a : ch.inv_nl;
    double2 s = make_double2(0.0, 0.0), t = make_double2(0.0, 0.0);
    df32 sr{0.f, 0.f}, si{0.f, 0.f};
    if (DFE && fabs(g) <= 64.0) {
      const float2 irf = (k + 1 < d) ? ch.inv_a_df : ch.inv_nl_df;
      const df32 gd = df_from_double(g), ird{irf.x, irf.y};
      const bool small = r <= (int64_t)(1 << 24);  // q exact in one float
      DfAcc as, at;
      for (int64_t q = q0 + lane; q < q1; q += kWarp) {
        df32 x;
        if (small) {
          x = df_mul_f(ird, (float)(int)q);
        } else {  // q < 2^31: q = qh + ql exactly, both floats
          const int qi = (int)q;
          const float qh = __int2float_rz(qi);
          x = df_mul(ird, df32{qh, __int2float_rn(qi - __float2int_rz(qh))});
        }
        const df32 e = df_exp(df_mul(gd, x), s_exp2);
        dacc_add(as, e);
        if constexpr (WITH_T) dacc_prod(at, e, x);
      }
      df32 sv = dacc_value(as), tv = dacc_value(at);
#pragma unroll
      for (int off = kWarp / 2; off > 0; off >>= 1) {
        sv = df_add(sv, df_shfl_down(sv, off));
        if constexpr (WITH_T) tv = df_add(tv, df_shfl_down(tv, off));
      }
      if (lane == 0) {
        partS[c] = make_double2(df_to_double(sv), 0.0);
        if constexpr (WITH_T) partT[c] = make_double2(df_to_double(tv), 0.0);
      }
      continue;
    }
    if constexpr (PREC == MDI_PREC_FP64 || PREC == MDI_PREC_DF64) {
      // FP64 terms: along the cluster they form a geometric progression,
      // e^{g (q + 32)/r} = e^{g q/r} R with R = e^{32 g/r} (complex for OSC), so each
      // lane steps its points by one multiply and takes a fresh exp (sincos) every
      // kAnchor points: a term's error stays below about 2 kAnchor ulps.
      const double gr = g * invr;
      if constexpr (FAM == MDI_FAM_OSC) {
        double rs, rc;
        if (gamma_g) {
          sincos(32.0 * gr, &rs, &rc);
        } else {
          rc = s_step[k].x;
          rs = s_step[k].y;
        }
        double2 E = make_double2(1.0, 0.0);
        int i = 0;
        for (int64_t q = q0 + lane; q < q1; q += kWarp, ++i) {
          if ((i & (kAnchor - 1)) == 0) {
            double es, ec;
            sincos(gr * (double)q, &es, &ec);
            E = make_double2(ec, es);
          }
          s = c_add(s, E);
          if constexpr (WITH_T) t = c_add(t, c_scale(E, (double)q * invr));
          E = make_double2(fma(E.x, rc, -E.y * rs), fma(E.x, rs, E.y * rc));
        }
      } else {
        const double R = gamma_g ? exp_tang64(32.0 * gr, s_exp2d) : s_step[k].x;
        double E = 1.0;
        int i = 0;
        for (int64_t q = q0 + lane; q < q1; q += kWarp, ++i) {
          if ((i & (kAnchor - 1)) == 0) E = exp_tang64(gr * (double)q, s_exp2d);
          s.x += E;
          if constexpr (WITH_T) t.x = fma(E, (double)q * invr, t.x);
          E *= R;
        }
      }
    } else for (int64_t q = q0 + lane; q < q1; q += kWarp) {
      const double x = (double)q * invr;
      const double arg = g * x;
      double2 e;
      if constexpr (FAM == MDI_FAM_OSC) {
        if constexpr (PREC == MDI_PREC_FP64) {
          double sn, cs;
          sincos(arg, &sn, &cs);
          e = make_double2(cs, sn);
        } else {
          float fs, fc;
          sincosf((float)arg, &fs, &fc);
          e = make_double2((double)fc, (double)fs);
        }
      } else if constexpr (TANG) {
        e = make_double2(exp_tang64(arg, s_exp2d), 0.0);
      } else {
        e = make_double2((double)expf((float)arg), 0.0);
      }
      if constexpr (PREC == MDI_PREC_FP32_EVAL_DF32) {
        sr = df_add(sr, df32{(float)e.x, 0.f});
        si = df_add(si, df32{(float)e.y, 0.f});
      } else {
        s = c_add(s, e);
      }
      if constexpr (WITH_T) t = c_add(t, c_scale(e, x));
    }
    if constexpr (PREC == MDI_PREC_FP32_EVAL_DF32) {
#pragma unroll
      for (int off = kWarp / 2; off > 0; off >>= 1) {
        sr = df_add(sr, df_shfl_down(sr, off));
        si = df_add(si, df_shfl_down(si, off));
      }
      s = make_double2(df_to_double(sr), df_to_double(si));
    } else if constexpr (FAM == MDI_FAM_OSC) {
      s = warp_sum(s);
    } else {  // real terms: the imaginary parts are zero
      s.x = warp_sum(s.x);
    }
    if constexpr (WITH_T) {
      if constexpr (FAM == MDI_FAM_OSC) t = warp_sum(t);
      else t.x = warp_sum(t.x);
    }
    if (lane == 0) {
      partS[c] = s;
      if constexpr (WITH_T) partT[c] = t;
    }
  }
}

// The same sums for levels of at most a few chunks: one thread per level, chunks
// added in order.
template <bool WITH_T>
__global__ void closed_reduce_small_kernel(int d, int64_t a, int64_t n_last, Chunks ch,
                                           const double2 *__restrict__ partS, const double2 *__restrict__ partT,
                                           double2 *__restrict__ S, double2 *__restrict__ T) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < d; k += gridDim.x * blockDim.x) {
    const int n = k < d - 1 ? ch.cpl : ch.cpl_last, base = chunk_base(k, d, ch.cpl);
    const double invr = (k + 1 < d) ? ch.inv_a : ch.inv_nl;
    double2 s = make_double2(0.0, 0.0), t = make_double2(0.0, 0.0);
    for (int j = 0; j < n; ++j) {
      s = c_add(s, partS[base + j]);
      if constexpr (WITH_T) t = c_add(t, partT[base + j]);
    }
    S[k] = c_scale(s, invr);
    if constexpr (WITH_T) T[k] = c_scale(t, invr);
  }
}

// Per-level sums (S_k, and T_k with WITH_T) of the chunk partials.
template <bool WITH_T>
static void launch_reduce(int d, int64_t a, int64_t n_last, const Chunks &ch, const double2 *partS,
                          const double2 *partT, double2 *S, double2 *T, cudaStream_t stream);

// S_k (and T_k) = (1/r_k) * (sum of the chunk sums of level k), one CTA per level:
// each thread adds a strided subset of the level's chunks, then a fixed tree.
constexpr int kReduceThreads = 128;
template <bool WITH_T>
__global__ void __launch_bounds__(kReduceThreads) closed_reduce_kernel(int d, int64_t a, int64_t n_last, Chunks ch,
                                                                       const double2 *__restrict__ partS,
                                                                       const double2 *__restrict__ partT,
                                                                       double2 *__restrict__ S,
                                                                       double2 *__restrict__ T) {
  __shared__ double2 s_red[kReduceThreads / kWarp];
  for (int k = blockIdx.x; k < d; k += gridDim.x) {
    const int n = k < d - 1 ? ch.cpl : ch.cpl_last, base = chunk_base(k, d, ch.cpl);
    const double invr = (k + 1 < d) ? ch.inv_a : ch.inv_nl;
    double2 s = make_double2(0.0, 0.0), t = make_double2(0.0, 0.0);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      s = c_add(s, partS[base + j]);
      if constexpr (WITH_T) t = c_add(t, partT[base + j]);
    }
    s = block_sum(s, s_red);
    if constexpr (WITH_T) t = block_sum(t, s_red);
    if (threadIdx.x == 0) {
      S[k] = c_scale(s, invr);
      if constexpr (WITH_T) T[k] = c_scale(t, invr);
    }
  }
}

template <bool WITH_T>
static void launch_reduce(int d, int64_t a, int64_t n_last, const Chunks &ch, const double2 *partS,
                          const double2 *partT, double2 *S, double2 *T, cudaStream_t stream) {
  if (ch.cpl <= 8 && ch.cpl_last <= 8)
    closed_reduce_small_kernel<WITH_T><<<std::max(1, std::min((d + 255) / 256, sm_count() * 4)), 256, 0, stream>>>(
        d, a, n_last, ch, partS, partT, S, T);
  else
    closed_reduce_kernel<WITH_T><<<std::max(1, std::min(d, sm_count() * 16)), kReduceThreads, 0, stream>>>(
        d, a, n_last, ch, partS, partT, S, T);
}

// S_k = (1/r_k) (sum of level k's chunk sums, in shared memory) for every level,
// by one CTA in a fixed order: one thread per level adding its chunks in order
// when levels have few chunks, else warp w takes levels w, w + nw, ... with its
// lanes adding a strided subset and an xor butterfly adding the lanes.  Real
// families (REAL) add real parts only: their imaginary parts are zero.
template <bool REAL>
__device__ __forceinline__ void level_sums(int d, const Chunks &ch, const double2 *part, double2 *__restrict__ S) {
  using V = typename std::conditional<REAL, double, double2>::type;
  const int lane = threadIdx.x & (kWarp - 1), warp = threadIdx.x / kWarp, nw = blockDim.x / kWarp;
  auto load = [&](int c) -> V {
    if constexpr (REAL) return part[c].x;
    else return part[c];
  };
  auto store = [&](int k, V v) {
    const double r = (k + 1 < d) ? ch.inv_a : ch.inv_nl;
    if constexpr (REAL) S[k] = make_double2(v * r, 0.0);
    else S[k] = c_scale(v, r);
  };
  if (ch.cpl <= 8 && ch.cpl_last <= 8) {
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
      const int n = k < d - 1 ? ch.cpl : ch.cpl_last, base = chunk_base(k, d, ch.cpl);
      V v = VOps<V>::zero();
      for (int j = 0; j < n; ++j) v = VOps<V>::add(v, load(base + j));
      store(k, v);
    }
  } else {
    for (int k = warp; k < d; k += nw) {
      const int n = k < d - 1 ? ch.cpl : ch.cpl_last, base = chunk_base(k, d, ch.cpl);
      V v = VOps<V>::zero();
      for (int j = lane; j < n; j += kWarp) v = VOps<V>::add(v, load(base + j));
      v = warp_sum(v);
      if (lane == 0) store(k, v);
    }
  }
}

// Steps 3 and 4 in one CTA when the chunk sums number at most kFinishMaxChunks:
// the CTA first copies every chunk sum into shared memory (all loads in flight at
// once: a level's sums read one after the other would each wait for L2), then
// forms S_k -- one thread per level adding its chunks in order when levels have
// few chunks, else warp w takes levels w, w + 8, ... with its lanes adding a
// strided subset and an xor butterfly adding the lanes (fixed orders either way)
// -- and multiplies the S_k by the fixed tree of product_body.
template <int FAM>
__device__ void product_body(int d, const double *__restrict__ params, const double2 *__restrict__ S,
                             double *__restrict__ out, typename FamTraits<FAM>::V *sW);
constexpr int kFinishThreads = 256;
template <int FAM>
__global__ void __launch_bounds__(kFinishThreads) closed_finish_kernel(int d, Chunks ch,
                                                                       const double *__restrict__ params,
                                                                       const double2 *__restrict__ partS,
                                                                       double2 *__restrict__ S,
                                                                       double *__restrict__ out) {
  extern __shared__ double2 s_part[];  // ch.total chunk sums
  __shared__ typename FamTraits<FAM>::V sW[kFinishThreads / kWarp];
  for (int c = threadIdx.x; c < ch.total; c += kFinishThreads) s_part[c] = partS[c];
  __syncthreads();
  level_sums<FAM != MDI_FAM_OSC>(d, ch, s_part, S);
  __syncthreads();  // the S_k written above are visible to the whole CTA
  product_body<FAM>(d, params, S, out, sW);
}

// out = Re(front * prod_k S_k) by a fixed tree: each thread multiplies a run of
// consecutive factors, the 32 runs of a warp are combined by an xor butterfly
// (IEEE multiplication commutes exactly, so every lane holds the same value), and
// thread 0 multiplies the warps' products in order.  Real families multiply reals.
constexpr int kProdThreads = 256;
template <int FAM>
__device__ void product_body(int d, const double *__restrict__ params, const double2 *__restrict__ S,
                             double *__restrict__ out, typename FamTraits<FAM>::V *sW) {
  using V = typename FamTraits<FAM>::V;
  const int per = (d + blockDim.x - 1) / blockDim.x;
  const int lo = min(d, (int)threadIdx.x * per), hi = min(d, lo + per);
  V p = VOps<V>::one();
  // __ldcg: S may have been written earlier in the same launch (closed_finish_kernel),
  // so it must not come through the non-coherent read-only path.
  for (int k = lo; k < hi; ++k) p = VOps<V>::mul(p, from2<V>(__ldcg(S + k)));
  for (int off = 1; off < kWarp; off <<= 1) {
    if constexpr (FAM == MDI_FAM_OSC) {
      const double2 o = make_double2(__shfl_xor_sync(0xffffffffu, p.x, off), __shfl_xor_sync(0xffffffffu, p.y, off));
      p = c_mul(p, o);
    } else {
      p *= __shfl_xor_sync(0xffffffffu, p, off);
    }
  }
  if ((threadIdx.x & (kWarp - 1)) == 0) sW[threadIdx.x / kWarp] = p;
  __syncthreads();
  if (threadIdx.x == 0) {
    // Warps past the last factor hold exactly 1, so leaving them out changes no bit.
    const int nw = min((int)(blockDim.x / kWarp), (d + per * kWarp - 1) / (per * kWarp));
    V K = sW[0];
    for (int w = 1; w < nw; ++w) K = VOps<V>::mul(K, sW[w]);
    if constexpr (FAM == MDI_FAM_OSC) {
      double sn, cs;
      sincos(kTwoPi * params[d], &sn, &cs);
      out[0] = cs * K.x - sn * K.y;
    } else {
      out[0] = K;
    }
  }
}
template <int FAM>
__global__ void __launch_bounds__(kProdThreads) closed_product_kernel(int d, const double *__restrict__ params,
                                                                      const double2 *__restrict__ S,
                                                                      double *__restrict__ out) {
  __shared__ typename FamTraits<FAM>::V sW[kProdThreads / kWarp];
  product_body<FAM>(d, params, S, out, sW);
}

// ---------------------------------------------------------------------------
// Workspace: gamma[d] | partS[chunks] | partT[chunks] | S[d] | T[d] | nu[d]
// ---------------------------------------------------------------------------
struct ClosedLayout {
  size_t gamma, partS, partT, S, T, nu, total;
};
static ClosedLayout closed_layout(int d, int64_t a, int64_t n_last, bool grad) {
  const Chunks ch = make_chunks(d, a, n_last);
  ClosedLayout L{};
  size_t off = 0;
  L.gamma = off;
  off += align_up(sizeof(double) * (size_t)d);
  L.partS = off;
  off += align_up(sizeof(double2) * (size_t)ch.total);
  L.partT = off;
  if (grad) off += align_up(sizeof(double2) * (size_t)ch.total);
  L.S = off;
  off += align_up(sizeof(double2) * (size_t)d);
  L.T = off;
  L.nu = off;
  if (grad) {
    off += align_up(sizeof(double2) * (size_t)d);
    L.nu = off;
    off += align_up(sizeof(double2) * (size_t)d);
  }
  L.total = off;
  return L;
}

static bool closed_sizes_ok(int d, int64_t a, int64_t n_last) {
  if (d < 1 || d > (1 << 20) || a < 1 || n_last < 1) return false;
  // chunk count must fit an int
  const int64_t q = chunk_q(d, a, n_last);
  return (double)(d - 1) * (double)((a + q - 1) / q) + (double)((n_last + q - 1) / q) < (double)(1 << 30);
}

size_t closed_workspace_bytes(int d, int64_t a, int64_t n_last) {
  return closed_sizes_ok(d, a, n_last) ? closed_layout(d, a, n_last, false).total : 0;
}

// Threads of the one-CTA scan: about 8 levels per thread, 32 to 1024.  The scan is
// FP64 work on one SM, so a block sized to d keeps small d from paying for 1024
// threads' tree steps.
static int scan_threads(int d) {
  const int t = ((d + 7) / 8 + kWarp - 1) / kWarp * kWarp;
  return std::max(kWarp, std::min(kScanThreads, t));
}

static int chunk_grid(const Chunks &ch) {
  const int warps_per_cta = kChunkThreads / kWarp;
  return std::max(1, std::min((ch.total + warps_per_cta - 1) / warps_per_cta, sm_count() * 8));
}

// Steps 1-3 (and 4 when `out` is given), see the top of this file.
template <int FAM, int PREC, bool WITH_T>
static mdi_status run_levels_sums(int d, int64_t a, int64_t n_last, const double *params, char *base,
                                  const ClosedLayout &L, double *out, cudaStream_t stream) {
  double *gamma = (double *)(base + L.gamma);
  double2 *partS = (double2 *)(base + L.partS), *partT = (double2 *)(base + L.partT);
  double2 *S = (double2 *)(base + L.S), *T = (double2 *)(base + L.T);
  const Chunks ch = make_chunks(d, a, n_last);
  mdi_status st;
  if (d > kWarpScanMaxD) {
    closed_scan_kernel<<<1, scan_threads(d), 0, stream>>>(d, ch.inv_a, params, gamma);
    if ((st = check_launch()) != MDI_OK) return st;
  }
  closed_chunk_kernel<FAM, PREC, WITH_T><<<chunk_grid(ch), kChunkThreads, 0, stream>>>(
      d, a, n_last, ch, d > kWarpScanMaxD ? gamma : nullptr, params, partS, partT);
  if ((st = check_launch()) != MDI_OK) return st;
  if (out && ch.total <= kFinishMaxChunks) {
    closed_finish_kernel<FAM><<<1, kFinishThreads, sizeof(double2) * ch.total, stream>>>(d, ch, params, partS, S, out);
    return check_launch();
  }
  launch_reduce<WITH_T>(d, a, n_last, ch, partS, partT, S, T, stream);
  if ((st = check_launch()) != MDI_OK || !out) return st;
  closed_product_kernel<FAM><<<1, kProdThreads, 0, stream>>>(d, params, S, out);
  return check_launch();
}

template <int FAM, int PREC>
static mdi_status run_closed(int d, int64_t a, int64_t n_last, const double *params, double *out, void *ws,
                             cudaStream_t stream) {
  const ClosedLayout L = closed_layout(d, a, n_last, false);
  return run_levels_sums<FAM, PREC, false>(d, a, n_last, params, (char *)ws, L, out, stream);
}

template <int FAM>
static mdi_status run_closed_p(int precision, int d, int64_t a, int64_t n_last, const double *params, double *out,
                               void *ws, cudaStream_t stream) {
  switch (precision) {
    case MDI_PREC_FP64: return run_closed<FAM, MDI_PREC_FP64>(d, a, n_last, params, out, ws, stream);
    case MDI_PREC_FP32_EVAL_FP64: return run_closed<FAM, MDI_PREC_FP32_EVAL_FP64>(d, a, n_last, params, out, ws, stream);
    case MDI_PREC_FP32_EVAL_DF32: return run_closed<FAM, MDI_PREC_FP32_EVAL_DF32>(d, a, n_last, params, out, ws, stream);
    default:  // DF64: double-float cluster sums for the exponential family, FP64 for the oscillatory one
      if constexpr (FAM == MDI_FAM_OSC) return run_closed<FAM, MDI_PREC_FP64>(d, a, n_last, params, out, ws, stream);
      else return run_closed<FAM, MDI_PREC_DF64>(d, a, n_last, params, out, ws, stream);
  }
}

mdi_status closed_launch(int family, int d, int64_t a, int64_t n_last, const double *params, int precision,
                         double *out, void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if (family != MDI_FAM_EXP && family != MDI_FAM_OSC) return MDI_EUNSUPPORTED;
  if (!closed_sizes_ok(d, a, n_last)) return MDI_EINVAL;
  if (precision < MDI_PREC_FP64 || precision > MDI_PREC_DF64) return MDI_EINVAL;
  if (precision == MDI_PREC_DF64 && (a >= (int64_t)1 << 31 || n_last >= (int64_t)1 << 31)) return MDI_EUNSUPPORTED;
  if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < closed_workspace_bytes(d, a, n_last))
    return MDI_EWORKSPACE;
  if (family == MDI_FAM_EXP) return run_closed_p<MDI_FAM_EXP>(precision, d, a, n_last, params, out, workspace, stream);
  return run_closed_p<MDI_FAM_OSC>(precision, d, a, n_last, params, out, workspace, stream);
}

// ---------------------------------------------------------------------------
// Paper-table mode: the tensor midpoint rule on the grid of eq. (3.5),
//     Q = Re(front * prod_i (1/n_i) sum_{k<n_i} phi_i((k + 1/2)/n_i)),
// with n_1 = ... = n_{d-1} = N and n_d = n_last: the rule whose errors the MDI-LR
// columns of the paper's Section 5 tables print (Tests 3-6).  Any product-form
// family.  Each axis factor is a level factor S_k of the pipeline above, so the
// chunking, the per-level reduction in chunk order and the fixed-tree product are
// shared; only the chunk sums differ.
// ---------------------------------------------------------------------------
template <int FAM>
__global__ void __launch_bounds__(kChunkThreads) midpoint_chunk_kernel(int d, int64_t N, int64_t n_last, Chunks ch,
                                                                       const double *__restrict__ params,
                                                                       double2 *__restrict__ partS) {
  const int lane = threadIdx.x & (kWarp - 1);
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
  const int nwarps = gridDim.x * blockDim.x / kWarp;
  for (int c = warp_global; c < ch.total; c += nwarps) {
    int k, j;
    if (c < (d - 1) * ch.cpl) {
      k = c / ch.cpl;
      j = c % ch.cpl;
    } else {
      k = d - 1;
      j = c - (d - 1) * ch.cpl;
    }
    const int64_t r = (k + 1 < d) ? N : n_last;
    const int64_t q0 = (int64_t)j * ch.q, q1 = min(r, q0 + ch.q);
    const double invr = (k + 1 < d) ? ch.inv_a : ch.inv_nl;
    const AxisParams ap = load_axis(params, d, k);
    double2 s = make_double2(0.0, 0.0);
    for (int64_t q = q0 + lane; q < q1; q += kWarp) s = c_add(s, as2(phi<FAM, false>(((double)q + 0.5) * invr, ap)));
    s = warp_sum(s);
    if (lane == 0) partS[c] = s;
  }
}

size_t midpoint_workspace_bytes(int d, int64_t N, int64_t n_last) { return closed_workspace_bytes(d, N, n_last); }

template <int FAM>
static mdi_status run_midpoint(int d, int64_t N, int64_t n_last, const double *params, double *out, void *ws,
                               cudaStream_t stream) {
  const ClosedLayout L = closed_layout(d, N, n_last, false);
  char *base = (char *)ws;
  double2 *partS = (double2 *)(base + L.partS), *S = (double2 *)(base + L.S);
  const Chunks ch = make_chunks(d, N, n_last);
  midpoint_chunk_kernel<FAM><<<chunk_grid(ch), kChunkThreads, 0, stream>>>(d, N, n_last, ch, params, partS);
  mdi_status st = check_launch();
  if (st != MDI_OK) return st;
  if (ch.total <= kFinishMaxChunks) {
    closed_finish_kernel<FAM><<<1, kFinishThreads, sizeof(double2) * ch.total, stream>>>(d, ch, params, partS, S, out);
    return check_launch();
  }
  launch_reduce<false>(d, N, n_last, ch, partS, partS, S, S, stream);
  if ((st = check_launch()) != MDI_OK) return st;
  closed_product_kernel<FAM><<<1, kProdThreads, 0, stream>>>(d, params, S, out);
  return check_launch();
}

mdi_status midpoint_launch(int family, int d, int64_t N, int64_t n_last, const double *params, double *out,
                           void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if (!closed_sizes_ok(d, N, n_last)) return MDI_EINVAL;
  if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < midpoint_workspace_bytes(d, N, n_last))
    return MDI_EWORKSPACE;
  switch (family) {
    case MDI_FAM_EXP: return run_midpoint<MDI_FAM_EXP>(d, N, n_last, params, out, workspace, stream);
    case MDI_FAM_OSC: return run_midpoint<MDI_FAM_OSC>(d, N, n_last, params, out, workspace, stream);
    case MDI_FAM_GAUSS: return run_midpoint<MDI_FAM_GAUSS>(d, N, n_last, params, out, workspace, stream);
    case MDI_FAM_PEAK: return run_midpoint<MDI_FAM_PEAK>(d, N, n_last, params, out, workspace, stream);
    default: return MDI_EINVAL;
  }
}

// ---------------------------------------------------------------------------
// Adjoint of the closed-state sweep.
//
// Q = front * prod_k S_k(gamma_k) with S_k(g) = (1/r_k) sum_q e^{iota g q / r_k}
// (iota = 1 for EXP, i for OSC) and gamma_j depending on c_k (k <= j) through
// dgamma_j/dc_k = a^{-(j-k)}.  With T_k = (1/r_k) sum_q (q/r_k) e^{iota gamma_k q/r_k}
// (so dS_k/dgamma_k = iota T_k) and nu_j = iota T_j prod_{i != j} S_i,
//     dQ/dc_k = front * mu_k,   mu_k = nu_k + mu_{k+1} / a,   mu_d = nu_d,
// i.e. the levels run in reverse.  The products prod_{i != j} S_i are formed from
// exclusive prefix and suffix products (no division by S_j), and the reverse
// recurrence, like the forward one, is a block-wide scan of affine maps.
// ---------------------------------------------------------------------------
template <int FAM>
__global__ void __launch_bounds__(kScanThreads) closed_grad_final_kernel(int d, double a,
                                                                         const double *__restrict__ params,
                                                                         const double2 *__restrict__ S,
                                                                         const double2 *__restrict__ T,
                                                                         double2 *__restrict__ nu,
                                                                         double *__restrict__ value,
                                                                         double *__restrict__ grad) {
  __shared__ double2 sP[kScanThreads], sR[kScanThreads];
  __shared__ double sA[kScanThreads];
  __shared__ double2 sB[kScanThreads];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int per = (d + nt - 1) / nt;
  const int lo = min(d, tid * per), hi = min(d, lo + per);
  const double2 iota = (FAM == MDI_FAM_OSC) ? make_double2(0.0, 1.0) : make_double2(1.0, 0.0);
  double2 front = make_double2(1.0, 0.0);
  if (FAM == MDI_FAM_OSC) {
    double sn, cs;
    sincos(kTwoPi * params[d], &sn, &cs);
    front = make_double2(cs, sn);
  }
  // Chunk products, then exclusive prefix (left) and suffix (right) products.
  double2 cp = make_double2(1.0, 0.0);
  for (int j = lo; j < hi; ++j) cp = c_mul(cp, S[j]);
  sP[tid] = cp;
  sR[tid] = cp;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {
    double2 pl = make_double2(1.0, 0.0), pr = make_double2(1.0, 0.0);
    if (tid >= off) pl = sP[tid - off];
    if (tid + off < nt) pr = sR[tid + off];
    __syncthreads();
    if (tid >= off) sP[tid] = c_mul(pl, sP[tid]);
    if (tid + off < nt) sR[tid] = c_mul(sR[tid], pr);
    __syncthreads();
  }
  const double2 left = tid > 0 ? sP[tid - 1] : make_double2(1.0, 0.0);
  const double2 right = tid + 1 < nt ? sR[tid + 1] : make_double2(1.0, 0.0);
  const double2 total = sP[nt - 1];
  // nu_j = iota T_j prod_{i<j} S_i prod_{i>j} S_i
  double2 R = right;
  for (int j = hi - 1; j >= lo; --j) {
    nu[j] = R;
    R = c_mul(S[j], R);
  }
  double2 Lp = left;
  for (int j = lo; j < hi; ++j) {
    nu[j] = c_mul(c_mul(iota, T[j]), c_mul(Lp, nu[j]));
    Lp = c_mul(Lp, S[j]);
  }
  // Reverse recurrence mu_j = nu_j + mu_{j+1}/a: composite map of the chunk, then an
  // inclusive scan from the right (later chunks applied first).
  const double inva = 1.0 / a;
  double A = 1.0;
  double2 Bc = make_double2(0.0, 0.0);
  for (int j = hi - 1; j >= lo; --j) {
    A *= inva;
    Bc = c_add(nu[j], c_scale(Bc, inva));
  }
  sA[tid] = A;
  sB[tid] = Bc;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {
    double pA = 1.0;
    double2 pB = make_double2(0.0, 0.0);
    const bool has = tid + off < nt;
    if (has) {
      pA = sA[tid + off];
      pB = sB[tid + off];
    }
    __syncthreads();
    if (has) {  // this chunk's map applied after the maps to its right
      const double cA = sA[tid];
      const double2 cB = sB[tid];
      sA[tid] = cA * pA;
      sB[tid] = c_add(c_scale(pB, cA), cB);
    }
    __syncthreads();
  }
  double2 mu = tid + 1 < nt ? sB[tid + 1] : make_double2(0.0, 0.0);  // mu at hi (0 past the last level)
  for (int j = hi - 1; j >= lo; --j) {
    mu = c_add(nu[j], c_scale(mu, inva));
    grad[j] = c_mul(front, mu).x;
    grad[d + j] = 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    const double2 fq = c_mul(front, total);
    if (value) *value = fq.x;
    if (FAM == MDI_FAM_OSC) grad[d] = -kTwoPi * fq.y;
  }
}

size_t closed_grad_workspace_bytes(int d, int64_t a, int64_t n_last) {
  return closed_sizes_ok(d, a, n_last) ? closed_layout(d, a, n_last, true).total : 0;
}

template <int FAM>
static mdi_status run_closed_grad(int d, int64_t a, int64_t n_last, const double *params, double *value,
                                  double *grad, void *ws, cudaStream_t stream) {
  const ClosedLayout L = closed_layout(d, a, n_last, true);
  char *base = (char *)ws;
  mdi_status st = run_levels_sums<FAM, MDI_PREC_FP64, true>(d, a, n_last, params, base, L, nullptr, stream);
  if (st != MDI_OK) return st;
  // One CTA of about d/8 threads: each takes a run of levels in order, and the
  // scans between runs take log2 of the thread count rounds (FP64 work on one SM).
  closed_grad_final_kernel<FAM><<<1, scan_threads(d), 0, stream>>>(d, (double)a, params, (const double2 *)(base + L.S),
                                                                (const double2 *)(base + L.T), (double2 *)(base + L.nu),
                                                                value, grad);
  return check_launch();
}

mdi_status closed_grad_launch(int family, int d, int64_t a, int64_t n_last, const double *params, double *value,
                              double *grad, void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if (family != MDI_FAM_EXP && family != MDI_FAM_OSC) return MDI_EUNSUPPORTED;
  if (!closed_sizes_ok(d, a, n_last)) return MDI_EINVAL;
  if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < closed_grad_workspace_bytes(d, a, n_last))
    return MDI_EWORKSPACE;
  if (family == MDI_FAM_EXP) return run_closed_grad<MDI_FAM_EXP>(d, a, n_last, params, value, grad, workspace, stream);
  return run_closed_grad<MDI_FAM_OSC>(d, a, n_last, params, value, grad, workspace, stream);
}

}  // namespace mdi
