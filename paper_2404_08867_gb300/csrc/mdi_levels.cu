// mdi_levels.cu -- node-state MDI-LR for ONE integral, parallel over levels,
// and its adjoint (the derivative of the rule with respect to c_j, w_j, u).
//
// With the node state (values of G_k at P Chebyshev points, read back by
// barycentric interpolation), level k < d of Algorithm 1 is a linear map of the
// node values:
//     G_k[p] = sum_t M_k[p][t] G_{k-1}[t],
//     M_k[p][t] = (1/a) sum_{q<a} phi_k(u_qp) l_t(u_qp),  u_qp = (q + xi_p)/a,
// and the last level is a row vector, Q = front * sum_t w[t] G_{d-1}[t] with
// w[t] = (1/n_last) sum_s phi_d(s/n_last) l_t(s/n_last), G_0 = 1.  The sweep is
// therefore a chain of P x P matrices whose construction -- where all the
// cluster evaluations are -- does not depend on the previous level.
//
// GB300 mapping (instead of walking the levels one by one on one SM):
//   K0  basis table l_t(u_qp) of this a (a*P*P entries).
//   K1  every M_k (and w) at once, one CTA per level, across the whole GPU.
//   K2  the levels are cut into groups of C (the checkpoint interval); the
//       group products R_g = M_top ... M_{gC+1} are formed on many SMs at once,
//       in two stages of about sqrt(C) operators when C >= 8 (and, for the
//       value alone with 16 or more groups, a third stage over the groups).
//   K3  one CTA runs the short chain over the groups forward (G at every group
//       boundary -- the checkpoints -- and the value) and, for the adjoint,
//       backward: lambda_{d-1} = front * w, lambda_{gC} = lambda_{top} R_g
//       (lambda_k = dQ/dG_k).  The sequential part is ceil((d-1)/C) steps, not d.
//   K4  (adjoint) each CTA takes a block of consecutive levels of one group,
//       recomputes their G_{k-1} from the checkpoint below and lambda_k from the
//       checkpoint above once for the block -- the level states are not all
//       stored -- and contracts
//           dQ/dtheta_k = lambda_k (dM_k/dtheta_k) G_{k-1}
//                       = (1/a) sum_{q,p} lambda_k[p] dphi_k(u_qp)/dtheta G~_{k-1}(u_qp),
//       theta_k = (c_k, w_k); level d uses the points s/n_last.  For OSC the
//       phase derivative dQ/du = Re(2 pi i Q) comes from K3.
#include <algorithm>
#include <atomic>

#include "mdi_common.cuh"
#include "mdi_exp2_table.inc"
#include "mdi_fp64.cuh"
#include "mdi_internal.h"
#include "mdi_nodes.cuh"

namespace mdi {

// FP64 pieces of the level kernels, built on the sweep's own exp and reciprocal
// (GB300's FP64 unit takes a warp instruction per ~64 cycles per sub-partition, and
// the library exp and IEEE division take several times their instruction count).

// 1/D for any D: the reciprocal of |D| with D's sign.
__device__ __forceinline__ double rcp_signed64(double D) {
  const double r = rcp_nr64(__hiloint2double(__double2hiint(D) & 0x7FFFFFFF, __double2loint(D)));
  return __hiloint2double(__double2hiint(r) ^ (__double2hiint(D) & (int)0x80000000), __double2loint(r));
}

// c_j, w_j and 1/c_j^2 of axis j (the reciprocal as rcp_nr64).
__device__ __forceinline__ AxisParams load_axis_lv(const double *params, int d, int j) {
  AxisParams p;
  p.c = params[j];
  p.w = params[d + j];
  p.ic2 = rcp_nr64(p.c * p.c);
  return p;
}

// phi_j(u): the formulas of phi64 with the own exp (table T) and reciprocal; in
// float when F32; OSC by sincos.
template <int FAM, bool F32>
__device__ __forceinline__ typename FamTraits<FAM>::V phi_lv(double u, const AxisParams &p, const double *T) {
  if constexpr (F32 || FAM == MDI_FAM_OSC) {
    return phi<FAM, F32>(u, p);
  } else if constexpr (FAM == MDI_FAM_EXP) {
    return exp_tang64(p.c * u, T);
  } else if constexpr (FAM == MDI_FAM_GAUSS) {
    const double t = p.c * (u - p.w);
    return exp_tang64(-t * t, T);
  } else {
    const double t = u - p.w;
    return rcp_nr64(fma(t, t, p.ic2));
  }
}

// phi_j and its derivatives in c_j and w_j (the formulas of phi_grad64) with the
// own exp and reciprocal; dcp = 2 / c_j^3, the PEAK factor of dc, per axis.
template <int FAM>
__device__ __forceinline__ PhiGrad<FAM> phi_grad_lv(double x, const AxisParams &p, double dcp, const double *T) {
  if constexpr (FAM == MDI_FAM_OSC) {
    return phi_grad64<FAM>(x, p);
  } else if constexpr (FAM == MDI_FAM_EXP) {
    const double e = exp_tang64(p.c * x, T);
    return {e, x * e, 0.0};
  } else if constexpr (FAM == MDI_FAM_GAUSS) {
    const double t = x - p.w, e = exp_tang64(-(p.c * t) * (p.c * t), T);
    return {e, -2.0 * p.c * t * t * e, 2.0 * p.c * p.c * t * e};
  } else {
    const double t = x - p.w, f = rcp_nr64(fma(t, t, p.ic2)), f2 = f * f;
    return {f, dcp * f2, 2.0 * t * f2};
  }
}

constexpr int kLvThreads = 256;
constexpr int kLvMaxPts = kNodesAMax * kNodesPMax;  // a*P <= 2048
constexpr int64_t kStepMaxRadix = 4096;              // a^m for the step-m operators

// Groups: g = 0..ng-1 covers levels gC+1 .. min((g+1)C, d-1); boundary b_g = gC
// for g < ng and b_ng = d-1.  gck[g] = G at b_g, lck[g] = lambda at b_g.
struct LevelsLayout {
  size_t table, M, runs, R, w, gck, lck, misc, total;
  int C, ng;  // checkpoint interval (= group length) and number of groups
  int r, nr;  // group products in two stages: runs of r levels, nr runs per group (nr = 1: one stage)
};

// Run length of the two-stage group products: about sqrt(C), which makes the
// r - 1 + ceil(C/r) - 1 products in sequence fewest, lengthened while the runs take
// more than 128 CTAs (one product per SM of GB300's 152) and the sequence does not
// grow.  One stage below C = 8.
static void group_runs(int C, int ng, int &r, int &nr) {
  r = C;
  nr = 1;
  if (C < 8) return;
  int s = 1;
  while (s * s < C) ++s;
  auto depth = [C](int x) { return x - 1 + (C + x - 1) / x - 1; };
  while (s + 1 < C && (int64_t)ng * ((C + s - 1) / s) > 128 && depth(s + 1) <= depth(s)) ++s;
  r = s;
  nr = (C + s - 1) / s;
}

static LevelsLayout levels_layout(int d, int64_t a, int P, int C) {
  LevelsLayout L{};
  L.C = C;
  L.ng = (d - 1 + C - 1) / C;
  group_runs(C, L.ng, L.r, L.nr);
  size_t off = 0;
  L.table = off;
  off += align_up(sizeof(double) * (size_t)a * P * P);
  L.M = off;
  off += align_up(sizeof(double2) * (size_t)std::max(d - 1, 1) * P * P);
  L.runs = off;
  if (C > 1 && L.nr > 1) off += align_up(sizeof(double2) * (size_t)std::max(L.ng, 1) * L.nr * P * P);
  L.R = off;
  if (C > 1) off += align_up(sizeof(double2) * (size_t)std::max(L.ng, 1) * P * P);
  L.w = off;
  off += align_up(sizeof(double2) * P);
  L.gck = off;
  off += align_up(sizeof(double2) * (size_t)(L.ng + 1) * P);
  L.lck = off;
  off += align_up(sizeof(double2) * (size_t)(L.ng + 1) * P);
  L.misc = off;
  off += align_up(4 * sizeof(double2));
  L.total = off;
  return L;
}

static int default_checkpoint(int d) {
  int c = 1;
  while ((int64_t)c * c < d) ++c;
  return c;
}

// K0: L[t][q*P + p] = l_t((q + xi_p)/a) for one a.  One warp per point u: lane t
// forms bw_t / (u - xi_t), a shuffle sum gives the denominator, so each lane takes
// two reciprocals (rcp_nr64: the FP64 unit is the scarce one on this chip).  DF
// writes each value as a float pair into the same 8-byte slot (the compensated
// double-float build reads it so).
template <bool DF>
__global__ void levels_table_kernel(int P, int a, double *__restrict__ L) {
  __shared__ double s_xi[kNodesPMax], s_bw[kNodesPMax];
  for (int t = threadIdx.x; t < P; t += blockDim.x) {
    s_xi[t] = cheb_node(t, P);
    s_bw[t] = cheb_weight(t, P);
  }
  __syncthreads();
  const int lane = threadIdx.x & (kWarp - 1);
  const int pt = (blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
  const int npts = a * P;
  if (pt >= npts) return;  // whole warps
  const int q = pt / P, p = pt % P;
  const double u = ((double)q + s_xi[p]) / (double)a;
  const bool on = lane < P;
  const double xi = on ? s_xi[lane] : 0.0;
  const unsigned hit = __ballot_sync(0xffffffffu, on && u == xi);
  const double r = (on && !hit) ? s_bw[lane] * rcp_signed64(u - xi) : 0.0;
  double den = r;
  for (int off = kWarp / 2; off > 0; off >>= 1) den += __shfl_xor_sync(0xffffffffu, den, off);
  if (on) {
    const double v = hit ? (lane == __ffs(hit) - 1 ? 1.0 : 0.0) : r * rcp_signed64(den);
    if constexpr (DF) {
      const float h = (float)v;
      reinterpret_cast<float2 *>(L)[(size_t)lane * npts + pt] = make_float2(h, (float)(v - (double)h));
    } else {
      L[(size_t)lane * npts + pt] = v;
    }
  }
}

// The last level's row w[t] = (1/n_last) sum_s phi_d(s/n_last) l_t(s/n_last), by
// one CTA: a group of GL lanes per point (lane t forms l_t, by the warp-per-point
// scheme of K0), partial rows in `part` (blockDim entries), w written by threads
// t < P.
template <int FAM, bool F32>
__device__ __forceinline__ void last_level_row(int d, int n_last, int P, const AxisParams &ap, const double *s_xi,
                                               const double *s_bw, const double *s_e64, double2 *part,
                                               double2 *__restrict__ w) {
  const int GL = P <= kWarp / 2 ? kWarp / 2 : kWarp;
  const int lane = threadIdx.x & (kWarp - 1), t = lane & (GL - 1);
  const int per_warp = kWarp / GL, nwarps = blockDim.x / kWarp;
  const unsigned gmask = GL == kWarp ? 0xffffffffu : (0xffffu << (lane & (kWarp / 2)));
  const bool on = t < P;
  const double xi = on ? s_xi[t] : 0.0, bw = on ? s_bw[t] : 0.0;
  double2 acc = make_double2(0.0, 0.0);
  for (int base = (threadIdx.x / kWarp) * per_warp; base < n_last; base += nwarps * per_warp) {
    const int s = base + lane / GL;  // whole warps run the loop and its shuffles
    const bool pt = s < n_last;
    const double u = (double)(pt ? s : 0) / (double)n_last;
    double l = (t == 0) ? 1.0 : 0.0;  // d = 1: G_0 = 1 is constant
    if (d > 1) {
      const unsigned hit = __ballot_sync(0xffffffffu, on && u == xi) & gmask;
      const double r = (on && !hit) ? bw * rcp_signed64(u - xi) : 0.0;
      double den = r;
      for (int off = 1; off < GL; off <<= 1) den += __shfl_xor_sync(0xffffffffu, den, off);
      l = hit ? ((on && u == xi) ? 1.0 : 0.0) : r * rcp_signed64(den);
    }
    if (pt && on) {
      const double2 f = as2(phi_lv<FAM, F32>(u, ap, s_e64));
      acc.x = fma(l, f.x, acc.x);
      if constexpr (FAM == MDI_FAM_OSC) acc.y = fma(l, f.y, acc.y);
    }
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < P) {
    double2 sum = make_double2(0.0, 0.0);
    for (int r = 0; r < (int)blockDim.x / GL; ++r) sum = c_add(sum, part[r * GL + threadIdx.x]);
    w[threadIdx.x] = c_scale(sum, 1.0 / (double)n_last);
  }
}

// K1: M_k for k = 1..d-1 (block k-1) and w (block d-1).  M is stored [k][t][p].
// PREC: FP64; FP32_EVAL_FP64 (phi in float); FP32_EVAL_DF32 (phi in float, the
// cluster sum of each entry as a Dot2 accumulation of the float-pair table values
// times the float phi values, rounded to double once per entry); DF64 (phi in
// double-float at the double coordinates -- FP64 for OSC -- and the same Dot2
// sums).  The products between levels and the last axis stay FP64.
template <int FAM, int PREC>
__global__ void __launch_bounds__(kLvThreads) levels_build_kernel(int d, int a, int n_last, int P,
                                                                  const double *__restrict__ prm,
                                                                  const double *__restrict__ L,
                                                                  double2 *__restrict__ M, double2 *__restrict__ w) {
  using V = typename FamTraits<FAM>::V;
  constexpr bool F32 = PREC == MDI_PREC_FP32_EVAL_FP64 || PREC == MDI_PREC_FP32_EVAL_DF32;
  constexpr bool DF = PREC == MDI_PREC_FP32_EVAL_DF32;
  constexpr bool D64 = PREC == MDI_PREC_DF64;
  __shared__ double s_xi[kNodesPMax], s_bw[kNodesPMax];
  __shared__ double2 s_f[DF || D64 ? 1 : kLvMaxPts];
  __shared__ float2 s_ff[DF ? kLvMaxPts : 1];
  __shared__ float4 s_fd[D64 ? kLvMaxPts : 1];  // (re.hi, re.lo, im.hi, im.lo)
  __shared__ float2 s_exp2[D64 ? kExpTable : 1];
  constexpr bool kExp64 = !F32 && FAM != MDI_FAM_OSC;  // phi_lv's table
  __shared__ double s_e64[kExp64 ? kExpTable : 1];
  __shared__ double2 s_part[kLvThreads];
  if constexpr (D64)
    for (int j = threadIdx.x; j < kExpTable; j += blockDim.x) s_exp2[j] = kExp2TableGen[j];
  if constexpr (kExp64)
    for (int j = threadIdx.x; j < kExpTable; j += blockDim.x) s_e64[j] = kExp2TableD[j];
  for (int t = threadIdx.x; t < P; t += blockDim.x) {
    s_xi[t] = cheb_node(t, P);
    s_bw[t] = cheb_weight(t, P);
  }
  __syncthreads();
  const int npts = a * P;
  const double inv_a = 1.0 / (double)a;
  // Block 0 takes the last level (w), whose points are the last axis' own, so that
  // it starts in the first wave.
  for (int b = blockIdx.x; b < d; b += gridDim.x) {
    const int lev = b == 0 ? d - 1 : b - 1;
    const AxisParams ap = load_axis_lv(prm, d, lev);
    if (lev < d - 1) {
      // level k = lev + 1 < d
      df32 cd{0.f, 0.f}, wd{0.f, 0.f}, icd{0.f, 0.f};
      if constexpr (D64 && FAM != MDI_FAM_OSC) {
        cd = df_from_double(prm[lev]);
        wd = df_from_double(prm[d + lev]);
        icd = df_rcp(df_sqr(cd));
      }
      for (int i = threadIdx.x; i < npts; i += blockDim.x) {
        const int q = i / P, p = i % P;
        const double u = ((double)q + s_xi[p]) * inv_a;
        if constexpr (D64) {
          if constexpr (FAM == MDI_FAM_OSC) {
            const double2 f = as2(phi<FAM, false>(u, ap));
            const df32 re = df_from_double(f.x), im = df_from_double(f.y);
            s_fd[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
          } else {
            const df32 f = phi_df<FAM>(df_from_double(u), make_float4(cd.hi, cd.lo, wd.hi, wd.lo),
                                       make_float2(icd.hi, icd.lo), s_exp2);
            s_fd[i] = make_float4(f.hi, f.lo, 0.f, 0.f);
          }
        } else {
          const double2 f = as2(phi_lv<FAM, F32>(u, ap, s_e64));
          if constexpr (DF) s_ff[i] = make_float2((float)f.x, (float)f.y);  // float values: exact
          else s_f[i] = f;
        }
      }
      __syncthreads();
      double2 *Mk = M + (size_t)lev * P * P;
      for (int o = threadIdx.x; o < P * P; o += blockDim.x) {
        const int t = o / P, p = o % P;
        if constexpr (DF || D64) {
          const float2 *Lt = reinterpret_cast<const float2 *>(L) + (size_t)t * npts + p;
          DfAcc ar, ai;
          for (int q = 0; q < a; ++q) {
            const float2 l = Lt[q * P];
            if constexpr (D64) {
              const float4 f = s_fd[q * P + p];
              dacc_prod(ar, df32{l.x, l.y}, df32{f.x, f.y});
              if constexpr (FAM == MDI_FAM_OSC) dacc_prod(ai, df32{l.x, l.y}, df32{f.z, f.w});
            } else {
              const float2 f = s_ff[q * P + p];
              dacc_prod(ar, df32{l.x, l.y}, df32{f.x, 0.f});
              if constexpr (FAM == MDI_FAM_OSC) dacc_prod(ai, df32{l.x, l.y}, df32{f.y, 0.f});
            }
          }
          const double im = FAM == MDI_FAM_OSC ? df_to_double(dacc_value(ai)) : 0.0;
          Mk[o] = c_scale(make_double2(df_to_double(dacc_value(ar)), im), inv_a);
        } else {
          const double *Lt = L + (size_t)t * npts + p;
          double2 acc = make_double2(0.0, 0.0);
          for (int q = 0; q < a; ++q) {
            const double l = Lt[q * P];
            const double2 f = s_f[q * P + p];
            acc.x = fma(l, f.x, acc.x);
            if constexpr (FAM == MDI_FAM_OSC) acc.y = fma(l, f.y, acc.y);
          }
          Mk[o] = c_scale(acc, inv_a);
        }
      }
      __syncthreads();
    } else {
      last_level_row<FAM, F32>(d, n_last, P, ap, s_xi, s_bw, s_e64, s_part, w);
      __syncthreads();
    }
  }
  (void)sizeof(V);
}

// Step size m of Algorithm 1 (m = 2, 3; forward value, FP64).  Operator j covers
// the cluster axes l0 = j m .. l0 + mj - 1 (0-based; mj = m, or the remainder for
// the last operator) and reads the previous state once, at the group's innermost
// coordinate:
//     M_j[p][t] = (1/a^mj) sum_{Q < a^mj} prod_{i < mj} phi_{l0+i}(x_i) l_t(x_0),
//     x_i = ((Q mod a^(mj-i)) + xi_p) / a^(mj-i),
// which is the affine recurrence x_i = (q_i + x_{i+1}) / a from x_mj = xi_p unrolled:
// the digit q_i of axis l0 + i weighs a^(mj-1-i) in Q (the innermost axis' digit
// is the most significant).  The a^mj tuples of each operator are cut into S
// slices, one CTA each (the work of an operator is a^mj P (mj phi + P) FP64
// operations: one SM per operator leaves most of the chip idle); CTA j S + s
// writes the slice's partial sums, and levels_step_sum_kernel adds the S partials
// of each entry in slice order.  The last CTA computes the last level's row w.
// The points (Q, p) go in tiles whose products of phi are staged in shared
// memory, and l_t(x_0) is read from the basis table of radix a^mj
// (levels_table_kernel with a^mj in place of a, so x_0 is the same double in both).
constexpr int kStepTile = 1024;          // points (Q, p) per tile
constexpr int kStepMaxEntries = 4;       // P*P <= kStepMaxEntries * kLvThreads
template <int FAM>
__global__ void __launch_bounds__(kLvThreads) levels_step_build_kernel(int d, int a, int n_last, int P, int m,
                                                                       int ns, int S, const double *__restrict__ prm,
                                                                       const double *__restrict__ Lm,
                                                                       const double *__restrict__ Lr,
                                                                       double2 *__restrict__ Mpart,
                                                                       double2 *__restrict__ w) {
  using V = typename FamTraits<FAM>::V;
  constexpr bool kExp64 = FAM != MDI_FAM_OSC;
  __shared__ double s_xi[kNodesPMax], s_bw[kNodesPMax];
  __shared__ double s_e64[kExp64 ? kExpTable : 1];
  __shared__ V s_f[kStepTile];
  __shared__ double2 s_part[kLvThreads];
  __shared__ AxisParams s_ap[3];
  __shared__ double s_inv[3];
  for (int t = threadIdx.x; t < P; t += blockDim.x) {
    s_xi[t] = cheb_node(t, P);
    s_bw[t] = cheb_weight(t, P);
  }
  if constexpr (kExp64)
    for (int j = threadIdx.x; j < kExpTable; j += blockDim.x) s_e64[j] = kExp2TableD[j];
  __syncthreads();
  const int tileQ = kStepTile / P;
  const int b = blockIdx.x;
  if (b < ns * S) {
    const int j = b / S, sl = b - j * S;
    const int l0 = j * m, mj = min(m, d - 1 - l0);
    int R = 1;
    for (int i = 0; i < mj; ++i) R *= a;
    const double *L = (mj == m) ? Lm : Lr;
    const int npts = R * P;
    const int Qb = (int)((int64_t)R * sl / S), Qe = (int)((int64_t)R * (sl + 1) / S);
    if (threadIdx.x < mj) {
      s_ap[threadIdx.x] = load_axis_lv(prm, d, l0 + threadIdx.x);
      int Ri = 1;
      for (int i = threadIdx.x; i < mj; ++i) Ri *= a;
      s_inv[threadIdx.x] = 1.0 / (double)Ri;  // 1 / a^(mj-ii)
    }
    V acc[kStepMaxEntries];
#pragma unroll
    for (int e = 0; e < kStepMaxEntries; ++e) acc[e] = VOps<V>::zero();
    __syncthreads();
    for (int Q0 = Qb; Q0 < Qe; Q0 += tileQ) {
      const int nq = min(tileQ, Qe - Q0);
      for (int i = threadIdx.x; i < nq * P; i += blockDim.x) {
        const int Q = Q0 + i / P, p = i % P;
        V prod = VOps<V>::one();
        int Ri = R;
        for (int ii = 0; ii < mj; ++ii) {  // x_ii = ((Q mod a^(mj-ii)) + xi_p) / a^(mj-ii)
          const double x = ((double)(Q % Ri) + s_xi[p]) * s_inv[ii];
          prod = VOps<V>::mul(prod, phi_lv<FAM, false>(x, s_ap[ii], s_e64));
          Ri /= a;
        }
        s_f[i] = prod;
      }
      __syncthreads();
#pragma unroll
      for (int e = 0; e < kStepMaxEntries; ++e) {
        const int o = threadIdx.x + e * kLvThreads;
        if (o < P * P) {
          const int t = o / P, p = o % P;
          const double *Lt = L + (size_t)t * npts + (size_t)Q0 * P + p;
          V a_e = acc[e];
          for (int q = 0; q < nq; ++q) a_e = VOps<V>::fma_s(Lt[(size_t)q * P], s_f[q * P + p], a_e);
          acc[e] = a_e;
        }
      }
      __syncthreads();
    }
    double2 *Mp = Mpart + (size_t)b * P * P;
#pragma unroll
    for (int e = 0; e < kStepMaxEntries; ++e) {
      const int o = threadIdx.x + e * kLvThreads;
      if (o < P * P) Mp[o] = as2(acc[e]);  // stored [t][p]; scaled by 1/a^mj in the sum
    }
  } else {
    last_level_row<FAM, false>(d, n_last, P, load_axis_lv(prm, d, d - 1), s_xi, s_bw, s_e64, s_part, w);
  }
}

// M_j = (1/a^mj) sum_s Mpart[j S + s], the slices in order (one thread per entry).
__global__ void levels_step_sum_kernel(int d, int a, int m, int ns, int S, int pp,
                                       const double2 *__restrict__ Mpart, double2 *__restrict__ M) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)ns * pp) return;
  const int j = (int)(idx / pp), o = (int)(idx - (int64_t)j * pp);
  const int mj = min(m, d - 1 - j * m);
  int R = 1;
  for (int i = 0; i < mj; ++i) R *= a;
  const double2 *src = Mpart + (size_t)j * S * pp + o;
  double2 acc = make_double2(0.0, 0.0);
  for (int s = 0; s < S; ++s) acc = c_add(acc, src[(size_t)s * pp]);
  M[idx] = c_scale(acc, 1.0 / (double)R);
}

// cp.async helpers for staging operators into shared memory (hardware
// wait_group, double-buffered), so no product waits on an L2 round trip.
constexpr int kChainMaxThreads = 8 * kNodesPMax;  // eight lanes per row of a P x P product

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Operators ops_first .. ops_first+cnt-1 (1-based) -> dst, one 16-byte copy each.
// Operators are stored [t][p]; `transpose` stages each one as [p][t], a thread
// taking the same entries (t, p) of every operator so that it divides by P once
// per entry rather than once per copy.
__device__ __forceinline__ void stage_ops(double2 *dst, const double2 *ops, int first, int cnt, int P, bool transpose) {
  const int pp = P * P;
  const double2 *src = ops + (size_t)(first - 1) * pp;
  if (!transpose) {
    for (int i = threadIdx.x; i < cnt * pp; i += blockDim.x) cp_async16(dst + i, src + i);
  } else {
    for (int e = threadIdx.x; e < pp; e += blockDim.x) {
      const int t = e / P, j = (e - t * P) * P + t;  // e = t*P + p -> p*P + t
      for (int lev = 0; lev < cnt; ++lev) cp_async16(dst + lev * pp + j, src + lev * pp + e);
    }
  }
  cp_async_commit();
}

// K2: R_g = M_hi ... M_lo for the levels lo = gC+1 .. hi = min((g+1)C, d-1) of
// each group g, in one or two stages of products of consecutive operators, one
// CTA per product:
//   stage 0, CTA b = g nr + j: the run of levels gC + 1 + j r .. min(gC + (j+1) r,
//     (g+1)C, d-1) of group g (an empty run of a short last group writes nothing);
//     with r = C, nr = 1 this is R_g itself;
//   stage 1, CTA g: the product of group g's run products g nr + 1 .. g nr + nr_g
//     (1-based; nr_g = ceil(len_g / r)).
// Two stages take r - 1 + nr - 1 products in sequence instead of C - 1, on nr times
// as many SMs (the FP64 unit of one SM takes about a microsecond per 16 x 16
// product).  Thread (p, t) forms entry (p, t) of each partial product R' = M_k R,
// R'[p][t] = sum_s M_k[p][s] R[s][t], from the operator staged in shared memory
// (the next one is in flight meanwhile) and R in shared memory, [s][t] row-major.
// Products are written [t][p] like the operators.
constexpr int kGroupMaxThreads = kNodesPMax * kNodesPMax;

template <int FAM>
__global__ void __launch_bounds__(kGroupMaxThreads) levels_group_kernel(int d, int P, int C, int r, int nr, int stage,
                                                                     const double2 *__restrict__ M,
                                                                     double2 *__restrict__ R) {
  extern __shared__ __align__(16) unsigned char group_smem[];
  const int pp = P * P;
  double2 *const sM = (double2 *)group_smem;  // two staged operators
  double2 *const sR = sM + 2 * pp;             // two partial products
  int lo, hi;
  if (stage == 0) {
    const int g = blockIdx.x / nr, j = blockIdx.x - g * nr;
    lo = g * C + 1 + j * r;
    hi = min(lo + r - 1, min((g + 1) * C, d - 1));
  } else {
    const int g = blockIdx.x, len = min((g + 1) * C, d - 1) - g * C;
    lo = g * nr + 1;
    hi = g * nr + (len + r - 1) / r;
  }
  if (lo > hi) return;  // the whole CTA, before any barrier
  const int g = blockIdx.x;  // the product written
  const int i = threadIdx.x, p = i / P, t = i % P;
  const bool on = i < pp;
  if (on) sR[p * P + t] = M[(size_t)(lo - 1) * pp + t * P + p];  // R = M_lo
  if (lo + 1 <= hi) stage_ops(sM, M, lo + 1, 1, P, false);
  int cur = 0;
  for (int k = lo + 1; k <= hi; ++k) {
    const int j = (k - lo - 1) & 1;
    if (k + 1 <= hi) {
      stage_ops(sM + (j ^ 1) * pp, M, k + 1, 1, P, false);
      cp_async_wait_prev();
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
    if (on) {
      const double2 *Mk = sM + j * pp;
      const double2 *Rc = sR + cur * pp;
      double2 acc = make_double2(0.0, 0.0);
      if constexpr (FAM == MDI_FAM_OSC) {
        for (int s = 0; s < P; ++s) acc = c_add(acc, c_mul(Mk[s * P + p], Rc[s * P + t]));
      } else {
        for (int s = 0; s < P; ++s) acc.x = fma(Mk[s * P + p].x, Rc[s * P + t].x, acc.x);
      }
      sR[(cur ^ 1) * pp + p * P + t] = acc;
    }
    cur ^= 1;
    __syncthreads();
  }
  if (on) R[(size_t)g * pp + t * P + p] = sR[cur * pp + p * P + t];
}

// Sum of v over aligned groups of G lanes (G a power of two <= 32); the result is
// valid in every lane of the group.
template <typename V> __device__ __forceinline__ V group_sum(V v, int G);
template <> __device__ __forceinline__ double group_sum<double>(double v, int G) {
  for (int off = 1; off < G; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off, G);
  return v;
}
template <> __device__ __forceinline__ double2 group_sum<double2>(double2 v, int G) {
  for (int off = 1; off < G; off <<= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, off, G);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, off, G);
  }
  return v;
}

// One entry of a level operator: real families read the real part only.
template <typename V> __device__ __forceinline__ V op_entry(const double2 *e);
template <> __device__ __forceinline__ double op_entry<double>(const double2 *e) {
  return reinterpret_cast<const double *>(e)[0];
}
template <> __device__ __forceinline__ double2 op_entry<double2>(const double2 *e) { return *e; }

// K3: the chain over the ng group operators (R_g, or M_k when C = 1), forward
// with a checkpoint at every group boundary and the value, backward for the
// adjoint.  One CTA: eight lanes per row of each matrix-vector product, each
// summing every eighth term, then three shuffle rounds (on GB300 a warp's FP64
// instruction holds its sub-partition's FP64 unit for about 64 cycles, so fewer,
// fuller warps finish a product sooner than one multiply per thread); the vector
// is double-buffered in shared memory, one barrier per product.  Each lane reads
// its entries of the operators straight from global memory into a ring of
// registers kChainAhead products ahead of their use, so no product waits on an L2
// round trip and nothing is staged through shared memory.  Real families use real
// arithmetic on the real parts (and load only those).  misc[0] = Q before the
// front factor.
constexpr int kChainAhead = 4;                  // products in flight per lane
constexpr int kChainMaxE = kNodesPMax / 8;      // entries per lane and product

template <int FAM>
__global__ void __launch_bounds__(kChainMaxThreads) levels_chain_kernel(int d, int ng, int P,
                                                                     const double *__restrict__ prm,
                                                                     const double2 *__restrict__ ops,
                                                                     const double2 *__restrict__ w,
                                                                     double2 *__restrict__ gck,
                                                                     double2 *__restrict__ lck,
                                                                     double2 *__restrict__ misc,
                                                                     double *__restrict__ value,
                                                                     double *__restrict__ grad, int adjoint) {
  using V = typename FamTraits<FAM>::V;
  using O = VOps<V>;
  __shared__ V s_v[2][kNodesPMax];  // the chain's vector, double-buffered
  const int row = threadIdx.x >> 3, part = threadIdx.x & 7;
  const bool rowok = row < P;
  const int p = threadIdx.x;
  const bool on = p < P;
  const size_t pp = (size_t)P * P;
  // This lane's entries of product st: forward, operator st + 1, row p and column
  // t at t*P + p; backward, operator ng - st transposed, row t and column p at
  // t*P + p.
  auto fetch = [&](bool fwd, int st, V(&e)[kChainMaxE]) {
    const double2 *Op = ops + (size_t)(fwd ? st : ng - 1 - st) * pp;
#pragma unroll
    for (int j = 0; j < kChainMaxE; ++j) {
      const int col = part + 8 * j;
      if (rowok && col < P) e[j] = op_entry<V>(Op + (fwd ? col * P + row : row * P + col));
    }
  };
  // The ng products in order; the new vector of product st goes to the checkpoint
  // st + 1 (forward) or ng - 1 - st (backward).  Returns the buffer holding the
  // last vector.
  auto run = [&](bool fwd, double2 *ck) -> int {
    int vb = 0;
    V ring[kChainAhead][kChainMaxE];
#pragma unroll
    for (int u = 0; u < kChainAhead; ++u)
#pragma unroll
      for (int j = 0; j < kChainMaxE; ++j) ring[u][j] = O::zero();
#pragma unroll
    for (int u = 0; u < kChainAhead; ++u)
      if (u < ng) fetch(fwd, u, ring[u]);
    for (int k0 = 0; k0 < ng; k0 += kChainAhead) {
#pragma unroll
      for (int u = 0; u < kChainAhead; ++u) {
        const int st = k0 + u;
        if (st < ng) {  // the same in every thread
          V acc = O::zero();
#pragma unroll
          for (int j = 0; j < kChainMaxE; ++j) {
            const int col = part + 8 * j;
            if (rowok && col < P) {
              if constexpr (FAM == MDI_FAM_OSC) acc = c_add(acc, c_mul(ring[u][j], s_v[vb][col]));
              else acc = fma(ring[u][j], s_v[vb][col], acc);
            }
          }
          acc = group_sum(acc, 8);
          if (st + kChainAhead < ng) fetch(fwd, st + kChainAhead, ring[u]);
          if (rowok && part == 0) {
            s_v[vb ^ 1][row] = acc;
            ck[(size_t)(fwd ? st + 1 : ng - 1 - st) * P + row] = as2(acc);
          }
          vb ^= 1;
          __syncthreads();
        }
      }
    }
    return vb;
  };
  if (on) {
    s_v[0][p] = O::one();
    gck[p] = as2(O::one());
  }
  __syncthreads();
  // Forward: S_k[p] = sum_t R_k[p][t] S_{k-1}[t], checkpoints gck[1..ng].
  const int vb = run(true, gck);
  // Q = front * sum_t w[t] G_{d-1}[t]
  double2 front = make_double2(1.0, 0.0);
  if (FAM == MDI_FAM_OSC) {
    double sn, cs;
    sincos(kTwoPi * prm[d], &sn, &cs);
    front = make_double2(cs, sn);
  }
  if (threadIdx.x < kWarp) {  // the P terms on the lanes of warp 0, then a shuffle sum
    const int t = threadIdx.x;
    double2 q = make_double2(0.0, 0.0);
    if (t < P) {
      if constexpr (FAM == MDI_FAM_OSC) q = c_mul(w[t], as2(s_v[vb][t]));
      else q.x = w[t].x * as2(s_v[vb][t]).x;  // real w and G
    }
    if constexpr (FAM == MDI_FAM_OSC) q = warp_sum(q);
    else q.x = warp_sum(q.x);
    if (t == 0) {
      misc[0] = q;
      const double2 fq = c_mul(front, q);
      if (value) *value = fq.x;
      if (adjoint && FAM == MDI_FAM_OSC) grad[d] = -kTwoPi * fq.y;  // dQ/du = Re(2 pi i front q)
    }
  }
  if (adjoint && FAM == MDI_FAM_OSC)
    for (int j = d + 1 + (int)threadIdx.x; j < 2 * d; j += blockDim.x) grad[j] = 0.0;
  if (!adjoint) return;
  __syncthreads();
  // lambda at b_ng = d-1 is front * w (real for real families: front = 1, w real).
  if (on) {
    const double2 l = c_mul(front, w[p]);
    s_v[0][p] = from2<V>(l);
    lck[(size_t)ng * P + p] = l;
  }
  __syncthreads();
  // Backward: Lambda_{k-1}[t] = sum_p Lambda_k[p] R_k[p][t], checkpoints lck[ng-1..0].
  run(false, lck);
}

// Product of a level operator (stored [t][p]: entry (p, t) at t*P + p) with a
// vector in shared memory: out[p] = sum_t Op[p][t] in[t], or with TRANSPOSE
// out[t] = sum_p in[p] Op[p][t].  Eight lanes per output, each summing every
// eighth term, then three shuffle rounds; the outputs are spread over P/4 warps
// so every SM sub-partition's FP64 unit takes a share (the FP64 rate of one warp
// is the bottleneck otherwise).  Threads past the last whole warp skip.
template <typename V, bool TRANSPOSE>
__device__ __forceinline__ void matvec8(const double2 *__restrict__ Op, const V *in, V *out, int P) {
  const int i = threadIdx.x, row = i >> 3, part = i & 7;
  if (i >= ((P * 8 + kWarp - 1) & ~(kWarp - 1))) return;
  V acc = VOps<V>::zero();
  if (row < P) {
    for (int t = part; t < P; t += 8) {
      const double2 m = TRANSPOSE ? Op[row * P + t] : Op[t * P + row];
      if constexpr (sizeof(V) == sizeof(double2)) acc = c_add(acc, c_mul(m, in[t]));
      else acc = fma(m.x, in[t], acc);
    }
  }
  acc = group_sum(acc, 8);
  if (row < P && part == 0) out[row] = acc;
}

// Operator entries for the recompute products of K4: a lane holds E entries of a
// row, the row spread over rec_lanes(E) lanes -- E = 2 (eight lanes per row) or
// E = 4 (four) up to P = 16, E = 8 (four) up to P = 32 -- so that a G product and a
// lambda product run side by side, each on at most 128 threads.  On GB300 a warp's
// FP64 instruction holds its sub-partition's FP64 unit for about 64 cycles: eight
// lanes per row (two FMAs and three shuffle rounds) give the shortest chain of
// dependent FP64 instructions per product, four lanes (four FMAs and two rounds on
// half the warps) leave the unit more room for the contractions of a block of
// levels running alongside.
__host__ __device__ constexpr int rec_lanes(int E) { return E == 2 ? 8 : 4; }
constexpr int kGradMaxLevels = 8;  // levels per CTA in K4


// A lane's entries (row, part + j rec_lanes(E)), j < E, of a level operator stored
// [t][p]: not TRANSPOSE, out[p] = sum_t Op[p][t] in[t] (row p, column t at t*P + p);
// TRANSPOSE, out[t] = sum_p in[p] Op[p][t] (row t, column p at t*P + p).
template <typename V, bool TRANSPOSE, int E>
__device__ __forceinline__ void op_fetch(const double2 *__restrict__ Op, int row, int part, int P, V (&e)[E]) {
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int col = part + j * rec_lanes(E);
    if (row < P && col < P) e[j] = op_entry<V>(Op + (TRANSPOSE ? row * P + col : col * P + row));
  }
}

// Per-level constants of K4: the axis, and 2 / c^3 (PEAK: d phi / dc = (2 / c^3) phi^2).
struct GradAxis {
  AxisParams ap;
  double dcp;
};

// K4: gradients of a block of consecutive levels of one checkpoint group, or of
// level d.  CTA b < ng nb takes block j = b mod nb of group g = b / nb, the levels
// klo = gC + 1 + jB .. khi = min(klo + B - 1, (g+1)C, d-1) (none for the short
// last group's spare blocks); the last CTA takes level d.  Every level of a group
// recomputes from the same checkpoints: G from G_gC up through the operators
// gC+1 .. khi-1 and lambda from lambda_top (top = min((g+1)C, d-1)) down through
// top .. klo+1, the states of the block's own levels kept in shared memory -- so a
// CTA of B levels takes one chain of each kind, not B, and no level state outside
// the block and the checkpoints is ever stored.  The two chains run side by side
// (one barrier per step of the longer), a lane holding its entries of the next
// operator in registers while it multiplies by the current one.  The phi
// derivatives at each thread's first point do not depend on the states and are
// evaluated before the chains, so their FP64 work fills the pipe while the
// products wait on one another.  Then, level by level,
//     dQ/dtheta_k = (1/a) sum_{q,p} lambda_k[p] dphi_k(u_qp)/dtheta G~_{k-1}(u_qp),
// warp sums per level into shared memory and one fixed-order sum at the end.  Real
// families run in real arithmetic (the operators' imaginary parts are zero).
template <int FAM, int E>
__global__ void __launch_bounds__(kLvThreads, 2) levels_grad_kernel(int d, int a, int n_last, int P, int C, int B,
                                                                 int nb, const double *__restrict__ prm,
                                                                 const double *__restrict__ L,
                                                                 const double2 *__restrict__ M,
                                                                 const double2 *__restrict__ gck,
                                                                 const double2 *__restrict__ lck,
                                                                 double *__restrict__ grad) {
  using V = typename FamTraits<FAM>::V;
  using O = VOps<V>;
  constexpr bool kExp64 = FAM != MDI_FAM_OSC;
  constexpr int kSlots = 2 + kGradMaxLevels;  // two chain temporaries, then the block's levels
  __shared__ double s_xi[kNodesPMax], s_bw[kNodesPMax];
  __shared__ double s_e64[kExp64 ? kExpTable : 1];
  __shared__ V s_g[kSlots][kNodesPMax], s_l[kSlots][kNodesPMax];
  __shared__ GradAxis s_ax[kGradMaxLevels];
  __shared__ double2 s_part[kGradMaxLevels][kLvThreads / kWarp];
  const int tid = threadIdx.x, lane = tid & (kWarp - 1), warp = tid / kWarp;
  const int ng = (d - 1 + C - 1) / C;
  const int npts = a * P;
  const double inv_a = 1.0 / (double)a;
  // This CTA's levels klo..khi, the checkpoint group g0 of G, and lambda's top.
  int g0, klo, khi, top = 0;
  const double2 *lsrc = nullptr;
  if ((int)blockIdx.x < ng * nb) {
    const int g = blockIdx.x / nb, j = blockIdx.x - g * nb;
    g0 = g;
    klo = g * C + 1 + j * B;
    top = min((g + 1) * C, d - 1);
    khi = min(klo + B - 1, top);
    if (klo > khi) return;  // the whole CTA, before any barrier
    lsrc = lck + (size_t)((g + 1) * C > d - 1 ? ng : g + 1) * P;
  } else {
    g0 = (d - 1) / C;
    klo = khi = d;
  }
  const int nlev = khi - klo + 1;
  for (int t = tid; t < P; t += blockDim.x) {
    s_xi[t] = cheb_node(t, P);
    s_bw[t] = cheb_weight(t, P);
  }
  if constexpr (kExp64)
    for (int j = tid; j < kExpTable; j += blockDim.x) s_e64[j] = kExp2TableD[j];
  if (tid < nlev) {
    const AxisParams ap = load_axis_lv(prm, d, klo + tid - 1);
    s_ax[tid] = GradAxis{ap, 2.0 * ap.ic2 * rcp_signed64(ap.c)};
  }
  double2 front = make_double2(1.0, 0.0);
  if (FAM == MDI_FAM_OSC) {
    double sn, cs;
    sincos(kTwoPi * prm[d], &sn, &cs);
    front = make_double2(cs, sn);
  }
  __syncthreads();
  // Level klo < d reads the points (q + xi_p)/a, level d the points s/n_last.
  const int npt = klo < d ? npts : n_last;
  auto point = [&](int k, int i) {
    return k < d ? ((double)(i / P) + s_xi[i % P]) * inv_a : (double)i / (double)n_last;
  };
  PhiGrad<FAM> pg0{};
  if (tid < npt) pg0 = phi_grad_lv<FAM>(point(klo, tid), s_ax[0].ap, s_ax[0].dcp, s_e64);

  // The chains.  G: vector i = G_{g0 C + i}, i = 0..nG, over the operators
  // g0 C + 1 + st; lambda: vector i = lambda_{top - i}, i = 0..nL, over the
  // transposed operators top - st.  The vectors of the block's levels (G_{k-1},
  // lambda_k for klo <= k <= khi) go to slots 2 + (k - klo), the others alternate
  // between slots 0 and 1.
  const int nG = (khi - 1) - g0 * C, gfirst = (klo - 1) - g0 * C;
  const int nL = klo < d ? top - klo : 0, lfirst = klo < d ? top - khi : 0;
  auto gslot = [&](int i) { return i >= gfirst ? 2 + (i - gfirst) : (i & 1); };
  auto lslot = [&](int i) { return i >= lfirst ? 2 + (top - i - klo) : (i & 1); };
  // Side 0 (G) and side 1 (lambda) take the first whole warps: for P = 16 warps 0-1
  // and 2-3, one per SM sub-partition, so that the two chains' FP64 instructions
  // queue on different units; the other warps sit the chains out.
  constexpr int LR = rec_lanes(E);
  const int side_threads = (P * LR + kWarp - 1) / kWarp * kWarp;
  const int side = tid / side_threads, li = tid % side_threads;
  const int row = li / LR, part = li % LR;
  const int mine = side == 0 ? nG : side == 1 ? nL : 0;
  const size_t pp = (size_t)P * P;
  // Operator of step st: G side g0 C + 1 + st, lambda side top - st (1-based).
  const double2 *op0 = side == 1 && top > 0 ? M + (size_t)(top - 1) * pp : M + (size_t)g0 * C * pp;
  const ptrdiff_t opstep = side == 1 ? -(ptrdiff_t)pp : (ptrdiff_t)pp;
  V cur[E], nxt[E];
#pragma unroll
  for (int j = 0; j < E; ++j) cur[j] = nxt[j] = O::zero();
  if (mine > 0) {
    if (side) op_fetch<V, true, E>(op0, row, part, P, cur);
    else op_fetch<V, false, E>(op0, row, part, P, cur);
  }
  if (tid < P) s_g[gslot(0)][tid] = from2<V>(gck[(size_t)g0 * P + tid]);
  if (klo < d && side == 1 && li < P) s_l[lslot(0)][li] = from2<V>(lsrc[li]);
  __syncthreads();
  const int nsteps = max(nG, nL);
  for (int st = 0; st < nsteps; ++st) {
    if (st < mine) {  // the same in every lane of a warp
      if (st + 1 < mine) {
        const double2 *op = op0 + (st + 1) * opstep;
        if (side) op_fetch<V, true, E>(op, row, part, P, nxt);
        else op_fetch<V, false, E>(op, row, part, P, nxt);
      }
      const V *in = side ? s_l[lslot(st)] : s_g[gslot(st)];
      V acc = O::zero();
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int col = part + j * LR;
        if (row < P && col < P) {
          if constexpr (FAM == MDI_FAM_OSC) acc = c_add(acc, c_mul(cur[j], in[col]));
          else acc = fma(cur[j], in[col], acc);
        }
      }
      acc = group_sum(acc, LR);
      if (row < P && part == 0) (side ? s_l[lslot(st + 1)] : s_g[gslot(st + 1)])[row] = acc;
#pragma unroll
      for (int j = 0; j < E; ++j) cur[j] = nxt[j];
    }
    __syncthreads();
  }

  // The contractions, level by level.
  for (int lv = 0; lv < nlev; ++lv) {
    const int k = klo + lv;
    const GradAxis ax = s_ax[lv];
    const V *g_k = s_g[2 + lv];  // G_{k-1}
    const V *l_k = s_l[2 + lv];  // lambda_k (k < d)
    V acc_c = O::zero(), acc_w = O::zero();
    if (k < d) {
      auto contract = [&](int i, const PhiGrad<FAM> &pg) {
        V g = O::one();
        if (k > 1) {
          g = O::zero();
          for (int t = 0; t < P; ++t) g = O::fma_s(L[(size_t)t * npts + i], g_k[t], g);
        }
        const V lg = O::mul(l_k[i % P], g);
        acc_c = O::add(acc_c, O::mul(lg, pg.dc));
        acc_w = O::add(acc_w, O::mul(lg, pg.dw));
      };
      const int i0 = lv == 0 ? tid + blockDim.x : tid;
      if (lv == 0 && tid < npts) contract(tid, pg0);
      for (int i = i0; i < npts; i += blockDim.x) contract(i, phi_grad_lv<FAM>(point(k, i), ax.ap, ax.dcp, s_e64));
    } else {
      // level d: Re(front (1/n_last) sum_s dphi_d(s/n_last) G~_{d-1}(s/n_last))
      auto contract = [&](double u, const PhiGrad<FAM> &pg) {
        V g = O::one();
        if (d > 1) {
          V num = O::zero();
          double den = 0.0;
          int hit = -1;
          for (int t = 0; t < P; ++t) {
            if (u == s_xi[t]) {
              hit = t;
              continue;
            }
            const double wt = s_bw[t] * rcp_signed64(u - s_xi[t]);
            den += wt;
            num = O::fma_s(wt, g_k[t], num);
          }
          g = hit >= 0 ? g_k[hit] : O::scale(num, rcp_signed64(den));
        }
        const V fg = from2<V>(c_mul(front, as2(g)));
        acc_c = O::add(acc_c, O::mul(fg, pg.dc));
        acc_w = O::add(acc_w, O::mul(fg, pg.dw));
      };
      if (tid < n_last) contract(point(d, tid), pg0);
      for (int i = tid + blockDim.x; i < n_last; i += blockDim.x) {
        const double u = point(d, i);
        contract(u, phi_grad_lv<FAM>(u, ax.ap, ax.dcp, s_e64));
      }
    }
    double2 both;
    if constexpr (FAM == MDI_FAM_OSC) both = as2(acc_c);  // complex: its real part is the gradient
    else both = make_double2(acc_c, acc_w);
    both = warp_sum(both);
    if (lane == 0) s_part[lv][warp] = both;
  }
  __syncthreads();
  if (tid < nlev) {
    const int k = klo + tid, nw = blockDim.x / kWarp;
    double2 tot = make_double2(0.0, 0.0);
    for (int w = 0; w < nw; ++w) tot = c_add(tot, s_part[tid][w]);
    const double scale = (k < d) ? inv_a : 1.0 / (double)n_last;
    grad[k - 1] = tot.x * scale;
    if (FAM != MDI_FAM_OSC) grad[d + k - 1] = tot.y * scale;
  }
}

// K4 for the step size m > 1: CTA j S + s takes slice s of operator k = j + 1,
// which contracts the axes l0 = j m .. l0 + mj - 1 over the a^mj digit tuples
// (Q, p) (the slices cut the tuples as in levels_step_build_kernel); the last CTA
// takes the last axis.  With G_{k-1} and lambda_k recomputed from the checkpoints
// as above (every slice of an operator recomputes the same two chains), each axis
// ii of the operator gets
//     dQ/dtheta_ii = (1/a^mj) sum_{Q,p} lambda_k[p] (prod_{jj != ii} phi_jj) dphi_ii/dtheta G~_{k-1}(x_0),
// the product rule over the tuple's factors (x_jj = ((Q mod a^(mj-jj)) + xi_p) /
// a^(mj-jj), as the operator's build), G~ read at x_0 from the radix-a^mj table.
// A slice writes its partial sums (c and w for each of its axes) to Gpart, and
// levels_step_grad_sum_kernel adds them in slice order.
constexpr int kStepMaxM = 3;
template <int FAM>
__global__ void __launch_bounds__(kLvThreads) levels_step_grad_kernel(int d, int a, int n_last, int P, int m, int ns,
                                                                      int S, int C, const double *__restrict__ prm,
                                                                      const double *__restrict__ Lm,
                                                                      const double *__restrict__ Lr,
                                                                      const double2 *__restrict__ M,
                                                                      const double2 *__restrict__ gck,
                                                                      const double2 *__restrict__ lck,
                                                                      double2 *__restrict__ Gpart,
                                                                      double *__restrict__ grad) {
  using V = typename FamTraits<FAM>::V;
  constexpr bool kExp64 = FAM != MDI_FAM_OSC;
  __shared__ double s_xi[kNodesPMax], s_bw[kNodesPMax];
  __shared__ double s_e64[kExp64 ? kExpTable : 1];
  __shared__ V s_g[2][kNodesPMax], s_l[2][kNodesPMax];
  __shared__ V s_red[kLvThreads / kWarp];
  __shared__ GradAxis s_ax[kStepMaxM];
  __shared__ double s_inv[kStepMaxM];
  for (int t = threadIdx.x; t < P; t += blockDim.x) {
    s_xi[t] = cheb_node(t, P);
    s_bw[t] = cheb_weight(t, P);
  }
  if constexpr (kExp64)
    for (int j = threadIdx.x; j < kExpTable; j += blockDim.x) s_e64[j] = kExp2TableD[j];
  const int ng = C > 1 ? (ns + C - 1) / C : ns;
  double2 front = make_double2(1.0, 0.0);
  if (FAM == MDI_FAM_OSC) {
    double sn, cs;
    sincos(kTwoPi * prm[d], &sn, &cs);
    front = make_double2(cs, sn);
  }
  const int tid = threadIdx.x;
  const int b = blockIdx.x < ns * S ? blockIdx.x / S : ns;  // operators applied before this unit
  const int sl = blockIdx.x < ns * S ? blockIdx.x - b * S : 0;
  // G after b operators, from the checkpoint at or below it (ping-pong buffers).
  const int j0 = b / C;
  int cg = 0;
  if (tid < P) s_g[0][tid] = from2<V>(gck[(size_t)j0 * P + tid]);
  __syncthreads();
  for (int op = j0 * C + 1; op <= b; ++op) {
    matvec8<V, false>(M + (size_t)(op - 1) * P * P, s_g[cg], s_g[cg ^ 1], P);
    cg ^= 1;
    __syncthreads();
  }
  const V *g_b = s_g[cg];
  if (b < ns) {
    const int k = b + 1, l0 = b * m, mj = min(m, d - 1 - l0);
    int R = 1;
    for (int i = 0; i < mj; ++i) R *= a;
    const double *L = (mj == m) ? Lm : Lr;
    const int npts = R * P;
    const int ib = (int)((int64_t)R * sl / S) * P, ie = (int)((int64_t)R * (sl + 1) / S) * P;
    // lambda_k from the checkpoint at or above it.
    int top = ((k + C - 1) / C) * C;
    const double2 *src;
    if (top > ns) {
      top = ns;
      src = lck + (size_t)ng * P;
    } else {
      src = lck + (size_t)(top / C) * P;
    }
    int cl = 0;
    if (tid < P) s_l[0][tid] = from2<V>(src[tid]);
    if (tid < mj) {
      const AxisParams ap = load_axis_lv(prm, d, l0 + tid);
      s_ax[tid] = GradAxis{ap, 2.0 * ap.ic2 * rcp_signed64(ap.c)};
      int Ri = 1;
      for (int i = tid; i < mj; ++i) Ri *= a;
      s_inv[tid] = 1.0 / (double)Ri;
    }
    __syncthreads();
    for (int op = top; op >= k + 1; --op) {
      matvec8<V, true>(M + (size_t)(op - 1) * P * P, s_l[cl], s_l[cl ^ 1], P);
      cl ^= 1;
      __syncthreads();
    }
    const V *l_k = s_l[cl];
    V acc_c[kStepMaxM], acc_w[kStepMaxM];
#pragma unroll
    for (int ii = 0; ii < kStepMaxM; ++ii) acc_c[ii] = acc_w[ii] = VOps<V>::zero();
    for (int i = ib + tid; i < ie; i += blockDim.x) {
      const int Q = i / P, p = i % P;
      PhiGrad<FAM> pg[kStepMaxM];
      int Ri = R;
#pragma unroll
      for (int ii = 0; ii < kStepMaxM; ++ii) {
        if (ii < mj) {
          const double x = ((double)(Q % Ri) + s_xi[p]) * s_inv[ii];
          pg[ii] = phi_grad_lv<FAM>(x, s_ax[ii].ap, s_ax[ii].dcp, s_e64);
          Ri /= a;
        }
      }
      V g = VOps<V>::one();
      if (b > 0) {
        g = VOps<V>::zero();
        for (int t = 0; t < P; ++t) g = VOps<V>::fma_s(L[(size_t)t * npts + i], g_b[t], g);
      }
      const V lg = VOps<V>::mul(l_k[p], g);
#pragma unroll
      for (int ii = 0; ii < kStepMaxM; ++ii) {
        if (ii < mj) {
          V others = lg;
#pragma unroll
          for (int jj = 0; jj < kStepMaxM; ++jj)
            if (jj < mj && jj != ii) others = VOps<V>::mul(others, pg[jj].f);
          acc_c[ii] = VOps<V>::add(acc_c[ii], VOps<V>::mul(others, pg[ii].dc));
          acc_w[ii] = VOps<V>::add(acc_w[ii], VOps<V>::mul(others, pg[ii].dw));
        }
      }
    }
#pragma unroll
    for (int ii = 0; ii < kStepMaxM; ++ii) {
      if (ii < mj) {  // mj is the same in every thread of the block
        const V tc = block_sum(acc_c[ii], s_red);
        const V tw = block_sum(acc_w[ii], s_red);
        if (tid == 0) Gpart[((size_t)blockIdx.x * kStepMaxM + ii)] = make_double2(as2(tc).x, as2(tw).x);
      }
    }
  } else {
    // last axis: dQ/dtheta_d = Re(front (1/n_last) sum_s dphi_d(s/n_last) G~(s/n_last))
    const AxisParams ap = load_axis_lv(prm, d, d - 1);
    const double dcp = 2.0 * ap.ic2 * rcp_signed64(ap.c);
    V acc_c = VOps<V>::zero(), acc_w = VOps<V>::zero();
    for (int s = tid; s < n_last; s += blockDim.x) {
      const double u = (double)s / (double)n_last;
      const PhiGrad<FAM> pg = phi_grad_lv<FAM>(u, ap, dcp, s_e64);
      V g = VOps<V>::one();
      if (d > 1) {
        V num = VOps<V>::zero();
        double den = 0.0;
        int hit = -1;
        for (int t = 0; t < P; ++t) {
          if (u == s_xi[t]) {
            hit = t;
            continue;
          }
          const double wt = s_bw[t] * rcp_signed64(u - s_xi[t]);
          den += wt;
          num = VOps<V>::fma_s(wt, g_b[t], num);
        }
        g = hit >= 0 ? g_b[hit] : VOps<V>::scale(num, rcp_signed64(den));
      }
      const V fg = from2<V>(c_mul(front, as2(g)));
      acc_c = VOps<V>::add(acc_c, VOps<V>::mul(fg, pg.dc));
      acc_w = VOps<V>::add(acc_w, VOps<V>::mul(fg, pg.dw));
    }
    const V tc = block_sum(acc_c, s_red);
    const V tw = block_sum(acc_w, s_red);
    if (tid == 0) {
      grad[d - 1] = as2(tc).x / (double)n_last;
      if (FAM != MDI_FAM_OSC) grad[2 * d - 1] = as2(tw).x / (double)n_last;
    }
  }
}

// The step-m gradients of the cluster axes: (1/a^mj) times the slices' partial
// sums, in slice order (one thread per axis).
template <int FAM>
__global__ void levels_step_grad_sum_kernel(int d, int a, int m, int ns, int S, const double2 *__restrict__ Gpart,
                                            double *__restrict__ grad) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;  // cluster axis 0 .. d-2
  if (l >= d - 1) return;
  const int j = l / m, ii = l - j * m, mj = min(m, d - 1 - j * m);
  int R = 1;
  for (int i = 0; i < mj; ++i) R *= a;
  double2 acc = make_double2(0.0, 0.0);
  for (int s = 0; s < S; ++s) acc = c_add(acc, Gpart[((size_t)(j * S + s) * kStepMaxM + ii)]);
  const double invR = 1.0 / (double)R;
  grad[l] = acc.x * invR;
  if (FAM != MDI_FAM_OSC) grad[d + l] = acc.y * invR;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
// The group kernel's dynamic shared-memory limit, set once per device
// (an attribute belongs to the device whose context sets it; setting it twice from
// racing threads is harmless).
template <int FAM> static mdi_status levels_kernel_attrs() {
  static std::atomic<int> done[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  cudaGetLastError();
  const bool cached = dev >= 0 && dev < 64;
  if (cached && done[dev].load(std::memory_order_acquire)) return MDI_OK;
  const cudaError_t e = cudaFuncSetAttribute(levels_group_kernel<FAM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(4 * sizeof(double2) * kNodesPMax * kNodesPMax));
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return MDI_ECUDA;
  }
  if (cached) done[dev].store(1, std::memory_order_release);
  return MDI_OK;
}

size_t levels_workspace_bytes(int d, int64_t a, const NodesConfig &cfg, int checkpoint) {
  const int C = checkpoint > 0 ? checkpoint : default_checkpoint(d);
  return levels_layout(d, a, cfg.P, C).total;
}

template <int FAM, int PREC>
static mdi_status run_levels(int d, int a, int n_last, const double *params, const NodesConfig &cfg, int C,
                             double *value, double *grad, void *ws, cudaStream_t stream) {
  const LevelsLayout Lo = levels_layout(d, a, cfg.P, C);
  char *base = (char *)ws;
  double *L = (double *)(base + Lo.table);
  double2 *M = (double2 *)(base + Lo.M), *w = (double2 *)(base + Lo.w);
  double2 *gck = (double2 *)(base + Lo.gck), *lck = (double2 *)(base + Lo.lck), *misc = (double2 *)(base + Lo.misc);
  const int P = cfg.P;
  constexpr bool kDfTable = PREC == MDI_PREC_FP32_EVAL_DF32 || PREC == MDI_PREC_DF64;
  levels_table_kernel<kDfTable><<<(a * P + 7) / 8, 8 * kWarp, 0, stream>>>(P, a, L);
  mdi_status st = check_launch();
  if (st != MDI_OK) return st;
  const int grid = std::min(d, sm_count() * 8);
  levels_build_kernel<FAM, PREC><<<grid, kLvThreads, 0, stream>>>(d, a, n_last, P, params, L, M, w);
  if ((st = check_launch()) != MDI_OK) return st;
  if ((st = levels_kernel_attrs<FAM>()) != MDI_OK) return st;
  // Group products (skipped when every group is one level: the operators are M).
  const double2 *ops = M;
  if (C > 1 && Lo.ng > 0) {
    double2 *R = (double2 *)(base + Lo.R);
    const size_t group_smem = 4 * sizeof(double2) * (size_t)P * P;
    const int gthreads = std::max(32, (P * P + 31) / 32 * 32);
    if (Lo.nr > 1) {
      double2 *runs = (double2 *)(base + Lo.runs);
      levels_group_kernel<FAM><<<Lo.ng * Lo.nr, gthreads, group_smem, stream>>>(d, P, C, Lo.r, Lo.nr, 0, M, runs);
      if ((st = check_launch()) != MDI_OK) return st;
      levels_group_kernel<FAM><<<Lo.ng, gthreads, group_smem, stream>>>(d, P, C, Lo.r, Lo.nr, 1, runs, R);
    } else {
      levels_group_kernel<FAM><<<Lo.ng, gthreads, group_smem, stream>>>(d, P, C, C, 1, 0, M, R);
    }
    if ((st = check_launch()) != MDI_OK) return st;
    ops = R;
  }
  // The value alone needs no checkpoints: with many groups, the chain runs over
  // products of about sqrt(ng) consecutive group products (one more product stage,
  // written over the level operators, which are no longer read), so the sequence of
  // dependent matrix-vector products is about 2 sqrt(ng) long instead of ng.
  int nchain = Lo.ng;
  if (!grad && C > 1 && Lo.ng >= 16) {
    int s = 1;
    while (s * s < Lo.ng) ++s;
    const int nsg = (Lo.ng + s - 1) / s;
    const size_t group_smem = 4 * sizeof(double2) * (size_t)P * P;
    const int gthreads = std::max(32, (P * P + 31) / 32 * 32);
    levels_group_kernel<FAM><<<nsg, gthreads, group_smem, stream>>>(Lo.ng + 1, P, s, s, 1, 0, ops, M);
    if ((st = check_launch()) != MDI_OK) return st;
    ops = M;
    nchain = nsg;
  }
  const int chain_threads = std::max(32, (8 * P + 31) / 32 * 32);
  levels_chain_kernel<FAM><<<1, chain_threads, 0, stream>>>(d, nchain, P, params, ops, w, gck, lck, misc, value, grad,
                                                            grad ? 1 : 0);
  if ((st = check_launch()) != MDI_OK) return st;
  if (grad) {
    // Blocks of B levels per CTA: one level each while the grid stays near 256 CTAs
    // (the contractions spread over every SM), more levels for deep chains (one
    // recompute serves them all).
    const int B = std::max(1, std::min({kGradMaxLevels, C, (d + 255) / 256}));
    const int nb = (C + B - 1) / B;
    const int grid = Lo.ng * nb + 1;
    if (P <= 16 && B == 1)
      levels_grad_kernel<FAM, 2><<<grid, kLvThreads, 0, stream>>>(d, a, n_last, P, C, B, nb, params, L, M, gck, lck,
                                                                   grad);
    else if (P <= 16)
      levels_grad_kernel<FAM, 4><<<grid, kLvThreads, 0, stream>>>(d, a, n_last, P, C, B, nb, params, L, M, gck, lck,
                                                                   grad);
    else
      levels_grad_kernel<FAM, 8><<<grid, kLvThreads, 0, stream>>>(d, a, n_last, P, C, B, nb, params, L, M, gck, lck,
                                                                   grad);
    st = check_launch();
  }
  return st;
}

// Step size m > 1: workspace | table of radix a^m | table of radix a^rem | M (ns
// operators) | their slices' partial sums | the gradient slices' partial sums | R
// | w | gck | lck | misc, with ns = ceil((d-1)/m) operators in groups of C, each
// cut into S slices of its tuples.
struct StepLayout {
  size_t Lm, Lr, M, Mpart, Gpart, R, w, gck, lck, misc, total;
  int ns, ng, C, Rm, Rr, S;
};
// Slices per step operator: about two CTAs per SM of a 152-SM GB300 over all
// operators, a slice holding at least 16 tuples.
static int step_slices(int ns, int Rm) {
  return std::max(1, std::min((304 + ns - 1) / std::max(ns, 1), Rm / 16));
}
static StepLayout step_layout(int d, int64_t a, int P, int m, int checkpoint) {
  StepLayout L{};
  L.ns = (d - 1 + m - 1) / m;
  L.C = checkpoint > 0 ? checkpoint : default_checkpoint(std::max(L.ns, 1));
  L.ng = L.C > 1 ? (L.ns + L.C - 1) / L.C : L.ns;
  const int rem = (d - 1) % m;
  L.Rm = 1;
  for (int i = 0; i < m; ++i) L.Rm *= (int)a;
  L.Rr = 1;
  for (int i = 0; i < rem; ++i) L.Rr *= (int)a;
  L.S = step_slices(L.ns, L.Rm);
  size_t off = 0;
  L.Lm = off;
  off += align_up(sizeof(double) * (size_t)L.Rm * P * P);
  L.Lr = off;
  if (rem) off += align_up(sizeof(double) * (size_t)L.Rr * P * P);
  L.M = off;
  off += align_up(sizeof(double2) * (size_t)std::max(L.ns, 1) * P * P);
  L.Mpart = off;
  off += align_up(sizeof(double2) * (size_t)std::max(L.ns, 1) * L.S * P * P);
  L.Gpart = off;
  off += align_up(sizeof(double2) * (size_t)std::max(L.ns, 1) * L.S * kStepMaxM);
  L.R = off;
  if (L.C > 1) off += align_up(sizeof(double2) * (size_t)std::max(L.ng, 1) * P * P);
  L.w = off;
  off += align_up(sizeof(double2) * P);
  L.gck = off;
  off += align_up(sizeof(double2) * (size_t)(L.ng + 1) * P);
  L.lck = off;
  off += align_up(sizeof(double2) * (size_t)(L.ng + 1) * P);
  L.misc = off;
  off += align_up(4 * sizeof(double2));
  L.total = off;
  return L;
}

static bool step_sizes_ok(int64_t a, int m) {
  int64_t R = 1;
  for (int i = 0; i < m; ++i) {
    R *= a;
    if (R > kStepMaxRadix) return false;
  }
  return true;
}

size_t levels_step_workspace_bytes(int d, int64_t a, const NodesConfig &cfg, int checkpoint) {
  if (cfg.step < 2 || !step_sizes_ok(a, cfg.step)) return 0;
  return step_layout(d, a, cfg.P, cfg.step, checkpoint).total;
}

template <int FAM>
static mdi_status run_levels_step(int d, int a, int n_last, const double *params, const NodesConfig &cfg,
                                  int checkpoint, double *value, double *grad, void *ws, cudaStream_t stream) {
  const int P = cfg.P, m = cfg.step;
  const StepLayout Lo = step_layout(d, a, P, m, checkpoint);
  char *base = (char *)ws;
  double *Lm = (double *)(base + Lo.Lm), *Lr = (double *)(base + Lo.Lr);
  double2 *M = (double2 *)(base + Lo.M), *w = (double2 *)(base + Lo.w);
  double2 *gck = (double2 *)(base + Lo.gck), *lck = (double2 *)(base + Lo.lck), *misc = (double2 *)(base + Lo.misc);
  levels_table_kernel<false><<<(Lo.Rm * P + 7) / 8, 8 * kWarp, 0, stream>>>(P, Lo.Rm, Lm);
  mdi_status st = check_launch();
  if (st != MDI_OK) return st;
  if ((d - 1) % m) {
    levels_table_kernel<false><<<(Lo.Rr * P + 7) / 8, 8 * kWarp, 0, stream>>>(P, Lo.Rr, Lr);
    if ((st = check_launch()) != MDI_OK) return st;
  }
  double2 *Mpart = (double2 *)(base + Lo.Mpart), *Gpart = (double2 *)(base + Lo.Gpart);
  levels_step_build_kernel<FAM><<<Lo.ns * Lo.S + 1, kLvThreads, 0, stream>>>(d, a, n_last, P, m, Lo.ns, Lo.S, params,
                                                                            Lm, Lr, Mpart, w);
  if ((st = check_launch()) != MDI_OK) return st;
  if (Lo.ns > 0) {
    const int64_t entries = (int64_t)Lo.ns * P * P;
    levels_step_sum_kernel<<<(unsigned)((entries + 255) / 256), 256, 0, stream>>>(d, a, m, Lo.ns, Lo.S, P * P, Mpart,
                                                                                M);
    if ((st = check_launch()) != MDI_OK) return st;
  }
  if ((st = levels_kernel_attrs<FAM>()) != MDI_OK) return st;
  // The operators play the levels' part in the group products and the chain: the
  // group kernel reads its "d - 1" as the operator count.
  const double2 *ops = M;
  if (Lo.C > 1 && Lo.ng > 0) {
    double2 *Rg = (double2 *)(base + Lo.R);
    const size_t group_smem = 4 * sizeof(double2) * (size_t)P * P;
    levels_group_kernel<FAM><<<Lo.ng, std::max(32, (P * P + 31) / 32 * 32), group_smem, stream>>>(
        Lo.ns + 1, P, Lo.C, Lo.C, 1, 0, M, Rg);
    if ((st = check_launch()) != MDI_OK) return st;
    ops = Rg;
  }
  const int chain_threads = std::max(32, (8 * P + 31) / 32 * 32);
  levels_chain_kernel<FAM><<<1, chain_threads, 0, stream>>>(d, Lo.ng, P, params, ops, w, gck, lck, misc, value, grad,
                                                            grad ? 1 : 0);
  if ((st = check_launch()) != MDI_OK || !grad) return st;
  levels_step_grad_kernel<FAM><<<Lo.ns * Lo.S + 1, kLvThreads, 0, stream>>>(d, a, n_last, P, m, Lo.ns, Lo.S, Lo.C,
                                                                           params, Lm, Lr, M, gck, lck, Gpart, grad);
  if ((st = check_launch()) != MDI_OK || d < 2) return st;
  levels_step_grad_sum_kernel<FAM><<<(d - 1 + 255) / 256, 256, 0, stream>>>(d, a, m, Lo.ns, Lo.S, Gpart, grad);
  return check_launch();
}

template <int FAM>
static mdi_status run_levels_p(int precision, int d, int a, int n_last, const double *params, const NodesConfig &cfg,
                               int C, double *value, double *grad, void *ws, cudaStream_t stream) {
  switch (precision) {
    case MDI_PREC_FP32_EVAL_FP64:
      return run_levels<FAM, MDI_PREC_FP32_EVAL_FP64>(d, a, n_last, params, cfg, C, value, grad, ws, stream);
    case MDI_PREC_FP32_EVAL_DF32:
      return run_levels<FAM, MDI_PREC_FP32_EVAL_DF32>(d, a, n_last, params, cfg, C, value, grad, ws, stream);
    case MDI_PREC_DF64:
      return run_levels<FAM, MDI_PREC_DF64>(d, a, n_last, params, cfg, C, value, grad, ws, stream);
    default: return run_levels<FAM, MDI_PREC_FP64>(d, a, n_last, params, cfg, C, value, grad, ws, stream);
  }
}

mdi_status levels_launch(int family, int d, int64_t a, int64_t n_last, const double *params, const NodesConfig &cfg,
                         int checkpoint, double *value, double *grad, void *workspace, size_t ws_bytes,
                         cudaStream_t stream) {
  if (d < 1 || d > (1 << 16) || a < 1 || a > kNodesAMax || n_last < 1 || n_last > 4096) return MDI_EUNSUPPORTED;
  if (cfg.P < 2 || cfg.P > kNodesPMax || (cfg.P & 1)) return MDI_EINVAL;
  if (grad && cfg.precision != MDI_PREC_FP64) return MDI_EUNSUPPORTED;
  if (cfg.step > 1) {  // Algorithm 1 with m = 2, 3 in FP64: value and adjoint
    if (cfg.precision != MDI_PREC_FP64 || !step_sizes_ok(a, cfg.step)) return MDI_EUNSUPPORTED;
    if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < levels_step_workspace_bytes(d, a, cfg, checkpoint))
      return MDI_EWORKSPACE;
    const int ai = (int)a, nl = (int)n_last;
    switch (family) {
      case MDI_FAM_EXP:
        return run_levels_step<MDI_FAM_EXP>(d, ai, nl, params, cfg, checkpoint, value, grad, workspace, stream);
      case MDI_FAM_OSC:
        return run_levels_step<MDI_FAM_OSC>(d, ai, nl, params, cfg, checkpoint, value, grad, workspace, stream);
      case MDI_FAM_GAUSS:
        return run_levels_step<MDI_FAM_GAUSS>(d, ai, nl, params, cfg, checkpoint, value, grad, workspace, stream);
      default:
        return run_levels_step<MDI_FAM_PEAK>(d, ai, nl, params, cfg, checkpoint, value, grad, workspace, stream);
    }
  }
  const int C = checkpoint > 0 ? checkpoint : default_checkpoint(d);
  if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < levels_layout(d, a, cfg.P, C).total)
    return MDI_EWORKSPACE;
  const int ai = (int)a, nl = (int)n_last;
  switch (family) {
    case MDI_FAM_EXP: return run_levels_p<MDI_FAM_EXP>(cfg.precision, d, ai, nl, params, cfg, C, value, grad,
                                                         workspace, stream);
    case MDI_FAM_OSC: return run_levels_p<MDI_FAM_OSC>(cfg.precision, d, ai, nl, params, cfg, C, value, grad,
                                                         workspace, stream);
    case MDI_FAM_GAUSS: return run_levels_p<MDI_FAM_GAUSS>(cfg.precision, d, ai, nl, params, cfg, C, value, grad,
                                                             workspace, stream);
    default: return run_levels_p<MDI_FAM_PEAK>(cfg.precision, d, ai, nl, params, cfg, C, value, grad, workspace,
                                               stream);
  }
}

}  // namespace mdi
