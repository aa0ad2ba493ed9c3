// mdi_closed.cu -- MDI-LR with the closed level state (MDI_STATE_CLOSED) for the
// exponential families EXP (phi_j = exp(c_j x)) and OSC (phi_j = exp(i c_j x)).
//
// With phi_k(x) = exp(c~_k x) (c~ = c or i c) the level recursion of Algorithm 1,
//     G_k(x) = (1/r_k) sum_{q<r_k} phi_k(u) G_{k-1}(u),   u = (q + x) / r_k,
// keeps the form G_k(x) = K_k exp(beta_k x):
//     gamma_k = beta_{k-1} + c~_k,   beta_k = gamma_k / r_k,
//     K_k = K_{k-1} S_k,  S_k = (1/r_k) sum_{q<r_k} exp(gamma_k q / r_k),
// and the rule is front * K_d (front = exp(2 pi i u) for OSC).  The cluster
// evaluation of level k is the sum S_k over its r_k points.
//
// GB300 mapping.  beta is an affine recurrence (beta_k = beta_{k-1}/r_k + c_k/r_k;
// for OSC the same real recurrence gives the imaginary part), so instead of
// walking the d levels one after the other on one SM, one CTA solves it with a
// block-wide scan of affine maps; then the cluster sums of all levels run at
// once across the whole GPU (one warp per level, lanes over q, shuffle
// reduction), each CTA multiplies its levels' S_k in level order, and one CTA
// multiplies the CTA partial products in order.  Three launches, independent of d.
#include <algorithm>

#include "mdi_common.cuh"
#include "mdi_internal.h"

namespace mdi {

constexpr int kScanThreads = 1024;
constexpr int kLevelThreads = 256;
constexpr int kLevelWarps = kLevelThreads / kWarp;

// gamma_k (real: the exponent rate, or its imaginary part for OSC) for k = 1..d.
__global__ void __launch_bounds__(kScanThreads) closed_scan_kernel(int d, double a, double n_last,
                                                                   const double *__restrict__ params,
                                                                   double *__restrict__ gamma) {
  __shared__ double sA[kScanThreads], sB[kScanThreads];
  const int per = (d + blockDim.x - 1) / blockDim.x;
  const int lo = threadIdx.x * per, hi = min(d - 1, lo + per);  // maps for levels lo+1..hi (k < d)
  // Composite of beta_k = beta_{k-1}/r + c_k/r over this thread's levels.
  double A = 1.0, B = 0.0;
  const double inva = 1.0 / a;
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
      double cA = sA[threadIdx.x], cB = sB[threadIdx.x];
      sA[threadIdx.x] = cA * pA;
      sB[threadIdx.x] = cA * pB + cB;
    }
    __syncthreads();
  }
  double beta = threadIdx.x == 0 ? 0.0 : sB[threadIdx.x - 1];  // beta at the start of the chunk
  for (int k = lo; k < min(d, lo + per); ++k) {
    double g = beta + params[k];
    gamma[k] = g;
    beta = g * inva;
  }
  (void)n_last;
}

template <int FAM, int PREC>
__global__ void __launch_bounds__(kLevelThreads) closed_level_kernel(int d, int64_t a, int64_t n_last,
                                                                     const double *__restrict__ gamma,
                                                                     typename FamTraits<FAM>::V *__restrict__ partial) {
  using V = typename FamTraits<FAM>::V;
  __shared__ V sS[kLevelWarps * 8];
  const int per_block = (d + gridDim.x - 1) / gridDim.x;
  const int k_lo = blockIdx.x * per_block, k_hi = min(d, k_lo + per_block);
  const int lane = threadIdx.x & (kWarp - 1), warp = threadIdx.x / kWarp;
  V prod = VOps<V>::one();
  // Levels of this block in chunks of kLevelWarps*8, product kept in level order.
  for (int base = k_lo; base < k_hi; base += kLevelWarps * 8) {
    const int cnt = min(kLevelWarps * 8, k_hi - base);
    for (int s = warp; s < cnt; s += kLevelWarps) {
      const int k = base + s;
      const int64_t r = (k + 1 < d) ? a : n_last;
      const double g = gamma[k], invr = 1.0 / (double)r;
      V acc = VOps<V>::zero();
      df32 acc_hi{0.f, 0.f}, acc_im{0.f, 0.f};
      for (int64_t q = lane; q < r; q += kWarp) {
        const double arg = g * (double)q * invr;
        if constexpr (FAM == MDI_FAM_OSC) {
          double sn, cs;
          if constexpr (PREC == MDI_PREC_FP64) {
            sincos(arg, &sn, &cs);
          } else {
            float fs, fc;
            sincosf((float)arg, &fs, &fc);
            sn = fs;
            cs = fc;
          }
          if constexpr (PREC == MDI_PREC_FP32_EVAL_DF32) {
            acc_hi = df_add(acc_hi, df32{(float)cs, 0.f});
            acc_im = df_add(acc_im, df32{(float)sn, 0.f});
          } else {
            acc = VOps<V>::add(acc, make_double2(cs, sn));
          }
        } else {
          if constexpr (PREC == MDI_PREC_FP64) {
            acc = VOps<V>::add(acc, exp(arg));
          } else if constexpr (PREC == MDI_PREC_FP32_EVAL_FP64) {
            acc = VOps<V>::add(acc, (double)expf((float)arg));
          } else {
            acc_hi = df_add(acc_hi, df32{expf((float)arg), 0.f});
          }
        }
      }
      if constexpr (PREC == MDI_PREC_FP32_EVAL_DF32) {
#pragma unroll
        for (int off = kWarp / 2; off > 0; off >>= 1) {
          acc_hi = df_add(acc_hi, df_shfl_down(acc_hi, off));
          if constexpr (FAM == MDI_FAM_OSC) acc_im = df_add(acc_im, df_shfl_down(acc_im, off));
        }
        if constexpr (FAM == MDI_FAM_OSC) acc = make_double2(df_to_double(acc_hi), df_to_double(acc_im));
        else acc = df_to_double(acc_hi);
      } else {
        acc = warp_sum(acc);
      }
      if (lane == 0) sS[s] = VOps<V>::scale(acc, invr);
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int s = 0; s < cnt; ++s) prod = VOps<V>::mul(prod, sS[s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = prod;
}

template <int FAM>
__global__ void closed_final_kernel(int nparts, int d, const double *__restrict__ params,
                                    const typename FamTraits<FAM>::V *__restrict__ partial, double *__restrict__ out) {
  using V = typename FamTraits<FAM>::V;
  if (threadIdx.x != 0) return;
  V K = VOps<V>::one();
  for (int i = 0; i < nparts; ++i) K = VOps<V>::mul(K, partial[i]);
  if constexpr (FAM == MDI_FAM_OSC) {
    double s, c;
    sincos(kTwoPi * params[d], &s, &c);
    out[0] = c * K.x - s * K.y;
  } else {
    out[0] = K;
  }
}

static int closed_grid(int d) {
  // One warp per level; at least a few levels per warp before adding CTAs.
  int want = (d + kLevelWarps * 2 - 1) / (kLevelWarps * 2);
  return std::max(1, std::min(want, sm_count() * 4));
}

size_t closed_workspace_bytes(int d) {
  return align_up(sizeof(double) * (size_t)d) + align_up(16 * (size_t)closed_grid(d));
}

template <int FAM, int PREC>
static mdi_status run_closed(int d, int64_t a, int64_t n_last, const double *params, double *out, void *ws,
                             cudaStream_t stream) {
  using V = typename FamTraits<FAM>::V;
  double *gamma = (double *)ws;
  V *partial = (V *)((char *)ws + align_up(sizeof(double) * (size_t)d));
  closed_scan_kernel<<<1, kScanThreads, 0, stream>>>(d, (double)a, (double)n_last, params, gamma);
  mdi_status st = check_launch();
  if (st != MDI_OK) return st;
  const int grid = closed_grid(d);
  closed_level_kernel<FAM, PREC><<<grid, kLevelThreads, 0, stream>>>(d, a, n_last, gamma, partial);
  if ((st = check_launch()) != MDI_OK) return st;
  closed_final_kernel<FAM><<<1, 32, 0, stream>>>(grid, d, params, partial, out);
  return check_launch();
}

template <int FAM>
static mdi_status run_closed_p(int precision, int d, int64_t a, int64_t n_last, const double *params, double *out,
                               void *ws, cudaStream_t stream) {
  switch (precision) {
    case MDI_PREC_FP64: return run_closed<FAM, MDI_PREC_FP64>(d, a, n_last, params, out, ws, stream);
    case MDI_PREC_FP32_EVAL_FP64: return run_closed<FAM, MDI_PREC_FP32_EVAL_FP64>(d, a, n_last, params, out, ws, stream);
    default: return run_closed<FAM, MDI_PREC_FP32_EVAL_DF32>(d, a, n_last, params, out, ws, stream);
  }
}

mdi_status closed_launch(int family, int d, int64_t a, int64_t n_last, const double *params, int precision,
                         double *out, void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if (family != MDI_FAM_EXP && family != MDI_FAM_OSC) return MDI_EUNSUPPORTED;
  if (d < 1 || d > (1 << 20) || a < 1 || n_last < 1) return MDI_EINVAL;
  if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < closed_workspace_bytes(d)) return MDI_EWORKSPACE;
  if (family == MDI_FAM_EXP) return run_closed_p<MDI_FAM_EXP>(precision, d, a, n_last, params, out, workspace, stream);
  return run_closed_p<MDI_FAM_OSC>(precision, d, a, n_last, params, out, workspace, stream);
}

}  // namespace mdi
