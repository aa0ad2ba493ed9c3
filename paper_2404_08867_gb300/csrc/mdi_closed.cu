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
  if (precision == MDI_PREC_DF64) return MDI_EUNSUPPORTED;
  if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < closed_workspace_bytes(d)) return MDI_EWORKSPACE;
  if (family == MDI_FAM_EXP) return run_closed_p<MDI_FAM_EXP>(precision, d, a, n_last, params, out, workspace, stream);
  return run_closed_p<MDI_FAM_OSC>(precision, d, a, n_last, params, out, workspace, stream);
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
__global__ void __launch_bounds__(kLevelThreads) closed_grad_level_kernel(int d, int64_t a, int64_t n_last,
                                                                          const double *__restrict__ gamma,
                                                                          double2 *__restrict__ S,
                                                                          double2 *__restrict__ T) {
  const int lane = threadIdx.x & (kWarp - 1);
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) / kWarp;
  const int nwarps = gridDim.x * blockDim.x / kWarp;
  for (int k = warp_global; k < d; k += nwarps) {
    const int64_t r = (k + 1 < d) ? a : n_last;
    const double g = gamma[k], invr = 1.0 / (double)r;
    double2 s = make_double2(0.0, 0.0), t = make_double2(0.0, 0.0);
    for (int64_t q = lane; q < r; q += kWarp) {
      const double x = (double)q * invr;
      double2 e;
      if constexpr (FAM == MDI_FAM_OSC) {
        double sn, cs;
        sincos(g * x, &sn, &cs);
        e = make_double2(cs, sn);
      } else {
        e = make_double2(exp(g * x), 0.0);
      }
      s = c_add(s, e);
      t = c_add(t, c_scale(e, x));
    }
    s = warp_sum(s);
    t = warp_sum(t);
    if (lane == 0) {
      S[k] = c_scale(s, invr);
      T[k] = c_scale(t, invr);
    }
  }
}

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

size_t closed_grad_workspace_bytes(int d) {
  return align_up(sizeof(double) * (size_t)d) + 3 * align_up(sizeof(double2) * (size_t)d);
}

template <int FAM>
static mdi_status run_closed_grad(int d, int64_t a, int64_t n_last, const double *params, double *value,
                                  double *grad, void *ws, cudaStream_t stream) {
  char *base = (char *)ws;
  double *gamma = (double *)base;
  double2 *S = (double2 *)(base + align_up(sizeof(double) * (size_t)d));
  double2 *T = S + 0;
  T = (double2 *)((char *)S + align_up(sizeof(double2) * (size_t)d));
  double2 *nu = (double2 *)((char *)T + align_up(sizeof(double2) * (size_t)d));
  closed_scan_kernel<<<1, kScanThreads, 0, stream>>>(d, (double)a, (double)n_last, params, gamma);
  mdi_status st = check_launch();
  if (st != MDI_OK) return st;
  const int grid = std::max(1, std::min((d + kLevelWarps - 1) / kLevelWarps, sm_count() * 8));
  closed_grad_level_kernel<FAM><<<grid, kLevelThreads, 0, stream>>>(d, a, n_last, gamma, S, T);
  if ((st = check_launch()) != MDI_OK) return st;
  closed_grad_final_kernel<FAM><<<1, kScanThreads, 0, stream>>>(d, (double)a, params, S, T, nu, value, grad);
  return check_launch();
}

mdi_status closed_grad_launch(int family, int d, int64_t a, int64_t n_last, const double *params, double *value,
                              double *grad, void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if (family != MDI_FAM_EXP && family != MDI_FAM_OSC) return MDI_EUNSUPPORTED;
  if (d < 1 || d > (1 << 20) || a < 1 || n_last < 1) return MDI_EINVAL;
  if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < closed_grad_workspace_bytes(d))
    return MDI_EWORKSPACE;
  if (family == MDI_FAM_EXP) return run_closed_grad<MDI_FAM_EXP>(d, a, n_last, params, value, grad, workspace, stream);
  return run_closed_grad<MDI_FAM_OSC>(d, a, n_last, params, value, grad, workspace, stream);
}

}  // namespace mdi
