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
//   K2  one CTA runs the P x P chain forward (G_k, checkpointed every C levels,
//       and the value) and, for the adjoint, backward:
//           lambda_{d-1} = front * w,   lambda_{k-1} = lambda_k M_k
//       (lambda_k = dQ/dG_k, checkpointed every C levels).
//   K3  (adjoint) one CTA per level k recomputes G_{k-1} from the checkpoint
//       below and lambda_k from the checkpoint above -- the level states are not
//       all stored -- and contracts
//           dQ/dtheta_k = lambda_k (dM_k/dtheta_k) G_{k-1}
//                       = (1/a) sum_{q,p} lambda_k[p] dphi_k(u_qp)/dtheta G~_{k-1}(u_qp),
//       theta_k = (c_k, w_k); level d uses the points s/n_last.  For OSC the
//       phase derivative dQ/du = Re(2 pi i Q) comes from K2.
#include <algorithm>

#include "mdi_common.cuh"
#include "mdi_internal.h"
#include "mdi_nodes.cuh"

namespace mdi {

constexpr int kLvThreads = 256;
constexpr int kLvMaxPts = kNodesAMax * kNodesPMax;  // a*P <= 2048

struct LevelsLayout {
  size_t table, M, w, gck, lck, misc, total;
  int C, nck;  // checkpoint interval and slots
};

static LevelsLayout levels_layout(int d, int64_t a, int P, int C) {
  LevelsLayout L{};
  L.C = C;
  L.nck = (d - 1) / C + 1;
  size_t off = 0;
  L.table = off;
  off += align_up(sizeof(double) * (size_t)a * P * P);
  L.M = off;
  off += align_up(sizeof(double2) * (size_t)std::max(d - 1, 1) * P * P);
  L.w = off;
  off += align_up(sizeof(double2) * P);
  L.gck = off;
  off += align_up(sizeof(double2) * (size_t)L.nck * P);
  L.lck = off;
  off += align_up(sizeof(double2) * (size_t)(L.nck + 1) * P);
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

// K0: L[t][q*P + p] = l_t((q + xi_p)/a) for one a.
__global__ void levels_table_kernel(int P, int a, double *__restrict__ L) {
  __shared__ double s_xi[kNodesPMax], s_bw[kNodesPMax];
  for (int t = threadIdx.x; t < P; t += blockDim.x) {
    s_xi[t] = cheb_node(t, P);
    s_bw[t] = cheb_weight(t, P);
  }
  __syncthreads();
  const int npts = a * P;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npts; i += gridDim.x * blockDim.x) {
    const int q = i / P, p = i % P;
    const double u = ((double)q + s_xi[p]) / (double)a;
    double den = 0.0;
    int hit = -1;
    for (int t = 0; t < P; ++t) {
      if (u == s_xi[t]) hit = t;
      else den += s_bw[t] / (u - s_xi[t]);
    }
    for (int t = 0; t < P; ++t)
      L[(size_t)t * npts + i] = hit >= 0 ? (t == hit ? 1.0 : 0.0) : (s_bw[t] / (u - s_xi[t])) / den;
  }
}

// Barycentric basis value l_t(u) with the nodes and weights in shared memory.
__device__ __forceinline__ double basis_at(const double *xi, const double *bw, int P, int t, double u) {
  double den = 0.0;
  for (int j = 0; j < P; ++j) {
    if (u == xi[j]) return j == t ? 1.0 : 0.0;
    den += bw[j] / (u - xi[j]);
  }
  return (bw[t] / (u - xi[t])) / den;
}

// K1: M_k for k = 1..d-1 (block k-1) and w (block d-1).  M is stored [k][t][p].
template <int FAM, bool F32>
__global__ void __launch_bounds__(kLvThreads) levels_build_kernel(int d, int a, int n_last, int P,
                                                                  const double *__restrict__ prm,
                                                                  const double *__restrict__ L,
                                                                  double2 *__restrict__ M, double2 *__restrict__ w) {
  using V = typename FamTraits<FAM>::V;
  __shared__ double s_xi[kNodesPMax], s_bw[kNodesPMax];
  __shared__ double2 s_f[kLvMaxPts];
  __shared__ double2 s_part[kLvThreads];
  for (int t = threadIdx.x; t < P; t += blockDim.x) {
    s_xi[t] = cheb_node(t, P);
    s_bw[t] = cheb_weight(t, P);
  }
  __syncthreads();
  const int npts = a * P;
  const double inv_a = 1.0 / (double)a;
  for (int lev = blockIdx.x; lev < d; lev += gridDim.x) {
    const AxisParams ap = load_axis(prm, d, lev);
    if (lev < d - 1) {
      // level k = lev + 1 < d
      for (int i = threadIdx.x; i < npts; i += blockDim.x) {
        const int q = i / P, p = i % P;
        s_f[i] = as2(phi<FAM, F32>(((double)q + s_xi[p]) * inv_a, ap));
      }
      __syncthreads();
      double2 *Mk = M + (size_t)lev * P * P;
      for (int o = threadIdx.x; o < P * P; o += blockDim.x) {
        const int t = o / P, p = o % P;
        const double *Lt = L + (size_t)t * npts + p;
        double2 acc = make_double2(0.0, 0.0);
        for (int q = 0; q < a; ++q) {
          const double l = Lt[q * P];
          const double2 f = s_f[q * P + p];
          acc.x = fma(l, f.x, acc.x);
          acc.y = fma(l, f.y, acc.y);
        }
        Mk[o] = c_scale(acc, inv_a);
      }
      __syncthreads();
    } else {
      // last level: w[t] = (1/n_last) sum_s phi_d(s/n_last) l_t(s/n_last)
      const int rows = blockDim.x / P;
      const int t = threadIdx.x % P, j = threadIdx.x / P;
      double2 acc = make_double2(0.0, 0.0);
      if (j < rows) {
        for (int s = j; s < n_last; s += rows) {
          const double u = (double)s / (double)n_last;
          const double2 f = as2(phi<FAM, F32>(u, ap));
          const double l = (d == 1) ? (t == 0 ? 1.0 : 0.0) : basis_at(s_xi, s_bw, P, t, u);
          acc.x = fma(l, f.x, acc.x);
          acc.y = fma(l, f.y, acc.y);
        }
      }
      s_part[threadIdx.x] = acc;
      __syncthreads();
      if (threadIdx.x < P) {
        double2 s = make_double2(0.0, 0.0);
        for (int r = 0; r < rows; ++r) s = c_add(s, s_part[r * P + threadIdx.x]);
        w[threadIdx.x] = c_scale(s, 1.0 / (double)n_last);
      }
      __syncthreads();
    }
  }
  (void)sizeof(V);
}

// K2: forward chain with checkpoints and the value; backward chain for the adjoint.
// One CTA of P threads.  misc[0] = complex Q before the front factor.
template <int FAM>
__global__ void levels_chain_kernel(int d, int P, int C, const double *__restrict__ prm,
                                    const double2 *__restrict__ M, const double2 *__restrict__ w,
                                    double2 *__restrict__ gck, double2 *__restrict__ lck, double2 *__restrict__ misc,
                                    double *__restrict__ value, double *__restrict__ grad, int adjoint) {
  __shared__ double2 s_v[kNodesPMax], s_n[kNodesPMax];
  const int p = threadIdx.x;
  const bool on = p < P;
  if (on) s_v[p] = make_double2(1.0, 0.0);
  __syncthreads();
  if (on) gck[p] = s_v[p];
  for (int k = 1; k < d; ++k) {
    const double2 *Mk = M + (size_t)(k - 1) * P * P;
    if (on) {
      double2 acc = make_double2(0.0, 0.0);
      for (int t = 0; t < P; ++t) acc = c_add(acc, c_mul(Mk[t * P + p], s_v[t]));
      s_n[p] = acc;
    }
    __syncthreads();
    if (on) {
      s_v[p] = s_n[p];
      if (k % C == 0) gck[(size_t)(k / C) * P + p] = s_n[p];
    }
    __syncthreads();
  }
  // Q = front * sum_t w[t] G_{d-1}[t]
  double2 front = make_double2(1.0, 0.0);
  if (FAM == MDI_FAM_OSC) {
    double sn, cs;
    sincos(kTwoPi * prm[d], &sn, &cs);
    front = make_double2(cs, sn);
  }
  if (threadIdx.x == 0) {
    double2 q = make_double2(0.0, 0.0);
    for (int t = 0; t < P; ++t) q = c_add(q, c_mul(w[t], s_v[t]));
    misc[0] = q;
    const double2 fq = c_mul(front, q);
    if (value) *value = fq.x;
    if (adjoint && FAM == MDI_FAM_OSC) {
      grad[d] = -kTwoPi * fq.y;  // dQ/du = Re(2 pi i front q)
      for (int j = d + 1; j < 2 * d; ++j) grad[j] = 0.0;
    }
  }
  if (!adjoint) return;
  __syncthreads();
  // lambda_{d-1} = front * w; lck[nck] holds it, lck[j] holds lambda_{jC}.
  const int nck = (d - 1) / C + 1;
  if (on) {
    s_v[p] = c_mul(front, w[p]);
    lck[(size_t)nck * P + p] = s_v[p];
    if ((d - 1) % C == 0) lck[(size_t)((d - 1) / C) * P + p] = s_v[p];
  }
  __syncthreads();
  for (int k = d - 1; k >= 1; --k) {  // lambda_{k-1} = lambda_k M_k
    const double2 *Mk = M + (size_t)(k - 1) * P * P;
    if (on) {
      double2 acc = make_double2(0.0, 0.0);
      for (int q = 0; q < P; ++q) acc = c_add(acc, c_mul(s_v[q], Mk[p * P + q]));
      s_n[p] = acc;
    }
    __syncthreads();
    if (on) {
      s_v[p] = s_n[p];
      if ((k - 1) % C == 0) lck[(size_t)((k - 1) / C) * P + p] = s_n[p];
    }
    __syncthreads();
  }
}

// K3: gradient of level k (block k-1, k = 1..d).
template <int FAM>
__global__ void __launch_bounds__(kLvThreads) levels_grad_kernel(int d, int a, int n_last, int P, int C,
                                                                 const double *__restrict__ prm,
                                                                 const double *__restrict__ L,
                                                                 const double2 *__restrict__ M,
                                                                 const double2 *__restrict__ gck,
                                                                 const double2 *__restrict__ lck,
                                                                 double *__restrict__ grad) {
  __shared__ double s_xi[kNodesPMax], s_bw[kNodesPMax];
  __shared__ double2 s_g[kNodesPMax], s_l[kNodesPMax], s_n[kNodesPMax];
  __shared__ double2 s_red[kLvThreads / kWarp];
  for (int t = threadIdx.x; t < P; t += blockDim.x) {
    s_xi[t] = cheb_node(t, P);
    s_bw[t] = cheb_weight(t, P);
  }
  const int nck = (d - 1) / C + 1;
  const int npts = a * P;
  const double inv_a = 1.0 / (double)a;
  double2 front = make_double2(1.0, 0.0);
  if (FAM == MDI_FAM_OSC) {
    double sn, cs;
    sincos(kTwoPi * prm[d], &sn, &cs);
    front = make_double2(cs, sn);
  }
  for (int k = blockIdx.x + 1; k <= d; k += gridDim.x) {
    // G_{k-1} from the checkpoint at or below it.
    const int j0 = (k - 1) / C;
    if (threadIdx.x < P) s_g[threadIdx.x] = gck[(size_t)j0 * P + threadIdx.x];
    __syncthreads();
    for (int m = j0 * C + 1; m <= k - 1; ++m) {
      const double2 *Mm = M + (size_t)(m - 1) * P * P;
      if (threadIdx.x < P) {
        double2 acc = make_double2(0.0, 0.0);
        for (int t = 0; t < P; ++t) acc = c_add(acc, c_mul(Mm[t * P + threadIdx.x], s_g[t]));
        s_n[threadIdx.x] = acc;
      }
      __syncthreads();
      if (threadIdx.x < P) s_g[threadIdx.x] = s_n[threadIdx.x];
      __syncthreads();
    }
    const int tid = threadIdx.x;
    double2 acc_c = make_double2(0.0, 0.0), acc_w = make_double2(0.0, 0.0);
    const AxisParams ap = load_axis(prm, d, k - 1);
    if (k < d) {
      // lambda_k from the checkpoint at or above it.
      int top = ((k + C - 1) / C) * C;
      const double2 *src;
      if (top > d - 1) {
        top = d - 1;
        src = lck + (size_t)nck * P;
      } else {
        src = lck + (size_t)(top / C) * P;
      }
      if (tid < P) s_l[tid] = src[tid];
      __syncthreads();
      for (int m = top; m >= k + 1; --m) {
        const double2 *Mm = M + (size_t)(m - 1) * P * P;
        if (tid < P) {
          double2 acc = make_double2(0.0, 0.0);
          for (int q = 0; q < P; ++q) acc = c_add(acc, c_mul(s_l[q], Mm[tid * P + q]));
          s_n[tid] = acc;
        }
        __syncthreads();
        if (tid < P) s_l[tid] = s_n[tid];
        __syncthreads();
      }
      for (int i = tid; i < npts; i += blockDim.x) {
        const int q = i / P, p = i % P;
        const double u = ((double)q + s_xi[p]) * inv_a;
        const PhiGrad<FAM> pg = phi_grad64<FAM>(u, ap);
        double2 g = make_double2(0.0, 0.0);
        if (k == 1) {
          g = make_double2(1.0, 0.0);
        } else {
          for (int t = 0; t < P; ++t) {
            const double l = L[(size_t)t * npts + i];
            g.x = fma(l, s_g[t].x, g.x);
            g.y = fma(l, s_g[t].y, g.y);
          }
        }
        const double2 lg = c_mul(s_l[p], g);
        acc_c = c_add(acc_c, c_mul(lg, as2(pg.dc)));
        acc_w = c_add(acc_w, c_mul(lg, as2(pg.dw)));
      }
    } else {
      // last level: dQ/dtheta_d = Re(front (1/n_last) sum_s dphi_d(s/n_last) G~_{d-1}(s/n_last))
      for (int s = tid; s < n_last; s += blockDim.x) {
        const double u = (double)s / (double)n_last;
        const PhiGrad<FAM> pg = phi_grad64<FAM>(u, ap);
        double2 g = make_double2(0.0, 0.0);
        if (d == 1) {
          g = make_double2(1.0, 0.0);
        } else {
          double den = 0.0;
          int hit = -1;
          for (int t = 0; t < P; ++t) {
            if (u == s_xi[t]) {
              hit = t;
              continue;
            }
            const double wt = s_bw[t] / (u - s_xi[t]);
            den += wt;
            g.x = fma(wt, s_g[t].x, g.x);
            g.y = fma(wt, s_g[t].y, g.y);
          }
          g = hit >= 0 ? s_g[hit] : c_scale(g, 1.0 / den);
        }
        const double2 fg = c_mul(front, g);
        acc_c = c_add(acc_c, c_mul(fg, as2(pg.dc)));
        acc_w = c_add(acc_w, c_mul(fg, as2(pg.dw)));
      }
    }
    const double2 tc = block_sum(acc_c, s_red);
    const double2 tw = block_sum(acc_w, s_red);
    if (tid == 0) {
      const double scale = (k < d) ? inv_a : 1.0 / (double)n_last;
      grad[k - 1] = tc.x * scale;
      if (FAM != MDI_FAM_OSC) grad[d + k - 1] = tw.x * scale;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
size_t levels_workspace_bytes(int d, int64_t a, const NodesConfig &cfg, int checkpoint) {
  const int C = checkpoint > 0 ? checkpoint : default_checkpoint(d);
  return levels_layout(d, a, cfg.P, C).total;
}

template <int FAM, bool F32>
static mdi_status run_levels(int d, int a, int n_last, const double *params, const NodesConfig &cfg, int C,
                             double *value, double *grad, void *ws, cudaStream_t stream) {
  const LevelsLayout Lo = levels_layout(d, a, cfg.P, C);
  char *base = (char *)ws;
  double *L = (double *)(base + Lo.table);
  double2 *M = (double2 *)(base + Lo.M), *w = (double2 *)(base + Lo.w);
  double2 *gck = (double2 *)(base + Lo.gck), *lck = (double2 *)(base + Lo.lck), *misc = (double2 *)(base + Lo.misc);
  const int P = cfg.P;
  levels_table_kernel<<<std::max(1, (a * P + 255) / 256), 256, 0, stream>>>(P, a, L);
  mdi_status st = check_launch();
  if (st != MDI_OK) return st;
  const int grid = std::min(d, sm_count() * 8);
  levels_build_kernel<FAM, F32><<<grid, kLvThreads, 0, stream>>>(d, a, n_last, P, params, L, M, w);
  if ((st = check_launch()) != MDI_OK) return st;
  levels_chain_kernel<FAM><<<1, 32, 0, stream>>>(d, P, C, params, M, w, gck, lck, misc, value, grad, grad ? 1 : 0);
  if ((st = check_launch()) != MDI_OK) return st;
  if (grad) {
    levels_grad_kernel<FAM><<<std::min(d, sm_count() * 8), kLvThreads, 0, stream>>>(d, a, n_last, P, C, params, L, M,
                                                                                    gck, lck, grad);
    st = check_launch();
  }
  return st;
}

mdi_status levels_launch(int family, int d, int64_t a, int64_t n_last, const double *params, const NodesConfig &cfg,
                         int checkpoint, double *value, double *grad, void *workspace, size_t ws_bytes,
                         cudaStream_t stream) {
  if (d < 1 || d > (1 << 16) || a < 1 || a > kNodesAMax || n_last < 1 || n_last > 4096) return MDI_EUNSUPPORTED;
  if (cfg.P < 2 || cfg.P > kNodesPMax || (cfg.P & 1)) return MDI_EINVAL;
  if (grad && cfg.precision != MDI_PREC_FP64) return MDI_EUNSUPPORTED;
  if (cfg.precision == MDI_PREC_FP32_EVAL_DF32 || cfg.precision == MDI_PREC_DF64) return MDI_EUNSUPPORTED;
  const int C = checkpoint > 0 ? checkpoint : default_checkpoint(d);
  if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < levels_layout(d, a, cfg.P, C).total)
    return MDI_EWORKSPACE;
  const bool f32 = cfg.precision == MDI_PREC_FP32_EVAL_FP64;
  const int ai = (int)a, nl = (int)n_last;
  switch (family) {
    case MDI_FAM_EXP:
      return f32 ? run_levels<MDI_FAM_EXP, true>(d, ai, nl, params, cfg, C, value, grad, workspace, stream)
                 : run_levels<MDI_FAM_EXP, false>(d, ai, nl, params, cfg, C, value, grad, workspace, stream);
    case MDI_FAM_OSC:
      return f32 ? run_levels<MDI_FAM_OSC, true>(d, ai, nl, params, cfg, C, value, grad, workspace, stream)
                 : run_levels<MDI_FAM_OSC, false>(d, ai, nl, params, cfg, C, value, grad, workspace, stream);
    case MDI_FAM_GAUSS:
      return f32 ? run_levels<MDI_FAM_GAUSS, true>(d, ai, nl, params, cfg, C, value, grad, workspace, stream)
                 : run_levels<MDI_FAM_GAUSS, false>(d, ai, nl, params, cfg, C, value, grad, workspace, stream);
    default:
      return f32 ? run_levels<MDI_FAM_PEAK, true>(d, ai, nl, params, cfg, C, value, grad, workspace, stream)
                 : run_levels<MDI_FAM_PEAK, false>(d, ai, nl, params, cfg, C, value, grad, workspace, stream);
  }
}

}  // namespace mdi
