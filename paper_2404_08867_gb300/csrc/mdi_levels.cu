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
// One CTA: P threads do the P x P products while all threads stage the operators
// of the next kChainLevels levels into shared memory with cp.async (hardware
// wait_group, double-buffered), so no level waits on an L2 round trip.  Real
// families use real arithmetic on the real parts.  misc[0] = Q before the front
// factor.
constexpr int kChainMaxThreads = 1024;  // P x G thread grid, G = the power of two >= P
constexpr int kChainSmem = 64 * 1024;  // two buffers of operators

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Operators M_first .. M_first+cnt-1 (1-based levels) -> dst, one 16-byte copy each.
// M is stored [t][p]; `transpose` stages each operator as [p][t].
__device__ __forceinline__ void stage_ops(double2 *dst, const double2 *M, int first, int cnt, int P, bool transpose) {
  const int n = cnt * P * P, pp = P * P;
  const double2 *src = M + (size_t)(first - 1) * pp;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int j = i;
    if (transpose) {
      const int lev = i / pp, e = i % pp;  // e = t*P + p
      j = lev * pp + (e % P) * P + e / P;
    }
    cp_async16(dst + j, src + i);
  }
  cp_async_commit();
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

// Lanes per row of the chain's thread grid: the power of two >= P.
__host__ __device__ __forceinline__ int chain_group(int P) {
  int g = 1;
  while (g < P) g <<= 1;
  return g;
}

static int chain_levels_per_chunk(int P) {
  return std::max(1, std::min(8, kChainSmem / 2 / (P * P * (int)sizeof(double2))));
}

template <int FAM>
__global__ void __launch_bounds__(kChainMaxThreads) levels_chain_kernel(int d, int P, int C, int LC,
                                                                     const double *__restrict__ prm,
                                                                     const double2 *__restrict__ M,
                                                                     const double2 *__restrict__ w,
                                                                     double2 *__restrict__ gck,
                                                                     double2 *__restrict__ lck,
                                                                     double2 *__restrict__ misc,
                                                                     double *__restrict__ value,
                                                                     double *__restrict__ grad, int adjoint) {
  using V = typename FamTraits<FAM>::V;
  extern __shared__ __align__(16) unsigned char chain_smem[];
  double2 *buf[2] = {(double2 *)chain_smem, (double2 *)chain_smem + (size_t)LC * P * P};
  __shared__ V s_v[kNodesPMax], s_n[kNodesPMax];
  // Thread grid: row = threadIdx.x / G, col = threadIdx.x % G; one product per thread,
  // summed over the G lanes of a row.
  const int G = chain_group(P);
  const int row = threadIdx.x / G, col = threadIdx.x % G;
  const bool cell = row < P && col < P;
  const int p = threadIdx.x;
  const bool on = p < P;
  auto mul = [](double2 m, V v) -> V {
    if constexpr (FAM == MDI_FAM_OSC) return c_mul(m, v);
    else return m.x * v;
  };
  if (on) s_v[p] = VOps<V>::one();
  __syncthreads();
  if (on) gck[p] = as2(s_v[p]);
  const int nlev = d - 1;
  const int nchunks = (nlev + LC - 1) / LC;
  // Forward: chunk c holds levels 1 + c*LC .. min(d-1, (c+1)*LC), staged as [p][t].
  // G_k[p] = sum_t M_k[p][t] G_{k-1}[t]: row = p, col = t.
  if (nchunks > 0) stage_ops(buf[0], M, 1, std::min(LC, nlev), P, true);
  for (int c = 0; c < nchunks; ++c) {
    const int k0 = 1 + c * LC, k1 = std::min(nlev, (c + 1) * LC);
    if (c + 1 < nchunks) {
      const int n0 = k1 + 1;
      stage_ops(buf[(c + 1) & 1], M, n0, std::min(LC, nlev - n0 + 1), P, true);
      cp_async_wait_prev();
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
    const double2 *B = buf[c & 1];
    for (int k = k0; k <= k1; ++k) {
      const double2 *Mk = B + (size_t)(k - k0) * P * P;
      V prod = cell ? mul(Mk[row * P + col], s_v[col]) : VOps<V>::zero();
      prod = group_sum(prod, G);
      if (cell && col == 0) {
        s_n[row] = prod;
        if (k % C == 0) gck[(size_t)(k / C) * P + row] = as2(prod);
      }
      __syncthreads();
      if (on) s_v[p] = s_n[p];
      __syncthreads();
    }
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
    for (int t = 0; t < P; ++t) q = c_add(q, c_mul(w[t], as2(s_v[t])));
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
  // lambda_{d-1} = front * w; lck[nck] holds it, lck[j] holds lambda_{jC}.  The
  // adjoint of a real family is real (front = 1, w real).
  const int nck = (d - 1) / C + 1;
  if (on) {
    const double2 l = c_mul(front, w[p]);
    s_v[p] = from2<V>(l);
    lck[(size_t)nck * P + p] = l;
    if ((d - 1) % C == 0) lck[(size_t)((d - 1) / C) * P + p] = l;
  }
  __syncthreads();
  // Backward: chunk c holds levels max(1, top - LC + 1) .. top, top = d-1 - c*LC,
  // staged as stored ([t][p]).  lambda_{k-1}[t] = sum_p lambda_k[p] M_k[p][t]:
  // row = t, col = p.
  if (nchunks > 0) {
    const int top = nlev, bot = std::max(1, top - LC + 1);
    stage_ops(buf[0], M, bot, top - bot + 1, P, false);
  }
  for (int c = 0; c < nchunks; ++c) {
    const int top = nlev - c * LC, bot = std::max(1, top - LC + 1);
    if (c + 1 < nchunks) {
      const int ntop = bot - 1, nbot = std::max(1, ntop - LC + 1);
      stage_ops(buf[(c + 1) & 1], M, nbot, ntop - nbot + 1, P, false);
      cp_async_wait_prev();
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
    const double2 *B = buf[c & 1];
    for (int k = top; k >= bot; --k) {
      const double2 *Mk = B + (size_t)(k - bot) * P * P;
      V prod = cell ? mul(Mk[row * P + col], s_v[col]) : VOps<V>::zero();
      prod = group_sum(prod, G);
      if (cell && col == 0) {
        s_n[row] = prod;
        if ((k - 1) % C == 0) lck[(size_t)((k - 1) / C) * P + row] = as2(prod);
      }
      __syncthreads();
      if (on) s_v[p] = s_n[p];
      __syncthreads();
    }
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
  static bool chain_attr = false;
  if (!chain_attr) {
    cudaError_t e = cudaFuncSetAttribute(levels_chain_kernel<FAM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kChainSmem);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return MDI_ECUDA;
    }
    chain_attr = true;
  }
  const int LC = chain_levels_per_chunk(P);
  const size_t chain_smem = 2 * (size_t)LC * P * P * sizeof(double2);
  const int chain_threads = std::max(32, (P * chain_group(P) + 31) / 32 * 32);
  levels_chain_kernel<FAM><<<1, chain_threads, chain_smem, stream>>>(d, P, C, LC, params, M, w, gck, lck, misc, value,
                                                                     grad, grad ? 1 : 0);
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
