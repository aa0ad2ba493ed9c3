// mdi_nodes.cu -- MDI-LR with the node level state (MDI_STATE_NODES), batched.
//
// The paper keeps each "symbolic function" g_{k-m} of eq. (4.4) symbolically; this
// library keeps the level state G_k(x) (x = the next original coordinate) at P
// Chebyshev points of the first kind on [0,1],
//     xi_p = (1 + cos(pi (2p+1) / (2P))) / 2,
// and reads it between them with the barycentric formula of the second kind
// (weights (-1)^p sin(pi (2p+1)/(2P)); Berrut & Trefethen, SIAM Review 46, 2004).
// Level k < d evaluates the cluster of the sweep,
//     G_k(xi_p) = (1/a) sum_{q<a} phi_k(u_qp) G_{k-1}(u_qp),  u_qp = (q + xi_p)/a,
// and the last level sums over the n_last points s/n_last of the last axis.
//
// GB300 mapping.  Integrals are independent, so a persistent grid of CTAs pulls
// them from an atomic counter (no waiting: a CTA that finds the queue empty
// exits).  A CTA sweeps its integral's d levels with the state in shared memory.
// Lanes are node-major: Q consecutive lanes serve node p and take the cluster
// points q = qs, qs + Q, ...; each point interpolates G_{k-1} (P multiply-adds
// against the basis table L_a[t][p*a + q] = l_t(u_qp), contiguous in q), multiplies
// by phi_k and accumulates; the Q lanes add their sums with shuffles and one lane
// writes G_k[p] into the other half of a double-buffered state, so a level costs
// one barrier.  The constants of 32 levels at a time are prepared by all threads
// together.  The basis tables depend only on (a, P) and are built once per workspace
// (mdi_lr_batched_prepare) for a = 1..64, together with the basis at the last
// axis' points s/a (used when n_last = a).  A CTA may stage its table in shared
// memory (fewer resident CTAs) or read it through L1 (more resident CTAs to hide
// the level barriers); the autotuner picks.
//
// Precision modes (mdi_precision):
//   FP64             everything in double;
//   FP32_EVAL_FP64   phi in float, interpolation and sums in double;
//   FP32_EVAL_DF32   phi in float, interpolation and the cluster sum in
//                    double-float (the state in double between levels for OSC,
//                    as float pairs for the real families);
//   DF64             coordinates, phi, interpolation, sums and the state in
//                    double-float (no FP64 instruction per cluster point or per
//                    level); OSC keeps phi in double.
// In every mode the real families use paired cluster points (sweep_paired,
// sweep_paired_fp64): by the symmetry of the nodes, one pass over a table of sums
// and differences of basis values interpolates the point u of node p and the
// point 1 - u of node P-1-p, lanes are pair-major, and the state is kept as sums
// and differences of mirrored nodes.  The single-precision-evaluation modes take
// phi at the float coordinate (q + xi_p)/a there, so both give phi the same floats.
#include <algorithm>
#include <atomic>

#include "mdi_common.cuh"
#include "mdi_fp64.cuh"
#include "mdi_internal.h"
#include "mdi_nodes.cuh"

namespace mdi {

constexpr int kNodesMaxBlock = 512;
constexpr int kNodesSmemTable = 64 * 1024;  // table bytes staged in shared memory

constexpr int kLvChunk = 32;  // levels whose constants are held in shared memory at once

// The threads sweeping one integral: the whole CTA, or one warp of it (the second
// phase of the hybrid schedule, where each warp of a two-warp CTA takes integrals
// of its own).  tid and size stand for threadIdx.x and blockDim.x inside a sweep;
// sync() is the team's barrier.
struct Team {
  int tid, size;
  __device__ __forceinline__ void sync() const {
    if (size == kWarp) __syncwarp();
    else __syncthreads();
  }
  static __device__ __forceinline__ Team block() { return Team{(int)threadIdx.x, (int)blockDim.x}; }
};

// Sum over the team, valid in its thread 0.
template <typename V> __device__ __forceinline__ V team_sum(V v, V *scratch, const Team &tm) {
  v = warp_sum(v);
  if (tm.size <= kWarp) return v;
  const int lane = tm.tid & (kWarp - 1), warp = tm.tid / kWarp, nwarps = (tm.size + kWarp - 1) / kWarp;
  if (lane == 0) scratch[warp] = v;
  tm.sync();
  V r = VOps<V>::zero();
  if (warp == 0) r = warp_sum(lane < nwarps ? scratch[lane] : VOps<V>::zero());
  tm.sync();
  return r;
}

// Per-axis constants of a level: c, w, 1/c^2 in double and as float pairs; c w and
// c (1 - w) for the FP64 sweep's affine arguments.
struct LevelConst {
  float4 cwf;  // (c.hi, c.lo, w.hi, w.lo)
  float2 ic;   // 1/c^2 as a float pair
  double c, w, ic2, cw, c1w;
  // FP64 Gaussian sweep, for lanes that step their points by Q (dq = (c/a) Q):
  double kap;  // exp(-2 dq^2), the recurrence's second ratio
  double eb;   // exp(2 (t_a - t_b) dq): the mirrored point's first ratio is rho_a eb
  int rec_ok;  // the arguments stay moderate on this level (the recurrence may run)
};

// Fixed part of the dynamic shared memory; the staged table (if any) follows it.
struct NodesShared {
  double xi[kNodesPMax], bw[kNodesPMax];
  double2 G[2][kNodesPMax];   // state at the nodes in double, double-buffered by level
  float4 Gdf[2][kNodesPMax];  // the state as float pairs (re.hi, re.lo, im.hi, im.lo)
  float2 xadf[kNodesPMax];    // xi_p / a as float pairs (DF64), per integral
  double2 red[kNodesMaxBlock / kWarp];
  float4 redf[kNodesMaxBlock / kWarp];
  union {
    float2 exp2tab[kExpTable];  // 2^(j/256) as float pairs (double-float exp, DF64)
    double exp2d[kExpTable];    // 2^(j/256) as doubles (FP64 exp)
  };
  double qd[kNodesAMax];      // q as a double, q < 64 (FP64)
  LevelConst lc[kLvChunk];    // constants of axes base .. base+kLvChunk-1
  float2 iadf;                // 1/a as a float pair (DF64)
  int inst;
  int pad;
};

// Constants common to every integral for P nodes, built once by the preparation
// and copied by each CTA (FP64 evaluation of them per CTA would queue on the
// FP64 pipe at every launch): the 2^(j/256) table of the double-float exp, the
// Chebyshev nodes and barycentric weights, and for every a the float pairs of 1/a
// and xi_p/a.
struct NodesConsts {
  float2 exp2tab[kExpTable];
  double exp2d[kExpTable];
  double xi[kNodesPMax], bw[kNodesPMax];
  float2 ia[kNodesAMax + 1];
  float2 xa[kNodesAMax + 1][kNodesPMax];
};

__global__ void nodes_consts_kernel(int P, NodesConsts *__restrict__ kc) {
  for (int j = threadIdx.x; j < kExpTable; j += blockDim.x) {
    kc->exp2tab[j] = exp2_table_entry(j);
    kc->exp2d[j] = kExp2TableD[j];
  }
  for (int t = threadIdx.x; t < P; t += blockDim.x) {
    kc->xi[t] = cheb_node(t, P);
    kc->bw[t] = cheb_weight(t, P);
  }
  for (int i = threadIdx.x; i <= kNodesAMax; i += blockDim.x) {
    const double v = i ? 1.0 / (double)i : 0.0;
    const float h = (float)v;
    kc->ia[i] = make_float2(h, (float)(v - (double)h));
  }
  for (int i = threadIdx.x; i < (kNodesAMax + 1) * P; i += blockDim.x) {
    const int a = i / P, t = i % P;
    const double v = a ? cheb_node(t, P) / (double)a : 0.0;
    const float h = (float)v;
    kc->xa[a][t] = make_float2(h, (float)(v - (double)h));
  }
}

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) / 16 * 16; }
static size_t nodes_smem_bytes(int block, int P, bool stage) {
  (void)block;
  (void)P;
  return align16(sizeof(NodesShared)) + (stage ? kNodesSmemTable : 0);
}

// Lanes per node: the largest power of two Q <= 32 with P*Q <= blockDim.
__device__ __forceinline__ int node_lanes(int B, int P) {
  int Q = 1;
  while (Q < kWarp && P * 2 * Q <= B) Q <<= 1;
  return Q;
}

// Table of parameter a (1-based) for P nodes, in 8-byte entries: the cluster basis
// L_a[t][p*a + q] = l_t((q + xi_p)/a) (a*P*P entries) followed by the last-axis
// basis F_a[t][s] = l_t(s/a) (a*P entries).  Even P keeps every block 16-byte
// aligned.
__host__ __device__ __forceinline__ size_t table_offset(int a, int P) {
  return (size_t)P * (P + 1) * (size_t)a * (size_t)(a - 1) / 2;
}
static size_t table_bytes(int P) { return 8 * table_offset(kNodesAMax + 1, P); }

template <bool DF>
__global__ void nodes_table_kernel(int P, void *__restrict__ table) {
  __shared__ double s_xi[kNodesPMax], s_bw[kNodesPMax];
  for (int t = threadIdx.x; t < P; t += blockDim.x) {
    s_xi[t] = cheb_node(t, P);
    s_bw[t] = cheb_weight(t, P);
  }
  __syncthreads();
  const size_t total_rows = (size_t)(P + 1) * kNodesAMax * (kNodesAMax + 1) / 2;  // sum_a a*(P+1)
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total_rows;
       g += (size_t)gridDim.x * blockDim.x) {
    int a = 1;
    size_t base = 0;
    while (base + (size_t)a * (P + 1) <= g) {
      base += (size_t)a * (P + 1);
      ++a;
    }
    const int i = (int)(g - base);  // i = p*a + q on the cluster part
    const bool last_axis = i >= a * P;
    double u;
    if (last_axis) u = (double)(i - a * P) / (double)a;                 // s / a
    else u = ((double)(i % a) + s_xi[i / a]) / (double)a;              // (q + xi_p) / a
    double den = 0.0;
    int hit = -1;
    for (int t = 0; t < P; ++t) {
      if (u == s_xi[t]) hit = t;
      else den += s_bw[t] / (u - s_xi[t]);
    }
    const size_t off = table_offset(a, P);
    for (int t = 0; t < P; ++t) {
      const double l = hit >= 0 ? (t == hit ? 1.0 : 0.0) : (s_bw[t] / (u - s_xi[t])) / den;
      const size_t idx = last_axis ? off + (size_t)a * P * P + (size_t)t * a + (i - a * P)
                                   : off + (size_t)t * a * P + i;
      if constexpr (DF) {
        const float h = (float)l;
        ((float2 *)table)[idx] = make_float2(h, (float)(l - (double)h));
      } else {
        ((double *)table)[idx] = l;
      }
    }
  }
}

// Paired cluster basis (DF64, real families).  The nodes are symmetric,
// xi_{P-1-p} = 1 - xi_p, and the barycentric weights are too up to one common sign,
// so l_t(1 - u) = l_{P-1-t}(u): the cluster point u = (q + xi_p)/a of node p and the
// point 1 - u = (a-1-q + xi_{P-1-p})/a of node P-1-p interpolate with the same basis
// values in reverse order.  For p < h = P/2 the table holds
//     Lpm[t][p*a + q] = (l_t(u) + l_{P-1-t}(u), l_t(u) - l_{P-1-t}(u)),  t < h,
// as two float pairs (DF64) or two doubles (FP64), one 16-byte entry; h*a*h
// entries per a, a = 1..64.
__host__ __device__ __forceinline__ size_t paired_offset(int a, int P) {
  const size_t h = (size_t)P / 2;
  return h * h * (size_t)a * (size_t)(a - 1) / 2;  // in 16-byte entries
}
static size_t paired_bytes(int P) { return 16 * paired_offset(kNodesAMax + 1, P); }

template <bool DF>
__global__ void nodes_paired_table_kernel(int P, float4 *__restrict__ table) {
  __shared__ double s_xi[kNodesPMax], s_bw[kNodesPMax];
  for (int t = threadIdx.x; t < P; t += blockDim.x) {
    s_xi[t] = cheb_node(t, P);
    s_bw[t] = cheb_weight(t, P);
  }
  __syncthreads();
  const int h = P / 2;
  const size_t total_rows = (size_t)h * kNodesAMax * (kNodesAMax + 1) / 2;  // sum_a a*h
  for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total_rows;
       g += (size_t)gridDim.x * blockDim.x) {
    int a = 1;
    size_t base = 0;
    while (base + (size_t)a * h <= g) {
      base += (size_t)a * h;
      ++a;
    }
    const int i = (int)(g - base);  // i = p*a + q, p < h
    const double u = ((double)(i % a) + s_xi[i / a]) / (double)a;
    double den = 0.0;
    int hit = -1;
    for (int t = 0; t < P; ++t) {
      if (u == s_xi[t]) hit = t;
      else den += s_bw[t] / (u - s_xi[t]);
    }
    auto basis = [&](int t) {
      return hit >= 0 ? (t == hit ? 1.0 : 0.0) : (s_bw[t] / (u - s_xi[t])) / den;
    };
    float4 *row = table + paired_offset(a, P);
    for (int t = 0; t < h; ++t) {
      const double lt = basis(t), lr = basis(P - 1 - t);
      const double vp = lt + lr, vm = lt - lr;
      if constexpr (DF) {
        const float ph = (float)vp, mh = (float)vm;
        row[(size_t)t * a * h + i] = make_float4(ph, (float)(vp - (double)ph), mh, (float)(vm - (double)mh));
      } else {
        reinterpret_cast<double2 *>(row)[(size_t)t * a * h + i] = make_double2(vp, vm);
      }
    }
  }
}

// Constants of axis j (0-based) for the level loop.  With DF, 1/c^2 is formed in
// double-float arithmetic (relative error about 2^-46) and its double copy is the
// sum of that pair: no FP64 division per level.
template <bool DF>
__device__ __forceinline__ void make_level_const(const double *__restrict__ prm, int d, int j, LevelConst &L) {
  const double c = prm[j], w = prm[d + j];
  const df32 cd = df_from_double(c), wd = df_from_double(w);
  df32 id;
  if constexpr (DF) {
    id = df_rcp(df_sqr(cd));
    L.ic2 = df_to_double(id);
  } else {
    L.ic2 = 1.0 / (c * c);
    id = df_from_double(L.ic2);
  }
  L.c = c;
  L.w = w;
  L.cw = c * w;
  L.c1w = c * (1.0 - w);
  L.cwf = make_float4(cd.hi, cd.lo, wd.hi, wd.lo);
  L.ic = make_float2(id.hi, id.lo);
}

// Fills sh.lc with the constants of axes base .. base+kLvChunk-1 (all threads).
// With a table T (the FP64 Gaussian sweep), also each level's kap for lanes that
// step their points by Q: dq = (c/a) Q, one exp per level and chunk rather than
// per level and lane.
template <bool DF = false>
__device__ __forceinline__ void load_level_chunk(LevelConst *lc, const double *__restrict__ prm, int d, int base,
                                                 const Team &tm = Team::block(), const double *T = nullptr,
                                                 double inv_a = 0.0, double Qd = 0.0) {
  const int n = min(kLvChunk, d - base);
  for (int j = tm.tid; j < n; j += tm.size) {
    LevelConst &L = lc[j];
    make_level_const<DF>(prm, d, base + j, L);
    if (T) {
      const double dq = (L.c * inv_a) * Qd;
      // |t| <= B at every cluster point of the level (t = c (u - w) and
      // c (u - 1 + w), u in [0, 1)); with |dq| (2B + |dq|) < 350 every factor, both
      // first ratios and eb stay in the normal range.
      const double B = fabs(L.c) * (fmax(fabs(L.w), fabs(1.0 - L.w)) + inv_a + 1.0);
      L.rec_ok = B < 20.0 && fabs(dq) * (2.0 * B + fabs(dq)) < 350.0;
      L.kap = exp_tang64(-2.0 * dq * dq, T);
      L.eb = exp_tang64(2.0 * (L.c1w - L.cw) * dq, T);  // t_a - t_b = c (1 - w) - c w
    }
  }
}

// The argument of phi at the cluster points u = q/a + x0 of one node is affine in
// q: t = s1 q + s0.  Per level and node:
//   GAUSS  t = c (u - w)  ->  s1 = c/a, s0 = c (x0 - w);   phi = exp(-t^2)
//   PEAK   t = u - w      ->  s1 = 1/a, s0 = x0 - w;       phi = 1 / (t^2 + 1/c^2)
//   EXP    t = c u        ->  s1 = c/a, s0 = c x0;         phi = exp(t)
template <int FAM>
__device__ __forceinline__ void phi_affine_coeffs(float4 cw, df32 ia, df32 x0, df32 &s1, df32 &s0) {
  const df32 c{cw.x, cw.y}, w{cw.z, cw.w};
  if constexpr (FAM == MDI_FAM_GAUSS) {
    s1 = df_mul(c, ia);
    s0 = df_mul(c, df_add(x0, df_neg(w)));
  } else if constexpr (FAM == MDI_FAM_PEAK) {
    s1 = ia;
    s0 = df_add(x0, df_neg(w));
  } else {
    s1 = df_mul(c, ia);
    s0 = df_mul(c, x0);
  }
}
// phi at the point q: one double-float multiply-add forms the argument.  The
// sloppy add suffices: phi depends on t through t^2 or exp(t), so only the
// absolute error of t (about 2^-48 |t| terms) matters.
template <int FAM>
__device__ __forceinline__ df32 phi_df_affine(df32 s1, df32 s0, float q, float2 ic, const float2 *tab) {
  const df32 t = df_add_sloppy(df_mul_f(s1, q), s0);
  if constexpr (FAM == MDI_FAM_GAUSS) return df_exp(df_neg(df_sqr(t)), tab);
  else if constexpr (FAM == MDI_FAM_PEAK) return df_rcp(df_add_sloppy(df_sqr(t), df32{ic.x, ic.y}));
  else return df_exp(t, tab);
}

__device__ __forceinline__ float4 split2(double2 g) {
  const float rh = (float)g.x, ih = (float)g.y;
  return make_float4(rh, (float)(g.x - (double)rh), ih, (float)(g.y - (double)ih));
}
__device__ __forceinline__ double2 join2(float4 v) {
  return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

// Block sum of double-float pairs (re, im); result valid in thread 0.
__device__ __forceinline__ float4 block_sum_df(df32 re, df32 im, float4 *scratch) {
  const int lane = threadIdx.x & (kWarp - 1), warp = threadIdx.x / kWarp;
  const int nwarps = (blockDim.x + kWarp - 1) / kWarp;
#pragma unroll
  for (int off = kWarp / 2; off > 0; off >>= 1) {
    re = df_add(re, df_shfl_down(re, off));
    im = df_add(im, df_shfl_down(im, off));
  }
  if (lane == 0) scratch[warp] = make_float4(re.hi, re.lo, im.hi, im.lo);
  __syncthreads();
  float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
  if (threadIdx.x == 0) {
    df32 sr{0.f, 0.f}, si{0.f, 0.f};
    for (int w = 0; w < nwarps; ++w) {
      sr = df_add(sr, df32{scratch[w].x, scratch[w].y});
      si = df_add(si, df32{scratch[w].z, scratch[w].w});
    }
    r = make_float4(sr.hi, sr.lo, si.hi, si.lo);
  }
  __syncthreads();
  return r;
}

// Sum of double-float pairs (re, im) over a team; result valid in its thread 0.
__device__ __forceinline__ float4 team_sum_df(df32 re, df32 im, float4 *scratch, const Team &tm) {
  if (tm.size > kWarp) return block_sum_df(re, im, scratch);
#pragma unroll
  for (int off = kWarp / 2; off > 0; off >>= 1) {
    re = df_add(re, df_shfl_down(re, off));
    im = df_add(im, df_shfl_down(im, off));
  }
  return make_float4(re.hi, re.lo, im.hi, im.lo);
}

// Sums over aligned groups of Q lanes (Q a power of two <= 32), valid in every lane.
__device__ __forceinline__ double2 lanes_sum(double2 v, int Q) {
  for (int off = 1; off < Q; off <<= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, off, Q);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, off, Q);
  }
  return v;
}
__device__ __forceinline__ df32 lanes_sum_df(df32 v, int Q) {
  for (int off = 1; off < Q; off <<= 1)
    v = df_add(v, df32{__shfl_xor_sync(0xffffffffu, v.hi, off, Q), __shfl_xor_sync(0xffffffffu, v.lo, off, Q)});
  return v;
}
// The same over Dot2 accumulators left unnormalised: the high parts are added
// with TwoSum, the low parts and the TwoSum errors with plain adds.
__device__ __forceinline__ DfAcc lanes_sum_acc(DfAcc v, int Q) {
  for (int off = 1; off < Q; off <<= 1) {
    const float os = __shfl_xor_sync(0xffffffffu, v.s, off, Q), oc = __shfl_xor_sync(0xffffffffu, v.c, off, Q);
    const df32 t = two_sum(v.s, os);
    v.s = t.hi;
    v.c = __fadd_rn(__fadd_rn(v.c, oc), t.lo);
  }
  return v;
}
// x + sg * y (sg = +1 or -1) of two Dot2 accumulators as a normalised double-float:
// the error is bounded relative to |x| + |y| (as a sloppy double-word add).
__device__ __forceinline__ df32 pair_combine(const DfAcc &x, const DfAcc &y, float sg) {
  const df32 t = two_sum(x.s, sg * y.s);
  return fast_two_sum(t.hi, __fadd_rn(__fmaf_rn(sg, y.c, x.c), t.lo));
}

// The last level of one integral, Q = (1/n_last) sum_s phi_d(s/n_last) G_{d-1}(s/n_last),
// with G_{d-1} in state buffer sb (sh.Gdf as float pairs in DF64, sh.G otherwise)
// and the level constants of the chunk holding axis d-2 in sh.lc.
template <int FAM, int PREC>
__device__ void last_level(NodesShared &sh, const void *__restrict__ Ftab, int P, int d, int a, int n_last,
                           const double *__restrict__ prm, double *__restrict__ out_slot, int sb,
                           const Team &tm = Team::block()) {
  using V = typename FamTraits<FAM>::V;
  constexpr bool F32 = (PREC == MDI_PREC_FP32_EVAL_FP64 || PREC == MDI_PREC_FP32_EVAL_DF32);
  constexpr bool DF = (PREC == MDI_PREC_FP32_EVAL_DF32 || PREC == MDI_PREC_DF64);
  constexpr bool CPLX = (FAM == MDI_FAM_OSC);
  constexpr bool DF64 = (PREC == MDI_PREC_DF64) && !CPLX;
  constexpr bool DFSTATE = (PREC == MDI_PREC_DF64);
  const int tid = tm.tid, B = tm.size;
  if (d > 1 && (d - 1) % kLvChunk == 0) {
    load_level_chunk<DFSTATE>(sh.lc, prm, d, d - 1, tm);
    tm.sync();
  }
  const LevelConst &LL = sh.lc[(d - 1) % kLvChunk];
  const bool tabulated = (n_last == a) && d > 1;
  if constexpr (DF64) {
    if (tabulated) {
      const df32 ia{sh.iadf.x, sh.iadf.y};
      df32 s1, s0;  // the last axis' points are s/a: no node offset
      phi_affine_coeffs<FAM>(LL.cwf, ia, df32{0.f, 0.f}, s1, s0);
      DfAcc acc;
      for (int s = tid; s < n_last; s += B) {
        const float2 *F = (const float2 *)Ftab + s;
        DfAcc ag;
#pragma unroll 4
        for (int t = 0; t < P; ++t) {
          const float2 l = F[(size_t)t * a];
          const float4 gt = sh.Gdf[sb][t];
          dacc_prod(ag, df32{l.x, l.y}, df32{gt.x, gt.y});
        }
        dacc_prod(acc, phi_df_affine<FAM>(s1, s0, (float)s, LL.ic, sh.exp2tab), dacc_value(ag));
      }
      const float4 tot = team_sum_df(dacc_value(acc), df32{0.f, 0.f}, sh.redf, tm);
      if (tid == 0) *out_slot = ((double)tot.x + (double)tot.y) / (double)n_last;
      tm.sync();
      return;
    }
  }
  if constexpr (DFSTATE) {  // double view of the state for the general last level
    if (tid < P) sh.G[sb][tid] = join2(sh.Gdf[sb][tid]);
    tm.sync();
  }
  const AxisParams ap{LL.c, LL.w, LL.ic2};
  const double inv_n = 1.0 / (double)n_last;
  V acc = VOps<V>::zero();
  for (int s = tid; s < n_last; s += B) {
    const double u = (double)s * inv_n;
    V g;
    if (d == 1) {
      g = VOps<V>::one();
    } else if (tabulated) {
      g = VOps<V>::zero();
      if constexpr (DF) {
        const float2 *F = (const float2 *)Ftab + s;
        for (int t = 0; t < P; ++t) {
          const float2 l = F[(size_t)t * a];
          g = VOps<V>::fma_s((double)l.x + (double)l.y, from2<V>(sh.G[sb][t]), g);
        }
      } else {
        const double *F = (const double *)Ftab + s;
        for (int t = 0; t < P; ++t) g = VOps<V>::fma_s(F[(size_t)t * a], from2<V>(sh.G[sb][t]), g);
      }
    } else {
      double den = 0.0;
      double2 num = make_double2(0.0, 0.0);
      int hit = -1;
      for (int t = 0; t < P; ++t) {
        if (u == sh.xi[t]) {
          hit = t;
          continue;
        }
        const double wt = sh.bw[t] / (u - sh.xi[t]);
        den += wt;
        num = make_double2(fma(wt, sh.G[sb][t].x, num.x), fma(wt, sh.G[sb][t].y, num.y));
      }
      g = hit >= 0 ? from2<V>(sh.G[sb][hit]) : from2<V>(c_scale(num, 1.0 / den));
    }
    acc = VOps<V>::add(acc, VOps<V>::mul(phi<FAM, F32 && !DFSTATE>(u, ap), g));
  }
  const V tot = team_sum(acc, (V *)sh.red, tm);
  if (tid == 0) {
    if constexpr (CPLX) {
      double sn, cs;
      sincos(kTwoPi * prm[d], &sn, &cs);
      *out_slot = (cs * tot.x - sn * tot.y) * inv_n;
    } else {
      *out_slot = tot * inv_n;
    }
  }
  tm.sync();
}


// ---------------------------------------------------------------------------
// One integral, swept by one CTA.  Ltab: the cluster basis of this a (shared or
// global memory); Ftab: the last-axis basis (global).
//
// Lanes are node-major: the Q = node_lanes(B, P) consecutive lanes of node p take
// the cluster points q = qs, qs + Q, ... and add their sums with shuffles, so a
// level ends with one barrier; the state is double-buffered by level parity.
// ---------------------------------------------------------------------------
// v 2^S for the power-of-two state scales, by adding S to the exponent field (exact;
// integer operations only -- the FP64 pipe is the scarce one); a result that
// would leave the normal range, and zero, subnormal or non-finite v, go through
// ldexp.
__device__ __forceinline__ double scale_pow2(double v, int S) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF), ne = e + S;
  if (e == 0 || e == 0x7FF || ne <= 0 || ne >= 0x7FF) return ldexp(v, S);
  return __longlong_as_double((b & ~(0x7FFll << 52)) | ((long long)ne << 52));
}
// Unbiased exponent of a normal, finite double (0 otherwise), from its bits.
__device__ __forceinline__ int exponent_of(double v) {
  const int e = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
  return (e == 0 || e == 0x7FF) ? 0 : e - 1023;
}

template <int FAM, int PREC>
__device__ void sweep_one(NodesShared &sh, const NodesConsts *__restrict__ kc, const void *__restrict__ Ltab,
                          const void *__restrict__ Ftab, int P, int d, int a, int n_last,
                          const double *__restrict__ prm, double *__restrict__ out_slot) {
  using V = typename FamTraits<FAM>::V;
  constexpr bool F32 = (PREC == MDI_PREC_FP32_EVAL_FP64 || PREC == MDI_PREC_FP32_EVAL_DF32);
  constexpr bool DF = (PREC == MDI_PREC_FP32_EVAL_DF32 || PREC == MDI_PREC_DF64);
  constexpr bool CPLX = (FAM == MDI_FAM_OSC);
  constexpr bool DF64 = (PREC == MDI_PREC_DF64) && !CPLX;  // OSC keeps phi in FP64 in this mode
  constexpr bool DFSTATE = (PREC == MDI_PREC_DF64);        // state kept as float pairs only
  const int tid = threadIdx.x, B = blockDim.x;
  const int Q = node_lanes(B, P);
  const int p = min(tid / Q, P - 1), qs = tid % Q;
  const bool act = tid < P * Q;
  const bool warp_act = (tid & ~(kWarp - 1)) < P * Q;  // this warp holds active lanes
  const int npts = a * P;

  if (tid < P) {
    sh.Gdf[0][tid] = make_float4(1.f, 0.f, 0.f, 0.f);
    sh.G[0][tid] = make_double2(1.0, 0.0);
    if (DFSTATE) sh.xadf[tid] = kc->xa[a][tid];
  }
  if (tid == 0 && DFSTATE) sh.iadf = kc->ia[a];
  load_level_chunk<DFSTATE>(sh.lc, prm, d, 0);
  __syncthreads();
  const double inv_a = 1.0 / (double)a;  // FP64 modes only (folded away in DF64)
  const double xi_p = sh.xi[p];
  // Single-precision evaluation with double-float contractions interpolates from
  // a float-pair copy of the state: it is kept as G 2^-S (a power of two per
  // level, from the first stored value's exponent) so that the copy stays inside
  // the float range whatever d; the result gets 2^S at the end.
  constexpr bool RESCALE = DF && !DFSTATE;
  int S = 0;

  for (int k = 1; k < d; ++k) {
    const int j = k - 1;  // axis of this level
    if (j > 0 && j % kLvChunk == 0) {  // next chunk of level constants
      load_level_chunk<DFSTATE>(sh.lc, prm, d, j);
      __syncthreads();
    }
    const LevelConst &L = sh.lc[j % kLvChunk];
    const int rb = (k - 1) & 1, wb = k & 1;
    double scale = 1.0;
    if constexpr (RESCALE) {
      if (k > 1) {
        const int sk = max(-100, min(100, exponent_of(sh.G[rb][0].x)));
        S += sk;
        scale = __longlong_as_double((long long)(1023 - sk) << 52);  // 2^-sk
      }
    }
    double2 acc = make_double2(0.0, 0.0);
    DfAcc dre, dim;
    if (act) {
      const df32 ia{sh.iadf.x, sh.iadf.y}, xa{sh.xadf[p].x, sh.xadf[p].y};
      const AxisParams ap{L.c, L.w, L.ic2};
      df32 s1{0.f, 0.f}, s0{0.f, 0.f};
      if constexpr (DF64) phi_affine_coeffs<FAM>(L.cwf, ia, xa, s1, s0);
      for (int q = qs; q < a; q += Q) {
        const int i = p * a + q;
        V f;
        df32 fdf{0.f, 0.f};
        if constexpr (DF64) {
          fdf = phi_df_affine<FAM>(s1, s0, (float)q, L.ic, sh.exp2tab);
        } else {
          f = phi<FAM, F32>(((double)q + xi_p) * inv_a, ap);
        }
        if constexpr (!DF) {
          V g;
          if (k == 1) {
            g = VOps<V>::one();
          } else {
            const double *Lt = (const double *)Ltab + i;
            g = VOps<V>::zero();
#pragma unroll 4
            for (int t = 0; t < P; ++t) g = VOps<V>::fma_s(Lt[(size_t)t * npts], from2<V>(sh.G[rb][t]), g);
          }
          acc = c_add(acc, as2(VOps<V>::mul(f, g)));
        } else {
          // Interpolation and cluster sum in double-float, Dot2-style accumulation.
          const float2 *Lt = (const float2 *)Ltab + i;
          df32 gr{1.f, 0.f}, gi{0.f, 0.f};
          if (k > 1) {
            DfAcc ar, ai;
#pragma unroll 4
            for (int t = 0; t < P; ++t) {
              const float2 l = Lt[(size_t)t * npts];
              const float4 gt = sh.Gdf[rb][t];
              dacc_prod(ar, df32{l.x, l.y}, df32{gt.x, gt.y});
              if constexpr (CPLX) dacc_prod(ai, df32{l.x, l.y}, df32{gt.z, gt.w});
            }
            gr = dacc_value(ar);
            if constexpr (CPLX) gi = dacc_value(ai);
          }
          if constexpr (CPLX) {
            const double2 f2 = as2(f);
            const df32 fr = (PREC == MDI_PREC_DF64) ? df_from_double(f2.x) : df32{(float)f2.x, 0.f};
            const df32 fi = (PREC == MDI_PREC_DF64) ? df_from_double(f2.y) : df32{(float)f2.y, 0.f};
            dacc_prod(dre, fr, gr);
            dacc_prod(dre, df_neg(fi), gi);
            dacc_prod(dim, fr, gi);
            dacc_prod(dim, fi, gr);
          } else if constexpr (DF64) {
            dacc_prod(dre, fdf, gr);
          } else {
            dacc_prod(dre, df32{(float)as2(f).x, 0.f}, gr);
          }
        }
      }
    }
    // The Q lanes of node p add their sums; lane qs = 0 writes the new state.
    if (warp_act) {
      if constexpr (DF) {
        const df32 sr = lanes_sum_df(dacc_value(dre), Q);
        const df32 si = CPLX ? lanes_sum_df(dacc_value(dim), Q) : df32{0.f, 0.f};
        if (act && qs == 0) {
          if constexpr (DFSTATE) {
            const df32 ia{sh.iadf.x, sh.iadf.y};
            const df32 gr = df_mul(sr, ia), gi = df_mul(si, ia);
            sh.Gdf[wb][p] = make_float4(gr.hi, gr.lo, gi.hi, gi.lo);
          } else {
            const double2 g = make_double2(df_to_double(sr) * (inv_a * scale), df_to_double(si) * (inv_a * scale));
            sh.G[wb][p] = g;
            sh.Gdf[wb][p] = split2(g);
          }
        }
      } else {
        const double2 s = lanes_sum(acc, Q);
        if (act && qs == 0) sh.G[wb][p] = c_scale(s, inv_a);
      }
    }
    __syncthreads();
  }

  // Last level: Q = (1/n_last) sum_s phi_d(s/n_last) G_{d-1}(s/n_last).
  last_level<FAM, PREC>(sh, Ftab, P, d, a, n_last, prm, out_slot, (d - 1) & 1);
  if constexpr (RESCALE)
    if (tid == 0 && S != 0) *out_slot = scale_pow2(*out_slot, S);  // the thread that wrote it
}

// ---------------------------------------------------------------------------
// One integral of a real family in DF64 with paired cluster points.  The state
// is kept as E_t = (G_t + G_{P-1-t})/2 and O_t = (G_t - G_{P-1-t})/2 (t < h, sh.Gdf
// as (E.hi, E.lo, O.hi, O.lo)).  With S+ = sum_t Lp[t] E_t and S- = sum_t Lm[t] O_t,
//     G(u) = S+ + S-,   G(1 - u) = S+ - S-,
// so one pass of h Dot2 pairs interpolates both points of a pair: P multiply-adds
// for two cluster points instead of 2P.  The two accumulators are combined with
// one TwoSum of their high parts and one add of their low parts (pair_combine),
// whose error is bounded relative to |S+| + |S-| -- the bound the accumulated
// sums carry already.  Lanes are pair-major: the Q lanes of
// pair pp take the points q of node pp (and a-1-q of node P-1-pp) and accumulate
// both nodes' sums.  The last level unpacks E, O into G and runs last_level.
// ---------------------------------------------------------------------------
// S+ and S- of one cluster point: h Dot2 pairs over the paired table column Lt
// (entries stride apart) and the state E, O.  H > 0 fixes h at compile time.
template <int H>
__device__ __forceinline__ void paired_dot(const float4 *__restrict__ Lt, int stride, const float4 *__restrict__ EO,
                                           int h, DfAcc &sp, DfAcc &sm) {
  if constexpr (H > 0) {
#pragma unroll
    for (int t = 0; t < H; ++t) {
      const float4 l = Lt[t * stride];
      const float4 eo = EO[t];
      dacc_prod(sp, df32{l.x, l.y}, df32{eo.x, eo.y});
      dacc_prod(sm, df32{l.z, l.w}, df32{eo.z, eo.w});
    }
  } else {
#pragma unroll 4
    for (int t = 0; t < h; ++t) {
      const float4 l = Lt[(size_t)t * stride];
      const float4 eo = EO[t];
      dacc_prod(sp, df32{l.x, l.y}, df32{eo.x, eo.y});
      dacc_prod(sm, df32{l.z, l.w}, df32{eo.z, eo.w});
    }
  }
}

// phi_j at a float coordinate, evaluated in float (the single-precision-evaluation
// modes of the paired sweeps): the formulas of phi32 with float parameters.
struct AxisF {
  float c, w, ic2;
};
template <int FAM>
__device__ __forceinline__ float phi_f(float u, const AxisF &p) {
  if constexpr (FAM == MDI_FAM_EXP) {
    return expf(p.c * u);
  } else if constexpr (FAM == MDI_FAM_GAUSS) {
    const float t = p.c * (u - p.w);
    return expf(-t * t);
  } else {
    const float t = u - p.w;
    return 1.0f / fmaf(t, t, p.ic2);
  }
}
// acc += f g for a float f and a double-float g: the exact product of f and g.hi,
// and f g.lo folded into the low sum.
__device__ __forceinline__ void dacc_prod_f(DfAcc &a, float f, df32 g) {
  const float p = __fmul_rn(f, g.hi);
  const float e = __fmaf_rn(f, g.hi, -p);
  const df32 t = two_sum(a.s, p);
  a.s = t.hi;
  a.c = __fadd_rn(a.c, __fmaf_rn(f, g.lo, __fadd_rn(e, t.lo)));
}

// PREC: MDI_PREC_DF64 (phi in double-float) or MDI_PREC_FP32_EVAL_DF32 (phi in
// float at the float coordinate (q + xi_p)/a, the rest as in DF64).
template <int FAM, int H, int PREC = MDI_PREC_DF64>
__device__ void sweep_paired(NodesShared &sh, const NodesConsts *__restrict__ kc, const float4 *__restrict__ Lpm,
                             const void *__restrict__ Ftab, int P, int d, int a, int n_last,
                             const double *__restrict__ prm, double *__restrict__ out_slot,
                             const Team &tm = Team::block()) {
  const int h = H > 0 ? H : P / 2;
  const int tid = tm.tid, B = tm.size;
  const int Q = node_lanes(B, h);
  const int pp = min(tid / Q, h - 1), pb = P - 1 - pp, qs = tid % Q;
  const bool act = tid < h * Q;
  const bool warp_act = (tid & ~(kWarp - 1)) < h * Q;
  const int npts_h = a * h;
  constexpr bool F32 = (PREC == MDI_PREC_FP32_EVAL_DF32);
  if (tid < h) sh.Gdf[0][tid] = make_float4(1.f, 0.f, 0.f, 0.f);  // G_0 = 1: E = 1, O = 0
  if (tid < P) sh.xadf[tid] = kc->xa[a][tid];
  if (tid == 0) sh.iadf = kc->ia[a];
  load_level_chunk<!F32>(sh.lc, prm, d, 0, tm);
  tm.sync();
  const df32 ia{sh.iadf.x, sh.iadf.y};
  const df32 ia2{0.5f * ia.hi, 0.5f * ia.lo};  // 1/(2a), exact halving
  // The stored state is G 2^-S: each level rescales its output by 2^-s, s the
  // exponent of the first stored value it reads, so that the float pairs hold one
  // level's growth whatever d (the product over levels leaves the float range,
  // e.g. 3.7e40 for d = 130).  Exact: powers of two; the result gets 2^S at the end.
  int S = 0;

  for (int k = 1; k < d; ++k) {
    const int j = k - 1;
    if (j > 0 && j % kLvChunk == 0) {
      load_level_chunk<!F32>(sh.lc, prm, d, j, tm);
      tm.sync();
    }
    const LevelConst &L = sh.lc[j % kLvChunk];
    const int rb = (k - 1) & 1, wb = k & 1;
    DfAcc acc_a, acc_b;
    if constexpr (F32) {
      if (act) {
        const AxisF af{(float)L.c, (float)L.w, (float)L.ic2};
        const float iaf = ia.hi, xaf = sh.xadf[pp].x, xbf = sh.xadf[pb].x;
        for (int q = qs; q < a; q += Q) {
          df32 ga{1.f, 0.f}, gb{1.f, 0.f};
          if (k > 1) {
            DfAcc sp, sm;
            paired_dot<H>(Lpm + pp * a + q, npts_h, sh.Gdf[rb], h, sp, sm);
            ga = pair_combine(sp, sm, 1.0f);
            gb = pair_combine(sp, sm, -1.0f);
          }
          dacc_prod_f(acc_a, phi_f<FAM>(fmaf((float)q, iaf, xaf), af), ga);
          dacc_prod_f(acc_b, phi_f<FAM>(fmaf((float)(a - 1 - q), iaf, xbf), af), gb);
        }
      }
    } else if (act) {
      const df32 xa{sh.xadf[pp].x, sh.xadf[pp].y}, xb{sh.xadf[pb].x, sh.xadf[pb].y};
      df32 s1a, s0a, s1b, s0b;
      phi_affine_coeffs<FAM>(L.cwf, ia, xa, s1a, s0a);
      phi_affine_coeffs<FAM>(L.cwf, ia, xb, s1b, s0b);
      for (int q = qs; q < a; q += Q) {
        df32 ga{1.f, 0.f}, gb{1.f, 0.f};
        if (k > 1) {
          DfAcc sp, sm;
          paired_dot<H>(Lpm + pp * a + q, npts_h, sh.Gdf[rb], h, sp, sm);
          ga = pair_combine(sp, sm, 1.0f);
          gb = pair_combine(sp, sm, -1.0f);
        }
        dacc_prod(acc_a, phi_df_affine<FAM>(s1a, s0a, (float)q, L.ic, sh.exp2tab), ga);
        dacc_prod(acc_b, phi_df_affine<FAM>(s1b, s0b, (float)(a - 1 - q), L.ic, sh.exp2tab), gb);
      }
    }
    // The read buffer rb is not written this level: its first value's exponent is
    // read here, after the cluster loop, so nothing extra stays live through it.
    int sk = 0;
    if (k > 1) {
      const int bits = __float_as_int(sh.Gdf[rb][0].x) & 0x7FFFFFFF;
      if (bits != 0 && bits < 0x7F800000) sk = max(-100, min(100, (bits >> 23) - 127));
    }
    S += sk;
    const float scale = __int_as_float((127 - sk) << 23);  // 2^-sk
    if (warp_act) {
      const DfAcc sa = lanes_sum_acc(acc_a, Q), sbv = lanes_sum_acc(acc_b, Q);
      if (act && qs == 0) {
        // E = (G_a + G_b)/2, O = (G_a - G_b)/2 with G = (1/a) * sum: one scale by
        // 2^-sk/(2a).
        const df32 ia2s{ia2.hi * scale, ia2.lo * scale};
        const df32 E = df_mul(pair_combine(sa, sbv, 1.0f), ia2s);
        const df32 O = df_mul(pair_combine(sa, sbv, -1.0f), ia2s);
        sh.Gdf[wb][pp] = make_float4(E.hi, E.lo, O.hi, O.lo);
      }
    }
    tm.sync();
  }
  // G_{d-1} from (E, O) into the other buffer, then the common last level.
  const int eb = (d - 1) & 1, gbuf = eb ^ 1;
  if (tid < P) {
    const int t = tid < h ? tid : P - 1 - tid;
    const float4 eo = sh.Gdf[eb][t];
    const df32 E{eo.x, eo.y}, O{eo.z, eo.w};
    const df32 v = tid < h ? df_add(E, O) : df_add(E, df_neg(O));
    sh.Gdf[gbuf][tid] = make_float4(v.hi, v.lo, 0.f, 0.f);
    if constexpr (F32) sh.G[gbuf][tid] = make_double2(df_to_double(v), 0.0);  // its last level reads doubles
  }
  tm.sync();
  last_level<FAM, PREC>(sh, Ftab, P, d, a, n_last, prm, out_slot, gbuf, tm);
  if (tid == 0 && S != 0) *out_slot = scale_pow2(*out_slot, S);  // the thread that wrote it
}

// phi_j in FP64 at the affine argument t of the point (see phi_affine_coeffs):
// Gaussian exp(-t^2), peak 1/(t^2 + 1/c^2), exponential exp(t).
template <int FAM>
__device__ __forceinline__ double phi_t64(double t, double ic2, const double *__restrict__ T) {
  if constexpr (FAM == MDI_FAM_GAUSS) return exp_tang64(-(t * t), T);
  else if constexpr (FAM == MDI_FAM_PEAK) return rcp_nr64(fma(t, t, ic2));
  else return exp_tang64(t, T);
}

// The same pairing in FP64 (real families): the state (E_t, O_t) in sh.G as
// doubles, the paired table as (Lp, Lm) doubles, phi in FP64.  P/2 fused
// multiply-adds per cluster point instead of P, on the FP64 pipe that bounds
// this mode.  F32 (MDI_PREC_FP32_EVAL_FP64): phi in float at the float coordinate
// (q + xi_p)/a, as the paired double-float sweep evaluates it.
template <int FAM, int H, bool F32 = false>
__device__ void sweep_paired_fp64(NodesShared &sh, const NodesConsts *__restrict__ kc,
                                  const double2 *__restrict__ Lpm, const void *__restrict__ Ftab, int P, int d, int a,
                                  int n_last, const double *__restrict__ prm, double *__restrict__ out_slot,
                                  const Team &tm = Team::block()) {
  const int h = H > 0 ? H : P / 2;
  const int tid = tm.tid, B = tm.size;
  const int Q = node_lanes(B, h);
  const int pp = min(tid / Q, h - 1), pb = P - 1 - pp, qs = tid % Q;
  const bool act = tid < h * Q;
  const bool warp_act = (tid & ~(kWarp - 1)) < h * Q;
  const int npts_h = a * h;
  if (tid < h) sh.G[0][tid] = make_double2(1.0, 0.0);  // G_0 = 1: E = 1, O = 0
  if (F32 && tid < P) sh.xadf[tid] = kc->xa[a][tid];
  const double inv_a = 1.0 / (double)a, half_inv_a = 0.5 * inv_a;
  constexpr bool REC = FAM == MDI_FAM_GAUSS && !F32;  // the recurrence's kap comes with the level constants
  const double *ktab = REC ? sh.exp2d : nullptr;
  load_level_chunk(sh.lc, prm, d, 0, tm, ktab, inv_a, (double)Q);
  tm.sync();
  const double xa = sh.xi[pp], xb = sh.xi[pb];
  const double x0 = xa * inv_a;  // xi_pp / a
  const float iaf = F32 ? kc->ia[a].x : 0.f, xaf = F32 ? sh.xadf[pp].x : 0.f, xbf = F32 ? sh.xadf[pb].x : 0.f;

  for (int k = 1; k < d; ++k) {
    const int j = k - 1;
    if (j > 0 && j % kLvChunk == 0) {
      load_level_chunk(sh.lc, prm, d, j, tm, ktab, inv_a, (double)Q);
      tm.sync();
    }
    const LevelConst &L = sh.lc[j % kLvChunk];
    const int rb = (k - 1) & 1, wb = k & 1;
    // phi's argument at the cluster points u_a = q/a + xi_pp/a of node pp and
    // u_b = 1 - u_a of node P-1-pp, as t = s1 q + s0:
    //   GAUSS  t = c (u - w)      (sign of t_b immaterial: phi depends on t^2)
    //   PEAK   t = u - w          (likewise)
    //   EXP    t = c u
    double s1a = 0.0, s0a = 0.0, s1b = 0.0, s0b = 0.0;
    if constexpr (!F32) {
      if constexpr (FAM == MDI_FAM_GAUSS) {  // c (x0 - w), c (x0 - (1 - w))
        s1a = s1b = L.c * inv_a;
        s0a = fma(L.c, x0, -L.cw);
        s0b = fma(L.c, x0, -L.c1w);
      } else if constexpr (FAM == MDI_FAM_PEAK) {
        s1a = s1b = inv_a;
        s0a = x0 - L.w;
        s0b = x0 - (1.0 - L.w);
      } else {
        s1a = L.c * inv_a;
        s1b = -s1a;
        s0a = L.c * x0;
        s0b = L.c - s0a;
      }
    }
    // Gaussian factors along a lane's points q = qs, qs + Q, ...: t steps by
    // dq = s1 Q, so phi(q + Q) = phi(q) rho(q) and rho(q + Q) = rho(q) kappa with
    // rho(q) = exp(-(2 t dq + dq^2)) and kappa = exp(-2 dq^2) -- two multiplies per
    // point after three exps per lane and level, against an exp per point: the
    // mirrored point's argument is t_b = t_a - (t_a - t_b) with a per-level
    // difference, so rho_b = rho_a exp(2 (t_a - t_b) dq), and that factor and kappa
    // come with the level's constants.  Taken when every lane has at least three
    // points and the level's arguments stay moderate (|t| <= B < 20,
    // |dq| (2B + |dq|) < 350: no factor or ratio leaves the normal range).  The k-th
    // factor's relative error is the rounding of the arguments carried along,
    // about (t0^2 + k |2 t0 dq| + k^2 dq^2) ulps -- the size of the direct exp's own
    // argument rounding, t_k^2 ulps -- plus about 3k ulps of products.
    bool rec = false;
    double fa = 0.0, fb = 0.0, rho_a = 0.0, rho_b = 0.0, kap = 0.0;
    if constexpr (FAM == MDI_FAM_GAUSS && !F32) {
      rec = (a + Q - 1) / Q >= 3 && L.rec_ok;
      if (rec && act) {
        const double dq = s1a * (double)Q;
        const double qd0 = sh.qd[qs];
        const double ta = fma(s1a, qd0, s0a), tb = fma(s1b, qd0, s0b);
        fa = exp_tang64(-(ta * ta), sh.exp2d);
        fb = exp_tang64(-(tb * tb), sh.exp2d);
        rho_a = exp_tang64(-fma(2.0 * ta, dq, dq * dq), sh.exp2d);
        rho_b = rho_a * L.eb;
        kap = L.kap;
      }
    }
    double acc_a = 0.0, acc_b = 0.0;
    if (act) {
      for (int q = qs; q < a; q += Q) {
        double ga = 1.0, gb = 1.0;
        if (k > 1) {
          const double2 *Lt = Lpm + pp * a + q;
          double sp = 0.0, sm = 0.0;
          if constexpr (H > 0) {
#pragma unroll
            for (int t = 0; t < H; ++t) {
              const double2 l = Lt[t * npts_h], eo = sh.G[rb][t];
              sp = fma(l.x, eo.x, sp);
              sm = fma(l.y, eo.y, sm);
            }
          } else {
#pragma unroll 4
            for (int t = 0; t < h; ++t) {
              const double2 l = Lt[(size_t)t * npts_h], eo = sh.G[rb][t];
              sp = fma(l.x, eo.x, sp);
              sm = fma(l.y, eo.y, sm);
            }
          }
          ga = sp + sm;
          gb = sp - sm;
        }
        if constexpr (F32) {
          const AxisF af{(float)L.c, (float)L.w, (float)L.ic2};
          acc_a = fma((double)phi_f<FAM>(fmaf((float)q, iaf, xaf), af), ga, acc_a);
          acc_b = fma((double)phi_f<FAM>(fmaf((float)(a - 1 - q), iaf, xbf), af), gb, acc_b);
        } else if (FAM == MDI_FAM_GAUSS && rec) {
          acc_a = fma(fa, ga, acc_a);
          acc_b = fma(fb, gb, acc_b);
          fa *= rho_a;
          rho_a *= kap;
          fb *= rho_b;
          rho_b *= kap;
        } else {
          // The arguments of both mirrored points are affine in q (u_b = 1 - u_a).
          const double qd = sh.qd[q];
          acc_a = fma(phi_t64<FAM>(fma(s1a, qd, s0a), L.ic2, sh.exp2d), ga, acc_a);
          acc_b = fma(phi_t64<FAM>(fma(s1b, qd, s0b), L.ic2, sh.exp2d), gb, acc_b);
        }
      }
    }
    if (warp_act) {
      const double2 s2 = lanes_sum(make_double2(acc_a, acc_b), Q);
      if (act && qs == 0) sh.G[wb][pp] = make_double2((s2.x + s2.y) * half_inv_a, (s2.x - s2.y) * half_inv_a);
    }
    tm.sync();
  }
  const int eb = (d - 1) & 1, gbuf = eb ^ 1;
  if (tid < P) {
    const int t = tid < h ? tid : P - 1 - tid;
    const double2 eo = sh.G[eb][t];
    sh.G[gbuf][tid] = make_double2(tid < h ? eo.x + eo.y : eo.x - eo.y, 0.0);
  }
  tm.sync();
  last_level<FAM, F32 ? MDI_PREC_FP32_EVAL_FP64 : MDI_PREC_FP64>(sh, Ftab, P, d, a, n_last, prm, out_slot, gbuf, tm);
}

// One integral of a real family on the paired sweep of a single-precision-
// evaluation mode; H > 0 fixes the number of node pairs at compile time.
template <int PREC, int H, int FAM>
__device__ __forceinline__ void paired_one(NodesShared &sh, const NodesConsts *__restrict__ kc, const void *C,
                                           const void *Ftab, int P, int d, int a, int n_last,
                                           const double *__restrict__ prm, double *out_slot, const Team &tm) {
  if constexpr (PREC == MDI_PREC_FP32_EVAL_DF32)
    sweep_paired<FAM, H, PREC>(sh, kc, (const float4 *)C, Ftab, P, d, a, n_last, prm, out_slot, tm);
  else
    sweep_paired_fp64<FAM, H, true>(sh, kc, (const double2 *)C, Ftab, P, d, a, n_last, prm, out_slot, tm);
}
template <int PREC, int H>
__device__ __forceinline__ void run_paired(NodesShared &sh, const NodesConsts *__restrict__ kc, const void *C,
                                           const void *Ftab, int P, int family, int d, int a, int n_last,
                                           const double *__restrict__ prm, double *out_slot, const Team &tm) {
  if (family == MDI_FAM_EXP) paired_one<PREC, H, MDI_FAM_EXP>(sh, kc, C, Ftab, P, d, a, n_last, prm, out_slot, tm);
  else if (family == MDI_FAM_GAUSS)
    paired_one<PREC, H, MDI_FAM_GAUSS>(sh, kc, C, Ftab, P, d, a, n_last, prm, out_slot, tm);
  else paired_one<PREC, H, MDI_FAM_PEAK>(sh, kc, C, Ftab, P, d, a, n_last, prm, out_slot, tm);
}

// One work item of the batched kernel: order slot `slot`, swept by team `tm` with
// state `sh`.  `whole` says the team is the whole CTA (which may stage the basis
// table in shared memory and runs every family); a one-warp team of the hybrid
// schedule runs the paired sweeps of the real families only.
template <int PREC>
__device__ __forceinline__ void nodes_item(int slot, const Team &tm, bool whole, NodesShared &sh,
                                           unsigned char *tab_smem, int &staged_a,
                                           const mdi_batch_desc *__restrict__ descs,
                                           const int32_t *__restrict__ order, int count,
                                           const mdi_batch_desc &single, const double *__restrict__ pool,
                                           long long pool_len, const void *__restrict__ tables,
                                           const float4 *__restrict__ paired, const NodesConsts *__restrict__ kc,
                                           int P, int stage, double *__restrict__ out, unsigned *__restrict__ counter,
                                           bool prepared) {
  const int inst = order ? order[slot] : slot;
  if (inst < 0 || inst >= count) {  // an order entry outside the batch is skipped
    if (tm.tid == 0) atomicOr(&counter[3], MDI_DEV_BAD_ORDER);
    return;
  }
  const mdi_batch_desc ds = descs ? descs[inst] : single;
  const int a = ds.a;
  const bool desc_ok = ds.family >= MDI_FAM_EXP && ds.family <= MDI_FAM_PEAK && ds.d >= 1 &&
                       ds.d <= MDI_BATCH_MAX_D && a >= 1 && a <= kNodesAMax && ds.n_last >= 1 &&
                       ds.n_last <= 4096 && ds.param_offset >= 0 && (whole || ds.family != MDI_FAM_OSC);
  // The integral's 2d parameters must lie inside the pool (no read past its end).
  const bool in_pool = desc_ok && ds.param_offset <= pool_len && 2ll * ds.d <= pool_len - ds.param_offset;
  if (!prepared || !in_pool) {
    if (tm.tid == 0) {
      out[inst] = __longlong_as_double(0x7ff8000000000000ll);  // NaN marks a rejected integral
      atomicOr(&counter[3], !prepared ? MDI_DEV_UNPREPARED : !desc_ok ? MDI_DEV_BAD_DESC : MDI_DEV_POOL_RANGE);
    }
    return;
  }
  // Basis tables of a: the cluster part (the paired one for real families),
  // staged in shared memory when asked and it fits, and the last-axis part.
  const bool use_paired = paired != nullptr && ds.family != MDI_FAM_OSC;
  const size_t tbytes = (size_t)a * P * P * 8;  // plain cluster part; a multiple of 16 for even P
  const unsigned char *gtab = (const unsigned char *)tables + table_offset(a, P) * 8;
  const void *Ftab = gtab + tbytes;
  const unsigned char *csrc = use_paired ? (const unsigned char *)(paired + paired_offset(a, P)) : gtab;
  const size_t cbytes = use_paired ? (size_t)a * P * P * 4 : tbytes;
  const void *C = csrc;
  if (whole && stage && cbytes <= (size_t)kNodesSmemTable && ds.d > 1) {
    const int key = 2 * a + (use_paired ? 1 : 0);
    if (staged_a != key) {
      const double2 *src = (const double2 *)csrc;
      double2 *dst = (double2 *)tab_smem;
      for (size_t i = threadIdx.x; i < cbytes / 16; i += blockDim.x) dst[i] = src[i];
      staged_a = key;
      __syncthreads();
    }
    C = tab_smem;
  }
  const double *prm = pool + ds.param_offset;
  double *out_slot = out + inst;
  if (use_paired) {
    // P = 16 (the default node count) runs with the pair loop fully unrolled.
    if constexpr (PREC == MDI_PREC_FP64) {
      // FP64 and DF64 spelled out: this form keeps their instantiations as
      // they were tuned (the FP64 one free of spills).
      const double2 *Lpm = (const double2 *)C;
      if (P == 16) {
        if (ds.family == MDI_FAM_EXP)
          sweep_paired_fp64<MDI_FAM_EXP, 8>(sh, nullptr, Lpm, Ftab, P, ds.d, a, ds.n_last, prm, out_slot, tm);
        else if (ds.family == MDI_FAM_GAUSS)
          sweep_paired_fp64<MDI_FAM_GAUSS, 8>(sh, nullptr, Lpm, Ftab, P, ds.d, a, ds.n_last, prm, out_slot, tm);
        else sweep_paired_fp64<MDI_FAM_PEAK, 8>(sh, nullptr, Lpm, Ftab, P, ds.d, a, ds.n_last, prm, out_slot, tm);
      } else {
        if (ds.family == MDI_FAM_EXP)
          sweep_paired_fp64<MDI_FAM_EXP, 0>(sh, nullptr, Lpm, Ftab, P, ds.d, a, ds.n_last, prm, out_slot, tm);
        else if (ds.family == MDI_FAM_GAUSS)
          sweep_paired_fp64<MDI_FAM_GAUSS, 0>(sh, nullptr, Lpm, Ftab, P, ds.d, a, ds.n_last, prm, out_slot, tm);
        else sweep_paired_fp64<MDI_FAM_PEAK, 0>(sh, nullptr, Lpm, Ftab, P, ds.d, a, ds.n_last, prm, out_slot, tm);
      }
    } else if constexpr (PREC == MDI_PREC_DF64) {
      const float4 *Lpm = (const float4 *)C;
      if (P == 16) {
        if (ds.family == MDI_FAM_EXP)
          sweep_paired<MDI_FAM_EXP, 8>(sh, kc, Lpm, Ftab, P, ds.d, a, ds.n_last, prm, out_slot, tm);
        else if (ds.family == MDI_FAM_GAUSS)
          sweep_paired<MDI_FAM_GAUSS, 8>(sh, kc, Lpm, Ftab, P, ds.d, a, ds.n_last, prm, out_slot, tm);
        else sweep_paired<MDI_FAM_PEAK, 8>(sh, kc, Lpm, Ftab, P, ds.d, a, ds.n_last, prm, out_slot, tm);
      } else {
        if (ds.family == MDI_FAM_EXP)
          sweep_paired<MDI_FAM_EXP, 0>(sh, kc, Lpm, Ftab, P, ds.d, a, ds.n_last, prm, out_slot, tm);
        else if (ds.family == MDI_FAM_GAUSS)
          sweep_paired<MDI_FAM_GAUSS, 0>(sh, kc, Lpm, Ftab, P, ds.d, a, ds.n_last, prm, out_slot, tm);
        else sweep_paired<MDI_FAM_PEAK, 0>(sh, kc, Lpm, Ftab, P, ds.d, a, ds.n_last, prm, out_slot, tm);
      }
    } else if (P == 16) {
      run_paired<PREC, 8>(sh, kc, C, Ftab, P, ds.family, ds.d, a, ds.n_last, prm, out_slot, tm);
    } else {
      run_paired<PREC, 0>(sh, kc, C, Ftab, P, ds.family, ds.d, a, ds.n_last, prm, out_slot, tm);
    }
    return;
  }
  switch (ds.family) {
    case MDI_FAM_EXP: sweep_one<MDI_FAM_EXP, PREC>(sh, kc, C, Ftab, P, ds.d, a, ds.n_last, prm, out_slot); break;
    case MDI_FAM_OSC: sweep_one<MDI_FAM_OSC, PREC>(sh, kc, C, Ftab, P, ds.d, a, ds.n_last, prm, out_slot); break;
    case MDI_FAM_GAUSS: sweep_one<MDI_FAM_GAUSS, PREC>(sh, kc, C, Ftab, P, ds.d, a, ds.n_last, prm, out_slot); break;
    default: sweep_one<MDI_FAM_PEAK, PREC>(sh, kc, C, Ftab, P, ds.d, a, ds.n_last, prm, out_slot); break;
  }
}

// Persistent batched kernel.  Order slots below `split` are swept by the whole
// CTA; from the first slot at or past it (hybrid schedule: two-warp CTAs with the
// tables read through L1) each warp takes slots of its own, with its own copy of
// the state (the second NodesShared).  split >= count: every slot by the whole
// CTA.
template <int PREC>
__global__ void __launch_bounds__(kNodesMaxBlock) nodes_batched_kernel(const mdi_batch_desc *__restrict__ descs,
                                                                       const int32_t *__restrict__ order, int count,
                                                                       mdi_batch_desc single,
                                                                       const double *__restrict__ pool,
                                                                       long long pool_len,
                                                                       const void *__restrict__ tables,
                                                                       const float4 *__restrict__ paired,
                                                                       const NodesConsts *__restrict__ kc, int P,
                                                                       int stage, int split, double *__restrict__ out,
                                                                       unsigned *__restrict__ counter,
                                                                       unsigned expect_tag) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  const bool hybrid = split < count;
  NodesShared &sh = *reinterpret_cast<NodesShared *>(dyn_smem);
  NodesShared &sh2 = *reinterpret_cast<NodesShared *>(dyn_smem + (hybrid ? align16(sizeof(NodesShared)) : 0));
  unsigned char *tab_smem = dyn_smem + align16(sizeof(NodesShared)) * (hybrid ? 2 : 1);
  for (int c = 0; c < (hybrid ? 2 : 1); ++c) {
    NodesShared &s = c ? sh2 : sh;
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
      s.xi[t] = kc->xi[t];
      s.bw[t] = kc->bw[t];
    }
    if (PREC == MDI_PREC_DF64)
      for (int j = threadIdx.x; j < kExpTable; j += blockDim.x) s.exp2tab[j] = kc->exp2tab[j];
    if (PREC == MDI_PREC_FP64) {
      for (int j = threadIdx.x; j < kExpTable; j += blockDim.x) s.exp2d[j] = kc->exp2d[j];
      for (int q = threadIdx.x; q < kNodesAMax; q += blockDim.x) s.qd[q] = (double)q;
    }
  }
  int staged_a = -1;
  // counter[0]: next work item; counter[1]: CTAs finished; counter[2]: preparation
  // tag; counter[3]: the device status word (MDI_DEV_* flags, OR-ed in).
  const bool prepared = counter[2] == expect_tag;
  int slot;
  while (true) {
    if (threadIdx.x == 0) sh.inst = (int)atomicAdd(&counter[0], 1u);
    __syncthreads();
    slot = sh.inst;
    __syncthreads();
    if (slot >= count || slot >= split) break;
    nodes_item<PREC>(slot, Team::block(), true, sh, tab_smem, staged_a, descs, order, count, single, pool, pool_len,
                     tables, paired, kc, P, stage, out, counter, prepared);
  }
  if (slot < count) {  // hybrid: slot is the first one past the split; warp 0 takes it
    {
      const int warp = threadIdx.x / kWarp, lane = threadIdx.x & (kWarp - 1);
      NodesShared &shw = warp == 0 ? sh : sh2;
      const Team tm{lane, kWarp};
      int mine = warp == 0 ? slot : -1;
      while (true) {
        if (mine < 0) {
          unsigned v = 0;
          if (lane == 0) v = atomicAdd(&counter[0], 1u);
          mine = (int)__shfl_sync(0xffffffffu, v, 0);
        }
        if (mine >= count) break;
        nodes_item<PREC>(mine, tm, false, shw, tab_smem, staged_a, descs, order, count, single, pool, pool_len,
                         tables, paired, kc, P, 0, out, counter, prepared);
        mine = -1;
      }
    }
    __syncthreads();
  }
  // The last CTA to finish re-arms the queue for the next call on this workspace.
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&counter[1], 1u) == gridDim.x - 1) {
      atomicExch(&counter[0], 0u);
      atomicExch(&counter[1], 0u);
    }
  }
}

// Zeroes the queue counters and the status word and stamps the preparation tag.
__global__ void nodes_arm_kernel(unsigned *counter, unsigned tag) {
  counter[0] = 0u;
  counter[1] = 0u;
  counter[2] = tag;
  counter[3] = 0u;
}

// Element-wise view of the FP64 exp and reciprocal of the paired sweep (tests
// compare them with CUDA's exp and IEEE division).
__global__ void fp64_phi_debug_kernel(int which, const double *__restrict__ x, double *__restrict__ y, int64_t n) {
  __shared__ double T[kExpTable];
  for (int j = threadIdx.x; j < kExpTable; j += blockDim.x) T[j] = kExp2TableD[j];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = which == 0 ? exp_tang64(x[i], T) : rcp_nr64(x[i]);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
NodesConfig nodes_config(const mdi_opts *opts) {
  NodesConfig c{16, 256, 0, MDI_PREC_FP64, 1, 1};
  if (opts) {
    if (opts->nodes) c.P = opts->nodes;
    if (opts->block) c.block = opts->block;
    c.ctas_per_sm = opts->ctas_per_sm;
    c.precision = opts->precision;
    c.stage = opts->table_in_l1 ? 0 : 1;
    c.step = opts->step > 1 ? opts->step : 1;
  }
  return c;
}

static bool config_ok(const NodesConfig &c) {
  if (c.P < 2 || c.P > kNodesPMax || (c.P & 1)) return false;  // even P keeps tables 16-byte aligned
  if (c.block < 32 || c.block > kNodesMaxBlock || c.block % 32 || c.block < c.P) return false;
  if (c.precision < MDI_PREC_FP64 || c.precision > MDI_PREC_DF64) return false;
  return c.ctas_per_sm >= 0 && c.ctas_per_sm <= 32;
}

// Double-float precision modes read the basis tables as float pairs.
static bool df_tables(const NodesConfig &c) {
  return c.precision == MDI_PREC_FP32_EVAL_DF32 || c.precision == MDI_PREC_DF64;
}

static size_t counter_bytes() { return align_up(4 * sizeof(unsigned)); }

// Every precision pairs the real families' cluster points (float-pair entries in
// the double-float modes, doubles otherwise).
static bool paired_tables(const NodesConfig &) { return true; }

// Tag stamped by the preparation: node count and table format.
static unsigned nodes_tag(const NodesConfig &c) {
  return 0x4D440000u | ((unsigned)c.P << 4) | (df_tables(c) ? 1u : 0u) | (paired_tables(c) ? 2u : 0u);
}

// Workspace: queue counters | basis tables | paired tables | NodesConsts.
static size_t consts_offset(const NodesConfig &cfg) {
  return counter_bytes() + align_up(table_bytes(cfg.P)) + (paired_tables(cfg) ? align_up(paired_bytes(cfg.P)) : 0);
}

size_t nodes_batched_workspace_bytes(int count, const NodesConfig &cfg) {
  (void)count;
  return consts_offset(cfg) + align_up(sizeof(NodesConsts));
}
size_t nodes_single_workspace_bytes(const NodesConfig &cfg) { return nodes_batched_workspace_bytes(1, cfg); }

static bool ws_ok(const void *ws, size_t bytes, const NodesConfig &cfg) {
  return ws && ((uintptr_t)ws % kAlign) == 0 && bytes >= nodes_batched_workspace_bytes(1, cfg);
}

mdi_status nodes_prepare(const NodesConfig &cfg, void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if (!config_ok(cfg)) return MDI_EINVAL;
  if (!ws_ok(workspace, ws_bytes, cfg)) return MDI_EWORKSPACE;
  unsigned *counter = (unsigned *)workspace;
  void *tables = (char *)workspace + counter_bytes();
  const int table_grid = sm_count() * 2;
  if (df_tables(cfg)) nodes_table_kernel<true><<<table_grid, 256, 0, stream>>>(cfg.P, tables);
  else nodes_table_kernel<false><<<table_grid, 256, 0, stream>>>(cfg.P, tables);
  mdi_status st = check_launch();
  if (st != MDI_OK) return st;
  if (paired_tables(cfg)) {
    float4 *paired = (float4 *)((char *)tables + align_up(table_bytes(cfg.P)));
    if (df_tables(cfg)) nodes_paired_table_kernel<true><<<table_grid, 256, 0, stream>>>(cfg.P, paired);
    else nodes_paired_table_kernel<false><<<table_grid, 256, 0, stream>>>(cfg.P, paired);
    if ((st = check_launch()) != MDI_OK) return st;
  }
  nodes_consts_kernel<<<1, 256, 0, stream>>>(cfg.P, (NodesConsts *)((char *)workspace + consts_offset(cfg)));
  if ((st = check_launch()) != MDI_OK) return st;
  nodes_arm_kernel<<<1, 1, 0, stream>>>(counter, nodes_tag(cfg));
  return check_launch();
}

// The hybrid schedule needs two-warp CTAs reading their tables through L1 (its
// one-warp teams run the paired sweeps of every precision).
static bool hybrid_ok(const NodesConfig &cfg) { return cfg.block == 2 * kWarp && !cfg.stage; }

template <int PREC>
static int resident_ctas(const NodesConfig &cfg, size_t smem, bool hybrid) {
  // Resident CTAs per SM for this (block, P, staging, schedule), queried once per
  // process (the GPUs one process drives are taken to be of one kind).
  static std::atomic<int> occ_cache[4][kNodesMaxBlock / 32 + 1][kNodesPMax / 2 + 1][2][2];
  std::atomic<int> &occ = occ_cache[PREC][cfg.block / 32][cfg.P / 2][cfg.stage ? 1 : 0][hybrid ? 1 : 0];
  int v = occ.load(std::memory_order_relaxed);
  if (v == 0) {
    int o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, nodes_batched_kernel<PREC>, cfg.block, smem);
    v = std::max(1, o);
    occ.store(v, std::memory_order_relaxed);
  }
  return v;
}

static size_t launch_smem(const NodesConfig &cfg, bool hybrid) {
  return nodes_smem_bytes(cfg.block, cfg.P, cfg.stage != 0) + (hybrid ? align16(sizeof(NodesShared)) : 0);
}

int nodes_workers(const NodesConfig &cfg) {
  const bool hybrid = hybrid_ok(cfg);
  const size_t smem = launch_smem(cfg, hybrid);
  int per_sm = cfg.ctas_per_sm;
  if (per_sm == 0) {
    switch (cfg.precision) {
      case MDI_PREC_FP64: per_sm = resident_ctas<MDI_PREC_FP64>(cfg, smem, hybrid); break;
      case MDI_PREC_FP32_EVAL_FP64: per_sm = resident_ctas<MDI_PREC_FP32_EVAL_FP64>(cfg, smem, hybrid); break;
      case MDI_PREC_FP32_EVAL_DF32: per_sm = resident_ctas<MDI_PREC_FP32_EVAL_DF32>(cfg, smem, hybrid); break;
      default: per_sm = resident_ctas<MDI_PREC_DF64>(cfg, smem, hybrid); break;
    }
  }
  return sm_count() * per_sm;
}

template <int PREC>
static mdi_status launch_nodes(const mdi_batch_desc *descs, const int32_t *order, int count, int split,
                               const mdi_batch_desc &single, const double *pool, int64_t pool_len,
                               const NodesConfig &cfg, double *out, void *ws, cudaStream_t stream) {
  unsigned *counter = (unsigned *)ws;
  void *tables = (char *)ws + counter_bytes();
  const bool hybrid = split < count && hybrid_ok(cfg);
  const int split_eff = hybrid ? std::max(split, 0) : count;
  const size_t smem = launch_smem(cfg, hybrid);
  // The dynamic shared-memory limit, set once per device and mode (an attribute
  // belongs to the device whose context sets it; racing threads set it twice, which
  // is harmless).
  static std::atomic<unsigned> attr_set[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  cudaGetLastError();
  const bool cached = dev >= 0 && dev < 64;
  if (!cached || !(attr_set[dev].load(std::memory_order_acquire) & (1u << PREC))) {
    cudaError_t e = cudaFuncSetAttribute(nodes_batched_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)nodes_smem_bytes(kNodesMaxBlock, 2, true));
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return MDI_ECUDA;
    }
    if (cached) attr_set[dev].fetch_or(1u << PREC, std::memory_order_release);
  }
  const int per_sm = cfg.ctas_per_sm ? cfg.ctas_per_sm : resident_ctas<PREC>(cfg, smem, hybrid);
  const int grid = std::max(1, std::min(count, sm_count() * per_sm));
  const float4 *paired = paired_tables(cfg) ? (const float4 *)((char *)tables + align_up(table_bytes(cfg.P))) : nullptr;
  const NodesConsts *kc = (const NodesConsts *)((char *)ws + consts_offset(cfg));
  nodes_batched_kernel<PREC><<<grid, cfg.block, smem, stream>>>(descs, order, count, single, pool,
                                                                 (long long)pool_len, tables, paired, kc, cfg.P,
                                                                 cfg.stage, split_eff, out, counter, nodes_tag(cfg));
  return check_launch();
}

static mdi_status dispatch_nodes(const mdi_batch_desc *descs, const int32_t *order, int count, int split,
                                 const mdi_batch_desc &single, const double *pool, int64_t pool_len,
                                 const NodesConfig &cfg, double *out, void *ws, cudaStream_t stream) {
  switch (cfg.precision) {
    case MDI_PREC_FP64:
      return launch_nodes<MDI_PREC_FP64>(descs, order, count, split, single, pool, pool_len, cfg, out, ws, stream);
    case MDI_PREC_FP32_EVAL_FP64:
      return launch_nodes<MDI_PREC_FP32_EVAL_FP64>(descs, order, count, split, single, pool, pool_len, cfg, out, ws,
                                                   stream);
    case MDI_PREC_FP32_EVAL_DF32:
      return launch_nodes<MDI_PREC_FP32_EVAL_DF32>(descs, order, count, split, single, pool, pool_len, cfg, out, ws,
                                                   stream);
    default:
      return launch_nodes<MDI_PREC_DF64>(descs, order, count, split, single, pool, pool_len, cfg, out, ws, stream);
  }
}

mdi_status nodes_batched_launch(const mdi_batch_desc *descs, const int32_t *order, int count, int split,
                                const double *param_pool, int64_t pool_len, const NodesConfig &cfg, double *out,
                                void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if (!descs || !param_pool || !out || count < 1) return MDI_EINVAL;
  if (!config_ok(cfg)) return MDI_EINVAL;
  if (!ws_ok(workspace, ws_bytes, cfg)) return MDI_EWORKSPACE;
  mdi_batch_desc none{};
  return dispatch_nodes(descs, order, count, split, none, param_pool, pool_len, cfg, out, workspace, stream);
}

size_t nodes_status_word_bytes() { return 4 * sizeof(unsigned); }

mdi_status fp64_phi_debug_launch(int which, const double *x, double *y, int64_t n, cudaStream_t stream) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8));
  fp64_phi_debug_kernel<<<grid, 256, 0, stream>>>(which, x, y, n);
  return check_launch();
}

mdi_status nodes_read_status(const void *workspace, bool clear, uint32_t *word, cudaStream_t stream) {
  unsigned *status = (unsigned *)workspace + 3;  // counter[3]
  cudaError_t e = cudaMemcpyAsync(word, status, sizeof(unsigned), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e == cudaSuccess && clear) e = cudaMemsetAsync(status, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return MDI_ECUDA;
  }
  return MDI_OK;
}

mdi_status nodes_single_launch(int family, int d, int64_t a, int64_t n_last, const double *params,
                               const NodesConfig &cfg, double *out, void *workspace, size_t ws_bytes,
                               cudaStream_t stream) {
  if (d < 1 || d > MDI_BATCH_MAX_D || a < 1 || a > kNodesAMax || n_last < 1 || n_last > 4096) return MDI_EUNSUPPORTED;
  mdi_status st = nodes_prepare(cfg, workspace, ws_bytes, stream);
  if (st != MDI_OK) return st;
  mdi_batch_desc one{family, d, (int32_t)a, (int32_t)n_last, 0, 0};
  return dispatch_nodes(nullptr, nullptr, 1, 1, one, params, 2 * (int64_t)d, cfg, out, workspace, stream);
}

}  // namespace mdi
