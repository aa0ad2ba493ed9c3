// mdi_nodes.cuh -- pieces of the node level state shared by the batched sweep
// (mdi_nodes.cu) and the level-parallel sweep and adjoint (mdi_levels.cu).
//
// The state G_k(x) is kept at P Chebyshev points of the first kind on [0,1],
//     xi_p = (1 + cos(pi (2p+1) / (2P))) / 2,
// and read between them with the barycentric formula of the second kind, whose
// weights for these points are (-1)^p sin(pi (2p+1) / (2P)) (Berrut & Trefethen,
// "Barycentric Lagrange interpolation", SIAM Review 46 (2004), Sec. 5).
#pragma once

#include "mdi_cheb_table.inc"
#include "mdi_common.cuh"

namespace mdi {

constexpr int kNodesAMax = 64;  // largest a with a basis table
constexpr int kNodesPMax = 32;
static_assert(kChebTablePMax >= kNodesPMax, "the generated node table covers every P");

// xi_p and the weight of node p of P, 0 <= p < P <= kNodesPMax: read from the
// table build.py writes from the definitions above (each value correctly
// rounded), rather than by cospi/sinpi in FP64 at the start of every CTA --
// about sixty FP64 instructions on the critical path of each, on a chip whose
// FP64 unit takes a warp instruction per ~64 cycles per sub-partition.
__device__ __forceinline__ double cheb_node(int p, int P) { return kChebXiGen[P * (P - 1) / 2 + p]; }
__device__ __forceinline__ double cheb_weight(int p, int P) { return kChebBwGen[P * (P - 1) / 2 + p]; }

__device__ __forceinline__ double2 as2(double v) { return make_double2(v, 0.0); }
__device__ __forceinline__ double2 as2(double2 v) { return v; }
template <typename V> __device__ __forceinline__ V from2(double2 v);
template <> __device__ __forceinline__ double from2<double>(double2 v) { return v.x; }
template <> __device__ __forceinline__ double2 from2<double2>(double2 v) { return v; }

// Derivatives of phi_j with respect to c_j (dc) and w_j (dw), with phi itself,
// from one evaluation of the transcendental part.  Complex for OSC.
template <int FAM> struct PhiGrad {
  typename FamTraits<FAM>::V f, dc, dw;
};

template <int FAM> __device__ __forceinline__ PhiGrad<FAM> phi_grad64(double x, const AxisParams &p);
template <> __device__ __forceinline__ PhiGrad<MDI_FAM_EXP> phi_grad64<MDI_FAM_EXP>(double x, const AxisParams &p) {
  const double e = exp(p.c * x);
  return {e, x * e, 0.0};
}
template <> __device__ __forceinline__ PhiGrad<MDI_FAM_OSC> phi_grad64<MDI_FAM_OSC>(double x, const AxisParams &p) {
  double s, c;
  sincos(p.c * x, &s, &c);
  // d/dc exp(i c x) = i x exp(i c x)
  return {make_double2(c, s), make_double2(-x * s, x * c), make_double2(0.0, 0.0)};
}
template <> __device__ __forceinline__ PhiGrad<MDI_FAM_GAUSS> phi_grad64<MDI_FAM_GAUSS>(double x, const AxisParams &p) {
  const double t = x - p.w, e = exp(-(p.c * t) * (p.c * t));
  return {e, -2.0 * p.c * t * t * e, 2.0 * p.c * p.c * t * e};
}
template <> __device__ __forceinline__ PhiGrad<MDI_FAM_PEAK> phi_grad64<MDI_FAM_PEAK>(double x, const AxisParams &p) {
  const double t = x - p.w, D = fma(t, t, p.ic2), f = 1.0 / D, f2 = f * f;
  return {f, 2.0 * p.ic2 / p.c * f2, 2.0 * t * f2};
}

// phi_j(u) in double-float arithmetic for the real families: cw = (c.hi, c.lo,
// w.hi, w.lo), ic = 1/c^2 as a float pair (PEAK), tab = the 2^(j/256) table of the
// double-float exp.
template <int FAM> __device__ __forceinline__ df32 phi_df(df32 u, float4 cw, float2 ic, const float2 *tab) {
  const df32 c{cw.x, cw.y}, w{cw.z, cw.w};
  if constexpr (FAM == MDI_FAM_EXP) {
    return df_exp(df_mul(c, u), tab);
  } else if constexpr (FAM == MDI_FAM_GAUSS) {
    const df32 t = df_mul(c, df_add(u, df_neg(w)));
    return df_exp(df_neg(df_sqr(t)), tab);
  } else {
    const df32 t = df_add(u, df_neg(w));
    return df_rcp(df_add(df_sqr(t), df32{ic.x, ic.y}));
  }
}

}  // namespace mdi
