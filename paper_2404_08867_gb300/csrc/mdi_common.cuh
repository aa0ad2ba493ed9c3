// mdi_common.cuh -- device helpers shared by the MDI-LR kernels (sm_103a).
//
// Integrand factors phi_j of the product-form families, complex arithmetic on
// double2, double-float ("df32": an unevaluated sum hi + lo of two floats)
// arithmetic, and warp/block reductions with a fixed summation tree so that every
// result is deterministic run to run.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mdi_lr.h"

namespace mdi {

constexpr int kWarp = 32;
constexpr double kTwoPi = 6.283185307179586476925286766559;

// ---------------------------------------------------------------------------
// Complex values as double2 (x = real, y = imaginary)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ double2 c_make(double re, double im) { return make_double2(re, im); }
__device__ __forceinline__ double2 c_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 c_mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 c_scale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// Generic value operations for V = double (real families) or double2 (OSC).
template <typename V> struct VOps;
template <> struct VOps<double> {
  __device__ static double zero() { return 0.0; }
  __device__ static double one() { return 1.0; }
  __device__ static double add(double a, double b) { return a + b; }
  __device__ static double mul(double a, double b) { return a * b; }
  __device__ static double scale(double a, double s) { return a * s; }
  __device__ static double fma_s(double s, double g, double acc) { return fma(s, g, acc); }
  __device__ static double shfl_down(double v, int off) { return __shfl_down_sync(0xffffffffu, v, off); }
};
template <> struct VOps<double2> {
  __device__ static double2 zero() { return make_double2(0.0, 0.0); }
  __device__ static double2 one() { return make_double2(1.0, 0.0); }
  __device__ static double2 add(double2 a, double2 b) { return c_add(a, b); }
  __device__ static double2 mul(double2 a, double2 b) { return c_mul(a, b); }
  __device__ static double2 scale(double2 a, double s) { return c_scale(a, s); }
  __device__ static double2 fma_s(double s, double2 g, double2 acc) {
    return make_double2(fma(s, g.x, acc.x), fma(s, g.y, acc.y));
  }
  __device__ static double2 shfl_down(double2 v, int off) {
    return make_double2(__shfl_down_sync(0xffffffffu, v.x, off), __shfl_down_sync(0xffffffffu, v.y, off));
  }
};

// ---------------------------------------------------------------------------
// Integrand families.  Per-axis constants are loaded once per level.
// ---------------------------------------------------------------------------
struct AxisParams {
  double c;    // c_j
  double w;    // w_j (GAUSS, PEAK)
  double ic2;  // 1 / c_j^2 (PEAK)
};

__device__ __forceinline__ AxisParams load_axis(const double *params, int d, int j) {
  AxisParams p;
  p.c = params[j];
  p.w = params[d + j];
  p.ic2 = 1.0 / (p.c * p.c);
  return p;
}

template <int FAM> struct FamTraits { using V = double; };
template <> struct FamTraits<MDI_FAM_OSC> { using V = double2; };

// phi_j(x) in double precision.
template <int FAM> __device__ __forceinline__ typename FamTraits<FAM>::V phi64(double x, const AxisParams &p);
template <> __device__ __forceinline__ double phi64<MDI_FAM_EXP>(double x, const AxisParams &p) { return exp(p.c * x); }
template <> __device__ __forceinline__ double2 phi64<MDI_FAM_OSC>(double x, const AxisParams &p) {
  double s, c;
  sincos(p.c * x, &s, &c);
  return make_double2(c, s);
}
template <> __device__ __forceinline__ double phi64<MDI_FAM_GAUSS>(double x, const AxisParams &p) {
  double t = p.c * (x - p.w);
  return exp(-t * t);
}
template <> __device__ __forceinline__ double phi64<MDI_FAM_PEAK>(double x, const AxisParams &p) {
  double t = x - p.w;
  return 1.0 / fma(t, t, p.ic2);
}

// phi_j(x) evaluated in float (argument rounded to float), returned widened.
template <int FAM> __device__ __forceinline__ typename FamTraits<FAM>::V phi32(double x, const AxisParams &p);
template <> __device__ __forceinline__ double phi32<MDI_FAM_EXP>(double x, const AxisParams &p) {
  return (double)expf((float)p.c * (float)x);
}
template <> __device__ __forceinline__ double2 phi32<MDI_FAM_OSC>(double x, const AxisParams &p) {
  float s, c;
  sincosf((float)p.c * (float)x, &s, &c);
  return make_double2((double)c, (double)s);
}
template <> __device__ __forceinline__ double phi32<MDI_FAM_GAUSS>(double x, const AxisParams &p) {
  float t = (float)p.c * ((float)x - (float)p.w);
  return (double)expf(-t * t);
}
template <> __device__ __forceinline__ double phi32<MDI_FAM_PEAK>(double x, const AxisParams &p) {
  float t = (float)x - (float)p.w;
  return (double)(1.0f / fmaf(t, t, (float)p.ic2));
}

template <int FAM, bool FP32EVAL>
__device__ __forceinline__ typename FamTraits<FAM>::V phi(double x, const AxisParams &p) {
  if constexpr (FP32EVAL) return phi32<FAM>(x, p);
  else return phi64<FAM>(x, p);
}

// Whole integrand from coordinates, for the lattice kernel: f(x) = Re(C prod phi_j).
// EXP/GAUSS accumulate the exponent and take one exp, as in the definitions.

// ---------------------------------------------------------------------------
// Double-float arithmetic on float pairs (hi, lo), |lo| <= ulp(hi)/2.
// Error-free transformations: Knuth's TwoSum, Dekker's Fast2Sum and the
// FMA-based TwoProd; pair addition and multiplication follow Joldes, Muller &
// Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 44 (2017), Algorithms 6 and 12.
// Explicit _rn intrinsics keep the compiler from contracting or reassociating.
// ---------------------------------------------------------------------------
struct df32 {
  float hi, lo;
};

__device__ __forceinline__ df32 df_make(float h, float l) { return df32{h, l}; }
__device__ __forceinline__ df32 two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df32{s, e};
}
__device__ __forceinline__ df32 fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return df32{s, e};
}
__device__ __forceinline__ df32 two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return df32{p, e};
}
__device__ __forceinline__ df32 df_add(df32 x, df32 y) {
  df32 s = two_sum(x.hi, y.hi);
  df32 t = two_sum(x.lo, y.lo);
  float c = __fadd_rn(s.lo, t.hi);
  df32 v = fast_two_sum(s.hi, c);
  float w = __fadd_rn(t.lo, v.lo);
  return fast_two_sum(v.hi, w);
}
__device__ __forceinline__ df32 df_mul(df32 x, df32 y) {
  df32 c = two_prod(x.hi, y.hi);
  float tl0 = __fmul_rn(x.lo, y.lo);
  float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
  float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
  float cl3 = __fadd_rn(c.lo, cl2);
  return fast_two_sum(c.hi, cl3);
}
__device__ __forceinline__ df32 df_from_double(double v) {
  float h = (float)v;
  return df32{h, (float)(v - (double)h)};
}
__device__ __forceinline__ double df_to_double(df32 v) { return (double)v.hi + (double)v.lo; }
__device__ __forceinline__ df32 df_shfl_down(df32 v, int off) {
  return df32{__shfl_down_sync(0xffffffffu, v.hi, off), __shfl_down_sync(0xffffffffu, v.lo, off)};
}
__device__ __forceinline__ df32 df_neg(df32 x) { return df32{-x.hi, -x.lo}; }
// x + y with the error bounded relative to |x| + |y| rather than |x + y|
// (Joldes, Muller & Popescu 2017, Algorithm 5, "sloppy" double-word addition):
// used where only the absolute error of the sum matters.
__device__ __forceinline__ df32 df_add_sloppy(df32 x, df32 y) {
  const df32 s = two_sum(x.hi, y.hi);
  const float v = __fadd_rn(x.lo, y.lo);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, v));
}

// Accumulator for sums of double-float products: Algorithm Dot2 of Ogita, Rump &
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005), extended
// to double-float operands.  The product of the high parts is split exactly
// (TwoProd), the high parts are added with TwoSum, and every low-order part (the
// product errors, the cross terms hi*lo, the TwoSum errors) is collected in one
// float, which is folded in once at the end.  About 12 float operations per term
// instead of about 30 for a renormalised double-float add after each product.
struct DfAcc {
  float s = 0.0f, c = 0.0f;
};
__device__ __forceinline__ void dacc_prod(DfAcc &a, df32 x, df32 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  const float e = __fmaf_rn(x.hi, y.hi, -p);
  const df32 t = two_sum(a.s, p);
  a.s = t.hi;
  // The term's low-order part first, then one addition into the running low sum,
  // so the chain carried from term to term is one add on each of s and c.
  const float lo = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, __fadd_rn(e, t.lo)));
  a.c = __fadd_rn(a.c, lo);
}
__device__ __forceinline__ void dacc_add(DfAcc &a, df32 x) {
  const df32 t = two_sum(a.s, x.hi);
  a.s = t.hi;
  a.c = __fadd_rn(a.c, __fadd_rn(x.lo, t.lo));
}
__device__ __forceinline__ df32 dacc_value(const DfAcc &a) { return two_sum(a.s, a.c); }
// Long per-thread sums run in chunks of kDfFlush steps (a term, or a pass of a
// few terms), each chunk's float-pair accumulator then moving into a double.  The
// pair's compensated sum loses up to about one unit of 2^-48 of the running total
// per term, so runs of thousands of terms (2^32 ghosts, lattices of up to 2^48
// points, 2^22 Korobov terms per thread) are cut short.
constexpr int kDfFlush = 128;
__device__ __forceinline__ void df_flush(DfAcc &acc, double &acc64) {
  acc64 += (double)acc.s + (double)acc.c;
  acc = DfAcc{};
}
// x * f for a double-float x and a float f (Joldes et al. 2017, Algorithm 9 without
// the final renormalisation of the error term).
__device__ __forceinline__ df32 df_mul_f(df32 x, float f) {
  df32 c = two_prod(x.hi, f);
  float cl = __fmaf_rn(x.lo, f, c.lo);
  return fast_two_sum(c.hi, cl);
}
__device__ __forceinline__ df32 df_sqr(df32 x) {
  df32 c = two_prod(x.hi, x.hi);
  float t = __fmul_rn(__fadd_rn(x.hi, x.hi), x.lo);
  return fast_two_sum(c.hi, __fadd_rn(c.lo, t));
}
__device__ __forceinline__ df32 df_from_float(float f) { return df32{f, 0.0f}; }

// exp(x) for a double-float x with -80 <= x <= 87 (below, the result flushes
// towards 0 as the float range does).  Table-driven reduction after P. T. P. Tang,
// "Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15 (1989): x = (256 k + j) ln2/256 + r with
// |r| <= ln2/512, the constant ln2/256 split Cody-Waite style into three floats
// (C1 with 9 significant bits, so n * C1 is exact for |n| < 2^15), then
// exp(r) = 1 + r + r^2/2 + r^3/6 (1 + r/4) with the last term (< 5e-10) in float,
// 2^(j/256) read as a float pair from `tab` (kExpTable entries built by
// exp2_table_entry), and the power 2^k applied exactly.
constexpr int kExpTable = 256;
struct DfExpConsts {
  // ln2/256 = C1 + C2 + C3 (residual 4.5e-23).
  static constexpr float C1 = 0.00270843505859375f;
  static constexpr float C2 = -8.2888453789564664476e-07f;
  static constexpr float C3 = 6.4320116005783627144e-15f;
  static constexpr float INV = 369.32993046757463f;  // 256 / ln2, only used to pick n
};
__device__ __forceinline__ float2 exp2_table_entry(int j) {
  const double v = exp2((double)j / (double)kExpTable);
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}
__device__ __forceinline__ df32 df_exp(df32 x, const float2 *__restrict__ tab) {
  const float n = rintf(x.hi * DfExpConsts::INV);
  // r = x - n ln2/256, accurate to about 2^-50 absolute
  const float t = __fmaf_rn(-n, DfExpConsts::C1, x.hi);  // exact: n*C1 exact, Sterbenz
  df32 r = two_sum(t, x.lo);
  r = df_add_sloppy(r, two_prod(-n, DfExpConsts::C2));  // absolute error ~2^-48 |n C2|
  r = fast_two_sum(r.hi, __fmaf_rn(-n, DfExpConsts::C3, r.lo));
  // exp(r): 1 + r (TwoSum) + r^2/2 (exact product of the high part plus cross term)
  const float h = 0.5f * r.hi;
  const float p2 = __fmul_rn(r.hi, h);
  const float e2 = __fmaf_rn(r.hi, h, -p2);
  const float cross = __fmul_rn(r.hi, r.lo);
  const float t3 = __fmul_rn(__fmul_rn(p2, r.hi), __fmaf_rn(r.hi, 1.0f / 12.0f, 1.0f / 3.0f));
  // |r.hi| <= ln2/512 < 1 and |p2| <= r^2/2 < |s1.hi|: both sums meet FastTwoSum's
  // ordering condition, so their errors are exact with three operations.
  const df32 s1 = fast_two_sum(1.0f, r.hi);
  const df32 s2 = fast_two_sum(s1.hi, p2);
  float lo = __fadd_rn(s1.lo, s2.lo);
  lo = __fadd_rn(lo, r.lo);
  lo = __fadd_rn(lo, __fadd_rn(e2, cross));
  lo = __fadd_rn(lo, t3);
  df32 e = fast_two_sum(s2.hi, lo);
  const int ni = (int)n;
  const int j = ni & (kExpTable - 1), k = ni >> 8;  // floor division for negative n
  const float2 tj = tab[j];
  e = df_mul(e, df32{tj.x, tj.y});
  const float sc = __int_as_float((max(k, -126) + 127) << 23);  // 2^k
  return df32{e.hi * sc, e.lo * sc};
}

// 1/x for a positive double-float x: float reciprocal refined by one
// Newton-Raphson step, y = y0 + y0 (1 - x y0) (quadratic convergence: the
// residual 2^-24 squares to 2^-48).  t = x y0 lies within 2^-22 of 1, so
// 1 - t.hi is exact (Sterbenz), and (1 - t.hi) - t.lo rounds only at 2^-24 of a
// residual that is itself below 2^-22.
__device__ __forceinline__ df32 df_rcp(df32 x) {
  const float y0 = __frcp_rn(x.hi);
  const df32 t = df_mul_f(x, y0);
  const float e = __fsub_rn(__fsub_rn(1.0f, t.hi), t.lo);
  return fast_two_sum(y0, __fmul_rn(y0, e));
}

// ---------------------------------------------------------------------------
// Exact lattice index arithmetic.
// ---------------------------------------------------------------------------
// (x * y) mod n for x, y < n < 2^63 by binary double-and-add: exact, no 128-bit type.
__device__ __forceinline__ uint64_t mulmod_u63(uint64_t x, uint64_t y, uint64_t n) {
  uint64_t r = 0;
  while (y) {
    if (y & 1ull) {
      r += x;
      if (r >= n) r -= n;
    }
    x += x;
    if (x >= n) x -= n;
    y >>= 1;
  }
  return r;
}

// Index run [j0, j1) of thread `tid` out of `nthreads` covering [0, n).
__device__ __forceinline__ void thread_run(uint64_t n, uint64_t tid, uint64_t nthreads, uint64_t &j0,
                                           uint64_t &j1) {
  uint64_t per = n / nthreads, extra = n % nthreads;
  j0 = tid * per + (tid < extra ? tid : extra);
  j1 = j0 + per + (tid < extra ? 1 : 0);
}

// ---------------------------------------------------------------------------
// Reductions with a fixed tree (deterministic).
// ---------------------------------------------------------------------------
template <typename V> __device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
  for (int off = kWarp / 2; off > 0; off >>= 1) v = VOps<V>::add(v, VOps<V>::shfl_down(v, off));
  return v;  // valid in lane 0
}

// Block sum; `scratch` holds blockDim.x / 32 values.  Result valid in thread 0.
template <typename V> __device__ __forceinline__ V block_sum(V v, V *scratch) {
  const int lane = threadIdx.x & (kWarp - 1), warp = threadIdx.x / kWarp;
  const int nwarps = (blockDim.x + kWarp - 1) / kWarp;
  v = warp_sum(v);
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  V r = VOps<V>::zero();
  if (warp == 0) {
    r = lane < nwarps ? scratch[lane] : VOps<V>::zero();
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// Host helpers shared by the .cu translation units.
// ---------------------------------------------------------------------------
void set_cuda_error(cudaError_t e);
inline mdi_status check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return MDI_ECUDA;
  }
  return MDI_OK;
}
int sm_count();

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

}  // namespace mdi
