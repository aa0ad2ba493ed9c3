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
