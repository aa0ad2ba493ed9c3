// mdi_fp64.cuh -- FP64 exp and reciprocal for kernels bound by GB300's FP64 pipe
// (2 DFMA lanes per SM per clock): fewer FP64 instructions than the general math
// library routines, within one unit in the last place of them (tests hold them to
// CUDA's exp and IEEE division through mdi_debug_fp64_phi), and without calls,
// which would cost the calling kernels registers.
#pragma once

#include "mdi_common.cuh"
#include "mdi_exp64_consts.inc"

namespace mdi {

// exp(x) in FP64 by a table-driven reduction (P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point arithmetic",
// ACM TOMS 15, 1989): x = (256 k + j) ln2/256 + r with |r| <= ln2/512, n = 256 k + j
// picked by the round-to-integer of adding 1.5 2^52 (n lands in the low word);
// ln2/256 = L1 + L2 with n L1 exact, so r = (x - n L1) - n L2 has one rounding;
// exp(r) - 1 = r + r^2 (1/2 + r (1/6 + r (1/24 + r/120))) (the next Taylor term
// is below 2^-66 relative); the result is 2^(j/256) (1 + (exp(r) - 1)) with the
// table entry read from `T` and 2^k put into its exponent field by an integer add.
// Ten FP64 operations.  Off the hot path (decided on the integer high word, so no
// FP64 compare): |x| >= 745.15 gives 0 or +inf (exp(-745.14) already rounds to
// 0) and NaN stays NaN, selected at the end rather than returned early; results
// outside the normal range apply 2^k as two normal factors.  No call into the
// math library and no early return: either made ptxas give the sweep kernel
// half its registers, with spills.
__device__ __forceinline__ double exp_tang64(double x, const double *__restrict__ T) {
  const int hx = __double2hiint(x), ax = hx & 0x7FFFFFFF;
  const bool big = ax >= 0x40874933;  // |x| >= 745.15, inf or NaN: result selected below
  const double xs = big ? 0.0 : x;
  const double shifted = fma(xs, kExp64Inv, 0x1.8p52);
  const int n = __double2loint(shifted);
  const double nd = shifted - 0x1.8p52;
  const double r = fma(-nd, kExp64L2, fma(-nd, kExp64L1, xs));
  const double p = fma(r, fma(r, fma(r, 1.0 / 120.0, 1.0 / 24.0), 1.0 / 6.0), 0.5);
  const double em1 = fma(r * r, p, r);
  const int k = n >> 8;  // floor(n / 256), -1076 <= k <= 1075
  const double tj = T[n & (kExpTable - 1)];
  double res;
  if (k >= -1021 && k <= 1023) {  // 2^k tj normal
    const double t = __longlong_as_double(__double_as_longlong(tj) + ((long long)k << 52));
    res = fma(t, em1, t);
  } else {
    const int h = k / 2;  // both 2^h and 2^(k-h) are normal: underflow or overflow
    res = fma(tj, em1, tj) * __longlong_as_double((long long)(h + 1023) << 52) *  // happens in the last product
          __longlong_as_double((long long)(k - h + 1023) << 52);
  }
  if (big) {
    const bool nan = ax > 0x7FF00000 || (ax == 0x7FF00000 && __double2loint(x) != 0);
    res = nan ? x : (hx < 0 ? 0.0 : __longlong_as_double(0x7FF0000000000000ll));
  }
  return res;
}

// 1/D for D > 0 in FP64: a float seed from D's leading 20 fraction bits (integer
// operations build the float and bring the seed back), the hardware's
// approximate float reciprocal, and one cubic Newton-Raphson step
// y = y0 (1 + e + e^2), e = 1 - D y0: the seed's relative error (below 2^-19)
// cubes to below 2^-57.  Three FP64 operations.  D outside [2^-120, 2^120] is first
// brought to [1, 2) by an exact power of two (its exponent field), and the result
// scaled back the same way (as two normal factors); D = 0, subnormal, infinite
// or NaN follow IEEE division's results (+inf, a huge value or +inf, 0, NaN).  No
// call into the math library (see exp_tang64).
__device__ __forceinline__ double rcp_nr64_core(double D, int e) {
  const int hi = __double2hiint(D);
  const float f = __int_as_float(((e + 127) << 23) | ((hi & 0xFFFFF) << 3));
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(f));
  const int yb = __float_as_int(yf);
  const double y0 = __hiloint2double(((((yb >> 23) & 0xFF) - 127 + 1023) << 20) | ((yb & 0x7FFFFF) >> 3),
                                     (yb & 7) << 29);
  const double er = fma(-D, y0, 1.0);
  return fma(y0, fma(er, er, er), y0);
}
__device__ __forceinline__ double rcp_nr64(double D) {
  const int hi = __double2hiint(D);
  int e = ((hi >> 20) & 0x7FF) - 1023;
  if (e >= -120 && e <= 120) return rcp_nr64_core(D, e);
  if (e == 1024) return D != D ? D : 0.0;  // inf -> 0, NaN -> NaN
  double post = 1.0;
  if (e == -1023) {  // zero or subnormal
    if (D == 0.0) return __longlong_as_double(0x7FF0000000000000ll);
    D *= 0x1p600;     // exact, now normal
    post = 0x1p600;
    e = ((__double2hiint(D) >> 20) & 0x7FF) - 1023;
  }
  // D = m 2^e with m in [1, 2): 1/D = (1/m) 2^-e
  const double m = __longlong_as_double((__double_as_longlong(D) & 0x800FFFFFFFFFFFFFll) | (1023ll << 52));
  const int h = -e / 2;
  return rcp_nr64_core(m, 0) * __longlong_as_double((long long)(h + 1023) << 52) *
         __longlong_as_double((long long)(-e - h + 1023) << 52) * post;
}

}  // namespace mdi
