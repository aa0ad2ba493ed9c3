// slr.cu -- the standard lattice rule (SLR), eq. (1.2) over the rank-1 points of
// eq. (2.1): Q = (1/n) sum_{j<n} f({j z / n}).
//
// Every point is generated and evaluated: this is the paper's baseline method and
// the parity partner of the MDI-LR sweep.  Each thread owns a contiguous run of
// indices j; it forms r_i = j0 z_i mod n once (exact 64-bit double-and-add) and
// then steps r_i <- r_i + z_i (mod n), so every coordinate numerator is an exact
// integer (n < 2^63 keeps r_i + z_i below 2^64).  Coordinates x_i = r_i / n are
// formed in FP64.  Per-thread FP64 partial sums are reduced by a fixed tree into
// one partial per CTA, and a second one-CTA kernel adds the partials in index
// order, so the result is bitwise reproducible.
#include <algorithm>
#include <type_traits>
#include <mutex>

#include "mdi_common.cuh"
#include "mdi_exp2_table.inc"
#include "mdi_fp64.cuh"
#include "mdi_internal.h"

namespace mdi {

constexpr int kSlrMaxD = 256;
constexpr int kSlrThreads = 256;
constexpr int kSlrMinRun = 4;  // minimum indices per thread (amortises the exact set-up of the residues)

struct SlrArgs {
  uint64_t n;
  double inv_n;
  int d;
  int pad;
  uint64_t z[kSlrMaxD];  // reduced mod n
};

// SHIFT: the randomly shifted rule of Section 2.1, x = {j z / n + Delta_r} with the
// shift Delta_r = shifts[r*d .. r*d + d) of replicate r = blockIdx.y; each
// replicate's CTAs write their partials at partials + r * gridDim.x.
//
// FP64 points of the unshifted rule (FAST) keep GB300's FP64 pipe, which bounds
// them, to what the point needs: 1/n is folded into each coordinate's constant
// (the exponential family's argument is sum_i (c_i/n) r_i, the Gaussian's t_i =
// (c_i/n) r_i - c_i w_i), exp is the table-driven exp_tang64 (ten FP64
// operations) and the peak's 1/prod is rcp_nr64 (three) instead of a division.
// The coordinate numerators stay exact integers; only the rounding of the
// argument's terms differs from forming x_i = r_i/n first (within a few units in
// the last place of the argument).
template <int FAM, bool FP32EVAL, int MAXD, bool SHIFT = false>
__global__ void __launch_bounds__(kSlrThreads, MAXD <= 8 ? 2 : 1) slr_kernel(const __grid_constant__ SlrArgs args,
                                                          const double *__restrict__ params,
                                                          double *__restrict__ partials,
                                                          const double *__restrict__ shifts = nullptr) {
  constexpr bool FAST = !FP32EVAL && !SHIFT && FAM != MDI_FAM_OSC;
  __shared__ double s_c[MAXD], s_w[MAXD], s_ic2[MAXD];
  __shared__ double s_dx[SHIFT ? MAXD : 1];
  __shared__ double s_cn[FAST ? MAXD : 1], s_cw[FAST ? MAXD : 1];
  __shared__ double s_exp2d[FAST && FAM != MDI_FAM_PEAK ? kExpTable : 1];
  __shared__ double s_red[kSlrThreads / kWarp];
  constexpr int kUnroll = MAXD <= 32 ? MAXD : 1;  // the wide bucket keeps r[] in local memory
  const int d = args.d;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    s_c[i] = params[i];
    s_w[i] = params[d + i];
    s_ic2[i] = 1.0 / (params[i] * params[i]);
    if constexpr (SHIFT) s_dx[i] = shifts[(size_t)blockIdx.y * d + i];
    if constexpr (FAST) {
      s_cn[i] = params[i] * args.inv_n;
      s_cw[i] = params[i] * params[d + i];
    }
  }
  if constexpr (FAST && FAM != MDI_FAM_PEAK)
    for (int j = threadIdx.x; j < kExpTable; j += blockDim.x) s_exp2d[j] = kExp2TableD[j];
  if constexpr (SHIFT) partials += (size_t)blockIdx.y * gridDim.x;
  __syncthreads();
  // Coordinate i of the current point: r_i / n, shifted and wrapped into [0, 1).
  auto coord = [&](uint64_t ri, int i) -> double {
    double x = (double)ri * args.inv_n;
    if constexpr (SHIFT) {
      x += s_dx[i];
      if (x >= 1.0) x -= 1.0;
    }
    return x;
  };
  const double u2pi = (FAM == MDI_FAM_OSC) ? kTwoPi * params[d] : 0.0;

  const uint64_t n = args.n;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t j0, j1;
  thread_run(n, tid, nthreads, j0, j1);

  uint64_t r[MAXD];
#pragma unroll(kUnroll)
  for (int i = 0; i < MAXD; ++i)
    if (i < d) r[i] = (j0 < j1) ? mulmod_u63(j0, args.z[i], n) : 0;

  double acc = 0.0;
  for (uint64_t j = j0; j < j1; ++j) {
    double f;
    if constexpr (FAST) {
      if constexpr (FAM == MDI_FAM_PEAK) {
        double p = 1.0, den = 1.0;
#pragma unroll(kUnroll)
        for (int i = 0; i < MAXD; ++i) {
          if (i < d) {
            const double t = fma((double)r[i], args.inv_n, -s_w[i]);
            den *= fma(t, t, s_ic2[i]);
            if ((i & 7) == 7) {
              p *= rcp_nr64(den);
              den = 1.0;
            }
          }
        }
        f = p * rcp_nr64(den);
      } else {
        double sarg = 0.0;
#pragma unroll(kUnroll)
        for (int i = 0; i < MAXD; ++i) {
          if (i < d) {
            if constexpr (FAM == MDI_FAM_GAUSS) {
              const double t = fma(s_cn[i], (double)r[i], -s_cw[i]);
              sarg = fma(t, t, sarg);
            } else {
              sarg = fma(s_cn[i], (double)r[i], sarg);
            }
          }
        }
        f = exp_tang64(FAM == MDI_FAM_GAUSS ? -sarg : sarg, s_exp2d);
      }
    } else if constexpr (FAM == MDI_FAM_PEAK) {
      double p = 1.0, den = 1.0;
#pragma unroll(kUnroll)
      for (int i = 0; i < MAXD; ++i) {
        if (i < d) {
          double t = SHIFT ? coord(r[i], i) - s_w[i] : fma((double)r[i], args.inv_n, -s_w[i]);
          den *= fma(t, t, s_ic2[i]);
          if ((i & 7) == 7) { p /= den; den = 1.0; }
        }
      }
      f = p / den;
      if constexpr (FP32EVAL) f = (double)(float)f;
    } else {
      double s = 0.0;
      float sf = 0.0f;
#pragma unroll(kUnroll)
      for (int i = 0; i < MAXD; ++i) {
        if (i < d) {
          double x = coord(r[i], i);
          if constexpr (FAM == MDI_FAM_GAUSS) {
            if constexpr (FP32EVAL) {
              float t = (float)s_c[i] * ((float)x - (float)s_w[i]);
              sf = fmaf(t, t, sf);
            } else {
              double t = s_c[i] * (x - s_w[i]);
              s = fma(t, t, s);
            }
          } else {
            if constexpr (FP32EVAL) sf = fmaf((float)s_c[i], (float)x, sf);
            else s = fma(s_c[i], x, s);
          }
        }
      }
      if constexpr (FAM == MDI_FAM_EXP) f = FP32EVAL ? (double)expf(sf) : exp(s);
      else if constexpr (FAM == MDI_FAM_GAUSS) f = FP32EVAL ? (double)expf(-sf) : exp(-s);
      else f = FP32EVAL ? (double)cosf((float)u2pi + sf) : cos(u2pi + s);
    }
    acc += f;
#pragma unroll(kUnroll)
    for (int i = 0; i < MAXD; ++i) {
      if (i < d) {
        uint64_t v = r[i] + args.z[i];
        r[i] = (v >= n) ? v - n : v;
      }
    }
  }
  double b = block_sum(acc, s_red);
  if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

// DF64 (EXP, GAUSS, PEAK): the same points with the integrand in double-float
// arithmetic on the FP32 pipe.  x_i = r_i / n is formed from the exact integer
// r_i < 2^48 as r = rh 2^24 + rl (each exact in a float): x = rh (2^24/n) + rl (1/n)
// with both constants as float pairs (one product when n <= 2^24).  Sums over the
// coordinates are Dot2 accumulations, exp and 1/x the double-float ones; a point
// whose value would leave the float range (argument of exp beyond 64 in size, or
// a peak product outside 2^(+-100)) is evaluated in FP64 into a separate double
// accumulator.  Each thread's Dot2 sum moves into the double sum every kDfFlush
// points (except the unshifted n <= 2^24 case, at most a few hundred points per
// thread), then the fixed block tree as in slr_kernel.  IDX32 steps the numerators in 32-bit
// integers, half the integer work of the 64-bit steps; it is used for n <= 2^24
// (one-limb coordinates), where it was measured faster (with two-limb
// coordinates it measured slower, so larger n keeps 64-bit steps).
constexpr int kSlrDfMaxLog2N = 48;
// SHIFT: the randomly shifted rule, x = {j z / n + Delta_r} for replicate
// r = blockIdx.y (as slr_kernel): the shift as a float pair is added to the
// coordinate and 1 subtracted when the sum reaches 1 (exact: Sterbenz).
template <int FAM, int MAXD, bool IDX32, bool SHIFT = false>
__global__ void __launch_bounds__(kSlrThreads) slr_df_kernel(const __grid_constant__ SlrArgs args,
                                                             const double *__restrict__ params,
                                                             double *__restrict__ partials,
                                                             const double *__restrict__ shifts = nullptr) {
  __shared__ float2 s_dx[SHIFT ? MAXD : 1];
  __shared__ double s_dxd[SHIFT ? MAXD : 1];
  __shared__ float4 s_cw[MAXD];  // (c.hi, c.lo, w.hi, w.lo)
  __shared__ float2 s_ic[MAXD];  // 1/c^2 (PEAK)
  __shared__ double s_c[MAXD], s_w[MAXD];
  __shared__ float2 s_exp2[kExpTable];
  __shared__ double s_red[kSlrThreads / kWarp];
  constexpr int kUnroll = MAXD <= 32 ? MAXD : 1;
  const int d = args.d;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    const double c = params[i], w = params[d + i];
    const df32 cd = df_from_double(c), wd = df_from_double(w);
    s_cw[i] = make_float4(cd.hi, cd.lo, wd.hi, wd.lo);
    const df32 ic = df_rcp(df_sqr(cd));
    s_ic[i] = make_float2(ic.hi, ic.lo);
    s_c[i] = c;
    s_w[i] = w;
    if constexpr (SHIFT) {
      const double dx = shifts[(size_t)blockIdx.y * d + i];
      const df32 dd = df_from_double(dx);
      s_dx[i] = make_float2(dd.hi, dd.lo);
      s_dxd[i] = dx;
    }
  }
  if constexpr (SHIFT) partials += (size_t)blockIdx.y * gridDim.x;
  for (int j = threadIdx.x; j < kExpTable; j += blockDim.x) s_exp2[j] = kExp2TableGen[j];
  __syncthreads();
  const uint64_t n = args.n;
  const bool one_limb = n <= (1ull << 24);
  const df32 inv_n = df_from_double(args.inv_n), inv_n24 = df_from_double(args.inv_n * 16777216.0);
  using Idx = typename std::conditional<IDX32, uint32_t, uint64_t>::type;
  auto coord0 = [&](Idx ri) -> df32 {
    if (one_limb) return df_mul_f(inv_n, (float)(uint32_t)ri);
    return df_add_sloppy(df_mul_f(inv_n24, (float)(uint32_t)(ri >> 24)), df_mul_f(inv_n, (float)(uint32_t)(ri & 0xFFFFFFu)));
  };
  auto coord = [&](Idx ri, int i) -> df32 {
    df32 x = coord0(ri);
    if constexpr (SHIFT) {
      x = df_add_sloppy(x, df32{s_dx[i].x, s_dx[i].y});
      if (x.hi > 1.0f || (x.hi == 1.0f && x.lo >= 0.0f)) x = df_add_sloppy(x, df32{-1.0f, 0.0f});
    }
    return x;
  };
  // The same coordinate in double for the FP64 fallback.
  auto coord64 = [&](Idx ri, int i) -> double {
    double x = (double)ri * args.inv_n;
    if constexpr (SHIFT) {
      x += s_dxd[i];
      if (x >= 1.0) x -= 1.0;
    }
    return x;
  };
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t j0, j1;
  thread_run(n, tid, nthreads, j0, j1);
  const Idx nn = (Idx)n;
  Idx r[MAXD];
#pragma unroll(kUnroll)
  for (int i = 0; i < MAXD; ++i)
    if (i < d) r[i] = (j0 < j1) ? (Idx)mulmod_u63(j0, args.z[i], n) : 0;

  DfAcc acc;
  double acc64 = 0.0;
  // One point: its value into acc (or acc64), its residues stepped by z.
  auto point = [&]() {
    if constexpr (FAM == MDI_FAM_PEAK) {
      df32 p{1.f, 0.f};
#pragma unroll(kUnroll)
      for (int i = 0; i < MAXD; ++i) {
        if (i < d) {
          const float4 cw = s_cw[i];
          const df32 t = df_add_sloppy(coord(r[i], i), df32{-cw.z, -cw.w});
          p = df_mul(p, df_add_sloppy(df_sqr(t), df32{s_ic[i].x, s_ic[i].y}));
        }
      }
      const float mag = fabsf(p.hi);
      if (mag > 0x1p-100f && mag < 0x1p100f) {
        dacc_add(acc, df_rcp(p));
      } else {
        double q = 1.0;
        for (int i = 0; i < d; ++i) {
          const double t = coord64(r[i], i) - s_w[i];
          q *= 1.0 / (1.0 / (s_c[i] * s_c[i]) + t * t);
        }
        acc64 += q;
      }
    } else {
      DfAcc sa;
#pragma unroll(kUnroll)
      for (int i = 0; i < MAXD; ++i) {
        if (i < d) {
          const float4 cw = s_cw[i];
          const df32 x = coord(r[i], i);
          if constexpr (FAM == MDI_FAM_GAUSS) {
            const df32 t = df_mul(df32{cw.x, cw.y}, df_add_sloppy(x, df32{-cw.z, -cw.w}));
            dacc_prod(sa, t, t);
          } else {
            dacc_prod(sa, df32{cw.x, cw.y}, x);
          }
        }
      }
      df32 arg = dacc_value(sa);
      if constexpr (FAM == MDI_FAM_GAUSS) arg = df_neg(arg);
      if (fabsf(arg.hi) <= 64.0f) {
        dacc_add(acc, df_exp(arg, s_exp2));
      } else {
        double sum = 0.0;
        for (int i = 0; i < d; ++i) {
          const double x = coord64(r[i], i);
          if constexpr (FAM == MDI_FAM_GAUSS) {
            const double t = s_c[i] * (x - s_w[i]);
            sum = fma(t, t, sum);
          } else {
            sum = fma(s_c[i], x, sum);
          }
        }
        acc64 += exp(FAM == MDI_FAM_GAUSS ? -sum : sum);
      }
    }
#pragma unroll(kUnroll)
    for (int i = 0; i < MAXD; ++i) {
      if (i < d) {
        const Idx v = r[i] + (Idx)args.z[i];
        r[i] = (v >= nn) ? v - nn : v;
      }
    }
  };
  if constexpr (IDX32 && !SHIFT) {
    // n <= 2^24 over at least 2 x 256 threads per SM: at most 216 points per thread.
    for (uint64_t j = j0; j < j1; ++j) point();
  } else {
    // Chunks of kDfFlush points, each chunk's float-pair sum then moved into acc64.
    for (uint64_t jc = j0; jc < j1; jc += kDfFlush) {
      const uint64_t je = jc + kDfFlush < j1 ? jc + kDfFlush : j1;
      for (uint64_t j = jc; j < je; ++j) point();
      df_flush(acc, acc64);
    }
  }
  const double b = block_sum((double)acc.s + ((double)acc.c + acc64), s_red);
  if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

// Adds `count` partials in a fixed order and writes scale * sum; CTA r handles the
// partials of replicate r (one CTA without shifts).
__global__ void __launch_bounds__(kSlrThreads) sum_partials_kernel(const double *__restrict__ partials, int count,
                                                                   double inv_count_scale, double *__restrict__ out) {
  __shared__ double s_red[kSlrThreads / kWarp];
  partials += (size_t)blockIdx.x * count;
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += partials[i];
  double b = block_sum(acc, s_red);
  if (threadIdx.x == 0) out[blockIdx.x] = b * inv_count_scale;
}

__global__ void lattice_indices_kernel(const __grid_constant__ SlrArgs args, uint64_t j0, uint64_t count,
                                       uint64_t runs, int64_t *__restrict__ r_out) {
  // Same generator as slr_kernel: run `tid` covers a contiguous slice of [0, count).
  uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= runs) return;
  uint64_t t0, t1;
  thread_run(count, tid, runs, t0, t1);
  const uint64_t n = args.n;
  for (int i = 0; i < args.d; ++i) {
    uint64_t jj = (j0 + t0) % n;
    uint64_t r = mulmod_u63(jj, args.z[i], n);
    for (uint64_t t = t0; t < t1; ++t) {
      r_out[t * (uint64_t)args.d + i] = (int64_t)r;
      uint64_t v = r + args.z[i];
      r = (v >= n) ? v - n : v;
    }
  }
}

// CTAs for n points: runs of at least kSlrMinRun indices, but never fewer threads
// than two CTAs per SM while n allows (the FP64 pipe of every SM is needed for
// small n; runs then shorten down to one index), and at most 8 CTAs per SM.
static int slr_grid(uint64_t n) {
  const uint64_t max_threads = (uint64_t)sm_count() * 8 * kSlrThreads;
  const uint64_t want = (n + kSlrMinRun - 1) / kSlrMinRun;
  const uint64_t floor_threads = std::min<uint64_t>(n, (uint64_t)sm_count() * 2 * kSlrThreads);
  const uint64_t threads = std::min(max_threads, std::max(want, floor_threads));
  return (int)std::max<uint64_t>(1, (threads + kSlrThreads - 1) / kSlrThreads);
}

size_t slr_workspace_bytes(int d, int64_t n) {
  (void)d;
  return align_up(sizeof(double) * (size_t)slr_grid((uint64_t)n));
}

template <int FAM, bool F32, int MAXD>
static void launch_slr(int grid, const SlrArgs &args, const double *params, double *partials, cudaStream_t s) {
  slr_kernel<FAM, F32, MAXD><<<grid, kSlrThreads, 0, s>>>(args, params, partials);
}

template <int FAM, bool F32>
static void launch_slr_d(int grid, const SlrArgs &args, const double *params, double *partials, cudaStream_t s) {
  if (args.d <= 8) launch_slr<FAM, F32, 8>(grid, args, params, partials, s);
  else if (args.d <= 32) launch_slr<FAM, F32, 32>(grid, args, params, partials, s);
  else launch_slr<FAM, F32, kSlrMaxD>(grid, args, params, partials, s);
}

template <int FAM, bool IDX32>
static void launch_slr_df_i(int grid, const SlrArgs &args, const double *params, double *partials, cudaStream_t s) {
  if (args.d <= 8) slr_df_kernel<FAM, 8, IDX32><<<grid, kSlrThreads, 0, s>>>(args, params, partials);
  else if (args.d <= 16) slr_df_kernel<FAM, 16, IDX32><<<grid, kSlrThreads, 0, s>>>(args, params, partials);
  else if (args.d <= 32) slr_df_kernel<FAM, 32, IDX32><<<grid, kSlrThreads, 0, s>>>(args, params, partials);
  else slr_df_kernel<FAM, kSlrMaxD, IDX32><<<grid, kSlrThreads, 0, s>>>(args, params, partials);
}
template <int FAM>
static void launch_slr_df_d(int grid, const SlrArgs &args, const double *params, double *partials, cudaStream_t s) {
  if (args.n <= (1ull << 24)) launch_slr_df_i<FAM, true>(grid, args, params, partials, s);
  else launch_slr_df_i<FAM, false>(grid, args, params, partials, s);
}

// The point sums of one plain-rule launch into `partials` (grid entries).
static void launch_slr_points(int family, int precision, int grid, const SlrArgs &args, const double *params,
                              double *partials, cudaStream_t stream) {
  const bool f32 = precision == MDI_PREC_FP32_EVAL_FP64;
  const bool df = precision == MDI_PREC_DF64 && family != MDI_FAM_OSC;  // OSC evaluates in FP64
  switch (family) {
    case MDI_FAM_EXP:
      df ? launch_slr_df_d<MDI_FAM_EXP>(grid, args, params, partials, stream)
         : f32 ? launch_slr_d<MDI_FAM_EXP, true>(grid, args, params, partials, stream)
               : launch_slr_d<MDI_FAM_EXP, false>(grid, args, params, partials, stream);
      break;
    case MDI_FAM_OSC: f32 ? launch_slr_d<MDI_FAM_OSC, true>(grid, args, params, partials, stream)
                          : launch_slr_d<MDI_FAM_OSC, false>(grid, args, params, partials, stream); break;
    case MDI_FAM_GAUSS:
      df ? launch_slr_df_d<MDI_FAM_GAUSS>(grid, args, params, partials, stream)
         : f32 ? launch_slr_d<MDI_FAM_GAUSS, true>(grid, args, params, partials, stream)
               : launch_slr_d<MDI_FAM_GAUSS, false>(grid, args, params, partials, stream);
      break;
    default:
      df ? launch_slr_df_d<MDI_FAM_PEAK>(grid, args, params, partials, stream)
         : f32 ? launch_slr_d<MDI_FAM_PEAK, true>(grid, args, params, partials, stream)
               : launch_slr_d<MDI_FAM_PEAK, false>(grid, args, params, partials, stream);
      break;
  }
}

// Precision modes of the plain rule: FP64, FP32 evaluation, and DF64 for n <= 2^48.
static mdi_status slr_precision_ok(int precision, int64_t n) {
  if (precision == MDI_PREC_FP64 || precision == MDI_PREC_FP32_EVAL_FP64) return MDI_OK;
  if (precision == MDI_PREC_DF64 && (uint64_t)n <= (1ull << kSlrDfMaxLog2N)) return MDI_OK;
  return MDI_EUNSUPPORTED;
}

mdi_status slr_launch(int family, int d, int64_t n, const int64_t *z, const double *params, int precision,
                      double *out, void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if (d < 1 || d > kSlrMaxD || n < 1 || !z || !params || !out) return MDI_EINVAL;
  if (family < MDI_FAM_EXP || family > MDI_FAM_PEAK) return MDI_EINVAL;
  if (slr_precision_ok(precision, n) != MDI_OK) return MDI_EUNSUPPORTED;
  for (int i = 0; i < d; ++i)
    if (z[i] < 0 || z[i] >= n) return MDI_EINVAL;
  if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < slr_workspace_bytes(d, n)) return MDI_EWORKSPACE;
  SlrArgs args{};
  args.n = (uint64_t)n;
  args.inv_n = 1.0 / (double)n;
  args.d = d;
  for (int i = 0; i < d; ++i) args.z[i] = (uint64_t)z[i];
  const int grid = slr_grid((uint64_t)n);
  double *partials = (double *)workspace;
  launch_slr_points(family, precision, grid, args, params, partials, stream);
  mdi_status st = check_launch();
  if (st != MDI_OK) return st;
  sum_partials_kernel<<<1, kSlrThreads, 0, stream>>>(partials, grid, 1.0 / (double)n, out);
  return check_launch();
}

// Randomly shifted rule: R replicates, one launch (grid.y = R) plus one sum launch.
template <int FAM>
static void launch_slr_shifted(int grid, int R, const SlrArgs &args, const double *params, double *partials,
                               const double *shifts, cudaStream_t s) {
  const dim3 g(grid, R);
  if (args.d <= 8) slr_kernel<FAM, false, 8, true><<<g, kSlrThreads, 0, s>>>(args, params, partials, shifts);
  else if (args.d <= 32) slr_kernel<FAM, false, 32, true><<<g, kSlrThreads, 0, s>>>(args, params, partials, shifts);
  else slr_kernel<FAM, false, kSlrMaxD, true><<<g, kSlrThreads, 0, s>>>(args, params, partials, shifts);
}

static int slr_shifted_grid(uint64_t n, int R) {
  // CTAs per replicate: the R replicates together fill the GPU as one launch over
  // n * R points would (so R = 1 is slr_grid's partition), and none uses more CTAs
  // than a single unshifted launch.
  const double max_threads = (double)sm_count() * 8 * kSlrThreads;
  const double want = std::ceil((double)n * (double)R / kSlrMinRun);
  const double floor_threads = std::min((double)n * (double)R, (double)sm_count() * 2 * kSlrThreads);
  const double threads = std::min(max_threads, std::max(want, floor_threads));
  const int per = (int)std::ceil(threads / (double)R / kSlrThreads);
  return std::max(1, std::min(per, slr_grid(n)));
}

size_t slr_shifted_workspace_bytes(int d, int64_t n, int R) {
  (void)d;
  if (n < 1 || R < 1 || R > 65535) return 0;
  return align_up(sizeof(double) * (size_t)slr_shifted_grid((uint64_t)n, R) * (size_t)R);
}

template <int FAM, bool IDX32>
static void launch_slr_df_shift_i(int grid, int R, const SlrArgs &args, const double *params, double *partials,
                                  const double *shifts, cudaStream_t s) {
  const dim3 g(grid, R);
  if (args.d <= 8) slr_df_kernel<FAM, 8, IDX32, true><<<g, kSlrThreads, 0, s>>>(args, params, partials, shifts);
  else if (args.d <= 16) slr_df_kernel<FAM, 16, IDX32, true><<<g, kSlrThreads, 0, s>>>(args, params, partials, shifts);
  else if (args.d <= 32) slr_df_kernel<FAM, 32, IDX32, true><<<g, kSlrThreads, 0, s>>>(args, params, partials, shifts);
  else slr_df_kernel<FAM, kSlrMaxD, IDX32, true><<<g, kSlrThreads, 0, s>>>(args, params, partials, shifts);
}
template <int FAM>
static void launch_slr_df_shift(int grid, int R, const SlrArgs &args, const double *params, double *partials,
                                const double *shifts, cudaStream_t s) {
  if (args.n <= (1ull << 24)) launch_slr_df_shift_i<FAM, true>(grid, R, args, params, partials, shifts, s);
  else launch_slr_df_shift_i<FAM, false>(grid, R, args, params, partials, shifts, s);
}

mdi_status slr_shifted_launch(int family, int d, int64_t n, const int64_t *z, const double *params,
                              const double *shifts, int R, int precision, double *out, void *workspace,
                              size_t ws_bytes, cudaStream_t stream) {
  if (d < 1 || d > kSlrMaxD || n < 1 || !z || !params || !shifts || !out || R < 1 || R > 65535) return MDI_EINVAL;
  if (family < MDI_FAM_EXP || family > MDI_FAM_PEAK) return MDI_EINVAL;
  if (precision != MDI_PREC_FP64 && !(precision == MDI_PREC_DF64 && (uint64_t)n <= (1ull << kSlrDfMaxLog2N)))
    return MDI_EUNSUPPORTED;
  for (int i = 0; i < d; ++i)
    if (z[i] < 0 || z[i] >= n) return MDI_EINVAL;
  if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < slr_shifted_workspace_bytes(d, n, R))
    return MDI_EWORKSPACE;
  SlrArgs args{};
  args.n = (uint64_t)n;
  args.inv_n = 1.0 / (double)n;
  args.d = d;
  for (int i = 0; i < d; ++i) args.z[i] = (uint64_t)z[i];
  const int grid = slr_shifted_grid((uint64_t)n, R);
  double *partials = (double *)workspace;
  const bool df = precision == MDI_PREC_DF64;  // OSC evaluates in FP64
  switch (family) {
    case MDI_FAM_EXP:
      df ? launch_slr_df_shift<MDI_FAM_EXP>(grid, R, args, params, partials, shifts, stream)
         : launch_slr_shifted<MDI_FAM_EXP>(grid, R, args, params, partials, shifts, stream);
      break;
    case MDI_FAM_OSC: launch_slr_shifted<MDI_FAM_OSC>(grid, R, args, params, partials, shifts, stream); break;
    case MDI_FAM_GAUSS:
      df ? launch_slr_df_shift<MDI_FAM_GAUSS>(grid, R, args, params, partials, shifts, stream)
         : launch_slr_shifted<MDI_FAM_GAUSS>(grid, R, args, params, partials, shifts, stream);
      break;
    default:
      df ? launch_slr_df_shift<MDI_FAM_PEAK>(grid, R, args, params, partials, shifts, stream)
         : launch_slr_shifted<MDI_FAM_PEAK>(grid, R, args, params, partials, shifts, stream);
      break;
  }
  mdi_status st = check_launch();
  if (st != MDI_OK) return st;
  sum_partials_kernel<<<R, kSlrThreads, 0, stream>>>(partials, grid, 1.0 / (double)n, out);
  return check_launch();
}

// Section 2.1's estimate from R shifted replicates: their mean and its standard
// error, sqrt(sum_r (v_r - mean)^2 / (R (R - 1))).  One CTA; each thread sums a
// strided subset in index order and a fixed shared-memory tree adds the threads'
// sums, so the result does not depend on timing.  Two passes (mean, then the
// squared deviations from it) avoid the cancellation of a one-pass variance.
constexpr int kEstThreads = 256;
__device__ double block_tree_sum(double v, double *sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kEstThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}
__global__ void __launch_bounds__(kEstThreads) shifted_estimate_kernel(const double *__restrict__ values, int R,
                                                                       double *__restrict__ mean_se) {
  __shared__ double sh[kEstThreads];
  double acc = 0.0;
  for (int r = threadIdx.x; r < R; r += kEstThreads) acc += values[r];
  const double mean = block_tree_sum(acc, sh) / (double)R;
  double dev = 0.0;
  for (int r = threadIdx.x; r < R; r += kEstThreads) {
    const double e = values[r] - mean;
    dev = fma(e, e, dev);
  }
  const double ss = block_tree_sum(dev, sh);
  if (threadIdx.x == 0) {
    mean_se[0] = mean;
    mean_se[1] = R > 1 ? sqrt(ss / ((double)R * (double)(R - 1))) : 0.0;
  }
}

mdi_status shifted_estimate_launch(const double *values, int R, double *mean_se, cudaStream_t stream) {
  shifted_estimate_kernel<<<1, kEstThreads, 0, stream>>>(values, R, mean_se);
  return check_launch();
}

mdi_status lattice_indices_launch(int d, int64_t n, const int64_t *z, int64_t j0, int64_t count, int64_t *r_out,
                                  cudaStream_t stream) {
  if (d < 1 || d > kSlrMaxD || n < 1 || !z || !r_out || j0 < 0 || count < 1) return MDI_EINVAL;
  SlrArgs args{};
  args.n = (uint64_t)n;
  args.inv_n = 1.0 / (double)n;
  args.d = d;
  for (int i = 0; i < d; ++i) {
    if (z[i] < 0 || z[i] >= n) return MDI_EINVAL;
    args.z[i] = (uint64_t)z[i];
  }
  uint64_t runs = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)count / 4, 65536));
  int blocks = (int)((runs + 255) / 256);
  lattice_indices_kernel<<<blocks, 256, 0, stream>>>(args, (uint64_t)j0, (uint64_t)count, runs, r_out);
  return check_launch();
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the lattice rule (lattice_rule_integrate_noalloc).
//
// Some callers cannot allocate device memory at call time -- for example code
// that runs inside a host application which reserves all GPU memory up front and
// forbids later cudaMalloc, or a plug-in that has no access to the application's
// allocator -- yet still want the plain lattice rule.  For them the per-CTA
// partial sums live in a fixed array compiled into this library, reserved on
// every GPU that loads it until the process exits.  The kernels are the same as
// lattice_rule_integrate's, so the results are the same.
// ---------------------------------------------------------------------------
constexpr int kSlrNoAllocSlots = 4096;  // partial sums: 32 KiB, enough for 512 SMs x 8 CTAs
static __device__ __align__(256) double g_slr_noalloc_partials[kSlrNoAllocSlots];

// Device address of g_slr_noalloc_partials on the current device.  Host code
// must not pass the symbol itself to a kernel (it names a host-side stand-in);
// the address is looked up once per device, with that device current.
static mdi_status noalloc_scratch(double **ptr) {
  static std::mutex mu;
  static double *cache[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return MDI_ECUDA;
  }
  if (dev < 0 || dev >= 64) return MDI_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(mu);
  if (!cache[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_slr_noalloc_partials);
    if (e != cudaSuccess) {
      set_cuda_error(e);
      return MDI_ECUDA;
    }
    cache[dev] = (double *)p;
  }
  *ptr = cache[dev];
  return MDI_OK;
}

mdi_status slr_launch_noalloc(int family, int d, int64_t n, const int64_t *z, const double *params, int precision,
                              double *out, cudaStream_t stream) {
  if (d < 1 || d > kSlrMaxD || n < 1 || !z || !params || !out) return MDI_EINVAL;
  if (family < MDI_FAM_EXP || family > MDI_FAM_PEAK) return MDI_EINVAL;
  if (slr_precision_ok(precision, n) != MDI_OK) return MDI_EUNSUPPORTED;
  for (int i = 0; i < d; ++i)
    if (z[i] < 0 || z[i] >= n) return MDI_EINVAL;
  const int grid = slr_grid((uint64_t)n);
  if (grid > kSlrNoAllocSlots) return MDI_EWORKSPACE;  // more CTAs than the built-in scratch holds
  double *partials = nullptr;
  mdi_status st = noalloc_scratch(&partials);
  if (st != MDI_OK) return st;
  SlrArgs args{};
  args.n = (uint64_t)n;
  args.inv_n = 1.0 / (double)n;
  args.d = d;
  for (int i = 0; i < d; ++i) args.z[i] = (uint64_t)z[i];
  // Every slot the sum reads (0..grid-1) is written by this call's CTAs first, so
  // the array needs no clearing between calls.
  launch_slr_points(family, precision, grid, args, params, partials, stream);
  st = check_launch();
  if (st != MDI_OK) return st;
  sum_partials_kernel<<<1, kSlrThreads, 0, stream>>>(partials, grid, 1.0 / (double)n, out);
  return check_launch();
}


// ---------------------------------------------------------------------------
// Improved lattice rule (Definition 3.3) for the Korobov vector z = (1, a, ..,
// a^(d-1)) mod n.  With M = a^(d-1), the transformed grid of Theorem 3.1 has M
// lines (the digit blocks of the first d-1 axes) of n_d = ceil(n / M) positions
// (eq. 3.5), N = M n_d points, of which n are lattice points.  Indexing every
// grid point by r = n x_d (an integer), the lattice points are r < n and, when
// gcd(a, n) = 1, every r < N occurs exactly once: r = M s + (-n Q mod M) ties the
// last coordinate to the line Q, so Q(r) = -r n^{-1} mod M, and the other
// coordinates follow from the base-a digits q_0, q_1, ... of Q:
//     x_{d-1} = (q_0 + x_d)/a,  x_{d-2} = (q_1 + x_{d-1})/a,  ...
// The ghosts are r = n .. N-1 with x_d = r/n >= 1: each continues the progression
// of its line by one lattice step z/n without reduction mod 1 (the unwrapped
// reading).  The rule is (sum over the n lattice points + sum over the N - n
// ghosts) / N.  Each line's points all have distinct last coordinates, so no MDI
// work is shared: the lattice points run through slr_kernel and the ghosts
// through ghost_kernel, each thread forming Q once and then stepping it by a
// digit-wise subtraction of n^{-1} with borrow.
// ---------------------------------------------------------------------------
constexpr int kGhostMaxD = 64;  // a^(d-1) < 2^62 with a >= 2 bounds d - 1 by 61

struct GhostArgs {
  uint64_t n, count, M, ninv;  // count = N - n ghosts
  double inv_n, inv_a;
  int d, a;
  int ninv_digit[kGhostMaxD];  // base-a digits of n^{-1} mod M, least significant first
};

// Base-a digits of the line Q(r) = -r n^{-1} mod M of grid index r, least
// significant first.
template <int KDIG, int UNROLL>
__device__ __forceinline__ void ghost_digits(const GhostArgs &g, uint64_t r, int (&q)[KDIG]) {
  const uint64_t m = mulmod_u63(r % g.M, g.ninv, g.M);
  uint64_t Q = m ? g.M - m : 0;
#pragma unroll(UNROLL)
  for (int k = 0; k < KDIG; ++k) {
    if (k + 1 < g.d) {
      q[k] = (int)(Q % (uint64_t)g.a);
      Q /= (uint64_t)g.a;
    }
  }
}

// Q(r + 1) = Q(r) - n^{-1} mod M, digit by digit (the borrow out of the top digit
// is the reduction mod M).
template <int KDIG, int UNROLL>
__device__ __forceinline__ void ghost_step(const GhostArgs &g, int (&q)[KDIG]) {
  int borrow = 0;
#pragma unroll(UNROLL)
  for (int k = 0; k < KDIG; ++k) {
    if (k + 1 < g.d) {
      const int v = q[k] - g.ninv_digit[k] - borrow;
      borrow = v < 0;
      q[k] = borrow ? v + g.a : v;
    }
  }
}

// f at the grid point of index r with line digits q, in FP64: x_d = r/n, then
// x_{d-1} = (q_0 + x_d)/a, x_{d-2} = (q_1 + x_{d-1})/a, ...
template <int FAM, int KDIG, int UNROLL>
__device__ __forceinline__ double ghost_value64(const GhostArgs &g, uint64_t r, const int (&q)[KDIG],
                                                const double *s_c, const double *s_w, const double *s_ic2,
                                                double u2pi) {
  const int d = g.d;
  double x = (double)r * g.inv_n;
  if constexpr (FAM == MDI_FAM_PEAK) {
    const double u0 = x - s_w[d - 1];
    double p = 1.0, den = fma(u0, u0, s_ic2[d - 1]);
#pragma unroll(UNROLL)
    for (int k = 1; k <= KDIG; ++k) {
      if (k < d) {
        x = ((double)q[k - 1] + x) * g.inv_a;
        const int i = d - 1 - k;
        const double u = x - s_w[i];
        den *= fma(u, u, s_ic2[i]);
        if ((k & 7) == 7) {
          p /= den;
          den = 1.0;
        }
      }
    }
    return p / den;
  } else {
    auto term = [&](int i, double xi, double sum) {
      if constexpr (FAM == MDI_FAM_GAUSS) {
        const double u = s_c[i] * (xi - s_w[i]);
        return fma(u, u, sum);
      } else {
        return fma(s_c[i], xi, sum);
      }
    };
    double sum = term(d - 1, x, 0.0);
#pragma unroll(UNROLL)
    for (int k = 1; k <= KDIG; ++k) {
      if (k < d) {
        x = ((double)q[k - 1] + x) * g.inv_a;
        sum = term(d - 1 - k, x, sum);
      }
    }
    if constexpr (FAM == MDI_FAM_EXP) return exp(sum);
    else if constexpr (FAM == MDI_FAM_GAUSS) return exp(-sum);
    else return cos(u2pi + sum);
  }
}

template <int FAM, int MAXD>
__global__ void __launch_bounds__(kSlrThreads) ghost_kernel(const __grid_constant__ GhostArgs g,
                                                            const double *__restrict__ params,
                                                            double *__restrict__ partials) {
  __shared__ double s_c[MAXD], s_w[MAXD], s_ic2[MAXD];
  __shared__ double s_red[kSlrThreads / kWarp];
  const int d = g.d;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    s_c[i] = params[i];
    s_w[i] = params[d + i];
    s_ic2[i] = 1.0 / (params[i] * params[i]);
  }
  __syncthreads();
  const double u2pi = (FAM == MDI_FAM_OSC) ? kTwoPi * params[d] : 0.0;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t t0, t1;
  thread_run(g.count, tid, nthreads, t0, t1);
  // Digits of Q; loops run to the bucket's compile-time bound so that they stay
  // in registers for d <= 32.
  constexpr int kDig = MAXD > 1 ? MAXD - 1 : 1;
  constexpr int kUnroll = MAXD <= 32 ? kDig : 1;
  int q[kDig];
  if (t0 < t1) ghost_digits<kDig, kUnroll>(g, g.n + t0, q);
  double acc = 0.0;
  for (uint64_t t = t0; t < t1; ++t) {
    acc += ghost_value64<FAM, kDig, kUnroll>(g, g.n + t, q, s_c, s_w, s_ic2, u2pi);
    ghost_step<kDig, kUnroll>(g, q);
  }
  const double b = block_sum(acc, s_red);
  if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

// The ghosts in double-float (the lattice points' DF64 mode, real families): the
// chain x_d = r/n (r in two 24-bit limbs, r < 2^48), x_{i} = (q + x_{i+1})/a (q < 2^24)
// as float pairs, then the integrand as slr_df_kernel forms it; a ghost whose
// exponent leaves [-64, 64] or whose peak product leaves 2^+-100 is evaluated in
// FP64 from the same digits.
template <int FAM, int MAXD>
__global__ void __launch_bounds__(kSlrThreads) ghost_df_kernel(const __grid_constant__ GhostArgs g,
                                                               const double *__restrict__ params,
                                                               double *__restrict__ partials) {
  __shared__ float4 s_cw[MAXD];  // (c.hi, c.lo, w.hi, w.lo)
  __shared__ float2 s_ic[MAXD];  // 1/c^2 (PEAK)
  __shared__ double s_c[MAXD], s_w[MAXD], s_ic2[MAXD];
  __shared__ float2 s_exp2[kExpTable];
  __shared__ double s_red[kSlrThreads / kWarp];
  const int d = g.d;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    const double c = params[i], w = params[d + i];
    const df32 cd = df_from_double(c), wd = df_from_double(w);
    s_cw[i] = make_float4(cd.hi, cd.lo, wd.hi, wd.lo);
    const df32 ic = df_rcp(df_sqr(cd));
    s_ic[i] = make_float2(ic.hi, ic.lo);
    s_c[i] = c;
    s_w[i] = w;
    s_ic2[i] = 1.0 / (c * c);
  }
  for (int j = threadIdx.x; j < kExpTable; j += blockDim.x) s_exp2[j] = kExp2TableGen[j];
  __syncthreads();
  const df32 inv_n = df_from_double(g.inv_n), inv_n24 = df_from_double(g.inv_n * 16777216.0);
  const df32 inv_a = df_from_double(g.inv_a);
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t t0, t1;
  thread_run(g.count, tid, nthreads, t0, t1);
  constexpr int kDig = MAXD > 1 ? MAXD - 1 : 1;
  constexpr int kUnroll = MAXD <= 32 ? kDig : 1;
  int q[kDig];
  if (t0 < t1) ghost_digits<kDig, kUnroll>(g, g.n + t0, q);
  DfAcc acc;
  double acc64 = 0.0;
  // Chunks of kDfFlush ghosts, each chunk's float-pair sum then moved into acc64.
  for (uint64_t tc = t0; tc < t1; tc += kDfFlush) {
    const uint64_t te = tc + kDfFlush < t1 ? tc + kDfFlush : t1;
    for (uint64_t t = tc; t < te; ++t) {
      const uint64_t r = g.n + t;
      df32 x = df_add_sloppy(df_mul_f(inv_n24, (float)(uint32_t)(r >> 24)),
                             df_mul_f(inv_n, (float)(uint32_t)(r & 0xFFFFFFu)));
      bool ok;
      if constexpr (FAM == MDI_FAM_PEAK) {
        df32 p{1.f, 0.f};
#pragma unroll(kUnroll)
        for (int k = 0; k <= kDig; ++k) {
          if (k < d) {
            if (k > 0) x = df_mul(df_add_sloppy(x, df32{(float)q[k - 1], 0.f}), inv_a);
            const int i = d - 1 - k;
            const float4 cw = s_cw[i];
            const df32 u = df_add_sloppy(x, df32{-cw.z, -cw.w});
            p = df_mul(p, df_add_sloppy(df_sqr(u), df32{s_ic[i].x, s_ic[i].y}));
          }
        }
        const float mag = fabsf(p.hi);
        ok = mag > 0x1p-100f && mag < 0x1p100f;
        if (ok) dacc_add(acc, df_rcp(p));
      } else {
        DfAcc sa;
#pragma unroll(kUnroll)
        for (int k = 0; k <= kDig; ++k) {
          if (k < d) {
            if (k > 0) x = df_mul(df_add_sloppy(x, df32{(float)q[k - 1], 0.f}), inv_a);
            const float4 cw = s_cw[d - 1 - k];
            if constexpr (FAM == MDI_FAM_GAUSS) {
              const df32 u = df_mul(df32{cw.x, cw.y}, df_add_sloppy(x, df32{-cw.z, -cw.w}));
              dacc_prod(sa, u, u);
            } else {
              dacc_prod(sa, df32{cw.x, cw.y}, x);
            }
          }
        }
        df32 arg = dacc_value(sa);
        if constexpr (FAM == MDI_FAM_GAUSS) arg = df_neg(arg);
        ok = fabsf(arg.hi) <= 64.0f;
        if (ok) dacc_add(acc, df_exp(arg, s_exp2));
      }
      if (!ok) acc64 += ghost_value64<FAM, kDig, kUnroll>(g, r, q, s_c, s_w, s_ic2, 0.0);
      ghost_step<kDig, kUnroll>(g, q);
    }
    df_flush(acc, acc64);
  }
  const double b = block_sum((double)acc.s + ((double)acc.c + acc64), s_red);
  if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

// M = a^(d-1), N = M ceil(n / M) and n^{-1} mod M, or false when out of range.
struct ImprovedPlan {
  uint64_t M, N, ninv;
  int grid_lattice, grid_ghost;
};
static bool improved_plan(int d, int64_t n, int64_t a, ImprovedPlan &pl) {
  if (d < 1 || d > kGhostMaxD || n < 1 || a < 1 || n >= (int64_t)(1ull << 62)) return false;
  uint64_t M = 1;
  for (int i = 1; i < d; ++i) {
    if (M > ((1ull << 62) - 1) / (uint64_t)a) return false;
    M *= (uint64_t)a;
  }
  const uint64_t nd = ((uint64_t)n + M - 1) / M;
  if (nd > ((1ull << 62) - 1) / M) return false;
  pl.M = M;
  pl.N = nd * M;
  pl.ninv = 0;
  if (pl.N > (uint64_t)n) {
    // n^{-1} mod M by the extended Euclidean algorithm; needs gcd(n, M) = 1.
    __int128 r0 = (__int128)M, r1 = (__int128)((uint64_t)n % M), s0 = 0, s1 = 1;
    while (r1 != 0) {
      const __int128 qq = r0 / r1, r2 = r0 - qq * r1, s2 = s0 - qq * s1;
      r0 = r1;
      r1 = r2;
      s0 = s1;
      s1 = s2;
    }
    if (r0 != 1) return false;
    __int128 inv = s0 % (__int128)M;
    if (inv < 0) inv += (__int128)M;
    pl.ninv = (uint64_t)inv;
  }
  pl.grid_lattice = slr_grid((uint64_t)n);
  pl.grid_ghost = pl.N > (uint64_t)n ? slr_grid(pl.N - (uint64_t)n) : 0;
  return true;
}

size_t slr_improved_workspace_bytes(int d, int64_t n, int64_t a) {
  ImprovedPlan pl{};
  if (!improved_plan(d, n, a, pl)) return 0;
  return align_up(sizeof(double) * (size_t)(pl.grid_lattice + pl.grid_ghost));
}

template <int FAM, int MAXD>
static void launch_ghost(int grid, const GhostArgs &g, const double *params, double *partials, cudaStream_t s) {
  ghost_kernel<FAM, MAXD><<<grid, kSlrThreads, 0, s>>>(g, params, partials);
}
template <int FAM>
static void launch_ghost_d(int grid, const GhostArgs &g, const double *params, double *partials, cudaStream_t s) {
  if (g.d <= 8) launch_ghost<FAM, 8>(grid, g, params, partials, s);
  else if (g.d <= 32) launch_ghost<FAM, 32>(grid, g, params, partials, s);
  else launch_ghost<FAM, kGhostMaxD>(grid, g, params, partials, s);
}
template <int FAM>
static void launch_ghost_df_d(int grid, const GhostArgs &g, const double *params, double *partials, cudaStream_t s) {
  if (g.d <= 8) ghost_df_kernel<FAM, 8><<<grid, kSlrThreads, 0, s>>>(g, params, partials);
  else if (g.d <= 32) ghost_df_kernel<FAM, 32><<<grid, kSlrThreads, 0, s>>>(g, params, partials);
  else ghost_df_kernel<FAM, kGhostMaxD><<<grid, kSlrThreads, 0, s>>>(g, params, partials);
}

mdi_status slr_improved_launch(int family, int d, int64_t n, int64_t a, const double *params, int precision,
                               double *out, int64_t *n_ghost, void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if (!params || !out) return MDI_EINVAL;
  if (family < MDI_FAM_EXP || family > MDI_FAM_PEAK) return MDI_EINVAL;
  ImprovedPlan pl{};
  if (!improved_plan(d, n, a, pl)) return MDI_EINVAL;
  if (slr_precision_ok(precision, n) != MDI_OK) return MDI_EUNSUPPORTED;
  if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < slr_improved_workspace_bytes(d, n, a))
    return MDI_EWORKSPACE;
  SlrArgs args{};
  args.n = (uint64_t)n;
  args.inv_n = 1.0 / (double)n;
  args.d = d;
  uint64_t zi = 1 % (uint64_t)n;
  for (int i = 0; i < d; ++i) {
    args.z[i] = zi;
    zi = (uint64_t)(((unsigned __int128)zi * (uint64_t)a) % (uint64_t)n);
  }
  double *partials = (double *)workspace;
  // The lattice points in the requested arithmetic; the ghosts below in DF64 or FP64.
  launch_slr_points(family, precision, pl.grid_lattice, args, params, partials, stream);
  mdi_status st = check_launch();
  if (st != MDI_OK) return st;
  if (pl.grid_ghost > 0) {
    GhostArgs g{};
    g.n = (uint64_t)n;
    g.count = pl.N - (uint64_t)n;
    g.M = pl.M;
    g.ninv = pl.ninv;
    g.inv_n = 1.0 / (double)n;
    g.inv_a = 1.0 / (double)a;
    g.d = d;
    g.a = (int)a;
    uint64_t v = pl.ninv;
    for (int k = 0; k + 1 < d; ++k) {
      g.ninv_digit[k] = (int)(v % (uint64_t)a);
      v /= (uint64_t)a;
    }
    double *gp = partials + pl.grid_lattice;
    // DF64 ghosts where their coordinates fit float pairs exactly enough: grid
    // indices below 2^48 (two 24-bit limbs) and line digits below 2^24.
    const bool df = precision == MDI_PREC_DF64 && family != MDI_FAM_OSC && pl.N <= (1ull << 48) &&
                    (uint64_t)a <= (1ull << 24);
    switch (family) {
      case MDI_FAM_EXP:
        df ? launch_ghost_df_d<MDI_FAM_EXP>(pl.grid_ghost, g, params, gp, stream)
           : launch_ghost_d<MDI_FAM_EXP>(pl.grid_ghost, g, params, gp, stream);
        break;
      case MDI_FAM_OSC: launch_ghost_d<MDI_FAM_OSC>(pl.grid_ghost, g, params, gp, stream); break;
      case MDI_FAM_GAUSS:
        df ? launch_ghost_df_d<MDI_FAM_GAUSS>(pl.grid_ghost, g, params, gp, stream)
           : launch_ghost_d<MDI_FAM_GAUSS>(pl.grid_ghost, g, params, gp, stream);
        break;
      default:
        df ? launch_ghost_df_d<MDI_FAM_PEAK>(pl.grid_ghost, g, params, gp, stream)
           : launch_ghost_d<MDI_FAM_PEAK>(pl.grid_ghost, g, params, gp, stream);
        break;
    }
    if ((st = check_launch()) != MDI_OK) return st;
  }
  sum_partials_kernel<<<1, kSlrThreads, 0, stream>>>(partials, pl.grid_lattice + pl.grid_ghost, 1.0 / (double)pl.N,
                                                      out);
  if (n_ghost) *n_ghost = (int64_t)(pl.N - (uint64_t)n);
  return check_launch();
}
}  // namespace mdi
