// lattice_search.cu -- generating-vector construction on the GPU (Section 2.2).
//
// Korobov search (Example 2): for every candidate a the criterion of eq. (2.4),
//     P_alpha(z(a)) = -1 + (1/n) sum_{k<n} prod_{j<d} (1 + C_alpha B_alpha({k a^j / n})),
// C_alpha = (-1)^(alpha/2+1) (2 pi)^alpha / alpha!, alpha = 2 or 4.
// CBC (Example 3): z_1 = 1 and, component by component, the z_s minimising the
// squared shift-averaged worst-case error of eq. (2.12) with product weights,
//     -prod_{j<=s} (1 + gamma_j beta) + (1/n) sum_k prod_{j<=s} (1 + gamma_j [B_2({k z_j/n}) + beta]).
//
// GB300 mapping.  Both are sums over k of per-k products, for every candidate:
// one CTA per candidate, each thread a run of consecutive k whose residues
// k z_j mod n are exact integers stepped by z_j (no division per point), FP64
// arithmetic, a fixed-tree block sum.  Even Bernoulli polynomials satisfy
// B(1 - x) = B(x), so the terms of k and n - k are equal: k runs over 1..(n-1)/2,
// doubled, plus k = 0 and (n even) k = n/2.  CBC keeps the running products
// p(k) = prod_{j<s} (...) of the components chosen so far in device memory (for
// k <= n/2, by the same symmetry) and searches z <= n/2 (E^2 of n - z equals that of
// z); each component is four launches -- its factor table, the candidates, a
// deterministic argmin (smallest z among equal values), the update of p -- with no
// host round trip.
//
// Factor tables (n <= 2^24).  A term's factor depends only on its residue r, and
// r and n - r share it, so T[r] = 1 + C B(r/n) (Korobov) or 1 + gamma_s (B_2(r/n) +
// beta) (CBC component s) for r <= n/2 is formed once, as a float pair, and every
// term becomes one table lookup and a double-float multiply on the FP32 pipe,
// accumulated with Dot2-style compensated sums; the running CBC products are
// float pairs too.  In these kernels thread t of B takes k = 1 + t, 1 + t + B, ...
// (residues stepped by B z_j mod n in 32 bits), so that a warp's loads of the
// first factor (z_1 = 1) and of p(k) fall on neighbouring entries.  Korobov
// searches with larger n (or d > 16) use the direct FP64 kernel; CBC is limited
// to n <= 2^24 (its work grows as d n^2 / 4).
#include <algorithm>
#include <cmath>

#include "mdi_common.cuh"
#include "mdi_internal.h"

namespace mdi {

constexpr int kSearchThreads = 256;
constexpr int kArgminThreads = 1024;
constexpr double kPi = 3.141592653589793238462643383279;

__device__ __forceinline__ uint64_t gcd_u64(uint64_t x, uint64_t y) {
  while (y) {
    const uint64_t t = x % y;
    x = y;
    y = t;
  }
  return x;
}

// B_alpha(x) for x in [0, 1): B_2 = y + 1/6, B_4 = y^2 - 1/30 with y = x (x - 1).
template <int ALPHA> __device__ __forceinline__ double bernoulli_even(double x) {
  const double y = x * (x - 1.0);
  if constexpr (ALPHA == 2) return y + 1.0 / 6.0;
  else return fma(y, y, -1.0 / 30.0);
}
template <int ALPHA> __host__ __device__ constexpr double p_alpha_coef() {
  return ALPHA == 2 ? 2.0 * kPi * kPi : -(2.0 * kPi) * (2.0 * kPi) * (2.0 * kPi) * (2.0 * kPi) / 24.0;
}

// ---------------------------------------------------------------------------
// Korobov criterion: values[t] = P_alpha(z(a_first + t)).
// ---------------------------------------------------------------------------
template <int ALPHA, int MAXD>
__global__ void __launch_bounds__(kSearchThreads, 4) korobov_criterion_kernel(int d, uint64_t n, uint64_t a_first,
                                                                           uint64_t count, double *__restrict__ values) {
  __shared__ uint64_t s_z[MAXD];
  __shared__ double s_red[kSearchThreads / kWarp];
  __shared__ int s_ok;
  constexpr int kUnroll = MAXD <= 16 ? MAXD : 1;  // the wide bucket keeps r[] in local memory
  constexpr double C = p_alpha_coef<ALPHA>();
  const double inv_n = 1.0 / (double)n;
  const uint64_t h = (n - 1) / 2;  // k = 1..h, each standing for k and n - k
  for (uint64_t t = blockIdx.x; t < count; t += gridDim.x) {
    const uint64_t a = a_first + t;
    if (threadIdx.x == 0) {
      const bool ok = a >= 1 && a < n && gcd_u64(a, n) == 1;
      if (ok) {
        uint64_t v = 1 % n;
        for (int j = 0; j < d; ++j) {
          s_z[j] = v;
          v = mulmod_u63(v, a, n);
        }
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) {
      if (threadIdx.x == 0) values[t] = INFINITY;
      __syncthreads();
      continue;
    }
    uint64_t k0, k1;
    thread_run(h, threadIdx.x, blockDim.x, k0, k1);
    k0 += 1;
    k1 += 1;
    uint64_t r[MAXD];
#pragma unroll(kUnroll)
    for (int j = 0; j < MAXD; ++j)
      if (j < d) r[j] = (k0 < k1) ? mulmod_u63(k0 % n, s_z[j], n) : 0;
    double acc = 0.0;
    for (uint64_t k = k0; k < k1; ++k) {
      double prod = 1.0;
#pragma unroll(kUnroll)
      for (int j = 0; j < MAXD; ++j) {
        if (j < d) {
          prod *= fma(C, bernoulli_even<ALPHA>((double)r[j] * inv_n), 1.0);
          r[j] += s_z[j];
          if (r[j] >= n) r[j] -= n;
        }
      }
      acc += prod;
    }
    acc = block_sum(acc, s_red);
    if (threadIdx.x == 0) {
      double p0 = 1.0, pm = 1.0;
      const double f0 = fma(C, bernoulli_even<ALPHA>(0.0), 1.0);
      for (int j = 0; j < d; ++j) {
        p0 *= f0;
        // k = n/2: (n/2) z_j mod n is 0 or n/2
        pm *= fma(C, bernoulli_even<ALPHA>((s_z[j] & 1ull) ? 0.5 : 0.0), 1.0);
      }
      const double S = p0 + 2.0 * acc + ((n % 2 == 0 && n > 1) ? pm : 0.0);
      values[t] = -1.0 + S * inv_n;
    }
    __syncthreads();
  }
}

// One CTA: the smallest value and the first index attaining it (+inf everywhere:
// index = count).  Fixed reduction tree, so the choice is deterministic.
__device__ __forceinline__ void argmin_block(const double *__restrict__ values, uint64_t count, double &best_v,
                                             uint64_t &best_i) {
  __shared__ double s_v[kArgminThreads];
  __shared__ uint64_t s_i[kArgminThreads];
  double v = INFINITY;
  uint64_t i = count;
  for (uint64_t t = threadIdx.x; t < count; t += blockDim.x) {
    const double x = values[t];
    if (x < v) {  // strided scan: the first hit of each thread is its smallest index
      v = x;
      i = t;
    }
  }
  s_v[threadIdx.x] = v;
  s_i[threadIdx.x] = i;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      const double ov = s_v[threadIdx.x + s];
      const uint64_t oi = s_i[threadIdx.x + s];
      if (ov < s_v[threadIdx.x] || (ov == s_v[threadIdx.x] && oi < s_i[threadIdx.x])) {
        s_v[threadIdx.x] = ov;
        s_i[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  best_v = s_v[0];
  best_i = s_i[0];
}

__global__ void __launch_bounds__(kArgminThreads) korobov_argmin_kernel(const double *__restrict__ values,
                                                                        uint64_t count, uint64_t a_first,
                                                                        int64_t *__restrict__ best_a) {
  double v;
  uint64_t i;
  argmin_block(values, count, v, i);
  if (threadIdx.x == 0) *best_a = (i < count && v < INFINITY) ? (int64_t)(a_first + i) : 0;
}

// ---------------------------------------------------------------------------
// CBC with product weights: the factor of a residue r for component s.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double cbc_factor(double g, double beta, uint64_t r, double inv_n) {
  return fma(g, bernoulli_even<2>((double)r * inv_n) + beta, 1.0);
}

__global__ void __launch_bounds__(kArgminThreads) cbc_select_kernel(int s, const double *__restrict__ vals,
                                                                    uint64_t count, uint64_t z_first,
                                                                    int64_t *__restrict__ z, double *__restrict__ e2) {
  double v;
  uint64_t i;
  argmin_block(vals, count, v, i);
  if (threadIdx.x == 0) {
    z[s] = (i < count) ? (int64_t)(z_first + i) : 0;
    e2[s] = v;
  }
}


// ---------------------------------------------------------------------------
// Factor-table kernels (double-float)
// ---------------------------------------------------------------------------
constexpr uint64_t kTableMaxN = 1ull << 24;

__device__ __forceinline__ float2 split_f2(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}
__device__ __forceinline__ uint64_t fold(uint64_t r, uint64_t n) { return r <= n - r ? r : n - r; }

template <int ALPHA>
__global__ void korobov_table_kernel(uint64_t n, float2 *__restrict__ T) {
  constexpr double C = p_alpha_coef<ALPHA>();
  const double inv_n = 1.0 / (double)n;
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= n / 2; r += (uint64_t)gridDim.x * blockDim.x)
    T[r] = split_f2(fma(C, bernoulli_even<ALPHA>((double)r * inv_n), 1.0));
}

template <int ALPHA, int MAXD>
__global__ void __launch_bounds__(kSearchThreads) korobov_table_criterion_kernel(int d, uint64_t n, uint64_t a_first,
                                                                                 uint64_t count,
                                                                                 const float2 *__restrict__ T,
                                                                                 double *__restrict__ values) {
  __shared__ uint64_t s_z[MAXD];
  __shared__ double s_red[kSearchThreads / kWarp];
  __shared__ int s_ok;
  constexpr int kUnroll = MAXD <= 16 ? MAXD : 1;
  constexpr double C = p_alpha_coef<ALPHA>();
  const uint64_t h = (n - 1) / 2;
  for (uint64_t t = blockIdx.x; t < count; t += gridDim.x) {
    const uint64_t a = a_first + t;
    if (threadIdx.x == 0) {
      const bool ok = a >= 1 && a < n && gcd_u64(a, n) == 1;
      if (ok) {
        uint64_t v = 1 % n;
        for (int j = 0; j < d; ++j) {
          s_z[j] = v;
          v = mulmod_u63(v, a, n);
        }
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) {
      if (threadIdx.x == 0) values[t] = INFINITY;
      __syncthreads();
      continue;
    }
    // Thread t takes k = 1 + t, 1 + t + B, ... (B threads): the lanes of a warp read
    // neighbouring entries for the first factor (z_1 = 1).  n <= 2^24 here, so
    // residues, steps and folds fit 32 bits (r + step < 2^25).
    const uint32_t n32 = (uint32_t)n, B = blockDim.x, h32 = (uint32_t)h;
    uint32_t r[MAXD], step[MAXD];
#pragma unroll(kUnroll)
    for (int j = 0; j < MAXD; ++j)
      if (j < d) {
        r[j] = (uint32_t)(((uint64_t)(1 + threadIdx.x) * s_z[j]) % n);
        step[j] = (uint32_t)(((uint64_t)B * s_z[j]) % n);
      }
    // The term of one k: the product of its d factors; steps the residues to k + B.
    auto term = [&]() -> df32 {
      const float2 f0 = T[r[0] <= n32 - r[0] ? r[0] : n32 - r[0]];
      df32 prod{f0.x, f0.y};
      r[0] += step[0];
      if (r[0] >= n32) r[0] -= n32;
#pragma unroll(kUnroll)
      for (int j = 1; j < MAXD; ++j) {
        if (j < d) {
          const float2 f = T[r[j] <= n32 - r[j] ? r[j] : n32 - r[j]];
          prod = df_mul(prod, df32{f.x, f.y});
          r[j] += step[j];
          if (r[j] >= n32) r[j] -= n32;
        }
      }
      return prod;
    };
    DfAcc acc;
    double acc64 = 0.0;
    uint32_t k = 1 + threadIdx.x;
    // Two terms per pass (twice the lookups in flight), added in the order of k;
    // chunks of kDfFlush passes, each chunk's float-pair sum then moved into acc64.
    while (k + B <= h32) {
      for (int c = 0; c < kDfFlush && k + B <= h32; ++c, k += 2 * B) {
        const df32 pa = term();
        const df32 pb = term();
        dacc_add(acc, pa);
        dacc_add(acc, pb);
      }
      df_flush(acc, acc64);
    }
    if (k <= h32) dacc_add(acc, term());
    const double tot = block_sum((double)acc.s + ((double)acc.c + acc64), s_red);
    if (threadIdx.x == 0) {
      double p0 = 1.0, pm = 1.0;
      const double f0 = fma(C, bernoulli_even<ALPHA>(0.0), 1.0);
      for (int j = 0; j < d; ++j) {
        p0 *= f0;
        pm *= fma(C, bernoulli_even<ALPHA>((s_z[j] & 1ull) ? 0.5 : 0.0), 1.0);
      }
      const double S = p0 + 2.0 * tot + ((n % 2 == 0 && n > 1) ? pm : 0.0);
      values[t] = -1.0 + S / (double)n;
    }
    __syncthreads();
  }
}

// CBC with factor tables: T[r] = 1 + gamma_s (B_2(r/n) + beta) for component s; the
// running products p(k) (k <= n/2) as float pairs.
__global__ void cbc_df_init_kernel(uint64_t half, float2 *__restrict__ p, double *__restrict__ pref) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= half; k += (uint64_t)gridDim.x * blockDim.x)
    p[k] = make_float2(1.f, 0.f);
  if (blockIdx.x == 0 && threadIdx.x == 0) pref[0] = 1.0;
}

__global__ void cbc_table_kernel(int s, uint64_t n, const double *__restrict__ gamma, double beta,
                                 float2 *__restrict__ T) {
  const double inv_n = 1.0 / (double)n, g = gamma[s];
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= n / 2; r += (uint64_t)gridDim.x * blockDim.x)
    T[r] = split_f2(cbc_factor(g, beta, r, inv_n));
}

__global__ void __launch_bounds__(kSearchThreads) cbc_df_candidates_kernel(int s, uint64_t n,
                                                                           const double *__restrict__ gamma,
                                                                           double beta, const float2 *__restrict__ p,
                                                                           const float2 *__restrict__ T,
                                                                           const double *__restrict__ pref,
                                                                           uint64_t z_first, uint64_t count,
                                                                           double *__restrict__ vals) {
  __shared__ double s_red[kSearchThreads / kWarp];
  const uint64_t h = (n - 1) / 2;
  for (uint64_t t = blockIdx.x; t < count; t += gridDim.x) {
    const uint64_t z = z_first + t;
    if (gcd_u64(z, n) != 1) {  // uniform across the CTA
      if (threadIdx.x == 0) vals[t] = INFINITY;
      continue;
    }
    // Thread t takes k = 1 + t, 1 + t + B, ... (B threads): the lanes of a warp read
    // neighbouring p[k].  n <= 2^24 here, so the residue, its step and fold fit
    // 32 bits (r + step < 2^25).
    const uint32_t n32 = (uint32_t)n, B = blockDim.x, h32 = (uint32_t)h;
    const uint32_t step = (uint32_t)(((uint64_t)B * z) % n);
    uint32_t r = (uint32_t)(((uint64_t)(1 + threadIdx.x) * z) % n);
    auto factor = [&]() -> float2 {
      const float2 f = T[r <= n32 - r ? r : n32 - r];
      r += step;
      if (r >= n32) r -= n32;
      return f;
    };
    DfAcc acc;
    double acc64 = 0.0;
    uint32_t k = 1 + threadIdx.x;
    // Four terms per pass (four lookups in flight), accumulated in the order of k;
    // chunks of kDfFlush passes, each chunk's float-pair sum then moved into acc64.
    while (k + 3 * B <= h32) {
      for (int c = 0; c < kDfFlush && k + 3 * B <= h32; ++c, k += 4 * B) {
        const float2 f0 = factor(), f1 = factor(), f2 = factor(), f3 = factor();
        const float2 p0 = p[k], p1 = p[k + B], p2 = p[k + 2 * B], p3 = p[k + 3 * B];
        dacc_prod(acc, df32{p0.x, p0.y}, df32{f0.x, f0.y});
        dacc_prod(acc, df32{p1.x, p1.y}, df32{f1.x, f1.y});
        dacc_prod(acc, df32{p2.x, p2.y}, df32{f2.x, f2.y});
        dacc_prod(acc, df32{p3.x, p3.y}, df32{f3.x, f3.y});
      }
      df_flush(acc, acc64);
    }
    for (; k <= h32; k += B) {
      const float2 pk = p[k], f = factor();
      dacc_prod(acc, df32{pk.x, pk.y}, df32{f.x, f.y});
    }
    const double tot = block_sum((double)acc.s + ((double)acc.c + acc64), s_red);
    if (threadIdx.x == 0) {
      const double inv_n = 1.0 / (double)n, g = gamma[s];
      const float2 p0 = p[0];
      double S = ((double)p0.x + (double)p0.y) * cbc_factor(g, beta, 0, inv_n) +
                 2.0 * tot;
      if (n % 2 == 0 && n > 1) {
        const float2 pm = p[n / 2];
        S += ((double)pm.x + (double)pm.y) * cbc_factor(g, beta, (z & 1ull) ? n / 2 : 0, inv_n);
      }
      vals[t] = -pref[0] * fma(g, beta, 1.0) + S * inv_n;
    }
    __syncthreads();
  }
}

__global__ void cbc_df_update_kernel(int s, uint64_t n, const double *__restrict__ gamma, double beta,
                                     const int64_t *__restrict__ z, const float2 *__restrict__ T,
                                     float2 *__restrict__ p, double *__restrict__ pref) {
  const uint64_t half = n / 2, zs = (uint64_t)z[s];
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= half; k += (uint64_t)gridDim.x * blockDim.x) {
    const float2 pk = p[k], f = T[fold((k * zs) % n, n)];
    const df32 v = df_mul(df32{pk.x, pk.y}, df32{f.x, f.y});
    p[k] = make_float2(v.hi, v.lo);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) pref[0] *= fma(gamma[s], beta, 1.0);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <int ALPHA>
static mdi_status korobov_dispatch(int d, uint64_t n, uint64_t a_first, uint64_t count, double *values,
                                   cudaStream_t stream) {
  const int grid = (int)std::min<uint64_t>(count, (uint64_t)sm_count() * 16);
  if (d <= 8) korobov_criterion_kernel<ALPHA, 8><<<grid, kSearchThreads, 0, stream>>>(d, n, a_first, count, values);
  else if (d <= 16)
    korobov_criterion_kernel<ALPHA, 16><<<grid, kSearchThreads, 0, stream>>>(d, n, a_first, count, values);
  else korobov_criterion_kernel<ALPHA, 256><<<grid, kSearchThreads, 0, stream>>>(d, n, a_first, count, values);
  return check_launch();
}

size_t korobov_workspace_bytes(int64_t n) {
  if (n < 1) return 0;
  return ((uint64_t)n <= kTableMaxN) ? align_up(sizeof(float2) * (size_t)(n / 2 + 1)) : kAlign;
}

mdi_status korobov_search_launch(int alpha, int d, int64_t n, int64_t a_first, int64_t count, double *values,
                                 int64_t *best_a, void *workspace, size_t ws_bytes, cudaStream_t stream) {
  if ((alpha != 2 && alpha != 4) || d < 1 || d > 256 || n < 1 || n > (INT64_C(1) << 62) || a_first < 0 ||
      count < 1 || !values || !best_a)
    return MDI_EINVAL;
  if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < korobov_workspace_bytes(n)) return MDI_EWORKSPACE;
  const uint64_t un = (uint64_t)n, ua = (uint64_t)a_first, uc = (uint64_t)count;
  mdi_status st;
  if (un <= kTableMaxN && d <= 16) {
    float2 *T = (float2 *)workspace;
    const int tgrid = (int)std::max<uint64_t>(1, std::min<uint64_t>((un / 2 + 256) / 256, (uint64_t)sm_count() * 8));
    if (alpha == 2) korobov_table_kernel<2><<<tgrid, 256, 0, stream>>>(un, T);
    else korobov_table_kernel<4><<<tgrid, 256, 0, stream>>>(un, T);
    if ((st = check_launch()) != MDI_OK) return st;
    const int grid = (int)std::min<uint64_t>(uc, (uint64_t)sm_count() * 16);
    if (alpha == 2) {
      if (d <= 8) korobov_table_criterion_kernel<2, 8><<<grid, kSearchThreads, 0, stream>>>(d, un, ua, uc, T, values);
      else korobov_table_criterion_kernel<2, 16><<<grid, kSearchThreads, 0, stream>>>(d, un, ua, uc, T, values);
    } else {
      if (d <= 8) korobov_table_criterion_kernel<4, 8><<<grid, kSearchThreads, 0, stream>>>(d, un, ua, uc, T, values);
      else korobov_table_criterion_kernel<4, 16><<<grid, kSearchThreads, 0, stream>>>(d, un, ua, uc, T, values);
    }
    st = check_launch();
  } else {
    st = alpha == 2 ? korobov_dispatch<2>(d, un, ua, uc, values, stream) : korobov_dispatch<4>(d, un, ua, uc, values, stream);
  }
  if (st != MDI_OK) return st;
  korobov_argmin_kernel<<<1, kArgminThreads, 0, stream>>>(values, uc, ua, best_a);
  return check_launch();
}

// Workspace: p[n/2+1] (float pairs) | T[n/2+1] (float pairs) | vals[n/2+1] | pref.
struct CbcLayout {
  size_t p, T, vals, pref, total;
};
static CbcLayout cbc_layout(int64_t n) {
  CbcLayout L{};
  const size_t m = (size_t)(n / 2 + 1);
  size_t off = 0;
  L.p = off;
  off += align_up(sizeof(float2) * m);
  L.T = off;
  off += align_up(sizeof(float2) * m);
  L.vals = off;
  off += align_up(sizeof(double) * m);
  L.pref = off;
  off += align_up(sizeof(double));
  L.total = off;
  return L;
}

size_t cbc_workspace_bytes(int64_t n) { return (n >= 2 && (uint64_t)n <= kTableMaxN) ? cbc_layout(n).total : 0; }

mdi_status cbc_launch(int d, int64_t n, const double *gamma, double beta, int64_t *z, double *e2, void *workspace,
                      size_t ws_bytes, cudaStream_t stream) {
  if (d < 1 || n < 2 || (uint64_t)n > kTableMaxN || !gamma || !z || !e2 || !std::isfinite(beta)) return MDI_EINVAL;
  if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < cbc_workspace_bytes(n)) return MDI_EWORKSPACE;
  const CbcLayout L = cbc_layout(n);
  char *base = (char *)workspace;
  float2 *p = (float2 *)(base + L.p), *T = (float2 *)(base + L.T);
  double *vals = (double *)(base + L.vals), *pref = (double *)(base + L.pref);
  const uint64_t un = (uint64_t)n, half = un / 2;
  const int upd_grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((half + 256) / 256, (uint64_t)sm_count() * 8));
  cbc_df_init_kernel<<<upd_grid, 256, 0, stream>>>(half, p, pref);
  mdi_status st = check_launch();
  if (st != MDI_OK) return st;
  for (int s = 0; s < d; ++s) {
    // z_1 = 1 is fixed (Example 3, step (i)); later components search 1..n/2.
    const uint64_t first = 1, count = (s == 0) ? 1 : std::max<uint64_t>(1, half);
    const int grid = (int)std::min<uint64_t>(count, (uint64_t)sm_count() * 16);
    cbc_table_kernel<<<upd_grid, 256, 0, stream>>>(s, un, gamma, beta, T);
    if ((st = check_launch()) != MDI_OK) return st;
    cbc_df_candidates_kernel<<<grid, kSearchThreads, 0, stream>>>(s, un, gamma, beta, p, T, pref, first, count, vals);
    if ((st = check_launch()) != MDI_OK) return st;
    cbc_select_kernel<<<1, kArgminThreads, 0, stream>>>(s, vals, count, first, z, e2);
    if ((st = check_launch()) != MDI_OK) return st;
    if (s + 1 < d) {
      cbc_df_update_kernel<<<upd_grid, 256, 0, stream>>>(s, un, gamma, beta, z, T, p, pref);
      if ((st = check_launch()) != MDI_OK) return st;
    }
  }
  return MDI_OK;
}

}  // namespace mdi
