// mdi_ridge.cu -- paper-table mode for a ridge integrand f(x) = (c0 + sum_i x_i)^(-p)
// (Test 7's f_6 is c0 = 1, p = d + 1) on the midpoint grid of eq. (3.5),
// n_1 = ... = n_{d-1} = N, n_d = n_last.
//
// Dimension iteration (Algorithm 1, m = 1, eq. 2.14c): once the first i axes are
// summed out, the symbolic function depends on them only through the digit sum
// S = k_1 + ... + k_i, so the level state is the weight of each S,
//     H_i[S] = (1/N) sum_{k<N} H_{i-1}[S - k],   H_0 = [1],
// a box convolution per axis (length i(N-1) + 1 after i axes), and
//     Q = sum_S H_{d-1}[S] (1/n_last) sum_{k<n_last} f at (S + (d-1)/2)/N + (k + 1/2)/n_last.
//
// GB300 mapping: one launch per axis, one thread per output weight (N-term sums
// in the oracle's order, so the weights are bitwise the same), then one launch in
// which every thread takes weights S and their n_last last-axis points, a block sum
// per CTA, and a one-CTA sum of the CTA partials in order.  The work is
// N^2 d^2 / 2 multiply-adds for the weights and about (d-1) N n_last powers.
#include <algorithm>
#include <cmath>

#include "mdi_common.cuh"
#include "mdi_internal.h"

namespace mdi {

constexpr int kRidgeThreads = 256;
constexpr uint64_t kRidgeMaxLen = 1ull << 26;

__global__ void ridge_init_kernel(double *__restrict__ h) { h[0] = 1.0; }

// H_out[S] = (1/N) sum_{k<N, 0<=S-k<len} H_in[S - k] for S < len + N - 1.
__global__ void __launch_bounds__(kRidgeThreads) ridge_level_kernel(uint64_t len, uint64_t N,
                                                                    const double *__restrict__ hin,
                                                                    double *__restrict__ hout) {
  const uint64_t nlen = len + N - 1;
  for (uint64_t S = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; S < nlen; S += (uint64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (uint64_t k = 0; k < N; ++k)
      if (S >= k && S - k < len) acc += hin[S - k];
    hout[S] = acc / (double)N;
  }
}

// Partial sums over S of H[S] (1/n_last) sum_k (c0 + base_S + (k + 1/2)/n_last)^(-p).
__global__ void __launch_bounds__(kRidgeThreads) ridge_last_kernel(int d, uint64_t len, uint64_t N, uint64_t n_last,
                                                                   double c0, double p,
                                                                   const double *__restrict__ h,
                                                                   double *__restrict__ partials) {
  __shared__ double s_red[kRidgeThreads / kWarp];
  double q = 0.0;
  for (uint64_t S = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; S < len; S += (uint64_t)gridDim.x * blockDim.x) {
    const double base = ((double)S + 0.5 * (double)(d - 1)) / (double)N;
    double inner = 0.0;
    for (uint64_t k = 0; k < n_last; ++k) inner += pow(c0 + base + ((double)k + 0.5) / (double)n_last, -p);
    q += h[S] * inner / (double)n_last;
  }
  q = block_sum(q, s_red);
  if (threadIdx.x == 0) partials[blockIdx.x] = q;
}

__global__ void __launch_bounds__(kRidgeThreads) ridge_sum_kernel(const double *__restrict__ partials, int count,
                                                                  double *__restrict__ out) {
  __shared__ double s_red[kRidgeThreads / kWarp];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += partials[i];
  acc = block_sum(acc, s_red);
  if (threadIdx.x == 0) out[0] = acc;
}

static uint64_t ridge_len(int d, int64_t N) { return (uint64_t)(d - 1) * (uint64_t)(N - 1) + 1; }

static int ridge_grid(uint64_t len) {
  return (int)std::max<uint64_t>(1, std::min<uint64_t>((len + kRidgeThreads - 1) / kRidgeThreads,
                                                       (uint64_t)sm_count() * 8));
}

// Workspace: two weight buffers of the final length, then the CTA partials.
size_t ridge_workspace_bytes(int d, int64_t N, int64_t n_last) {
  if (d < 1 || N < 1 || n_last < 1 || (double)(d - 1) * (double)(N - 1) + 1.0 > (double)kRidgeMaxLen) return 0;
  const uint64_t L = ridge_len(d, N);
  return 2 * align_up(sizeof(double) * (size_t)L) + align_up(sizeof(double) * (size_t)ridge_grid(L));
}

mdi_status ridge_launch(int d, int64_t N, int64_t n_last, double c0, double p, double *out, void *workspace,
                        size_t ws_bytes, cudaStream_t stream) {
  if (d < 1 || N < 1 || n_last < 1 || !out || !(c0 > 0.0) || !std::isfinite(c0) || !std::isfinite(p))
    return MDI_EINVAL;
  const size_t need = ridge_workspace_bytes(d, N, n_last);
  if (need == 0) return MDI_EINVAL;
  if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < need) return MDI_EWORKSPACE;
  const uint64_t L = ridge_len(d, N);
  char *base = (char *)workspace;
  double *buf[2] = {(double *)base, (double *)(base + align_up(sizeof(double) * (size_t)L))};
  double *partials = (double *)(base + 2 * align_up(sizeof(double) * (size_t)L));
  ridge_init_kernel<<<1, 1, 0, stream>>>(buf[0]);
  mdi_status st = check_launch();
  if (st != MDI_OK) return st;
  uint64_t len = 1;
  int cur = 0;
  for (int i = 1; i < d; ++i) {
    const uint64_t nlen = len + (uint64_t)N - 1;
    ridge_level_kernel<<<ridge_grid(nlen), kRidgeThreads, 0, stream>>>(len, (uint64_t)N, buf[cur], buf[cur ^ 1]);
    if ((st = check_launch()) != MDI_OK) return st;
    cur ^= 1;
    len = nlen;
  }
  const int grid = ridge_grid(len);
  ridge_last_kernel<<<grid, kRidgeThreads, 0, stream>>>(d, len, (uint64_t)N, (uint64_t)n_last, c0, p, buf[cur],
                                                        partials);
  if ((st = check_launch()) != MDI_OK) return st;
  ridge_sum_kernel<<<1, kRidgeThreads, 0, stream>>>(partials, grid, out);
  return check_launch();
}

}  // namespace mdi
