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
// GB300 mapping: the d - 1 box convolutions run in ONE launch of a thread-block
// cluster (16 CTAs where the GPU allows it, else 8), each CTA holding a slice of
// the histogram in shared memory: per level the CTA forms its weights from
// power-of-two window sums (a few additions per weight instead of N - 1); every
// K levels it stores its last K (N - 1) weights into the next CTA's shared memory
// and a cluster barrier follows, the CTAs recomputing the halo in between.  (A histogram too long for
// the cluster's shared memory takes one launch per axis instead, with N-term sums
// in the oracle's order, so its weights are bitwise the oracle's.)  Then one launch over every (S, k) pair of the last axis -- the whole
// GPU -- with a block sum per CTA, and a one-CTA sum of the CTA partials in order.
// The work is N^2 d^2 / 2 additions for the weights and about (d-1) N n_last
// powers.
#include <algorithm>
#include <atomic>
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

// Thread-block cluster primitives (PTX): this CTA's rank in its cluster, a
// cluster-wide barrier (release/acquire: shared-memory stores before it, local or
// remote, are seen by every CTA after it), and stores into another CTA's shared
// memory at the address mapa gives for its copy of a local variable.
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_map(const void *local, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(local);
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_store(unsigned addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

// H_{d-1} by d - 1 box convolutions in one cluster of cs CTAs.  CTA c holds the
// weights S in [c W, (c + 1) W) in two level buffers, each preceded by a halo of
// K (N - 1) entries.  Every K levels the CTAs exchange: each sends its last
// K (N - 1) weights into the next CTA's receive buffer through distributed shared
// memory, a cluster barrier follows, and each copies what it received into its
// halo (CTA 0's halo stays zero: S < 0).  In between, a CTA recomputes the part of
// the previous CTA's slice that its own next levels read -- the halo shrinks by
// N - 1 per level -- so the cluster passes one barrier per K levels instead of one
// per level; a recomputed weight is bitwise the owner's (the same operations on
// the same inputs).  Weights past a level's length are never written and stay
// zero.  Receive buffers alternate between exchanges, so a CTA that runs ahead
// never overwrites one its neighbour has not copied yet (that takes passing the
// next barrier).  Every CTA passes the same barriers, and the last remote store
// comes before the last barrier, so no CTA leaves while another may still write
// its shared memory.  W >= K (N - 1).
//
// A level's N-term window sums are built from power-of-two windows, as N's binary
// digits: p_1 = H_{i-1}, p_2s[x] = p_s[x] + p_s[x - s], and each set bit s of N adds
// p_s[x - m] to the partial window of the bits below it (m of them), so a weight
// costs floor(log2 N) + popcount(N) - 1 additions instead of N - 1 (4 for N = 16),
// then one multiply by 1/N.  The terms are the oracle's, all positive, summed in a
// tree order: each weight is within about (log2 N + 2) units in the last place of
// the oracle's sequential sum.  Two more buffers hold the p_s.
__global__ void __launch_bounds__(kRidgeThreads) ridge_cluster_kernel(int d, int N, int W, int K, double inv_n,
                                                                      double *__restrict__ hout) {
  extern __shared__ double s_h[];  // [4][K (N - 1) + W]: levels i - 1 and i, two p_s buffers; [2][K (N - 1)] receive
  const int c = (int)cluster_rank(), cs = (int)gridDim.x;
  const int H = N - 1, KH = K * H, stride = KH + W, S0 = c * W;
  double *const recv = s_h + 4 * stride;
  for (int i = threadIdx.x; i < 4 * stride + 2 * KH; i += blockDim.x) s_h[i] = 0.0;
  cluster_barrier();  // every buffer is zero before any remote store lands
  if (c == 0 && threadIdx.x == 0) s_h[KH] = 1.0;  // H_0 = [1]
  __syncthreads();
  double *tmp[2] = {s_h + 2 * stride + KH, s_h + 3 * stride + KH};
  int cur = 0, ex = 0;
  for (int i = 1; i < d; ++i) {
    const int j = (i - 1) % K;
    double *const Pb = s_h + cur * stride + KH;  // H_{i-1} at local positions -KH .. W-1
    if (j == 0) {
      double *const rb = recv + (ex & 1) * KH;
      if (c + 1 < cs)
        for (int t = threadIdx.x; t < KH; t += blockDim.x) cluster_store(cluster_map(rb + t, c + 1), Pb[W - KH + t]);
      cluster_barrier();
      if (c > 0)
        for (int t = threadIdx.x; t < KH; t += blockDim.x) Pb[t - KH] = rb[t];
      __syncthreads();
      ++ex;
    }
    const int len = i * H + 1;          // weights of level i: S < len
    const int lo = -(K - 1 - j) * H;    // what the levels up to the next exchange read
    const int hi = min(W, len - S0);
    const double *P = Pb;
    double *out = s_h + (cur ^ 1) * stride + KH;
    int m = 0, t = 0;
    for (int span = 1; span <= N; span <<= 1) {
      if (N & span) {  // window of offsets [m, m + span) joins the partial sum
        const bool last = m + span == N, first = m == 0;
        for (int x = lo + (int)threadIdx.x; x < hi; x += blockDim.x) {
          double v = first ? P[x - m] : out[x] + P[x - m];
          out[x] = last ? v * inv_n : v;
        }
        m += span;
      }
      if (2 * span <= N) {  // p_2s on the positions the remaining bits read
        double *Pn = tmp[t];
        for (int x = lo + (int)threadIdx.x - (N - 2 * span); x < hi; x += blockDim.x) Pn[x] = P[x] + P[x - span];
        P = Pn;
        t ^= 1;
      }
      __syncthreads();
    }
    cur ^= 1;
  }
  const int len = (d - 1) * H + 1;
  const double *fin = s_h + cur * stride + KH;
  for (int s = threadIdx.x; s < min(W, len - S0); s += blockDim.x) hout[S0 + s] = fin[s];
}

// Partial sums of H[S] (1/n_last) (c0 + base_S + (k + 1/2)/n_last)^(-p) over the
// (S, k) pairs, one pair per thread and step, so the whole GPU shares the powers.
__global__ void __launch_bounds__(kRidgeThreads) ridge_last_kernel(int d, uint64_t len, uint64_t N, uint64_t n_last,
                                                                   double c0, double p,
                                                                   const double *__restrict__ h,
                                                                   double *__restrict__ partials) {
  __shared__ double s_red[kRidgeThreads / kWarp];
  double q = 0.0;
  const uint64_t total = len * n_last;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t S = e / n_last, k = e % n_last;
    const double base = ((double)S + 0.5 * (double)(d - 1)) / (double)N;
    q += h[S] * pow(c0 + base + ((double)k + 0.5) / (double)n_last, -p) / (double)n_last;
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

// The cluster path: at most kRidgeClusterSmem bytes of shared memory per CTA, and
// at most kRidgeMaxK levels between exchanges.
constexpr size_t kRidgeClusterSmem = 200 * 1024;
constexpr uint64_t kRidgeMaxK = 8;
static size_t ridge_cluster_smem(uint64_t W, int64_t N, uint64_t K) {
  const uint64_t KH = K * (uint64_t)(N - 1);
  return sizeof(double) * (4 * (KH + W) + 2 * KH);
}

// Largest cluster the GPU runs ridge_cluster_kernel in (16, else 8), once per
// device; 0 if neither launches.
static int ridge_cluster_size() {
  static std::atomic<int> cache[64];  // 0: not asked yet, -1: no cluster runs
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;  // the per-level launches
  const int known = cache[dev].load(std::memory_order_relaxed);
  if (known != 0) return known > 0 ? known : 0;
  int best = -1;
  if (cudaFuncSetAttribute(ridge_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
      cudaFuncSetAttribute(ridge_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kRidgeClusterSmem) == cudaSuccess) {
    for (int cs : {16, 8}) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cs);
      cfg.blockDim = dim3(kRidgeThreads);
      cfg.dynamicSmemBytes = kRidgeClusterSmem;
      cudaLaunchAttribute attr;
      attr.id = cudaLaunchAttributeClusterDimension;
      attr.val.clusterDim.x = cs;
      attr.val.clusterDim.y = 1;
      attr.val.clusterDim.z = 1;
      cfg.attrs = &attr;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, ridge_cluster_kernel, &cfg) == cudaSuccess && n > 0) {
        best = cs;
        break;
      }
    }
  }
  cudaGetLastError();  // a refused query leaves no error behind
  cache[dev].store(best, std::memory_order_relaxed);
  return best > 0 ? best : 0;
}

// Workspace: two weight buffers of the final length (the cluster path uses the
// first for H_{d-1}), then the last launch's CTA partials.
size_t ridge_workspace_bytes(int d, int64_t N, int64_t n_last) {
  if (d < 1 || N < 1 || n_last < 1 || (double)(d - 1) * (double)(N - 1) + 1.0 > (double)kRidgeMaxLen) return 0;
  const uint64_t L = ridge_len(d, N);
  if ((double)L * (double)n_last > 0x1p62) return 0;  // the last launch counts (S, k) pairs in 64 bits
  return 2 * align_up(sizeof(double) * (size_t)L) + align_up(sizeof(double) * (size_t)ridge_grid(L * (uint64_t)n_last));
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
  mdi_status st = MDI_OK;
  uint64_t len = L;
  int cur = 0;
  // The cluster path: cs CTAs of W >= N - 1 weights each, two buffers and halos
  // within the shared-memory budget.
  const int cmax = N > 1 ? ridge_cluster_size() : 0;
  int cs = 0;
  uint64_t W = 0;
  uint64_t K = 1;  // levels per exchange
  if (cmax > 0 && N <= 4096) {
    cs = (int)std::min<uint64_t>((uint64_t)cmax, std::max<uint64_t>(1, L / (uint64_t)(N - 1)));
    W = (L + cs - 1) / cs;
    K = std::max<uint64_t>(1, std::min<uint64_t>(kRidgeMaxK, W / (uint64_t)(N - 1)));
    if (W < (uint64_t)(N - 1) || ridge_cluster_smem(W, N, K) > kRidgeClusterSmem) cs = 0;
  }
  if (cs > 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kRidgeThreads);
    cfg.dynamicSmemBytes = ridge_cluster_smem(W, N, K);
    cfg.stream = stream;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = cs;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    const cudaError_t e =
        cudaLaunchKernelEx(&cfg, ridge_cluster_kernel, d, (int)N, (int)W, (int)K, 1.0 / (double)N, buf[0]);
    if (e != cudaSuccess) {  // a cluster the GPU refuses now: the per-level launches below
      cudaGetLastError();
      cs = 0;
    }
  }
  if (cs == 0) {
    ridge_init_kernel<<<1, 1, 0, stream>>>(buf[0]);
    if ((st = check_launch()) != MDI_OK) return st;
    len = 1;
    for (int i = 1; i < d; ++i) {
      const uint64_t nlen = len + (uint64_t)N - 1;
      ridge_level_kernel<<<ridge_grid(nlen), kRidgeThreads, 0, stream>>>(len, (uint64_t)N, buf[cur], buf[cur ^ 1]);
      if ((st = check_launch()) != MDI_OK) return st;
      cur ^= 1;
      len = nlen;
    }
  }
  const int grid = ridge_grid(len * (uint64_t)n_last);
  ridge_last_kernel<<<grid, kRidgeThreads, 0, stream>>>(d, len, (uint64_t)N, (uint64_t)n_last, c0, p, buf[cur],
                                                        partials);
  if ((st = check_launch()) != MDI_OK) return st;
  ridge_sum_kernel<<<1, kRidgeThreads, 0, stream>>>(partials, grid, out);
  return check_launch();
}

}  // namespace mdi
