// mdi_exact.cu -- MDI-LR with the exact level state (MDI_STATE_EXACT).
//
// Level k = 1..d of Algorithm 1 (m = 1) contracts the first remaining
// transformed coordinate with r_k points (r_k = a for k < d, r_d = n_last).  The
// state after level k, G_k, is needed at the parents x = m / M_k, m < M_k, with
// M_0 = n = n_last a^(d-1) and M_k = M_{k-1} / r_k, and satisfies (eq. (4.4) with
// equal weights 1/r_k)
//     G_k[m] = (1/r_k) sum_{q<r_k} phi_k((q M_k + m) / M_{k-1}) G_{k-1}[q M_k + m].
// The entries of G_{k-1} that feed G_k[m] all share m's residue modulo M_k, so a
// run of levels k0+1..k1 splits into independent residue classes rr < M_{k1}:
// one CTA keeps the T = M_{k0} / M_{k1} entries of a class in shared memory,
// contracts all the levels of the run there (each level in place, one barrier
// per level), and writes a single value of G_{k1}.  A run is as many levels as
// fit a 32 KiB tile, so a lattice of n points takes about log(n)/log(tile)
// launches, and only the table between runs touches global memory.
#include <algorithm>
#include <vector>

#include "mdi_common.cuh"
#include "mdi_internal.h"

namespace mdi {

constexpr int kExactThreads = 256;
constexpr size_t kExactTileBytes = 32 * 1024;
constexpr int64_t kExactMaxN = int64_t(1) << 40;

struct ExactPass {
  int k0, k1;      // levels k0+1 .. k1 (1-based)
  int64_t tile;    // T = M_{k0} / M_{k1}
  int64_t classes; // M_{k1}
};

struct ExactArgs {
  int d, k0, k1;
  int64_t a, n_last;
  int64_t classes;  // M_{k1}
  int64_t tile;     // T
  int64_t m_k0;     // M_{k0}
};

template <int FAM, bool F32>
__global__ void __launch_bounds__(kExactThreads) exact_pass_kernel(const ExactArgs args,
                                                                   const double *__restrict__ params,
                                                                   const typename FamTraits<FAM>::V *__restrict__ in,
                                                                   typename FamTraits<FAM>::V *__restrict__ out_table,
                                                                   double *__restrict__ out_final) {
  using V = typename FamTraits<FAM>::V;
  __shared__ V tile[kExactTileBytes / sizeof(V)];
  const int64_t T = args.tile, Mk1 = args.classes;
  for (int64_t rr = blockIdx.x; rr < Mk1; rr += gridDim.x) {
    for (int64_t t = threadIdx.x; t < T; t += blockDim.x)
      tile[t] = in ? in[rr + t * Mk1] : VOps<V>::one();
    __syncthreads();
    int64_t curT = T, Mprev = args.m_k0;  // M_{k-1} at the current level
    for (int k = args.k0 + 1; k <= args.k1; ++k) {
      const int64_t r = (k < args.d) ? args.a : args.n_last;
      const int64_t newT = curT / r;
      const AxisParams ap = load_axis(params, args.d, k - 1);
      const double invM = 1.0 / (double)Mprev, invr = 1.0 / (double)r;
      for (int64_t tp = threadIdx.x; tp < newT; tp += blockDim.x) {
        V acc = VOps<V>::zero();
        for (int64_t q = 0; q < r; ++q) {
          const int64_t t = tp + q * newT;
          const double x = (double)(rr + t * Mk1) * invM;
          acc = VOps<V>::add(acc, VOps<V>::mul(phi<FAM, F32>(x, ap), tile[t]));
        }
        tile[tp] = VOps<V>::scale(acc, invr);
      }
      __syncthreads();
      curT = newT;
      Mprev /= r;
    }
    if (threadIdx.x == 0) {
      if (out_final) {
        if constexpr (FAM == MDI_FAM_OSC) {
          double s, c;
          sincos(kTwoPi * params[args.d], &s, &c);
          out_final[0] = c * tile[0].x - s * tile[0].y;
        } else {
          out_final[0] = tile[0];
        }
      } else {
        out_table[rr] = tile[0];
      }
    }
    __syncthreads();
  }
}

// Splits levels 1..d into runs whose tiles fit in shared memory.
static bool plan_exact(int family, int d, int64_t a, int64_t n_last, std::vector<ExactPass> &passes, int64_t &n) {
  const int64_t tile_max = (int64_t)(kExactTileBytes / (family == MDI_FAM_OSC ? 16 : 8));
  n = n_last;
  for (int k = 1; k < d; ++k) {
    if (n > kExactMaxN / a) return false;
    n *= a;
  }
  if (n > kExactMaxN) return false;
  passes.clear();
  int64_t M = n;
  int k0 = 0;
  while (k0 < d) {
    int64_t T = 1;
    int k1 = k0;
    while (k1 < d) {
      int64_t r = (k1 + 1 < d) ? a : n_last;
      if (T * r > tile_max) break;
      T *= r;
      ++k1;
    }
    if (k1 == k0) return false;  // a single radix exceeds the tile
    passes.push_back(ExactPass{k0, k1, T, M / T});
    M /= T;
    k0 = k1;
  }
  return true;
}

size_t exact_workspace_bytes(int family, int d, int64_t a, int64_t n_last) {
  std::vector<ExactPass> passes;
  int64_t n;
  if (d < 1 || a < 1 || n_last < 1 || !plan_exact(family, d, a, n_last, passes, n)) return 0;
  int64_t biggest = 1;
  for (size_t i = 0; i + 1 < passes.size(); ++i) biggest = std::max(biggest, passes[i].classes);
  return 2 * align_up((size_t)biggest * 16);
}

template <int FAM, bool F32>
static mdi_status run_exact(const std::vector<ExactPass> &passes, int d, int64_t a, int64_t n_last,
                            const double *params, double *out, void *workspace, cudaStream_t stream) {
  using V = typename FamTraits<FAM>::V;
  int64_t biggest = 1;
  for (size_t i = 0; i + 1 < passes.size(); ++i) biggest = std::max(biggest, passes[i].classes);
  V *buf[2] = {(V *)workspace, (V *)((char *)workspace + align_up((size_t)biggest * 16))};
  const V *in = nullptr;
  int64_t Mk0 = 1;
  for (const auto &p : passes) Mk0 *= p.tile;  // = n
  const int max_grid = sm_count() * 16;
  for (size_t i = 0; i < passes.size(); ++i) {
    const ExactPass &p = passes[i];
    ExactArgs args{d, p.k0, p.k1, a, n_last, p.classes, p.tile, Mk0};
    const bool last = (i + 1 == passes.size());
    V *dst = last ? nullptr : buf[i & 1];
    int grid = (int)std::min<int64_t>(p.classes, max_grid);
    exact_pass_kernel<FAM, F32><<<grid, kExactThreads, 0, stream>>>(args, params, in, dst, last ? out : nullptr);
    mdi_status st = check_launch();
    if (st != MDI_OK) return st;
    in = dst;
    Mk0 = p.classes;
  }
  return MDI_OK;
}

mdi_status exact_launch(int family, int d, int64_t a, int64_t n_last, const double *params, int precision,
                        double *out, void *workspace, size_t ws_bytes, cudaStream_t stream) {
  std::vector<ExactPass> passes;
  int64_t n;
  if (!plan_exact(family, d, a, n_last, passes, n)) return MDI_EOVERFLOW;
  if (precision != MDI_PREC_FP64 && precision != MDI_PREC_FP32_EVAL_FP64) return MDI_EUNSUPPORTED;
  size_t need = exact_workspace_bytes(family, d, a, n_last);
  if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < need) return MDI_EWORKSPACE;
  const bool f32 = precision == MDI_PREC_FP32_EVAL_FP64;
  switch (family) {
    case MDI_FAM_EXP:
      return f32 ? run_exact<MDI_FAM_EXP, true>(passes, d, a, n_last, params, out, workspace, stream)
                 : run_exact<MDI_FAM_EXP, false>(passes, d, a, n_last, params, out, workspace, stream);
    case MDI_FAM_OSC:
      return f32 ? run_exact<MDI_FAM_OSC, true>(passes, d, a, n_last, params, out, workspace, stream)
                 : run_exact<MDI_FAM_OSC, false>(passes, d, a, n_last, params, out, workspace, stream);
    case MDI_FAM_GAUSS:
      return f32 ? run_exact<MDI_FAM_GAUSS, true>(passes, d, a, n_last, params, out, workspace, stream)
                 : run_exact<MDI_FAM_GAUSS, false>(passes, d, a, n_last, params, out, workspace, stream);
    default:
      return f32 ? run_exact<MDI_FAM_PEAK, true>(passes, d, a, n_last, params, out, workspace, stream)
                 : run_exact<MDI_FAM_PEAK, false>(passes, d, a, n_last, params, out, workspace, stream);
  }
}

}  // namespace mdi
