// api.cu -- the C ABI of include/mdi_lr.h: argument checks, state selection,
// workspace sizing and the host-side batch scheduler.  Every compute step runs in
// the kernels of slr.cu, mdi_exact.cu, mdi_closed.cu and mdi_nodes.cu.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>
#include <queue>
#include <cmath>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mdi_common.cuh"
#include "mdi_internal.h"

namespace mdi {

static thread_local std::string g_last_cuda_error;

// One NVTX range per compute call of the ABI, named after it, so a profiler can
// attribute the kernels it sees to calls (header-only NVTX 3: without an attached
// tool a push or pop is a pointer check).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

void set_cuda_error(cudaError_t e) {
  g_last_cuda_error = std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e);
}

int sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

static bool family_ok(int f) { return f >= MDI_FAM_EXP && f <= MDI_FAM_PEAK; }

static bool opts_ok(const mdi_opts *o) {
  if (!o) return true;
  if (o->state < MDI_STATE_AUTO || o->state > MDI_STATE_NODES) return false;
  if (o->precision < MDI_PREC_FP64 || o->precision > MDI_PREC_DF64) return false;
  if (o->nodes < 0 || o->block < 0 || o->ctas_per_sm < 0 || o->checkpoint < 0) return false;
  if (o->table_in_l1 != 0 && o->table_in_l1 != 1) return false;
  return o->step >= 0 && o->step <= 3;
}



static int resolve_state(int family, const mdi_opts *o) {
  int s = o ? o->state : MDI_STATE_AUTO;
  if (s != MDI_STATE_AUTO) return s;
  return (family == MDI_FAM_EXP || family == MDI_FAM_OSC) ? MDI_STATE_CLOSED : MDI_STATE_NODES;
}

// Estimated FP64-equivalent operations of one node-state integral (scheduler cost).
static double nodes_cost(const mdi_batch_desc &d, int P) {
  const double phi_cost = (d.family == MDI_FAM_PEAK) ? 8.0 : 20.0;
  return (double)(d.d - 1) * d.a * P * (P + phi_cost) + (double)d.n_last * (2.0 * P + phi_cost);
}

// One node-state integral runs parallel over levels (mdi_levels.cu) when it has
// enough levels to fill several SMs; short ones take one CTA of the batched kernel.
static bool use_levels(int d) { return d >= 8; }

static bool desc_ok(const mdi_batch_desc &d) {
  return family_ok(d.family) && d.d >= 1 && d.d <= MDI_BATCH_MAX_D && d.a >= 1 && d.a <= 64 && d.n_last >= 1 &&
         d.n_last <= 4096 && d.param_offset >= 0 && d.reserved == 0;
}

// The 2*d parameters of a descriptor lie inside a pool of pool_len doubles.
static bool desc_in_pool(const mdi_batch_desc &d, int64_t pool_len) {
  return d.param_offset <= pool_len && 2 * (int64_t)d.d <= pool_len - d.param_offset;
}

// x * y mod m for 0 <= x, y < m < 2^63, exact through a 128-bit product.
static int64_t mulmod(int64_t x, int64_t y, int64_t m) {
  return (int64_t)((unsigned __int128)(uint64_t)x * (uint64_t)y % (unsigned __int128)(uint64_t)m);
}

// A generating vector handed to an MDI-LR call (Algorithm 2's z) must be Example
// 2's Korobov vector for (a, n = n_last a^(d-1)): the sweep's digits describe that
// lattice only.  NULL selects it.
static mdi_status check_korobov_z(int d, int64_t a, int64_t n_last, const int64_t *z) {
  if (!z) return MDI_OK;
  unsigned __int128 n = (unsigned __int128)n_last;
  const unsigned __int128 limit = ((unsigned __int128)1 << 63) - 1;
  for (int i = 1; i < d; ++i) {
    n *= (unsigned __int128)a;
    if (n > limit) return MDI_EOVERFLOW;
  }
  const int64_t nn = (int64_t)n;
  int64_t v = 1 % nn;
  for (int i = 0; i < d; ++i) {
    if (z[i] != v) return MDI_EUNSUPPORTED;
    v = mulmod(v, a % nn, nn);
  }
  return MDI_OK;
}

}  // namespace mdi

using namespace mdi;

extern "C" {

const char *mdi_status_string(mdi_status s) {
  switch (s) {
    case MDI_OK: return "MDI_OK: success";
    case MDI_EINVAL: return "MDI_EINVAL: invalid argument";
    case MDI_EUNSUPPORTED: return "MDI_EUNSUPPORTED: combination not provided by this library";
    case MDI_EOVERFLOW: return "MDI_EOVERFLOW: lattice size exceeds the exact integer range";
    case MDI_ECUDA: return "MDI_ECUDA: CUDA runtime error";
    case MDI_EWORKSPACE: return "MDI_EWORKSPACE: workspace missing, misaligned or too small";
  }
  return "unknown mdi_status";
}

const char *mdi_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

int32_t mdi_abi_version(void) { return MDI_ABI_VERSION; }

mdi_status lattice_rule_workspace_size(int32_t d, int64_t n, size_t *bytes) {
  if (!bytes || d < 1 || n < 1) return MDI_EINVAL;
  *bytes = slr_workspace_bytes(d, n);
  return MDI_OK;
}

mdi_status lattice_rule_integrate(int32_t family, int32_t d, int64_t n, const int64_t *z, const double *params,
                                  int32_t precision, double *out, void *workspace, size_t ws_bytes,
                                  mdi_stream_t stream) {
  NvtxRange nvtx_scope("lattice_rule_integrate");
  if (!family_ok(family)) return MDI_EINVAL;
  return slr_launch(family, d, n, z, params, precision, out, workspace, ws_bytes, (cudaStream_t)stream);
}

mdi_status lattice_rule_shifted_workspace_size(int32_t d, int64_t n, int32_t R, size_t *bytes) {
  if (!bytes || d < 1 || n < 1 || R < 1) return MDI_EINVAL;
  *bytes = slr_shifted_workspace_bytes(d, n, R);
  return *bytes ? MDI_OK : MDI_EINVAL;
}

mdi_status lattice_rule_integrate_shifted(int32_t family, int32_t d, int64_t n, const int64_t *z,
                                          const double *params, const double *shifts, int32_t R,
                                          int32_t precision, double *out, void *workspace, size_t ws_bytes,
                                          mdi_stream_t stream) {
  NvtxRange nvtx_scope("lattice_rule_integrate_shifted");
  if (!family_ok(family)) return MDI_EINVAL;
  return slr_shifted_launch(family, d, n, z, params, shifts, R, precision, out, workspace, ws_bytes,
                            (cudaStream_t)stream);
}

mdi_status lattice_rule_improved_workspace_size(int32_t d, int64_t n, int64_t a, size_t *bytes) {
  if (!bytes) return MDI_EINVAL;
  *bytes = slr_improved_workspace_bytes(d, n, a);
  return *bytes ? MDI_OK : MDI_EINVAL;
}

mdi_status lattice_rule_integrate_improved(int32_t family, int32_t d, int64_t n, int64_t a, const double *params,
                                           int32_t precision, double *out, int64_t *n_ghost, void *workspace,
                                           size_t ws_bytes, mdi_stream_t stream) {
  NvtxRange nvtx_scope("lattice_rule_integrate_improved");
  if (!family_ok(family)) return MDI_EINVAL;
  return slr_improved_launch(family, d, n, a, params, precision, out, n_ghost, workspace, ws_bytes,
                             (cudaStream_t)stream);
}

mdi_status lattice_korobov_vector(int32_t d, int64_t a, int64_t n, int64_t *z) {
  if (d < 1 || n < 1 || a < 0 || !z) return MDI_EINVAL;
  int64_t v = 1 % n;
  const int64_t am = a % n;
  for (int32_t i = 0; i < d; ++i) {
    z[i] = v;
    v = mulmod(v, am, n);
  }
  return MDI_OK;
}

mdi_status lattice_shifted_estimate(const double *values, int32_t R, double *mean_se, mdi_stream_t stream) {
  NvtxRange nvtx_scope("lattice_shifted_estimate");
  if (!values || !mean_se || R < 1 || R > 65535) return MDI_EINVAL;
  return shifted_estimate_launch(values, R, mean_se, (cudaStream_t)stream);
}

mdi_status mdi_peak_probe(int32_t kind, int32_t iters, double *sink, mdi_stream_t stream) {
  if ((kind != 0 && kind != 1) || iters < 1 || iters > (1 << 20) || !sink) return MDI_EINVAL;
  return peak_probe_launch(kind, iters, sink, (cudaStream_t)stream);
}

int64_t mdi_peak_probe_threads(int32_t kind) {
  if (kind != 0 && kind != 1) return 0;
  return peak_probe_threads(kind);
}

mdi_status lattice_rule_integrate_noalloc(int32_t family, int32_t d, int64_t n, const int64_t *z, const double *params,
                                          int32_t precision, double *out, mdi_stream_t stream) {
  NvtxRange nvtx_scope("lattice_rule_integrate_noalloc");
  if (!family_ok(family)) return MDI_EINVAL;
  return slr_launch_noalloc(family, d, n, z, params, precision, out, (cudaStream_t)stream);
}

mdi_status mdi_lr_workspace_size(int32_t family, int32_t d, int64_t a, int64_t n_last, const mdi_opts *opts,
                                 size_t *bytes) {
  if (!bytes || !family_ok(family) || d < 1 || a < 1 || n_last < 1 || !opts_ok(opts)) return MDI_EINVAL;
  switch (resolve_state(family, opts)) {
    case MDI_STATE_EXACT: {
      size_t b = exact_workspace_bytes(family, d, a, n_last);
      if (b == 0) return MDI_EOVERFLOW;
      *bytes = b;
      return MDI_OK;
    }
    case MDI_STATE_CLOSED:
      if (family != MDI_FAM_EXP && family != MDI_FAM_OSC) return MDI_EUNSUPPORTED;
      *bytes = closed_workspace_bytes(d, a, n_last);
      if (*bytes == 0) return MDI_EINVAL;
      return MDI_OK;
    default: {
      const NodesConfig cfg = nodes_config(opts);
      if (cfg.step > 1) {
        *bytes = levels_step_workspace_bytes(d, a, cfg, opts->checkpoint);
        return *bytes ? MDI_OK : MDI_EUNSUPPORTED;
      }
      *bytes = use_levels(d) ? levels_workspace_bytes(d, a, cfg, opts ? opts->checkpoint : 0)
                                  : nodes_single_workspace_bytes(cfg);
      return MDI_OK;
    }
  }
}

mdi_status mdi_lr_integrate(int32_t family, int32_t d, int64_t a, int64_t n_last, const int64_t *z,
                            const double *params, const mdi_opts *opts, double *out, void *workspace,
                            size_t ws_bytes, mdi_stream_t stream) {
  NvtxRange nvtx_scope("mdi_lr_integrate");
  if (!family_ok(family) || d < 1 || a < 1 || n_last < 1 || !params || !out || !opts_ok(opts)) return MDI_EINVAL;
  if (mdi_status zs = check_korobov_z(d, a, n_last, z); zs != MDI_OK) return zs;
  const int precision = opts ? opts->precision : MDI_PREC_FP64;
  cudaStream_t s = (cudaStream_t)stream;
  switch (resolve_state(family, opts)) {
    case MDI_STATE_EXACT: return exact_launch(family, d, a, n_last, params, precision, out, workspace, ws_bytes, s);
    case MDI_STATE_CLOSED: return closed_launch(family, d, a, n_last, params, precision, out, workspace, ws_bytes, s);
    default: {
      const NodesConfig cfg = nodes_config(opts);
      if (use_levels(d) || cfg.step > 1)
        return levels_launch(family, d, a, n_last, params, cfg, opts ? opts->checkpoint : 0, out, nullptr, workspace,
                             ws_bytes, s);
      return nodes_single_launch(family, d, a, n_last, params, cfg, out, workspace, ws_bytes, s);
    }
  }
}

mdi_status mdi_lr_grad_workspace_size(int32_t family, int32_t d, int64_t a, int64_t n_last, const mdi_opts *opts,
                                      size_t *bytes) {
  if (!bytes || !family_ok(family) || d < 1 || a < 1 || n_last < 1 || !opts_ok(opts)) return MDI_EINVAL;
  switch (resolve_state(family, opts)) {
    case MDI_STATE_EXACT: return MDI_EUNSUPPORTED;
    case MDI_STATE_CLOSED:
      if (family != MDI_FAM_EXP && family != MDI_FAM_OSC) return MDI_EUNSUPPORTED;
      *bytes = closed_grad_workspace_bytes(d, a, n_last);
      if (*bytes == 0) return MDI_EINVAL;
      return MDI_OK;
    default:
      if (opts && opts->step > 1) {
        *bytes = levels_step_workspace_bytes(d, a, nodes_config(opts), opts->checkpoint);
        return *bytes ? MDI_OK : MDI_EUNSUPPORTED;
      }
      *bytes = levels_workspace_bytes(d, a, nodes_config(opts), opts ? opts->checkpoint : 0);
      return MDI_OK;
  }
}

mdi_status mdi_lr_grad(int32_t family, int32_t d, int64_t a, int64_t n_last, const int64_t *z, const double *params,
                       const mdi_opts *opts, double *value, double *grad, void *workspace, size_t ws_bytes,
                       mdi_stream_t stream) {
  NvtxRange nvtx_scope("mdi_lr_grad");
  if (!family_ok(family) || d < 1 || a < 1 || n_last < 1 || !params || !grad || !opts_ok(opts)) return MDI_EINVAL;
  if (mdi_status zs = check_korobov_z(d, a, n_last, z); zs != MDI_OK) return zs;
  const int precision = opts ? opts->precision : MDI_PREC_FP64;
  if (precision != MDI_PREC_FP64) return MDI_EUNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  switch (resolve_state(family, opts)) {
    case MDI_STATE_EXACT: return MDI_EUNSUPPORTED;
    case MDI_STATE_CLOSED: return closed_grad_launch(family, d, a, n_last, params, value, grad, workspace, ws_bytes, s);
    default:
      return levels_launch(family, d, a, n_last, params, nodes_config(opts), opts ? opts->checkpoint : 0, value, grad,
                           workspace, ws_bytes, s);
  }
}

mdi_status mdi_lr_batched_workspace_size(int32_t count, const mdi_opts *opts, size_t *bytes) {
  if (!bytes || count < 1 || !opts_ok(opts)) return MDI_EINVAL;
  *bytes = nodes_batched_workspace_bytes(count, nodes_config(opts));
  return MDI_OK;
}

mdi_status mdi_lr_batched_prepare(const mdi_opts *opts, void *workspace, size_t ws_bytes, mdi_stream_t stream) {
  NvtxRange nvtx_scope("mdi_lr_batched_prepare");
  if (!opts_ok(opts)) return MDI_EINVAL;
  return nodes_prepare(nodes_config(opts), workspace, ws_bytes, (cudaStream_t)stream);
}

mdi_status mdi_lr_integrate_batched(const mdi_batch_desc *descs, const int32_t *order, int32_t count, int32_t split,
                                    const double *param_pool, int64_t pool_len, const mdi_opts *opts, double *out,
                                    void *workspace, size_t ws_bytes, mdi_stream_t stream) {
  NvtxRange nvtx_scope("mdi_lr_integrate_batched");
  if (!opts_ok(opts) || pool_len < 0 || split < 0) return MDI_EINVAL;
  if (opts && opts->state != MDI_STATE_AUTO && opts->state != MDI_STATE_NODES) return MDI_EUNSUPPORTED;
  if (opts && opts->step > 1) return MDI_EUNSUPPORTED;
  return nodes_batched_launch(descs, order, count, split, param_pool, pool_len, nodes_config(opts), out, workspace,
                              ws_bytes, (cudaStream_t)stream);
}

mdi_status mdi_get_device_status(const void *workspace, size_t ws_bytes, int32_t clear, uint32_t *flags,
                                 mdi_stream_t stream) {
  if (!workspace || ((uintptr_t)workspace % kAlign) != 0 || ws_bytes < nodes_status_word_bytes()) return MDI_EINVAL;
  uint32_t word = 0;
  mdi_status st = nodes_read_status(workspace, clear != 0, &word, (cudaStream_t)stream);
  if (st != MDI_OK) return st;
  if (flags) *flags = word;
  return word ? MDI_EINVAL : MDI_OK;
}

// Time of one node-state integral on a team of `warps` warps (1 or 2) of the paired
// sweep, in units of one FP64 warp instruction of the FP64 sweep (the other
// precisions' sweeps have the same passes and are scheduled with the same model):
// each of the d-1 cluster
// levels takes ceil(a / lanes_per_pair) passes (8 node pairs share the team's
// lanes), a pass costs each warp the interpolation of one point pair (P/2 fused
// multiply-adds for each of the pair's two sums, their sum and difference, two
// accumulations) and two evaluations of phi; the first level has no
// interpolation; each level adds its constants and sums; the last axis is small.
// The FP64 sweep steps a Gaussian's factors by a recurrence when a lane has at
// least three points (two multiplies per factor after three exps per level; the
// model takes its argument guard as met).
static double team_time(const mdi_batch_desc &d, int P, int warps, bool fp64) {
  const double phi = d.family == MDI_FAM_PEAK ? 5.0 : 12.0;  // FP64 operations of one phi
  const int lanes_per_pair = 4 * warps;
  const double passes = std::ceil((double)d.a / lanes_per_pair);
  const bool rec = fp64 && d.family == MDI_FAM_GAUSS && passes >= 3.0;
  const double pphi = rec ? 2.0 : phi;
  const double pair = (double)P + 4.0 + 2.0 * pphi, first = 2.0 + 2.0 * pphi;
  const double level = 10.0 + (rec ? 3.0 * phi + 6.0 : 0.0);
  const double last = std::ceil((double)d.n_last / (kWarp * warps)) * ((double)P + phi);
  if (d.d < 2) return last;
  return (double)(d.d - 2) * (passes * pair + level) + passes * first + level + last;
}

// Makespan of the hybrid schedule in the order `idx`: `ctas` two-warp CTAs take
// the first `split` integrals as whole teams (longest first, each to the CTA that
// frees first), then every warp takes the rest on its own.
static double hybrid_makespan(const std::vector<double> &t2, const std::vector<double> &t1,
                              const std::vector<int32_t> &idx, int split, int ctas) {
  std::priority_queue<double, std::vector<double>, std::greater<double>> free_at;
  for (int c = 0; c < ctas; ++c) free_at.push(0.0);
  for (int i = 0; i < split; ++i) {
    const double t0 = free_at.top();
    free_at.pop();
    free_at.push(t0 + t2[(size_t)idx[(size_t)i]]);
  }
  std::priority_queue<double, std::vector<double>, std::greater<double>> warps;
  double end = 0.0;
  while (!free_at.empty()) {
    warps.push(free_at.top());
    warps.push(free_at.top());
    end = std::max(end, free_at.top());
    free_at.pop();
  }
  for (size_t i = (size_t)split; i < idx.size(); ++i) {
    const double t0 = warps.top();
    warps.pop();
    const double t = t0 + t1[(size_t)idx[i]];
    end = std::max(end, t);
    warps.push(t);
  }
  return end;
}

mdi_status mdi_batch_plan(const mdi_batch_desc *descs, int32_t count, int64_t pool_len, const mdi_opts *opts,
                          int32_t *order, int32_t *split) {
  if (!descs || !order || count < 1 || pool_len < 0 || !opts_ok(opts)) return MDI_EINVAL;
  const NodesConfig cfg = nodes_config(opts);
  const int P = cfg.P;
  std::vector<double> cost((size_t)count);
  bool all_real = true;
  for (int32_t i = 0; i < count; ++i) {
    if (!desc_ok(descs[i]) || !desc_in_pool(descs[i], pool_len)) return MDI_EINVAL;
    cost[(size_t)i] = nodes_cost(descs[i], P);
    all_real = all_real && descs[i].family != MDI_FAM_OSC;
  }
  // The hybrid schedule's launches order by the modelled time of a one-warp team
  // (which knows the passes per level and the FP64 sweep's Gaussian recurrence);
  // the rest by the estimated operations.
  const bool hybrid = all_real && cfg.block == 2 * kWarp && !cfg.stage;
  const bool fp64 = cfg.precision == MDI_PREC_FP64;
  std::vector<double> t1, t2;
  if (hybrid) {
    t1.resize((size_t)count);
    t2.resize((size_t)count);
    for (int32_t i = 0; i < count; ++i) {
      t1[(size_t)i] = team_time(descs[i], P, 1, fp64);
      t2[(size_t)i] = team_time(descs[i], P, 2, fp64);
      cost[(size_t)i] = t1[(size_t)i];
    }
  }
  std::vector<int32_t> idx((size_t)count);
  std::iota(idx.begin(), idx.end(), 0);
  // Longest processing time first; equal costs grouped by a, then by index.
  std::stable_sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) {
    if (cost[(size_t)x] != cost[(size_t)y]) return cost[(size_t)x] > cost[(size_t)y];
    return descs[x].a < descs[y].a;
  });
  std::memcpy(order, idx.data(), sizeof(int32_t) * (size_t)count);
  if (split) {
    *split = count;  // whole CTAs throughout unless the hybrid schedule applies and pays
    if (hybrid) {
      const int ctas = std::max(1, nodes_workers(cfg));
      double best = hybrid_makespan(t2, t1, idx, count, ctas);
      for (int k = 0; k < 40; ++k) {
        const int sp = (int)((int64_t)count * k / 40);
        const double m = hybrid_makespan(t2, t1, idx, sp, ctas);
        if (m < best) {
          best = m;
          *split = sp;
        }
      }
    }
  }
  return MDI_OK;
}

mdi_status mdi_midpoint_workspace_size(int32_t d, int64_t N, int64_t n_last, size_t *bytes) {
  if (!bytes || d < 1 || N < 1 || n_last < 1) return MDI_EINVAL;
  *bytes = midpoint_workspace_bytes(d, N, n_last);
  return *bytes ? MDI_OK : MDI_EINVAL;
}

mdi_status mdi_midpoint_integrate(int32_t family, int32_t d, int64_t N, int64_t n_last, const double *params,
                                  double *out, void *workspace, size_t ws_bytes, mdi_stream_t stream) {
  NvtxRange nvtx_scope("mdi_midpoint_integrate");
  if (!family_ok(family) || d < 1 || N < 1 || n_last < 1 || !params || !out) return MDI_EINVAL;
  return midpoint_launch(family, d, N, n_last, params, out, workspace, ws_bytes, (cudaStream_t)stream);
}

mdi_status lattice_korobov_search_workspace_size(int64_t n, size_t *bytes) {
  if (!bytes) return MDI_EINVAL;
  *bytes = korobov_workspace_bytes(n);
  return *bytes ? MDI_OK : MDI_EINVAL;
}

mdi_status lattice_korobov_search(int32_t alpha, int32_t d, int64_t n, int64_t a_first, int64_t count,
                                  double *values, int64_t *best_a, void *workspace, size_t ws_bytes,
                                  mdi_stream_t stream) {
  NvtxRange nvtx_scope("lattice_korobov_search");
  return korobov_search_launch(alpha, d, n, a_first, count, values, best_a, workspace, ws_bytes,
                               (cudaStream_t)stream);
}

mdi_status lattice_cbc_workspace_size(int64_t n, size_t *bytes) {
  if (!bytes) return MDI_EINVAL;
  *bytes = cbc_workspace_bytes(n);
  return *bytes ? MDI_OK : MDI_EINVAL;
}

mdi_status lattice_cbc(int32_t d, int64_t n, const double *gamma, double beta, int64_t *z, double *e2,
                       void *workspace, size_t ws_bytes, mdi_stream_t stream) {
  NvtxRange nvtx_scope("lattice_cbc");
  return cbc_launch(d, n, gamma, beta, z, e2, workspace, ws_bytes, (cudaStream_t)stream);
}

mdi_status mdi_midpoint_ridge_workspace_size(int32_t d, int64_t N, int64_t n_last, size_t *bytes) {
  if (!bytes) return MDI_EINVAL;
  *bytes = ridge_workspace_bytes(d, N, n_last);
  return *bytes ? MDI_OK : MDI_EINVAL;
}

mdi_status mdi_midpoint_ridge(int32_t d, int64_t N, int64_t n_last, double c0, double power, double *out,
                              void *workspace, size_t ws_bytes, mdi_stream_t stream) {
  NvtxRange nvtx_scope("mdi_midpoint_ridge");
  return ridge_launch(d, N, n_last, c0, power, out, workspace, ws_bytes, (cudaStream_t)stream);
}

mdi_status mdi_debug_fp64_phi(int32_t which, const double *x, double *y, int64_t n, mdi_stream_t stream) {
  if ((which != 0 && which != 1) || !x || !y || n < 1) return MDI_EINVAL;
  return fp64_phi_debug_launch(which, x, y, n, (cudaStream_t)stream);
}

mdi_status mdi_debug_lattice_indices(int32_t d, int64_t n, const int64_t *z, int64_t j0, int64_t count,
                                     int64_t *r_out, mdi_stream_t stream) {
  return lattice_indices_launch(d, n, z, j0, count, r_out, (cudaStream_t)stream);
}

}  // extern "C"
