// mdi_internal.h -- launchers behind the C ABI (one per kernel family).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "mdi_lr.h"

namespace mdi {

// slr.cu
size_t slr_workspace_bytes(int d, int64_t n);
mdi_status slr_launch(int family, int d, int64_t n, const int64_t *z, const double *params, int precision,
                      double *out, void *workspace, size_t ws_bytes, cudaStream_t stream);
mdi_status slr_launch_noalloc(int family, int d, int64_t n, const int64_t *z, const double *params, int precision,
                              double *out, cudaStream_t stream);
mdi_status lattice_indices_launch(int d, int64_t n, const int64_t *z, int64_t j0, int64_t count, int64_t *r_out,
                                  cudaStream_t stream);

// slr.cu: mean and standard error of shifted-rule replicates (Section 2.1)
mdi_status shifted_estimate_launch(const double *values, int R, double *mean_se, cudaStream_t stream);

// probe.cu: FMA throughput probe (measurement aid)
mdi_status peak_probe_launch(int kind, int iters, double *sink, cudaStream_t stream);
int64_t peak_probe_threads(int kind);

// mdi_exact.cu
size_t exact_workspace_bytes(int family, int d, int64_t a, int64_t n_last);
mdi_status exact_launch(int family, int d, int64_t a, int64_t n_last, const double *params, int precision,
                        double *out, void *workspace, size_t ws_bytes, cudaStream_t stream);

// mdi_closed.cu
size_t closed_workspace_bytes(int d, int64_t a, int64_t n_last);  // 0 when the sizes are out of range
mdi_status closed_launch(int family, int d, int64_t a, int64_t n_last, const double *params, int precision,
                         double *out, void *workspace, size_t ws_bytes, cudaStream_t stream);

// slr.cu: randomly shifted lattice rule, R replicates
size_t slr_shifted_workspace_bytes(int d, int64_t n, int R);  // 0 when out of range
size_t slr_improved_workspace_bytes(int d, int64_t n, int64_t a);  // 0 when out of range
mdi_status slr_improved_launch(int family, int d, int64_t n, int64_t a, const double *params, int precision,
                               double *out, int64_t *n_ghost, void *workspace, size_t ws_bytes, cudaStream_t stream);
mdi_status slr_shifted_launch(int family, int d, int64_t n, const int64_t *z, const double *params,
                              const double *shifts, int R, int precision, double *out, void *workspace,
                              size_t ws_bytes, cudaStream_t stream);

// mdi_ridge.cu: paper-table mode for (c0 + sum x_i)^(-p), histogram state
size_t ridge_workspace_bytes(int d, int64_t N, int64_t n_last);  // 0 when out of range
mdi_status ridge_launch(int d, int64_t N, int64_t n_last, double c0, double p, double *out, void *workspace,
                        size_t ws_bytes, cudaStream_t stream);

// lattice_search.cu
size_t korobov_workspace_bytes(int64_t n);  // 0 when n is out of range
mdi_status korobov_search_launch(int alpha, int d, int64_t n, int64_t a_first, int64_t count, double *values,
                                 int64_t *best_a, void *workspace, size_t ws_bytes, cudaStream_t stream);
size_t cbc_workspace_bytes(int64_t n);  // 0 when n is out of range
mdi_status cbc_launch(int d, int64_t n, const double *gamma, double beta, int64_t *z, double *e2, void *workspace,
                      size_t ws_bytes, cudaStream_t stream);

// Paper-table mode: tensor midpoint rule on the grid (N, ..., N, n_last).
size_t midpoint_workspace_bytes(int d, int64_t N, int64_t n_last);  // 0 when the sizes are out of range
mdi_status midpoint_launch(int family, int d, int64_t N, int64_t n_last, const double *params, double *out,
                           void *workspace, size_t ws_bytes, cudaStream_t stream);

size_t closed_grad_workspace_bytes(int d, int64_t a, int64_t n_last);
mdi_status closed_grad_launch(int family, int d, int64_t a, int64_t n_last, const double *params, double *value,
                              double *grad, void *workspace, size_t ws_bytes, cudaStream_t stream);

// mdi_nodes.cu
struct NodesConfig {
  int P;            // nodes per state
  int block;        // threads per CTA
  int ctas_per_sm;  // persistent CTAs per SM
  int precision;    // mdi_precision
  int stage;        // 1: stage each integral's basis table in shared memory; 0: read it through L1
  int step;         // m of Algorithm 1 (1, 2, 3)
};
NodesConfig nodes_config(const mdi_opts *opts);
size_t nodes_batched_workspace_bytes(int count, const NodesConfig &cfg);
mdi_status nodes_prepare(const NodesConfig &cfg, void *workspace, size_t ws_bytes, cudaStream_t stream);
mdi_status nodes_batched_launch(const mdi_batch_desc *descs, const int32_t *order, int count, int split,
                                const double *param_pool, int64_t pool_len, const NodesConfig &cfg, double *out,
                                void *workspace, size_t ws_bytes, cudaStream_t stream);
// Persistent CTAs one batched launch with this configuration keeps resident.
int nodes_workers(const NodesConfig &cfg);
// Device status word of a batched workspace (MDI_DEV_* flags): bytes needed to
// hold it, and a stream-ordered read (waits for the stream), optionally cleared.
size_t nodes_status_word_bytes();
mdi_status fp64_phi_debug_launch(int which, const double *x, double *y, int64_t n, cudaStream_t stream);
mdi_status nodes_read_status(const void *workspace, bool clear, uint32_t *word, cudaStream_t stream);
// Single integral through the batched machinery (descriptor built on the device).
size_t nodes_single_workspace_bytes(const NodesConfig &cfg);
mdi_status nodes_single_launch(int family, int d, int64_t a, int64_t n_last, const double *params,
                               const NodesConfig &cfg, double *out, void *workspace, size_t ws_bytes,
                               cudaStream_t stream);

// mdi_levels.cu: one integral, node state, parallel over levels (forward and adjoint)
size_t levels_workspace_bytes(int d, int64_t a, const NodesConfig &cfg, int checkpoint);
// Step size m = cfg.step > 1 (forward, FP64): 0 when a^m exceeds the table limit.
size_t levels_step_workspace_bytes(int d, int64_t a, const NodesConfig &cfg, int checkpoint);
mdi_status levels_launch(int family, int d, int64_t a, int64_t n_last, const double *params, const NodesConfig &cfg,
                         int checkpoint, double *value, double *grad, void *workspace, size_t ws_bytes,
                         cudaStream_t stream);

}  // namespace mdi
