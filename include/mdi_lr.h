/*
 * mdi_lr.h -- C ABI of the GB300 (sm_103a) MDI-LR library.
 *
 * The library evaluates rank-1 lattice rules for integrals over [0,1]^d
 * (Zhong & Feng, "An efficient implementation algorithm for quasi-Monte Carlo
 * approximations of high-dimensional integrals"):
 *   - lattice_rule_integrate: the standard lattice rule (SLR), eq. (1.2) with the
 *     points x_j = {j z / n} of eq. (2.1), every point generated and evaluated;
 *   - mdi_lr_integrate: the MDI-LR algorithm (Algorithm 2 calling Algorithm 1 with
 *     m = 1) on the Korobov lattice z = (1, a, ..., a^(d-1)) (Example 2) with
 *     n = n_last * a^(d-1) points, which the affine map of Theorem 3.1 turns into
 *     a tensor-product grid with a points on each transformed axis and n_last on
 *     the last (Lemma 3.2; no point has to be added, n* = 0).  For these n the
 *     MDI-LR value equals the SLR value on the same lattice.
 *
 * Integrands are product-form families f(x) = Re(C prod_j phi_j(x_j)):
 *   MDI_FAM_EXP    f = exp(sum_j c_j x_j)                 (Tests 2, 4, 7: f_1)
 *   MDI_FAM_OSC    f = cos(2 pi u + sum_j c_j x_j)         (Tests 5-7: cos(2 pi + 2 sum x))
 *   MDI_FAM_GAUSS  f = exp(-sum_j c_j^2 (x_j - w_j)^2)     (Tests 3, 5-7: Gaussian)
 *   MDI_FAM_PEAK   f = prod_j 1 / (c_j^-2 + (x_j - w_j)^2)  (Tests 4-7: product peak)
 * Parameters live in DEVICE memory as 2*d doubles: params[j] = c_j and
 * params[d + j] = w_j (j < d); for MDI_FAM_OSC params[d] = u and the rest of the
 * second half is ignored.
 *
 * Conventions for every call:
 *   - The caller owns all memory.  Device buffers (params, out, workspace) are
 *     plain device pointers (e.g. from a framework allocator); host arrays are read
 *     before the call returns.  The library allocates no device memory.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL means the legacy default
 *     stream) and the call returns without synchronising.  Results are valid once
 *     the stream reaches them.  Launch sequences contain no host synchronisation
 *     and no pageable copies, so they can be captured into a CUDA graph.
 *   - Scratch memory comes from `workspace` (device, 256-byte aligned, at least the
 *     size the matching *_workspace_size call returns).  Two calls that overlap on
 *     the GPU must not share a workspace.
 *   - Errors are returned as mdi_status.  Argument errors are detected on the host
 *     before anything is enqueued.  MDI_ECUDA means a launch was rejected by the
 *     CUDA runtime (the message is available from mdi_last_cuda_error()).
 */
#ifndef MDI_LR_H
#define MDI_LR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *mdi_stream_t; /* identical to cudaStream_t */

typedef enum {
  MDI_OK = 0,
  MDI_EINVAL = 1,        /* an argument is out of range or a pointer is NULL */
  MDI_EUNSUPPORTED = 2,  /* valid for the method, not provided by this library */
  MDI_EOVERFLOW = 3,     /* a lattice size does not fit the exact integer range */
  MDI_ECUDA = 4,         /* the CUDA runtime rejected a launch or copy */
  MDI_EWORKSPACE = 5     /* workspace NULL, misaligned or smaller than required */
} mdi_status;

typedef enum { MDI_FAM_EXP = 0, MDI_FAM_OSC = 1, MDI_FAM_GAUSS = 2, MDI_FAM_PEAK = 3 } mdi_family;

/* Representation of the level state ("symbolic function" g_{k-m} of eq. (4.4),
 * which the paper leaves unspecified):
 *   MDI_STATE_EXACT  the value at every parent the lattice needs, n a/(a-1)
 *                    evaluations in all; exact, exponential in d.
 *   MDI_STATE_CLOSED G_k(x) = K_k exp(beta_k x); exact, for EXP and OSC only.
 *   MDI_STATE_NODES  values at P Chebyshev points, read back by barycentric
 *                    interpolation; O(d a P^2), for every family.  A single
 *                    integral with d >= 8 runs level-parallel (every level's
 *                    P x P operator at once, then grouped products in FP64) in
 *                    every precision mode; d < 8 runs the levels in order in
 *                    one CTA.
 *   MDI_STATE_AUTO   CLOSED for EXP/OSC, NODES otherwise. */
typedef enum { MDI_STATE_AUTO = 0, MDI_STATE_EXACT = 1, MDI_STATE_CLOSED = 2, MDI_STATE_NODES = 3 } mdi_state;

/* Arithmetic of a call:
 *   MDI_PREC_FP64             every step in IEEE double.
 *   MDI_PREC_FP32_EVAL_FP64   integrand factors phi_j in float, everything else double.
 *   MDI_PREC_FP32_EVAL_DF32   phi_j in float; level contractions (interpolation and
 *                             the sum over the cluster) in double-float pairs of
 *                             floats; level states, cross-level products, the final
 *                             sum and coordinates in double (the batched node
 *                             state's real families keep their state as float
 *                             pairs, scaled by a power of two per level).
 *   In both single-precision-evaluation modes the batched node state's real
 *   families take phi_j at the float coordinate (q + xi_p)/a, so both modes give
 *   phi_j the same floats.
 *   MDI_PREC_DF64            FP64-class results without the FP64 pipe, for the
 *                             node state (batched kernel; single integrals, where
 *                             the level-parallel path keeps the products between
 *                             levels in FP64): coordinates, phi (own double-float exp
 *                             and reciprocal), interpolation and cluster sums in
 *                             double-float pairs of floats (about 48 significant
 *                             bits); FP64 only between levels and on the last
 *                             axis.  OSC keeps phi in FP64.  GB300 runs FP32 64x
 *                             faster than FP64.  The node state's values may leave
 *                             the float range (the state is kept scaled by powers
 *                             of two), but each factor phi_j must not: EXP needs
 *                             |c_j| <= 80, GAUSS c_j^2 (x - w_j)^2 <= 80 and PEAK
 *                             c_j <= 2^60 on [0, 1]; beyond that use MDI_PREC_FP64.  Closed state (forward): the
 *                             cluster sums of the exponential family in
 *                             double-float (own exp, Dot2 sums) on levels with
 *                             |gamma_k| <= 64, other levels and everything else
 *                             in FP64; a and
 *                             n_last below 2^31; OSC in FP64.  Other states and
 *                             gradients: MDI_EUNSUPPORTED. */
typedef enum {
  MDI_PREC_FP64 = 0,
  MDI_PREC_FP32_EVAL_FP64 = 1,
  MDI_PREC_FP32_EVAL_DF32 = 2,
  MDI_PREC_DF64 = 3
} mdi_precision;

typedef struct {
  int32_t state;       /* mdi_state */
  int32_t precision;   /* mdi_precision */
  int32_t nodes;       /* P for MDI_STATE_NODES, 2..32; 0 selects 16 */
  int32_t block;       /* threads per CTA for the node-state kernels (32..512, a
                          multiple of 32 and at least P); 0 selects the library
                          default */
  int32_t ctas_per_sm; /* resident CTAs per SM for persistent grids; 0 = default */
  int32_t checkpoint;  /* level-checkpoint interval of the adjoint; 0 = ceil(sqrt(d)) */
  int32_t table_in_l1; /* node-state kernels: 0 = stage each integral's basis table in
                          shared memory (when it fits 64 KiB), 1 = read it through L1
                          (less shared memory, more resident CTAs) */
  int32_t step;        /* m of Algorithm 1: transformed axes contracted per iteration,
                          0 or 1 (the paper's choice, m = 1), 2 or 3.  With the exact
                          and closed states every m gives the same sum; with the node
                          state, m > 1 reads the state once per m levels (Algorithm 1,
                          eq. 2.14c: the factors of the m axes multiplied over the
                          a^m digit tuples), for single integrals in FP64 with
                          a^m <= 4096, value (mdi_lr_integrate) and gradient
                          (mdi_lr_grad); other uses MDI_EUNSUPPORTED */
} mdi_opts;

/* ---------------------------------------------------------------------------
 * Standard lattice rule, eq. (1.2) with the rank-1 points of eq. (2.1).
 *   d        dimension, 1..256
 *   n        number of points, 1 <= n < 2^63
 *   z        HOST array of d generating-vector entries, 0 <= z_i < n (any vector;
 *            the paper's gcd(z_i, n) = 1 is not required)
 *   params   DEVICE, 2*d doubles (see above)
 *   precision MDI_PREC_FP64, MDI_PREC_FP32_EVAL_FP64, or MDI_PREC_DF64 (n <= 2^48:
 *            coordinates, integrand and per-thread sums in double-float pairs of
 *            floats from the exact integer numerators; a point whose value would
 *            leave the float range, and the OSC family, in FP64; larger n:
 *            MDI_EUNSUPPORTED)
 *   out      DEVICE, 1 double: Q = (1/n) sum_{j<n} f((j z mod n) / n)
 * Indices j z_i mod n are exact 64-bit integers; the sum is a fixed-order
 * (deterministic) FP64 reduction.
 * ------------------------------------------------------------------------- */
mdi_status lattice_rule_integrate(int32_t family, int32_t d, int64_t n, const int64_t *z,
                                  const double *params, int32_t precision, double *out,
                                  void *workspace, size_t ws_bytes, mdi_stream_t stream);
mdi_status lattice_rule_workspace_size(int32_t d, int64_t n, size_t *bytes);

/* Example 2's Korobov generating vector, z_i = a^(i-1) mod n for i = 1..d, in exact
 * integer arithmetic (128-bit products), written to z (HOST, d int64): the z that
 * lattice_rule_integrate and lattice_rule_integrate_shifted take for a Korobov
 * lattice.  Host only, nothing is enqueued.  MDI_EINVAL unless 1 <= d, 1 <= n < 2^63,
 * 0 <= a and z != NULL. */
mdi_status lattice_korobov_vector(int32_t d, int64_t a, int64_t n, int64_t *z);

/* lattice_rule_integrate without a workspace, for callers that cannot allocate
 * device memory when they call (for instance code inside an application that
 * reserves all GPU memory at start-up and forbids later allocation, or a plug-in
 * without access to its host's allocator).  The paper has no counterpart: this is
 * a packaging variant of the lattice rule above, with the same arguments minus
 * the workspace and the same result.
 *   - Scratch: a fixed 4096-slot (32 KiB) array of partial sums built into this
 *     library; every GPU that loads the library holds it until the process exits.
 *     A launch that would need more slots (GPUs with more than 512 SMs) returns
 *     MDI_EWORKSPACE.  Nothing is allocated or freed by the call.
 *   - Set-up: the first call on each device looks up the array's device address
 *     (with that device current); make that first call before any stream capture.
 *   - All calls share the array.  Each call overwrites every slot it reads, so no
 *     clearing is needed, but calls that overlap on the GPU (other streams, other
 *     host threads) race on it and must be serialised by the caller.
 *   - The looked-up address is kept for the life of the process: after a
 *     cudaDeviceReset on a device, this entry point must not be called on it
 *     again. */
mdi_status lattice_rule_integrate_noalloc(int32_t family, int32_t d, int64_t n, const int64_t *z,
                                          const double *params, int32_t precision, double *out,
                                          mdi_stream_t stream);

/* ---------------------------------------------------------------------------
 * Randomly shifted lattice rule (Section 2.1: P + Delta = {{t + Delta} : t in P}),
 * R shifts in one call:
 *     out[r] = (1/n) sum_{j<n} f({j z / n + Delta_r}),  r < R,
 * the replicates of the randomly shifted rule whose mean estimates the integral and
 * whose spread estimates its error (the mean square error over uniform shifts is
 * bounded by the shift-averaged worst-case error, eq. 2.12).
 *   shifts   DEVICE, R*d doubles, Delta_r = shifts[r*d .. r*d + d), each in [0, 1)
 *   out      DEVICE, R doubles
 *   R        1..65535
 *   precision MDI_PREC_FP64, or MDI_PREC_DF64 (n <= 2^48; the shifted coordinate
 *            {r/n + Delta} as a float pair, the rest as the plain rule's DF64 mode;
 *            OSC in FP64); others MDI_EUNSUPPORTED
 * Other arguments and the index arithmetic as lattice_rule_integrate.  Two
 * launches on `stream`.  MDI_EINVAL for bad sizes; MDI_EWORKSPACE for a missing,
 * misaligned or short workspace (lattice_rule_shifted_workspace_size).
 * ------------------------------------------------------------------------- */
mdi_status lattice_rule_integrate_shifted(int32_t family, int32_t d, int64_t n, const int64_t *z,
                                          const double *params, const double *shifts, int32_t R,
                                          int32_t precision, double *out, void *workspace, size_t ws_bytes,
                                          mdi_stream_t stream);
mdi_status lattice_rule_shifted_workspace_size(int32_t d, int64_t n, int32_t R, size_t *bytes);

/* The estimate of Section 2.1 from R replicates of the randomly shifted rule:
 *     mean_se[0] = (1/R) sum_r values[r],
 *     mean_se[1] = sqrt(sum_r (values[r] - mean)^2 / (R (R - 1)))   (0 for R = 1),
 * the integral's estimate and its standard error.  values and mean_se are DEVICE
 * pointers (R and 2 doubles); one single-CTA launch on `stream` with fixed-order
 * sums.  MDI_EINVAL unless 1 <= R <= 65535 and both pointers are non-NULL. */
mdi_status lattice_shifted_estimate(const double *values, int32_t R, double *mean_se, mdi_stream_t stream);

/* ---------------------------------------------------------------------------
 * Improved lattice rule (Definition 3.3, Section 2.2.2) for the Korobov vector
 * z = (1, a, ..., a^(d-1)) mod n and general n.  The transformed grid of
 * Theorem 3.1 has M = a^(d-1) lines of n_d = ceil(n / M) positions (eq. 3.5); the
 * n lattice points fill it except for n* = M n_d - n positions, one on each short
 * line.  Each is filled by the point that continues its line by one lattice step
 * z/n, not reduced mod 1 (so its last coordinate is >= 1):
 *     out = (sum_{j<n} f({j z / n}) + sum_{ghosts} f(x_g)) / (n + n*).
 * With a^(d-1) | n there are no ghosts and this is lattice_rule_integrate.
 *   d        1..64;  a >= 1 with a^(d-1) * ceil(n / a^(d-1)) < 2^62
 *   n        1 <= n < 2^62; gcd(a, n) = 1 unless a^(d-1) divides n
 *   params   DEVICE, the family's parameters as lattice_rule_integrate
 *   precision  mdi_precision, as lattice_rule_integrate (MDI_PREC_DF64: n <= 2^48);
 *            the n* ghosts take DF64 too when n + n* <= 2^48 and a <= 2^24 (real
 *            families), FP64 otherwise
 *   out      DEVICE, 1 double
 *   n_ghost  HOST, optional (may be NULL): receives n*
 * Three launches on `stream` (lattice points, ghosts, ordered sum).
 * MDI_EINVAL for bad sizes or a common factor of a and n with ghosts present;
 * MDI_EUNSUPPORTED for a precision the lattice points cannot take;
 * MDI_EWORKSPACE for a missing, misaligned or short workspace
 * (lattice_rule_improved_workspace_size).
 * ------------------------------------------------------------------------- */
mdi_status lattice_rule_integrate_improved(int32_t family, int32_t d, int64_t n, int64_t a, const double *params,
                                           int32_t precision, double *out, int64_t *n_ghost, void *workspace,
                                           size_t ws_bytes, mdi_stream_t stream);
mdi_status lattice_rule_improved_workspace_size(int32_t d, int64_t n, int64_t a, size_t *bytes);

/* ---------------------------------------------------------------------------
 * MDI-LR, Algorithm 2 (Section 4) with m = 1 on the Korobov lattice.  The
 * algorithm's inputs are f, Omega = [0,1]^d, d, the Korobov parameter a and n;
 * its generating vector is Example 2's z = (1, a, ..., a^(d-1)) mod n.
 *   d        dimension, >= 1 (EXACT: n <= 2^40; CLOSED: d <= 2^20; NODES: d <= 2^20)
 *   a        Korobov parameter = points per transformed axis 1..d-1, a >= 1
 *            (NODES: a <= 64, EXACT: a <= 4096)
 *   n_last   points on the last transformed axis (n_d of eq. (3.5)), >= 1;
 *            n = n_last * a^(d-1); Lemma 3.2's equal-N case is n_last = a
 *   z        HOST, d int64 entries, or NULL.  NULL means Example 2's Korobov vector
 *            for (a, n), which MDI-LR never forms (for large d, n exceeds every
 *            integer type; the sweep works on the digits of the transformed grid).
 *            A non-NULL z is checked against that vector: n must be below 2^63
 *            (MDI_EOVERFLOW otherwise: such a z cannot be written in int64), and
 *            z_i must equal a^(i-1) mod n for every i (MDI_EUNSUPPORTED otherwise:
 *            another vector needs the ghost points of Definition 3.3, see
 *            lattice_rule_integrate_improved, or the plain rule).
 *   params   DEVICE, 2*d doubles
 *   opts     HOST, may be NULL (all defaults)
 *   out      DEVICE, 1 double
 * ------------------------------------------------------------------------- */
mdi_status mdi_lr_integrate(int32_t family, int32_t d, int64_t a, int64_t n_last, const int64_t *z,
                            const double *params, const mdi_opts *opts, double *out,
                            void *workspace, size_t ws_bytes, mdi_stream_t stream);
mdi_status mdi_lr_workspace_size(int32_t family, int32_t d, int64_t a, int64_t n_last,
                                 const mdi_opts *opts, size_t *bytes);

/* ---------------------------------------------------------------------------
 * Derivative of the MDI-LR value with respect to the integrand parameters
 * (the adjoint sweep; the paper computes values only, this is an extension).
 *   grad     DEVICE, 2*d doubles: grad[j] = dQ/dc_j, grad[d+j] = dQ/dw_j; for
 *            MDI_FAM_EXP the w entries are 0, for MDI_FAM_OSC grad[d] = dQ/du and
 *            the rest of the second half is 0.  Q is the rule's own value, so this
 *            is the exact derivative of the computed number, not of the integral.
 *   value    DEVICE, 1 double, or NULL: receives Q as well.
 *   z        HOST or NULL, checked as for mdi_lr_integrate.
 *   opts     state CLOSED (EXP, OSC) or NODES (any family; AUTO picks as in
 *            mdi_lr_integrate); precision must be MDI_PREC_FP64.
 * CLOSED: the levels run in reverse as an affine recurrence, dQ/dc_k =
 * front * mu_k, mu_k = nu_k + mu_{k+1}/a, solved by a block-wide scan.
 * NODES (d <= 65536, a <= 64, n_last <= 4096): every level's P x P operator is
 * built in parallel, one CTA runs the forward and the reverse (adjoint) chains
 * keeping level states only every opts->checkpoint levels (0: ceil(sqrt(d))),
 * and the levels' contributions are then formed in parallel, each CTA taking a
 * block of consecutive levels of one checkpoint group and recomputing their
 * states once from the nearest checkpoints.  With opts->step = m > 1 the same
 * runs over the step-m operators (one per m axes), and each operator's m axes
 * take their derivatives by the product rule over the a^m digit tuples, which
 * are cut into slices on separate CTAs.
 * ------------------------------------------------------------------------- */
mdi_status mdi_lr_grad(int32_t family, int32_t d, int64_t a, int64_t n_last, const int64_t *z,
                       const double *params, const mdi_opts *opts, double *value, double *grad, void *workspace,
                       size_t ws_bytes, mdi_stream_t stream);
mdi_status mdi_lr_grad_workspace_size(int32_t family, int32_t d, int64_t a, int64_t n_last,
                                      const mdi_opts *opts, size_t *bytes);

/* ---------------------------------------------------------------------------
 * Many independent MDI-LR integrals in one launch sequence (node state for every
 * family, or closed state for EXP/OSC instances when opts->state is
 * MDI_STATE_AUTO).  One descriptor per integral:
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t family;       /* mdi_family */
  int32_t d;            /* 1..MDI_BATCH_MAX_D */
  int32_t a;            /* 1..64 */
  int32_t n_last;       /* 1..4096 */
  int64_t param_offset; /* index into param_pool of this integral's 2*d doubles */
  int64_t reserved;     /* must be 0 */
} mdi_batch_desc;       /* 32 bytes */

#define MDI_BATCH_MAX_D 65536

/* One-time set-up of a workspace for mdi_lr_integrate_batched: builds the
 * barycentric basis tables l_t((q + xi_p)/a) for a = 1..64 and the P of opts (they
 * depend on nothing else) and the paired table l_t +- l_{P-1-t} that the real
 * families' sweeps use (float pairs in the double-float modes, doubles
 * otherwise) -- and the constants every
 * integral shares (the Chebyshev nodes and weights, xi_p/a and 1/a as float
 * pairs, the 2^(j/256) table of the double-float exp), zeroes the work-queue
 * counters and stamps a tag naming opts->nodes and the table format of
 * opts->precision.  Enqueued on `stream`; a
 * prepared workspace serves any number of batched calls with the same nodes and
 * precision.  Call it again after a batched call failed to launch. */
mdi_status mdi_lr_batched_prepare(const mdi_opts *opts, void *workspace, size_t ws_bytes, mdi_stream_t stream);

/*   descs      DEVICE, count descriptors
 *   order      DEVICE, count int32 instance indices in the order CTAs should pick
 *              them up (from mdi_batch_plan), or NULL for 0..count-1
 *   count      number of integrals, >= 1
 *   split      hybrid schedule (from mdi_batch_plan): order slots below split are
 *              swept by whole CTAs, later ones by single warps, each with a state
 *              of its own (so the largest integrals, which come first, finish
 *              sooner, and the rest run at the lane efficiency of one warp).  It is
 *              honoured with 64-thread CTAs (opts->block = 64) and the tables read
 *              through L1 (opts->table_in_l1 = 1), and treated as count otherwise;
 *              split >= count means whole CTAs throughout.  An oscillatory integral
 *              past the split is rejected (NaN, MDI_DEV_BAD_DESC)
 *   param_pool DEVICE doubles
 *   pool_len   number of doubles in param_pool: descriptor i reads
 *              param_pool[param_offset, param_offset + 2 d), which must lie inside it
 *   out        DEVICE, count doubles; out[i] belongs to descs[i]
 *   workspace  prepared by mdi_lr_batched_prepare with the same nodes/precision
 * One kernel launch: a persistent grid of CTAs takes integrals from an atomic
 * counter in the workspace; the last CTA to finish re-arms the counter.  The
 * descriptors live in device memory, so the host cannot check them: the kernel
 * does.  A descriptor outside the limits above, or whose parameters leave the
 * pool, yields NaN in its output and sets a flag in the workspace's device status
 * word; an order entry outside 0..count-1 is skipped (that entry only) and flagged;
 * an unprepared workspace yields NaN everywhere and is flagged.  Read and clear the
 * flags with mdi_get_device_status. */
mdi_status mdi_lr_integrate_batched(const mdi_batch_desc *descs, const int32_t *order, int32_t count,
                                    int32_t split, const double *param_pool, int64_t pool_len, const mdi_opts *opts,
                                    double *out, void *workspace, size_t ws_bytes, mdi_stream_t stream);
mdi_status mdi_lr_batched_workspace_size(int32_t count, const mdi_opts *opts, size_t *bytes);

/* Host-side scheduler: writes into order (HOST, count int32) a processing order
 * for mdi_lr_integrate_batched -- longest estimated work first, ties grouped by a
 * so that consecutive pick-ups share their interpolation table -- and into *split
 * (HOST, may be NULL) the hybrid schedule's split for these opts: for batches of
 * real families with opts->block = 64 and tables through L1 the work is a
 * modelled time per integral for one- and two-warp teams (passes per level, the
 * precision's phi), the order is by the one-warp time, and the planner simulates
 * the persistent launch (the resident CTAs of this GPU taking the order) for 41
 * splits and keeps the shortest; otherwise the work is an operation count and
 * the split is count.  descs is a HOST copy of the descriptor table;
 * pool_len the number of doubles of the parameter pool the batch will read.
 * Returns MDI_EINVAL on an invalid descriptor or one whose 2*d parameters leave
 * the pool. */
mdi_status mdi_batch_plan(const mdi_batch_desc *descs, int32_t count, int64_t pool_len, const mdi_opts *opts,
                          int32_t *order, int32_t *split);

/* Flags of the device status word of a batched workspace (bitwise OR). */
#define MDI_DEV_BAD_DESC 1u    /* a descriptor outside the limits (its output is NaN) */
#define MDI_DEV_BAD_ORDER 2u   /* an order entry outside 0..count-1 (skipped) */
#define MDI_DEV_UNPREPARED 4u  /* the workspace was not prepared for these opts (NaN) */
#define MDI_DEV_POOL_RANGE 8u  /* a descriptor's parameters leave the pool (NaN) */

/* Reads the device status word of a workspace prepared by mdi_lr_batched_prepare:
 * enqueues a 4-byte device-to-host copy on `stream` and waits for the stream (this
 * call, unlike the compute calls, synchronises, so it cannot be captured in a CUDA
 * graph).  With clear != 0 the word is zeroed afterwards, in stream order.
 *   flags   HOST, may be NULL: receives the MDI_DEV_* bits seen since the
 *           preparation or the last clear
 * Returns MDI_OK when no flag is set, MDI_EINVAL when one is (or for a NULL,
 * misaligned or short workspace), MDI_ECUDA if the copy fails. */
mdi_status mdi_get_device_status(const void *workspace, size_t ws_bytes, int32_t clear, uint32_t *flags,
                                 mdi_stream_t stream);

/* ---------------------------------------------------------------------------
 * Paper-table mode for the ridge integrand f(x) = (c0 + sum_i x_i)^(-power) of
 * Test 7 (f_6: c0 = 1, power = d + 1) on the same midpoint grid (n_1 = ... =
 * n_{d-1} = N, n_d = n_last), by the dimension iteration of Algorithm 1 with m = 1:
 * after i axes the symbolic function depends only on the digit sum
 * S = k_1 + ... + k_i, so its state is the weight H_i[S] of each sum,
 * H_i[S] = (1/N) sum_{k<N} H_{i-1}[S - k]; then
 *     Q = sum_S H_{d-1}[S] (1/n_last) sum_{k<n_last} f at (S + (d-1)/2)/N + (k + 1/2)/n_last.
 *   out        DEVICE, one double
 *   workspace  DEVICE, >= mdi_midpoint_ridge_workspace_size bytes, 256-byte aligned
 * Three launches on `stream`, FP64: the d - 1 levels in one thread-block cluster
 * (the histogram split over its CTAs' shared memory, halos exchanged and a
 * cluster barrier every K <= 8 levels; d + 1 plain launches instead when the
 * histogram does not fit), every (S, k)
 * pair of the last axis, and the sum of the partials.  MDI_EINVAL unless d, N,
 * n_last >= 1, c0 > 0 and power finite, (d-1)(N-1) + 1 <= 2^26 and
 * ((d-1)(N-1) + 1) n_last <= 2^62; MDI_EWORKSPACE for a bad workspace.  f_6's integral is 1/(d+1)!, which leaves the double range near
 * d = 170.
 * ------------------------------------------------------------------------- */
mdi_status mdi_midpoint_ridge(int32_t d, int64_t N, int64_t n_last, double c0, double power, double *out,
                              void *workspace, size_t ws_bytes, mdi_stream_t stream);
mdi_status mdi_midpoint_ridge_workspace_size(int32_t d, int64_t N, int64_t n_last, size_t *bytes);

/* ---------------------------------------------------------------------------
 * Generating-vector construction (Section 2.2), FP64.
 *
 * Korobov search, Example 2: for a = a_first .. a_first + count - 1,
 *     values[t] = P_alpha(z(a)) = -1 + (1/n) sum_{k<n} prod_{j<d} (1 + C B_alpha({k a^j / n})),
 * the finite form of eq. (2.4), C = (-1)^(alpha/2+1) (2 pi)^alpha / alpha!,
 * alpha = 2 (B_2 = x^2 - x + 1/6) or 4 (B_4 = x^4 - 2x^3 + x^2 - 1/30).  A candidate
 * with a < 1, a >= n or gcd(a, n) > 1 is not admissible: +inf.  best_a[0] = the
 * smallest a attaining the least value (0 if none is admissible).  P_alpha is the
 * same for a and n - a, and for a and its inverse mod n.
 *   values     DEVICE, count doubles;  best_a  DEVICE, one int64
 *   workspace  DEVICE, >= lattice_korobov_search_workspace_size(n) bytes, 256-byte
 *              aligned (for n <= 2^24 and d <= 16 a table of the factors
 *              1 + C B_alpha(r/n), r <= n/2, as float pairs; the terms are then
 *              double-float products of table entries)
 * Two or three launches on `stream`.  MDI_EINVAL unless alpha is 2 or 4,
 * 1 <= d <= 256, 1 <= n <= 2^62, a_first >= 0 and count >= 1; MDI_EWORKSPACE for a
 * bad workspace.  Work: count * n * d / 2.
 * ------------------------------------------------------------------------- */
mdi_status lattice_korobov_search(int32_t alpha, int32_t d, int64_t n, int64_t a_first, int64_t count,
                                  double *values, int64_t *best_a, void *workspace, size_t ws_bytes,
                                  mdi_stream_t stream);
mdi_status lattice_korobov_search_workspace_size(int64_t n, size_t *bytes);

/* Component-by-component construction, Example 3, with product weights: z[0] = 1
 * and, for s = 1..d-1, z[s] = the z in {1 <= z <= n-1, gcd(z, n) = 1} minimising the
 * (s+1)-dimensional squared shift-averaged worst-case error of eq. (2.12),
 *     -prod_j (1 + gamma_j beta) + (1/n) sum_{k<n} prod_j (1 + gamma_j [B_2({k z_j/n}) + beta]),
 * with the earlier components held fixed; e2[s] = that minimum (e2[0]: z_1 = 1
 * alone).  beta = 0 for the unanchored weighted Sobolev space, c^2 - c + 1/3 for the
 * one anchored at c (Remark after eq. 2.12).  The error of n - z equals that of z;
 * the search takes z <= n/2 and, among equal values, the smallest z.
 *   gamma      DEVICE, d doubles;  z  DEVICE, d int64;  e2  DEVICE, d doubles
 *   workspace  DEVICE, >= lattice_cbc_workspace_size(n) bytes, 256-byte aligned
 * About 4d launches on `stream`, no host synchronisation; each component's factors
 * 1 + gamma_s (B_2(r/n) + beta), r <= n/2, are tabulated as float pairs and the
 * running products kept as float pairs (double-float arithmetic).  MDI_EINVAL
 * unless d >= 1, 2 <= n <= 2^24 and beta is finite; MDI_EWORKSPACE for a bad
 * workspace.  Work: d * n^2 / 4.
 * ------------------------------------------------------------------------- */
mdi_status lattice_cbc(int32_t d, int64_t n, const double *gamma, double beta, int64_t *z, double *e2,
                       void *workspace, size_t ws_bytes, mdi_stream_t stream);
mdi_status lattice_cbc_workspace_size(int64_t n, size_t *bytes);

/* ---------------------------------------------------------------------------
 * Paper-table mode: the tensor midpoint rule on the grid of eq. (3.5),
 *     Q = Re(front * prod_{i=1}^{d} (1/n_i) sum_{k<n_i} phi_i((k + 1/2)/n_i)),
 * n_1 = ... = n_{d-1} = N, n_d = n_last, front = exp(2 pi i u) for OSC.  This is
 * the rule whose relative errors the MDI-LR columns of Section 5 (Tables 2-1 to
 * 3-3) print, with n_last = N or N + 1; the text's reading of MDI-LR (the
 * transformed-lattice sum) is mdi_lr_integrate.  FP64.
 *   family     EXP, OSC, GAUSS or PEAK (params as for mdi_lr_integrate)
 *   params     DEVICE, 2*d doubles
 *   out        DEVICE, one double
 *   workspace  DEVICE, >= mdi_midpoint_workspace_size bytes, 256-byte aligned
 * Three launches on `stream` (per-axis chunk sums across the GPU, per-axis
 * reduction in chunk order, one fixed-tree product); no allocation.
 * MDI_EINVAL for a bad family, d < 1, N < 1, n_last < 1 or a grid whose chunk
 * count exceeds 2^30; MDI_EWORKSPACE for a missing, misaligned or short
 * workspace.
 * ------------------------------------------------------------------------- */
mdi_status mdi_midpoint_integrate(int32_t family, int32_t d, int64_t N, int64_t n_last, const double *params,
                                  double *out, void *workspace, size_t ws_bytes, mdi_stream_t stream);
mdi_status mdi_midpoint_workspace_size(int32_t d, int64_t N, int64_t n_last, size_t *bytes);

/* ---------------------------------------------------------------------------
 * Bit-exact view of the on-the-fly index generator used by the lattice kernel:
 * r_out[t*d + i] = (j0 + t) z_i mod n for t < count (DEVICE, count*d int64),
 * produced by the same incremental exact arithmetic the kernel uses.
 * ------------------------------------------------------------------------- */
mdi_status mdi_debug_lattice_indices(int32_t d, int64_t n, const int64_t *z, int64_t j0,
                                     int64_t count, int64_t *r_out, mdi_stream_t stream);

/* ---------------------------------------------------------------------------
 * Measurement aid (the paper has no counterpart): a dependency-free fused
 * multiply-add loop that keeps one arithmetic pipe busy, so that a benchmark can
 * measure the pipe's throughput on the running GPU and clock.
 *   kind   0: FP64 (DFMA), 1: FP32 (FFMA)
 *   iters  loop trips per thread, 1..2^20; each trip issues 16 independent FMAs
 *   sink   DEVICE, one double; written only if the chains' sum hits a value it
 *          never reaches, a condition the compiler cannot decide, so every FMA
 *          must run
 * One launch of mdi_peak_probe_threads(kind) threads on `stream`, each doing
 * 16 * iters FMAs, i.e. 32 * iters flops per thread.  MDI_EINVAL for a bad kind,
 * iters or sink.
 * ------------------------------------------------------------------------- */
mdi_status mdi_peak_probe(int32_t kind, int32_t iters, double *sink, mdi_stream_t stream);
/* Threads one mdi_peak_probe launch runs on the current device (0 for a bad kind). */
int64_t mdi_peak_probe_threads(int32_t kind);

/* Test hook (the paper has no counterpart): y[i] = the FP64 batched node-state
 * sweep's own exp(x[i]) (which = 0: Tang's table-driven method) or 1/x[i]
 * (which = 1: float seed and one cubic Newton-Raphson step; x[i] > 0), so tests can
 * hold them to CUDA's exp and IEEE division.  x, y: DEVICE, n doubles.  One
 * launch on `stream`; MDI_EINVAL for a bad `which`, pointer or n < 1. */
mdi_status mdi_debug_fp64_phi(int32_t which, const double *x, double *y, int64_t n, mdi_stream_t stream);

const char *mdi_status_string(mdi_status status);
/* Text of the last CUDA error seen by this library on the calling host thread. */
const char *mdi_last_cuda_error(void);
/* ABI version of this header (bumped on any incompatible change). */
int32_t mdi_abi_version(void);
#define MDI_ABI_VERSION 2

#ifdef __cplusplus
}
#endif
#endif /* MDI_LR_H */
