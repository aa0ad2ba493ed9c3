"""GB300 (sm_103a) MDI-LR: fast rank-1 lattice rules for high-dimensional integrals.

Thin Python binding of the C ABI in ``include/mdi_lr.h`` (same names).  Every
step of the computation runs in the CUDA kernels of ``libmdilr.so``; this module
only marshals arguments: it takes torch tensors for device memory, passes their
pointers and torch's current CUDA stream, and allocates workspaces through torch.

The method is that of Zhong & Feng: the standard lattice rule (eq. (1.2) over the
points of eq. (2.1)) and its fast evaluation MDI-LR (Algorithm 2 calling
Algorithm 1 with m = 1) on the Korobov lattice z = (1, a, ..., a^(d-1)) with
n = n_last * a^(d-1) points.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import _ffi
from ._ffi import BATCH_DESC_DTYPE, FAMILY, PRECISION, STATE, MdiError, MdiOpts

__all__ = [
    "lattice_rule_integrate", "lattice_rule_workspace_size", "lattice_rule_integrate_noalloc", "mdi_lr_integrate", "mdi_lr_workspace_size",
    "mdi_lr_integrate_batched", "mdi_lr_batched_workspace_size", "mdi_lr_batched_prepare", "mdi_batch_plan", "mdi_debug_lattice_indices",
    "mdi_lr_grad", "mdi_lr_grad_workspace_size", "MDILR", "mdi_lr", "make_batch_descs", "MdiError", "FAMILY", "STATE", "PRECISION", "BATCH_DESC_DTYPE", "library_path",
    "mdi_midpoint_integrate", "mdi_midpoint_workspace_size", "mdi_midpoint_ridge", "lattice_korobov_search", "lattice_cbc",
    "lattice_cbc_workspace_size", "lattice_korobov_search_workspace_size", "lattice_rule_integrate_shifted", "lattice_rule_shifted_workspace_size",
    "lattice_rule_integrate_improved", "lattice_rule_improved_workspace_size", "korobov_vector",
    "shifted_estimate", "mdi_get_device_status", "mdi_peak_probe", "mdi_peak_probe_threads",
]


def library_path() -> str:
    return _ffi.LIB_PATH


def _fam(f) -> int:
    return FAMILY[f] if isinstance(f, str) else int(f)


def _prec(p) -> int:
    return PRECISION[p] if isinstance(p, str) else int(p)


def _state(s) -> int:
    return STATE[s] if isinstance(s, str) else int(s)


def _stream(stream) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev_f64(t: torch.Tensor, name: str) -> torch.Tensor:
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    return t


def _opts(state="auto", precision="fp64", nodes=0, block=0, ctas_per_sm=0, checkpoint=0, table_in_l1=0,
          step=0) -> MdiOpts:
    o = MdiOpts()
    o.state, o.precision, o.nodes, o.block = _state(state), _prec(precision), int(nodes), int(block)
    o.ctas_per_sm, o.checkpoint, o.table_in_l1 = int(ctas_per_sm), int(checkpoint), int(bool(table_in_l1))
    o.step = int(step)
    return o


def _workspace(nbytes: int, device, workspace: Optional[torch.Tensor]) -> torch.Tensor:
    if workspace is not None:
        if workspace.numel() * workspace.element_size() < nbytes:
            raise ValueError(f"workspace too small: need {nbytes} bytes")
        return workspace
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


# ---------------------------------------------------------------------------
# Standard lattice rule
# ---------------------------------------------------------------------------
def lattice_rule_workspace_size(d: int, n: int) -> int:
    b = ctypes.c_size_t()
    _ffi.check(_ffi.load().lattice_rule_workspace_size(d, n, ctypes.byref(b)), "lattice_rule_workspace_size")
    return b.value


def lattice_rule_integrate(family, params: torch.Tensor, n: int, z: Sequence[int], precision="fp64",
                           out: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None,
                           stream=None) -> torch.Tensor:
    """Q = (1/n) sum_{j<n} f({j z / n}) on the GPU; ``params`` holds 2*d doubles
    (c then w; for "osc" params[d] = u).  Returns a 1-element float64 CUDA tensor."""
    _dev_f64(params, "params")
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.int64))
    d = int(zz.size)
    if params.numel() < 2 * d:
        raise ValueError("params must hold 2*d doubles")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=params.device)
    ws = _workspace(lattice_rule_workspace_size(d, n), params.device, workspace)
    st = _ffi.load().lattice_rule_integrate(_fam(family), d, int(n), zz.ctypes.data_as(ctypes.c_void_p),
                                            ctypes.c_void_p(params.data_ptr()), _prec(precision),
                                            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                            ws.numel(), _stream(stream))
    _ffi.check(st, "lattice_rule_integrate")
    return out


def lattice_rule_shifted_workspace_size(d: int, n: int, R: int) -> int:
    b = ctypes.c_size_t()
    _ffi.check(_ffi.load().lattice_rule_shifted_workspace_size(d, n, R, ctypes.byref(b)),
               "lattice_rule_shifted_workspace_size")
    return b.value


def lattice_rule_integrate_shifted(family, params: torch.Tensor, n: int, z: Sequence[int], shifts: torch.Tensor,
                                   out: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None,
                                   stream=None, precision="fp64") -> torch.Tensor:
    """R replicates of the randomly shifted rule, (1/n) sum_j f({j z/n + Delta_r}):
    ``shifts`` is an (R, d) float64 CUDA tensor of shifts in [0, 1).  Returns R values."""
    _dev_f64(params, "params")
    _dev_f64(shifts, "shifts")
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.int64))
    d = int(zz.size)
    if params.numel() < 2 * d or shifts.dim() != 2 or shifts.shape[1] != d:
        raise ValueError("params must hold 2*d doubles and shifts must be (R, d)")
    R = int(shifts.shape[0])
    if out is None:
        out = torch.empty(R, dtype=torch.float64, device=params.device)
    ws = _workspace(lattice_rule_shifted_workspace_size(d, n, R), params.device, workspace)
    st = _ffi.load().lattice_rule_integrate_shifted(_fam(family), d, int(n), zz.ctypes.data_as(ctypes.c_void_p),
                                                    ctypes.c_void_p(params.data_ptr()),
                                                    ctypes.c_void_p(shifts.data_ptr()), R, _prec(precision),
                                                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                                    ws.numel(), _stream(stream))
    _ffi.check(st, "lattice_rule_integrate_shifted")
    return out


def korobov_vector(d: int, a: int, n: int) -> np.ndarray:
    """The Korobov generating vector of Example 2, z_j = a^(j-1) mod n (j = 1..d),
    from the library's exact integer routine: the z argument of the lattice-rule
    calls (int64 numpy array)."""
    z = np.zeros(int(d), dtype=np.int64)
    _ffi.check(_ffi.load().lattice_korobov_vector(int(d), int(a), int(n), z.ctypes.data_as(ctypes.c_void_p)),
               "lattice_korobov_vector")
    return z


def lattice_rule_improved_workspace_size(d: int, n: int, a: int) -> int:
    b = ctypes.c_size_t()
    _ffi.check(_ffi.load().lattice_rule_improved_workspace_size(d, int(n), int(a), ctypes.byref(b)),
               "lattice_rule_improved_workspace_size")
    return b.value


def lattice_rule_integrate_improved(family, params: torch.Tensor, d: int, n: int, a: int, precision="fp64",
                                    out: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None,
                                    stream=None):
    """Improved lattice rule (Definition 3.3) on the Korobov lattice z = (1, a, ..)
    for general n: the n lattice points plus the n* points completing the
    transformed tensor grid, weight 1/(n + n*).  ``precision``: "fp64",
    "fp32_eval_fp64" (the lattice points; ghosts in FP64) or "df64" (both, where
    the ghosts' coordinates fit float pairs; see the C header).
    Returns (1-element float64 CUDA tensor, n*)."""
    _dev_f64(params, "params")
    if params.numel() < 2 * d:
        raise ValueError("params must hold 2*d doubles")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=params.device)
    ws = _workspace(lattice_rule_improved_workspace_size(d, n, a), params.device, workspace)
    ng = ctypes.c_int64()
    st = _ffi.load().lattice_rule_integrate_improved(_fam(family), d, int(n), int(a),
                                                     ctypes.c_void_p(params.data_ptr()), _prec(precision),
                                                     ctypes.c_void_p(out.data_ptr()), ctypes.byref(ng),
                                                     ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream))
    _ffi.check(st, "lattice_rule_integrate_improved")
    return out, ng.value


def shifted_estimate(values: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None):
    """(mean, standard error) of R shifted-rule replicates (a float64 CUDA tensor),
    computed on the device by the library: the estimate of the integral and of its
    error.  Returns two 0-dim views of one 2-element float64 CUDA tensor."""
    _dev_f64(values, "values")
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device=values.device)
    _ffi.check(_ffi.load().lattice_shifted_estimate(ctypes.c_void_p(values.data_ptr()), int(values.numel()),
                                                    ctypes.c_void_p(out.data_ptr()), _stream(stream)),
               "lattice_shifted_estimate")
    return out[0], out[1]


def lattice_rule_integrate_noalloc(family, params: torch.Tensor, n: int, z: Sequence[int], precision="fp64",
                                   out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """The lattice rule through the C entry point that takes no workspace: for
    callers that cannot allocate device memory at call time.  Its scratch is a
    fixed array inside the library shared by all calls, so calls that overlap on
    the GPU race; the first call on a device should precede any stream capture.
    ``out`` must be supplied by such callers (it is only allocated here when
    omitted, for convenience)."""
    _dev_f64(params, "params")
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.int64))
    d = int(zz.size)
    if params.numel() < 2 * d:
        raise ValueError("params must hold 2*d doubles")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=params.device)
    st = _ffi.load().lattice_rule_integrate_noalloc(_fam(family), d, int(n), zz.ctypes.data_as(ctypes.c_void_p),
                                                    ctypes.c_void_p(params.data_ptr()), _prec(precision),
                                                    ctypes.c_void_p(out.data_ptr()), _stream(stream))
    _ffi.check(st, "lattice_rule_integrate_noalloc")
    return out


# ---------------------------------------------------------------------------
# MDI-LR, one integral
# ---------------------------------------------------------------------------
def mdi_lr_workspace_size(family, d: int, a: int, n_last: int, **opts) -> int:
    b = ctypes.c_size_t()
    o = _opts(**opts)
    _ffi.check(_ffi.load().mdi_lr_workspace_size(_fam(family), d, a, n_last, ctypes.byref(o), ctypes.byref(b)),
               "mdi_lr_workspace_size")
    return b.value


def _host_z(z):
    """(keep-alive array, pointer) of an optional host generating vector."""
    if z is None:
        return None, ctypes.c_void_p(0)
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.int64))
    return zz, zz.ctypes.data_as(ctypes.c_void_p)


def mdi_lr_integrate(family, params: torch.Tensor, d: int, a: int, n_last: Optional[int] = None,
                     out: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None, stream=None,
                     z: Optional[Sequence[int]] = None, **opts) -> torch.Tensor:
    """MDI-LR value on the Korobov lattice with a points per transformed axis and
    n_last (default a) on the last one; ``z`` (optional) is Algorithm 2's
    generating vector, which must be Example 2's Korobov vector for (a, n); opts:
    state, precision, nodes, block, ctas_per_sm, checkpoint, step (Algorithm 1's m).
    Returns a 1-element float64 CUDA tensor."""
    _dev_f64(params, "params")
    n_last = a if n_last is None else n_last
    if params.numel() < 2 * d:
        raise ValueError("params must hold 2*d doubles")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=params.device)
    o = _opts(**opts)
    zz, zp = _host_z(z)
    ws = _workspace(mdi_lr_workspace_size(family, d, a, n_last, **opts), params.device, workspace)
    st = _ffi.load().mdi_lr_integrate(_fam(family), d, a, n_last, zp, ctypes.c_void_p(params.data_ptr()),
                                      ctypes.byref(o), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream))
    _ffi.check(st, "mdi_lr_integrate")
    return out


def mdi_lr_grad_workspace_size(family, d: int, a: int, n_last: int, **opts) -> int:
    b = ctypes.c_size_t()
    o = _opts(**opts)
    _ffi.check(_ffi.load().mdi_lr_grad_workspace_size(_fam(family), d, a, n_last, ctypes.byref(o), ctypes.byref(b)),
               "mdi_lr_grad_workspace_size")
    return b.value


def mdi_lr_grad(family, params: torch.Tensor, d: int, a: int, n_last: Optional[int] = None,
                value: Optional[torch.Tensor] = None, grad: Optional[torch.Tensor] = None,
                workspace: Optional[torch.Tensor] = None, stream=None, z: Optional[Sequence[int]] = None, **opts):
    """(value, grad): the MDI-LR value and its derivative with respect to the 2*d
    parameters, from the adjoint sweep on the GPU (FP64).  opts: state
    ("auto", "closed", "nodes"), nodes, checkpoint."""
    _dev_f64(params, "params")
    n_last = a if n_last is None else n_last
    if value is None:
        value = torch.empty(1, dtype=torch.float64, device=params.device)
    if grad is None:
        grad = torch.empty(2 * d, dtype=torch.float64, device=params.device)
    o = _opts(**opts)
    zz, zp = _host_z(z)
    ws = _workspace(mdi_lr_grad_workspace_size(family, d, a, n_last, **opts), params.device, workspace)
    st = _ffi.load().mdi_lr_grad(_fam(family), d, a, n_last, zp, ctypes.c_void_p(params.data_ptr()), ctypes.byref(o),
                                 ctypes.c_void_p(value.data_ptr()), ctypes.c_void_p(grad.data_ptr()),
                                 ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream))
    _ffi.check(st, "mdi_lr_grad")
    return value, grad


class MDILR(torch.autograd.Function):
    """Differentiable MDI-LR value.  When the parameters need a gradient and the
    call is in FP64 (the adjoint's arithmetic), the forward pass runs the adjoint
    call itself -- one sweep forward with checkpoints, the levels in reverse,
    states recomputed from the checkpoints -- which returns the value and dQ/dtheta
    together, and keeps only the 2d-long gradient; the backward pass scales it by
    the incoming gradient.  Otherwise the forward pass runs the plain sweep and the
    backward pass the adjoint call."""

    @staticmethod
    def forward(ctx, params, family, d, a, n_last, opts):
        ctx.meta = (family, d, a, n_last, dict(opts))
        p = params.detach().contiguous()
        if ctx.needs_input_grad[0] and opts.get("precision", "fp64") == "fp64":
            value, g = mdi_lr_grad(family, p, d, a, n_last, **opts)
            ctx.save_for_backward(g)
            ctx.fused = True
            return value.reshape(())
        ctx.save_for_backward(params)
        ctx.fused = False
        return mdi_lr_integrate(family, p, d, a, n_last, **opts).reshape(())

    @staticmethod
    def backward(ctx, grad_out):
        (saved,) = ctx.saved_tensors
        if ctx.fused:
            return saved * grad_out, None, None, None, None, None
        family, d, a, n_last, opts = ctx.meta
        opts = {k: v for k, v in opts.items() if k != "precision"}
        _, g = mdi_lr_grad(family, saved.detach().contiguous(), d, a, n_last, **opts)
        return g * grad_out, None, None, None, None, None


def mdi_lr(family, params: torch.Tensor, d: int, a: int, n_last: Optional[int] = None, **opts) -> torch.Tensor:
    """MDI-LR value as a 0-dim tensor that autograd can differentiate with respect
    to ``params`` (2*d float64 on the GPU)."""
    return MDILR.apply(params, family, d, a, a if n_last is None else n_last, opts)


# ---------------------------------------------------------------------------
# Batched MDI-LR
# ---------------------------------------------------------------------------
def make_batch_descs(families, ds, as_, n_lasts, param_offsets) -> np.ndarray:
    """Host descriptor table (numpy structured array laid out as mdi_batch_desc)."""
    n = len(ds)
    descs = np.zeros(n, dtype=BATCH_DESC_DTYPE)
    descs["family"] = [_fam(f) for f in families]
    descs["d"], descs["a"], descs["n_last"] = ds, as_, n_lasts
    descs["param_offset"] = param_offsets
    return descs


def mdi_batch_plan(descs: np.ndarray, pool_len: int, **opts):
    """(order, split): the library's host scheduler -- longest-first processing
    order and the hybrid schedule's split for these opts (count when whole CTAs
    are kept throughout); ``pool_len``: doubles in the parameter pool the batch
    reads."""
    descs = np.ascontiguousarray(descs, dtype=BATCH_DESC_DTYPE)
    order = np.zeros(descs.size, dtype=np.int32)
    split = ctypes.c_int32(0)
    o = _opts(**opts)
    _ffi.check(_ffi.load().mdi_batch_plan(descs.ctypes.data_as(ctypes.c_void_p), descs.size, int(pool_len),
                                          ctypes.byref(o), order.ctypes.data_as(ctypes.c_void_p),
                                          ctypes.byref(split)), "mdi_batch_plan")
    return order, int(split.value)


def mdi_lr_batched_workspace_size(count: int, **opts) -> int:
    b = ctypes.c_size_t()
    o = _opts(**opts)
    _ffi.check(_ffi.load().mdi_lr_batched_workspace_size(count, ctypes.byref(o), ctypes.byref(b)),
               "mdi_lr_batched_workspace_size")
    return b.value


def mdi_lr_batched_prepare(workspace: Optional[torch.Tensor] = None, device="cuda", stream=None,
                           **opts) -> torch.Tensor:
    """Returns a workspace prepared for batched calls with these opts (basis
    tables built, queue armed).  Reuse it for every call with the same opts."""
    ws = _workspace(mdi_lr_batched_workspace_size(1, **opts), device, workspace)
    o = _opts(**opts)
    _ffi.check(_ffi.load().mdi_lr_batched_prepare(ctypes.byref(o), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                                  _stream(stream)), "mdi_lr_batched_prepare")
    return ws


def mdi_lr_integrate_batched(descs: torch.Tensor, param_pool: torch.Tensor, count: int,
                             order: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None,
                             workspace: Optional[torch.Tensor] = None, stream=None, split: Optional[int] = None,
                             **opts) -> torch.Tensor:
    """``descs``: uint8 CUDA tensor holding ``count`` mdi_batch_desc records
    (``torch.from_numpy(make_batch_descs(...).view(np.uint8)).cuda()``); ``order``:
    optional int32 CUDA tensor from mdi_batch_plan; ``split``: the hybrid
    schedule's split from mdi_batch_plan (default: whole CTAs throughout);
    ``workspace``: from mdi_lr_batched_prepare with the same opts (prepared here
    when omitted).  Returns ``count`` float64 values."""
    if not (descs.is_cuda and descs.dtype == torch.uint8 and descs.numel() >= 32 * count):
        raise TypeError("descs must be a uint8 CUDA tensor of count*32 bytes")
    _dev_f64(param_pool, "param_pool")
    if order is not None and not (order.is_cuda and order.dtype == torch.int32 and order.numel() >= count):
        raise TypeError("order must be an int32 CUDA tensor of count entries")
    if out is None:
        out = torch.empty(count, dtype=torch.float64, device=param_pool.device)
    if workspace is None:
        workspace = mdi_lr_batched_prepare(device=param_pool.device, stream=stream, **opts)
    o = _opts(**opts)
    st = _ffi.load().mdi_lr_integrate_batched(
        ctypes.c_void_p(descs.data_ptr()), ctypes.c_void_p(order.data_ptr() if order is not None else 0), count,
        int(count if split is None else split), ctypes.c_void_p(param_pool.data_ptr()), int(param_pool.numel()),
        ctypes.byref(o),
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), _stream(stream))
    _ffi.check(st, "mdi_lr_integrate_batched")
    return out


def mdi_get_device_status(workspace: torch.Tensor, clear: bool = False, stream=None) -> int:
    """The MDI_DEV_* flags of a batched workspace's device status word (0: no
    integral rejected since the preparation or the last clear).  Waits for the
    stream; ``clear`` zeroes the word afterwards."""
    flags = ctypes.c_uint32(0)
    st = _ffi.load().mdi_get_device_status(ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), int(bool(clear)),
                                           ctypes.byref(flags), _stream(stream))
    if st not in (_ffi.MDI_OK, _ffi.MDI_EINVAL) or (st == _ffi.MDI_EINVAL and flags.value == 0):
        _ffi.check(st, "mdi_get_device_status")
    return flags.value


def mdi_peak_probe_threads(kind: str) -> int:
    """Threads of one mdi_peak_probe launch ("fp64" or "fp32")."""
    return int(_ffi.load().mdi_peak_probe_threads({"fp64": 0, "fp32": 1}[kind]))


def mdi_peak_probe(kind: str, iters: int, sink: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """One launch of the library's FMA throughput probe ("fp64": DFMA, "fp32": FFMA):
    mdi_peak_probe_threads(kind) threads, 16 * iters FMAs each."""
    if sink is None:
        sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    _ffi.check(_ffi.load().mdi_peak_probe({"fp64": 0, "fp32": 1}[kind], int(iters), ctypes.c_void_p(sink.data_ptr()),
                                          _stream(stream)), "mdi_peak_probe")
    return sink


def mdi_debug_fp64_phi(which: str, x: torch.Tensor, stream=None) -> torch.Tensor:
    """The FP64 batched sweep's own exp ("exp") or reciprocal ("rcp") of every
    element of a float64 CUDA tensor (test hook)."""
    _dev_f64(x, "x")
    y = torch.empty_like(x)
    _ffi.check(_ffi.load().mdi_debug_fp64_phi({"exp": 0, "rcp": 1}[which], ctypes.c_void_p(x.data_ptr()),
                                              ctypes.c_void_p(y.data_ptr()), int(x.numel()), _stream(stream)),
               "mdi_debug_fp64_phi")
    return y


def mdi_debug_lattice_indices(n: int, z: Sequence[int], j0: int, count: int, device="cuda",
                              stream=None) -> torch.Tensor:
    """(count, d) int64 CUDA tensor of (j0 + t) z_i mod n from the kernel's generator."""
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.int64))
    d = int(zz.size)
    out = torch.empty((count, d), dtype=torch.int64, device=device)
    st = _ffi.load().mdi_debug_lattice_indices(d, int(n), zz.ctypes.data_as(ctypes.c_void_p), int(j0), int(count),
                                               ctypes.c_void_p(out.data_ptr()), _stream(stream))
    _ffi.check(st, "mdi_debug_lattice_indices")
    return out


# ---------------------------------------------------------------------------
# Paper-table mode: tensor midpoint rule on the grid (N, ..., N, n_last)
# ---------------------------------------------------------------------------
def mdi_midpoint_workspace_size(d: int, N: int, n_last: int) -> int:
    b = ctypes.c_size_t()
    _ffi.check(_ffi.load().mdi_midpoint_workspace_size(d, N, n_last, ctypes.byref(b)), "mdi_midpoint_workspace_size")
    return b.value


def mdi_midpoint_integrate(family, params: torch.Tensor, d: int, N: int, n_last: Optional[int] = None,
                           out: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None,
                           stream=None) -> torch.Tensor:
    """prod_i (1/n_i) sum_k phi_i((k + 1/2)/n_i) (real part, times exp(2 pi i u) for
    OSC) on the grid n_1 = ... = n_{d-1} = N, n_d = n_last (default N): the rule
    the paper's tables print.  Returns a 1-element float64 CUDA tensor."""
    _dev_f64(params, "params")
    n_last = N if n_last is None else n_last
    if params.numel() < 2 * d:
        raise ValueError("params must hold 2*d doubles")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=params.device)
    ws = _workspace(mdi_midpoint_workspace_size(d, N, n_last), params.device, workspace)
    st = _ffi.load().mdi_midpoint_integrate(_fam(family), d, N, n_last, ctypes.c_void_p(params.data_ptr()),
                                            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                            ws.numel(), _stream(stream))
    _ffi.check(st, "mdi_midpoint_integrate")
    return out


def mdi_midpoint_ridge(d: int, N: int, n_last: Optional[int] = None, c0: float = 1.0,
                       power: Optional[float] = None, out: Optional[torch.Tensor] = None,
                       workspace: Optional[torch.Tensor] = None, device="cuda", stream=None) -> torch.Tensor:
    """Midpoint rule on the grid (N, ..., N, n_last) for (c0 + sum x_i)^(-power)
    (default power = d + 1: Test 7's f_6), by the dimension iteration with a
    partial-sum histogram state.  Returns a 1-element float64 CUDA tensor."""
    n_last = N if n_last is None else n_last
    power = float(d + 1) if power is None else float(power)
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=device)
    b = ctypes.c_size_t()
    _ffi.check(_ffi.load().mdi_midpoint_ridge_workspace_size(d, N, n_last, ctypes.byref(b)),
               "mdi_midpoint_ridge_workspace_size")
    ws = _workspace(b.value, out.device, workspace)
    st = _ffi.load().mdi_midpoint_ridge(d, N, n_last, float(c0), power, ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream))
    _ffi.check(st, "mdi_midpoint_ridge")
    return out


# ---------------------------------------------------------------------------
# Generating-vector construction (Section 2.2)
# ---------------------------------------------------------------------------
def lattice_korobov_search_workspace_size(n: int) -> int:
    b = ctypes.c_size_t()
    _ffi.check(_ffi.load().lattice_korobov_search_workspace_size(n, ctypes.byref(b)),
               "lattice_korobov_search_workspace_size")
    return b.value


def lattice_korobov_search(n: int, d: int, alpha: int = 2, a_first: int = 1, count: Optional[int] = None,
                           values: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None,
                           device="cuda", stream=None):
    """(values, best_a): P_alpha(z(a)) of eq. (2.4) for a = a_first .. a_first + count - 1
    (default: every a in 1..n-1; +inf where gcd(a, n) > 1) and the smallest a attaining
    the least value, both as CUDA tensors (float64, int64[1])."""
    count = (n - a_first) if count is None else count
    if values is None:
        values = torch.empty(count, dtype=torch.float64, device=device)
    best = torch.zeros(1, dtype=torch.int64, device=values.device)
    ws = _workspace(lattice_korobov_search_workspace_size(n), values.device, workspace)
    st = _ffi.load().lattice_korobov_search(alpha, d, n, a_first, count, ctypes.c_void_p(values.data_ptr()),
                                            ctypes.c_void_p(best.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                            ws.numel(), _stream(stream))
    _ffi.check(st, "lattice_korobov_search")
    return values, best


def lattice_cbc_workspace_size(n: int) -> int:
    b = ctypes.c_size_t()
    _ffi.check(_ffi.load().lattice_cbc_workspace_size(n, ctypes.byref(b)), "lattice_cbc_workspace_size")
    return b.value


def lattice_cbc(n: int, gamma: torch.Tensor, beta: float = 0.0, workspace: Optional[torch.Tensor] = None,
                stream=None):
    """(z, e2): the component-by-component generating vector of Example 3 for the
    product weights ``gamma`` (float64 CUDA tensor of d entries) and the squared
    shift-averaged worst-case error of eq. (2.12) after each component."""
    _dev_f64(gamma, "gamma")
    d = gamma.numel()
    z = torch.zeros(d, dtype=torch.int64, device=gamma.device)
    e2 = torch.zeros(d, dtype=torch.float64, device=gamma.device)
    ws = _workspace(lattice_cbc_workspace_size(n), gamma.device, workspace)
    st = _ffi.load().lattice_cbc(d, n, ctypes.c_void_p(gamma.data_ptr()), float(beta), ctypes.c_void_p(z.data_ptr()),
                                 ctypes.c_void_p(e2.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                 _stream(stream))
    _ffi.check(st, "lattice_cbc")
    return z, e2
