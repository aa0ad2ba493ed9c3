"""TEST INFRASTRUCTURE ONLY: Python access to the plain FP64 CPU oracle.

The oracle (``mdi_oracle.c``) is a slow, obviously-correct restatement of the
MDI-LR method of Zhong & Feng: the standard lattice rule of eq. (2.1)/(1.2), the
transformed-grid rule of Lemma 3.2, the level sweeps of Algorithm 1 (m = 1)
inside Algorithm 2, the tensor midpoint rule that reproduces the paper's printed
MDI-LR error columns, the exact integrals of the test integrands, and the
generating-vector criteria of Section 2.2 (P_alpha of eq. (2.4) with the Korobov
search of Example 2, the shift-averaged worst-case error of eq. (2.12) with the
component-by-component construction of Example 3).  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this module.  It shares no code with the CUDA library.

Family names used here: ``"exp"``, ``"osc"``, ``"gauss"``, ``"peak"`` (product
form, parameters ``c`` and ``w`` of length d; for ``"osc"`` ``w[0]`` is the phase
``u``) and ``"t1"``, ``"sinsq"``, ``"altsq"``, ``"ridge"`` (the paper's
non-product test integrands, brute-force rules only).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mdi_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

FAMILY = {"exp": 0, "osc": 1, "gauss": 2, "peak": 3,
          "t1": 10, "sinsq": 11, "altsq": 12, "ridge": 13}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (no fused multiply-add
    contraction, so x86 and Arm hosts give the same bits)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D = ctypes.c_double
            I = ctypes.c_int
            U = ctypes.c_uint64
            P = ctypes.c_void_p
            sig = {
                "or_korobov_z": (I, [I, U, U, P]),
                "or_lattice_indices": (I, [I, U, P, U, U, P]),
                "or_slr": (D, [I, I, U, P, P, P]),
                "or_improved": (D, [I, I, U, U, P, P, P]),
                "or_slr_grad": (I, [I, I, U, P, P, P, P]),
                "or_grid_sizes": (I, [I, U, P, P]),
                "or_affine_y": (I, [I, U, P, P]),
                "or_grid_korobov": (D, [I, I, U, U, P, P]),
                "or_mdi_exact": (D, [I, I, U, U, P, P]),
                "or_mdi_closed": (D, [I, I, U, U, P, P]),
                "or_mdi_closed_grad": (I, [I, I, U, U, P, P, P]),
                "or_mdi_nodes": (D, [I, I, U, U, I, P, P]),
                "or_mdi_nodes_step": (D, [I, I, U, U, I, I, P, P]),
                "or_mdi_nodes_states": (I, [I, I, U, U, I, P, P, P]),
                "or_mdi_nodes_grad": (I, [I, I, U, U, I, P, P, P, I, P]),
                "or_mdi_nodes_step_grad": (I, [I, I, U, U, I, I, P, P, P, I, P]),
                "or_bary_matrix": (I, [I, U, P]),
                "or_midpoint_grid": (D, [I, I, P, P, P]),
                "or_midpoint_product": (D, [I, I, P, P, P]),
                "or_closed_form": (D, [I, I, P, P]),
                "or_closed_form_grad": (I, [I, I, P, P, P]),
                "or_slr_shifted": (D, [I, I, U, P, P, P, P]),
                "or_midpoint_ridge": (D, [I, U, U, D, D]),
                "or_p_alpha": (D, [I, I, U, P]),
                "or_korobov_search": (I, [I, I, U, U, U, P, P]),
                "or_wce2_shift": (D, [I, U, P, P, D]),
                "or_cbc": (I, [I, U, P, D, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _f64(x, d):
    a = np.zeros(d, dtype=np.float64) if x is None else np.ascontiguousarray(x, dtype=np.float64)
    if a.size < d:
        a = np.concatenate([a, np.zeros(d - a.size)])
    return a


def _u64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint64))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _fam(family):
    return FAMILY[family] if isinstance(family, str) else int(family)


def korobov_z(d: int, a: int, n: int) -> np.ndarray:
    z = np.zeros(d, dtype=np.uint64)
    _load().or_korobov_z(d, a, n, _p(z))
    return z


def lattice_indices(d, n, z, j0, count) -> np.ndarray:
    z = _u64(z)
    r = np.zeros((count, d), dtype=np.uint64)
    _load().or_lattice_indices(d, n, _p(z), j0, count, _p(r))
    return r


def slr(family, d, n, z, c, w=None) -> float:
    z, c, w = _u64(z), _f64(c, d), _f64(w, d)
    return _load().or_slr(_fam(family), d, n, _p(z), _p(c), _p(w))


def improved_rule(family, d, n, a, c, w=None):
    """Improved lattice rule of Definition 3.3 on z = (1, a, ..) by brute force:
    (value, n*), ghosts by the unwrapped line extension."""
    c, w = _f64(c, d), _f64(w, d)
    ns = ctypes.c_uint64()
    v = _load().or_improved(_fam(family), d, n, a, _p(c), _p(w), ctypes.byref(ns))
    return v, ns.value


def slr_grad(family, d, n, z, c, w=None) -> np.ndarray:
    z, c, w = _u64(z), _f64(c, d), _f64(w, d)
    g = np.zeros(2 * d)
    assert _load().or_slr_grad(_fam(family), d, n, _p(z), _p(c), _p(w), _p(g)) == 0
    return g


def grid_sizes(d, n, z) -> np.ndarray:
    z = _u64(z)
    out = np.zeros(d, dtype=np.uint64)
    _load().or_grid_sizes(d, n, _p(z), _p(out))
    return out


def affine_y(d, n, z) -> np.ndarray:
    z = _u64(z)
    y = np.zeros((n, d))
    _load().or_affine_y(d, n, _p(z), _p(y))
    return y


def grid_korobov(family, d, a, nd, c, w=None) -> float:
    c, w = _f64(c, d), _f64(w, d)
    return _load().or_grid_korobov(_fam(family), d, a, nd, _p(c), _p(w))


def mdi_exact(family, d, a, nd, c, w=None) -> float:
    c, w = _f64(c, d), _f64(w, d)
    return _load().or_mdi_exact(_fam(family), d, a, nd, _p(c), _p(w))


def mdi_closed(family, d, a, nd, c, w=None) -> float:
    c, w = _f64(c, d), _f64(w, d)
    return _load().or_mdi_closed(_fam(family), d, a, nd, _p(c), _p(w))


def mdi_closed_grad(family, d, a, nd, c, w=None) -> np.ndarray:
    c, w = _f64(c, d), _f64(w, d)
    g = np.zeros(2 * d)
    assert _load().or_mdi_closed_grad(_fam(family), d, a, nd, _p(c), _p(w), _p(g)) == 0
    return g


def mdi_nodes(family, d, a, nd, P, c, w=None) -> float:
    c, w = _f64(c, d), _f64(w, d)
    return _load().or_mdi_nodes(_fam(family), d, a, nd, P, _p(c), _p(w))


def mdi_nodes_step(family, d, a, nd, P, m, c, w=None) -> float:
    """Node-state sweep with step size m of Algorithm 1: m transformed axes
    contracted per iteration (m = 1 is mdi_nodes)."""
    c, w = _f64(c, d), _f64(w, d)
    return _load().or_mdi_nodes_step(_fam(family), d, a, nd, P, m, _p(c), _p(w))


def mdi_nodes_states(family, d, a, nd, P, c, w=None) -> np.ndarray:
    """Complex node states G_0..G_{d-1} (rows) and G_d in row d, column 0."""
    c, w = _f64(c, d), _f64(w, d)
    s = np.zeros((d + 1, P, 2))
    assert _load().or_mdi_nodes_states(_fam(family), d, a, nd, P, _p(c), _p(w), _p(s)) == 0
    return s[..., 0] + 1j * s[..., 1]


def mdi_nodes_grad(family, d, a, nd, P, c, w=None, which=None) -> np.ndarray:
    c, w = _f64(c, d), _f64(w, d)
    which = np.arange(2 * d, dtype=np.int32) if which is None else np.ascontiguousarray(which, dtype=np.int32)
    g = np.zeros(which.size)
    assert _load().or_mdi_nodes_grad(_fam(family), d, a, nd, P, _p(c), _p(w), _p(which),
                                     int(which.size), _p(g)) == 0
    return g


def mdi_nodes_step_grad(family, d, a, nd, P, m, c, w=None, which=None) -> np.ndarray:
    """Derivative of the step-m node-state sweep (forward mode), entries as
    mdi_nodes_grad."""
    c, w = _f64(c, d), _f64(w, d)
    which = np.arange(2 * d, dtype=np.int32) if which is None else np.ascontiguousarray(which, dtype=np.int32)
    g = np.zeros(which.size)
    assert _load().or_mdi_nodes_step_grad(_fam(family), d, a, nd, P, m, _p(c), _p(w), _p(which),
                                          int(which.size), _p(g)) == 0
    return g


def bary_matrix(P, a) -> np.ndarray:
    L = np.zeros((a, P, P))
    _load().or_bary_matrix(P, a, _p(L))
    return L


def midpoint_grid(family, d, Nd, c=None, w=None) -> float:
    Nd, c, w = _u64(Nd), _f64(c, d), _f64(w, d)
    return _load().or_midpoint_grid(_fam(family), d, _p(Nd), _p(c), _p(w))


def midpoint_product(family, d, Nd, c, w=None) -> float:
    Nd, c, w = _u64(Nd), _f64(c, d), _f64(w, d)
    return _load().or_midpoint_product(_fam(family), d, _p(Nd), _p(c), _p(w))


def midpoint_ridge(d, N, n_last, c0=1.0, p=None) -> float:
    """Tensor midpoint rule for (c0 + sum x_i)^(-p) (default p = d + 1, Test 7's f_6)
    by the dimension iteration with a partial-sum histogram state."""
    return _load().or_midpoint_ridge(d, N, n_last, c0, float(d + 1) if p is None else float(p))


def closed_form(family, d, c, w=None) -> float:
    c, w = _f64(c, d), _f64(w, d)
    return _load().or_closed_form(_fam(family), d, _p(c), _p(w))


def closed_form_grad(family, d, c, w=None) -> np.ndarray:
    c, w = _f64(c, d), _f64(w, d)
    g = np.zeros(2 * d)
    assert _load().or_closed_form_grad(_fam(family), d, _p(c), _p(w), _p(g)) == 0
    return g


def mdi_lr(family, d, a, nd, c, w=None, state="auto", P=16) -> float:
    """The oracle's MDI-LR value for one instance: the exact level sweep where the
    lattice is small enough to enumerate, the closed state for the exponential
    families, the node state otherwise (the same choice the device makes for
    ``state="auto"``)."""
    if state == "exact":
        return mdi_exact(family, d, a, nd, c, w)
    if state == "closed":
        return mdi_closed(family, d, a, nd, c, w)
    if state == "nodes":
        return mdi_nodes(family, d, a, nd, P, c, w)
    if family in ("exp", "osc"):
        return mdi_closed(family, d, a, nd, c, w)
    return mdi_nodes(family, d, a, nd, P, c, w)


# ---------------------------------------------------------------------------
# Randomly shifted lattice rule (Section 2.1)
# ---------------------------------------------------------------------------
def slr_shifted(family, d, n, z, c, w=None, shift=None) -> float:
    z, c, w, sh = _u64(z), _f64(c, d), _f64(w, d), _f64(shift, d)
    return _load().or_slr_shifted(_fam(family), d, n, _p(z), _p(c), _p(w), _p(sh))


# ---------------------------------------------------------------------------
# Generating-vector criteria and searches (Section 2.2)
# ---------------------------------------------------------------------------
def p_alpha(alpha, d, n, z) -> float:
    z = _u64(z)
    return _load().or_p_alpha(alpha, d, n, _p(z))


def korobov_search(alpha, d, n, a_first, count):
    """(values, best_a): P_alpha(z(a)) for a = a_first .. a_first + count - 1 (+inf for
    inadmissible a) and the first a attaining the minimum."""
    vals = np.zeros(count)
    best = np.zeros(1, dtype=np.uint64)
    assert _load().or_korobov_search(alpha, d, n, a_first, count, _p(vals), _p(best)) == 0
    return vals, int(best[0])


def wce2_shift(d, n, z, gamma, beta=0.0) -> float:
    z, g = _u64(z), _f64(gamma, d)
    return _load().or_wce2_shift(d, n, _p(z), _p(g), beta)


def cbc(d, n, gamma, beta=0.0):
    """(z, e2): the component-by-component vector and the squared shift-averaged
    worst-case error after each component."""
    g = _f64(gamma, d)
    z = np.zeros(d, dtype=np.uint64)
    e2 = np.zeros(d)
    assert _load().or_cbc(d, n, _p(g), beta, _p(z), _p(e2)) == 0
    return z, e2
