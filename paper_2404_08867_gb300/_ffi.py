"""ctypes declarations of the C ABI in include/mdi_lr.h (no computation here)."""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmdilr.so")

MDI_OK, MDI_EINVAL, MDI_EUNSUPPORTED, MDI_EOVERFLOW, MDI_ECUDA, MDI_EWORKSPACE = range(6)
ABI_VERSION = 2
# Flags of the batched workspace's device status word (MDI_DEV_*).
DEV_FLAGS = {"bad_desc": 1, "bad_order": 2, "unprepared": 4, "pool_range": 8}
FAMILY = {"exp": 0, "osc": 1, "gauss": 2, "peak": 3}
STATE = {"auto": 0, "exact": 1, "closed": 2, "nodes": 3}
PRECISION = {"fp64": 0, "fp32_eval_fp64": 1, "fp32_eval_df32": 2, "df64": 3}

# Every symbol include/mdi_lr.h declares, with its ctypes signature.
_c = ctypes
_P = _c.c_void_p
_I32 = _c.c_int32
_I64 = _c.c_int64
_SZ = _c.c_size_t


class MdiOpts(ctypes.Structure):
    _fields_ = [("state", _I32), ("precision", _I32), ("nodes", _I32), ("block", _I32),
                ("ctas_per_sm", _I32), ("checkpoint", _I32), ("table_in_l1", _I32), ("step", _I32)]


BATCH_DESC_DTYPE = np.dtype([("family", np.int32), ("d", np.int32), ("a", np.int32), ("n_last", np.int32),
                             ("param_offset", np.int64), ("reserved", np.int64)])
assert BATCH_DESC_DTYPE.itemsize == 32

SIGNATURES = {
    "lattice_rule_integrate": (_I32, [_I32, _I32, _I64, _P, _P, _I32, _P, _P, _SZ, _P]),
    "lattice_rule_workspace_size": (_I32, [_I32, _I64, _c.POINTER(_SZ)]),
    "lattice_rule_integrate_noalloc": (_I32, [_I32, _I32, _I64, _P, _P, _I32, _P, _P]),
    "lattice_rule_integrate_shifted": (_I32, [_I32, _I32, _I64, _P, _P, _P, _I32, _I32, _P, _P, _SZ, _P]),
    "lattice_rule_shifted_workspace_size": (_I32, [_I32, _I64, _I32, _c.POINTER(_SZ)]),
    "lattice_rule_integrate_improved": (_I32, [_I32, _I32, _I64, _I64, _P, _I32, _P, _c.POINTER(_I64), _P, _SZ, _P]),
    "lattice_rule_improved_workspace_size": (_I32, [_I32, _I64, _I64, _c.POINTER(_SZ)]),
    "mdi_lr_integrate": (_I32, [_I32, _I32, _I64, _I64, _P, _P, _c.POINTER(MdiOpts), _P, _P, _SZ, _P]),
    "mdi_lr_workspace_size": (_I32, [_I32, _I32, _I64, _I64, _c.POINTER(MdiOpts), _c.POINTER(_SZ)]),
    "mdi_lr_grad": (_I32, [_I32, _I32, _I64, _I64, _P, _P, _c.POINTER(MdiOpts), _P, _P, _P, _SZ, _P]),
    "mdi_lr_grad_workspace_size": (_I32, [_I32, _I32, _I64, _I64, _c.POINTER(MdiOpts), _c.POINTER(_SZ)]),
    "mdi_lr_integrate_batched": (_I32, [_P, _P, _I32, _I32, _P, _I64, _c.POINTER(MdiOpts), _P, _P, _SZ, _P]),
    "mdi_lr_batched_workspace_size": (_I32, [_I32, _c.POINTER(MdiOpts), _c.POINTER(_SZ)]),
    "mdi_lr_batched_prepare": (_I32, [_c.POINTER(MdiOpts), _P, _SZ, _P]),
    "mdi_batch_plan": (_I32, [_P, _I32, _I64, _c.POINTER(MdiOpts), _P, _P]),
    "mdi_get_device_status": (_I32, [_P, _SZ, _I32, _c.POINTER(_c.c_uint32), _P]),
    "lattice_korobov_vector": (_I32, [_I32, _I64, _I64, _P]),
    "lattice_shifted_estimate": (_I32, [_P, _I32, _P, _P]),
    "mdi_peak_probe": (_I32, [_I32, _I32, _P, _P]),
    "mdi_peak_probe_threads": (_I64, [_I32]),
    "mdi_debug_lattice_indices": (_I32, [_I32, _I64, _P, _I64, _I64, _P, _P]),
    "mdi_debug_fp64_phi": (_I32, [_I32, _P, _P, _I64, _P]),
    "mdi_midpoint_integrate": (_I32, [_I32, _I32, _I64, _I64, _P, _P, _P, _SZ, _P]),
    "lattice_korobov_search": (_I32, [_I32, _I32, _I64, _I64, _I64, _P, _P, _P, _SZ, _P]),
    "lattice_korobov_search_workspace_size": (_I32, [_I64, _c.POINTER(_SZ)]),
    "lattice_cbc": (_I32, [_I32, _I64, _P, _c.c_double, _P, _P, _P, _SZ, _P]),
    "lattice_cbc_workspace_size": (_I32, [_I64, _c.POINTER(_SZ)]),
    "mdi_midpoint_workspace_size": (_I32, [_I32, _I64, _I64, _c.POINTER(_SZ)]),
    "mdi_midpoint_ridge": (_I32, [_I32, _I64, _I64, _c.c_double, _c.c_double, _P, _P, _SZ, _P]),
    "mdi_midpoint_ridge_workspace_size": (_I32, [_I32, _I64, _I64, _c.POINTER(_SZ)]),
    "mdi_status_string": (_c.c_char_p, [_I32]),
    "mdi_last_cuda_error": (_c.c_char_p, []),
    "mdi_abi_version": (_I32, []),
}

_lock = threading.Lock()
_lib = None


def load():
    """Loads libmdilr.so.  There is no fallback: without the built library every
    call fails loudly (build it with ``python -m paper_2404_08867_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing; build it with "
                                   "`python -m paper_2404_08867_gb300.build` (nvcc, sm_103a)")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            if lib.mdi_abi_version() != ABI_VERSION:
                raise RuntimeError("libmdilr.so ABI version mismatch; rebuild it")
            _lib = lib
    return _lib


class MdiError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.mdi_status_string(status).decode()
        if status == MDI_ECUDA:
            msg += " (" + lib.mdi_last_cuda_error().decode() + ")"
        super().__init__(f"{where}: {msg}")
        self.status = status


def check(status: int, where: str) -> None:
    if status != MDI_OK:
        raise MdiError(status, where)
