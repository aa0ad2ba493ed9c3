"""The lattice rule's allocation-free entry point (lattice_rule_integrate_noalloc).

It exists for callers that cannot allocate device memory when they call, e.g.
code inside an application that reserves all GPU memory at start-up, or a
plug-in without access to its host's allocator.  Its scratch is a fixed array
inside the library that every call shares.  This file is collected last so that
a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle as o
import paper_2404_08867_gb300 as mdi
from paper_2404_08867_gb300 import _ffi, inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12  # the FP64 parity tolerance of the other GPU tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_08867_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _noalloc_call(family, params, n, z, out, precision="fp64"):
    """Straight through the C ABI: no workspace argument exists."""
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.int64))
    st = _ffi.load().lattice_rule_integrate_noalloc(
        _ffi.FAMILY[family], int(zz.size), int(n), zz.ctypes.data_as(ctypes.c_void_p),
        ctypes.c_void_p(params.data_ptr()), _ffi.PRECISION[precision], ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _ffi.check(st, "lattice_rule_integrate_noalloc")
    return out


# Each arithmetic mode of the lattice rule against the workspace entry point in the
# same mode: both evaluate the same points in the same arithmetic, so they differ
# only by the order of the partial sums (1e-12, the FP64 parity tolerance).
@pytest.mark.parametrize("precision", ["fp64", "fp32_eval_fp64", "df64"])
def test_noalloc_matches_workspace_entry_point_two_calls_in_a_row(precision):
    # Call 1: large lattice (every scratch slot of the launch in use);
    # call 2: small lattice right after, reusing the same built-in array.
    cases = [("gauss", 6, 1_000_001, 10), ("exp", 4, 65536, inputs.SMALL_SLR_A)]
    for fam, d, n, a in cases:
        params = torch.as_tensor(inputs.random_product(fam, d, seed=n)).cuda()
        z = o.korobov_z(d, a, n).astype(np.int64)
        ref = mdi.lattice_rule_integrate(fam, params, n, z, precision=precision).item()
        got = _noalloc_call(fam, params, n, z, torch.empty(1, dtype=torch.float64, device="cuda"),
                            precision).item()
        assert abs(got - ref) <= TOL * abs(ref), (fam, n, precision, got, ref)


def test_noalloc_repeated_calls_agree():
    params = torch.as_tensor(inputs.random_product("peak", 5, seed=3)).cuda()
    z = o.korobov_z(5, 7, 300007).astype(np.int64)
    ref = mdi.lattice_rule_integrate("peak", params, 300007, z).item()
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    _noalloc_call("peak", params, 300007, z, out[0:1])
    _noalloc_call("peak", params, 300007, z, out[1:2])
    vals = out.cpu().numpy()
    assert abs(vals[0] - ref) <= TOL * abs(ref) and abs(vals[1] - ref) <= TOL * abs(ref)
