"""Host-side checks of the C ABI: the library loads, exports every symbol that
include/mdi_lr.h declares, validates arguments before touching the GPU, and its
scheduler orders work longest-first.  No kernel runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2404_08867_gb300 import _ffi
import paper_2404_08867_gb300 as mdi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mdi_lr.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2404_08867_gb300 import build
    build.build()
    return _ffi.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|mdi_status|int32_t|int64_t)\s*(\w+)\s*\(", text,
                                 flags=re.M)))


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for must in ("lattice_rule_integrate", "mdi_lr_integrate", "mdi_lr_integrate_batched", "mdi_batch_plan"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert names, "no declarations parsed"
    for name in names:
        assert hasattr(lib, name), f"libmdilr.so does not export {name}"
        assert name in _ffi.SIGNATURES, f"binding has no signature for {name}"


def test_abi_version_and_status_strings(lib):
    assert lib.mdi_abi_version() == _ffi.ABI_VERSION == 2
    for code in range(6):
        s = lib.mdi_status_string(code).decode()
        assert s.startswith("MDI_")
    assert b"unknown" in lib.mdi_status_string(99)


def test_batch_desc_layout():
    assert _ffi.BATCH_DESC_DTYPE.itemsize == 32
    assert ctypes.sizeof(_ffi.MdiOpts) == 32


def _null():
    return ctypes.c_void_p(0)


def test_lattice_rule_rejects_bad_arguments(lib):
    z = np.array([1, 5, 25], dtype=np.int64)
    zp = z.ctypes.data_as(ctypes.c_void_p)
    fake = ctypes.c_void_p(0x1000)
    # d out of range, n < 1, null device pointers, z_i >= n, unknown family
    assert lib.lattice_rule_integrate(0, 0, 100, zp, fake, 0, fake, fake, 4096, _null()) == _ffi.MDI_EINVAL
    assert lib.lattice_rule_integrate(0, 3, 0, zp, fake, 0, fake, fake, 4096, _null()) == _ffi.MDI_EINVAL
    assert lib.lattice_rule_integrate(0, 3, 100, zp, _null(), 0, fake, fake, 4096, _null()) == _ffi.MDI_EINVAL
    assert lib.lattice_rule_integrate(0, 3, 20, zp, fake, 0, fake, fake, 4096, _null()) == _ffi.MDI_EINVAL
    assert lib.lattice_rule_integrate(7, 3, 100, zp, fake, 0, fake, fake, 4096, _null()) == _ffi.MDI_EINVAL
    assert lib.lattice_rule_integrate(0, 3, 100, zp, fake, 2, fake, fake, 4096, _null()) == _ffi.MDI_EUNSUPPORTED
    # workspace missing or misaligned
    assert lib.lattice_rule_integrate(0, 3, 100, zp, fake, 0, fake, _null(), 4096, _null()) == _ffi.MDI_EWORKSPACE
    assert lib.lattice_rule_integrate(0, 3, 100, zp, fake, 0, fake, ctypes.c_void_p(0x1008), 4096,
                                      _null()) == _ffi.MDI_EWORKSPACE


def test_mdi_rejects_bad_arguments(lib):
    fake = ctypes.c_void_p(0x1000)
    o = _ffi.MdiOpts()
    assert lib.mdi_lr_integrate(0, 0, 16, 16, _null(), fake, ctypes.byref(o), fake, fake, 1 << 20, _null()) == _ffi.MDI_EINVAL
    assert lib.mdi_lr_integrate(0, 4, 0, 16, _null(), fake, ctypes.byref(o), fake, fake, 1 << 20, _null()) == _ffi.MDI_EINVAL
    o.step = 4  # Algorithm 1's m is 1, 2 or 3
    assert lib.mdi_lr_integrate(0, 4, 16, 16, _null(), fake, ctypes.byref(o), fake, fake, 1 << 20, _null()) == _ffi.MDI_EINVAL
    o.step = -1
    assert lib.mdi_lr_integrate(0, 4, 16, 16, _null(), fake, ctypes.byref(o), fake, fake, 1 << 20, _null()) == _ffi.MDI_EINVAL
    o = _ffi.MdiOpts()
    o.state = _ffi.STATE["closed"]
    assert lib.mdi_lr_integrate(2, 4, 16, 16, _null(), fake, ctypes.byref(o), fake, fake, 1 << 20,
                                _null()) == _ffi.MDI_EUNSUPPORTED
    o.state = _ffi.STATE["exact"]
    b = ctypes.c_size_t()
    assert lib.mdi_lr_workspace_size(2, 20, 16, 16, ctypes.byref(o), ctypes.byref(b)) == _ffi.MDI_EOVERFLOW
    assert lib.mdi_lr_workspace_size(2, 4, 16, 16, ctypes.byref(o), ctypes.byref(b)) == _ffi.MDI_OK
    o.state = _ffi.STATE["nodes"]
    o.nodes = 15  # odd P is refused
    assert lib.mdi_lr_integrate(2, 4, 16, 16, _null(), fake, ctypes.byref(o), fake, fake, 1 << 30, _null()) == _ffi.MDI_EINVAL
    o.nodes = 16
    assert lib.mdi_lr_integrate(2, 4, 65, 16, _null(), fake, ctypes.byref(o), fake, fake, 1 << 30,
                                _null()) == _ffi.MDI_EUNSUPPORTED


def test_batch_plan_is_longest_first_permutation(lib):
    rng = np.random.default_rng(1)
    n = 500
    a = rng.integers(8, 33, n)
    descs = mdi.make_batch_descs(["gauss"] * n, rng.integers(6, 21, n), a, a, np.arange(n) * 40)
    order, split = mdi.mdi_batch_plan(descs, 40 * n)
    assert split == n  # default 256-thread CTAs: whole CTAs throughout
    assert sorted(order.tolist()) == list(range(n))
    # one family, n_last = a: the work is dominated by the (d - 1) * a cluster points;
    # the last axis adds less than 3 such units for a <= 32
    work = (descs["d"][order] - 1) * descs["a"][order]
    assert np.all(np.diff(work) <= 3)
    assert work[0] == work.max() and work[-1] <= work.min() + 3
    bad = descs.copy()
    bad["a"][3] = 65
    with pytest.raises(mdi.MdiError):
        mdi.mdi_batch_plan(bad, 40 * n)


def test_workspace_queries(lib):
    assert mdi.lattice_rule_workspace_size(4, 65536) >= 8
    assert mdi.mdi_lr_workspace_size("exp", 1000, 16, 16, state="closed") >= 8 * 1000
    assert mdi.mdi_lr_batched_workspace_size(4096, nodes=16) > 4 * 2**20


def test_new_entry_points_validate_before_launching(lib):
    """The paper-table, ridge, shifted-rule and search entry points refuse bad
    arguments and workspaces with status codes, before any launch (no GPU here)."""
    fake = ctypes.c_void_p(0x1000)
    E, W = _ffi.MDI_EINVAL, _ffi.MDI_EWORKSPACE
    # tensor midpoint rule: family, d, N, n_last, workspace
    assert lib.mdi_midpoint_integrate(7, 4, 8, 8, fake, fake, fake, 1 << 20, _null()) == E
    assert lib.mdi_midpoint_integrate(2, 0, 8, 8, fake, fake, fake, 1 << 20, _null()) == E
    assert lib.mdi_midpoint_integrate(2, 4, 0, 8, fake, fake, fake, 1 << 20, _null()) == E
    assert lib.mdi_midpoint_integrate(2, 4, 8, 8, fake, fake, _null(), 1 << 20, _null()) == W
    assert lib.mdi_midpoint_integrate(2, 4, 8, 8, fake, fake, ctypes.c_void_p(0x1008), 1 << 20, _null()) == W
    # ridge: c0 > 0, finite power, sizes
    assert lib.mdi_midpoint_ridge(4, 8, 8, 0.0, 5.0, fake, fake, 1 << 20, _null()) == E
    assert lib.mdi_midpoint_ridge(4, 8, 8, 1.0, float("inf"), fake, fake, 1 << 20, _null()) == E
    assert lib.mdi_midpoint_ridge(4, 8, 8, 1.0, 5.0, fake, fake, 8, _null()) == W
    b = ctypes.c_size_t()
    assert lib.mdi_midpoint_ridge_workspace_size(1 << 20, 1 << 20, 8, ctypes.byref(b)) == E  # histogram > 2^26
    # shifted rule: R range, z range
    z = (ctypes.c_int64 * 2)(1, 5)
    zp = ctypes.cast(z, ctypes.c_void_p)
    assert lib.lattice_rule_integrate_shifted(0, 2, 11, zp, fake, fake, 0, 0, fake, fake, 1 << 20, _null()) == E
    assert lib.lattice_rule_integrate_shifted(0, 2, 11, zp, fake, fake, 70000, 0, fake, fake, 1 << 20, _null()) == E
    assert lib.lattice_rule_integrate_shifted(0, 2, 5, zp, fake, fake, 2, 0, fake, fake, 1 << 20, _null()) == E  # z >= n
    # precision: FP64 or DF64 only, DF64 up to 2^48 points
    assert lib.lattice_rule_integrate_shifted(0, 2, 11, zp, fake, fake, 2, 1, fake, fake, 1 << 20,
                                              _null()) == _ffi.MDI_EUNSUPPORTED
    # Korobov search: alpha, d, count, workspace
    assert lib.lattice_korobov_search(3, 4, 101, 1, 10, fake, fake, fake, 1 << 20, _null()) == E
    assert lib.lattice_korobov_search(2, 257, 101, 1, 10, fake, fake, fake, 1 << 20, _null()) == E
    assert lib.lattice_korobov_search(2, 4, 101, 1, 0, fake, fake, fake, 1 << 20, _null()) == E
    assert lib.lattice_korobov_search(2, 4, 101, 1, 10, fake, fake, _null(), 1 << 20, _null()) == W
    # CBC: n range (tabulated factors, n <= 2^24), beta finite, workspace
    assert lib.lattice_cbc(4, 1, fake, 0.0, fake, fake, fake, 1 << 20, _null()) == E
    assert lib.lattice_cbc(4, (1 << 24) + 1, fake, 0.0, fake, fake, fake, 1 << 30, _null()) == E
    assert lib.lattice_cbc(4, 101, fake, float("nan"), fake, fake, fake, 1 << 20, _null()) == E
    assert lib.lattice_cbc(4, 101, fake, 0.0, fake, fake, fake, 8, _null()) == W
    assert lib.lattice_cbc_workspace_size((1 << 24) + 1, ctypes.byref(b)) == E


def test_improved_rule_and_df64_modes_validate_before_launching(lib):
    """The improved lattice rule refuses bad sizes, a common factor of a and n with
    ghosts present, and bad workspaces; the plain rule's double-float mode refuses
    n beyond 2^48; the closed state's double-float mode refuses a >= 2^31.  All
    before any launch (no GPU here)."""
    fake = ctypes.c_void_p(0x1000)
    E, W, U = _ffi.MDI_EINVAL, _ffi.MDI_EWORKSPACE, _ffi.MDI_EUNSUPPORTED
    b = ctypes.c_size_t()
    ng = ctypes.c_int64(-1)
    # improved rule: family, d range, n < 1, a^(d-1) beyond 2^62, gcd(a, n) > 1 with ghosts
    assert lib.lattice_rule_integrate_improved(7, 3, 100, 7, fake, 0, fake, ctypes.byref(ng), fake, 1 << 20, _null()) == E
    assert lib.lattice_rule_integrate_improved(0, 0, 100, 7, fake, 0, fake, None, fake, 1 << 20, _null()) == E
    assert lib.lattice_rule_integrate_improved(0, 65, 100, 2, fake, 0, fake, None, fake, 1 << 20, _null()) == E
    assert lib.lattice_rule_integrate_improved(0, 3, 0, 7, fake, 0, fake, None, fake, 1 << 20, _null()) == E
    assert lib.lattice_rule_integrate_improved(0, 41, 1000, 3, fake, 0, fake, None, fake, 1 << 20, _null()) == E
    assert lib.lattice_rule_integrate_improved(0, 3, 150, 10, fake, 0, fake, None, fake, 1 << 20, _null()) == E
    assert lib.lattice_rule_integrate_improved(0, 3, 100, 7, _null(), 0, fake, None, fake, 1 << 20, _null()) == E
    assert ng.value == -1  # nothing written on refusal
    # workspace: missing, misaligned, short
    assert lib.lattice_rule_integrate_improved(0, 3, 100, 7, fake, 0, fake, None, _null(), 1 << 20, _null()) == W
    assert lib.lattice_rule_integrate_improved(0, 3, 100, 7, fake, 0, fake, None, ctypes.c_void_p(0x1008), 1 << 20,
                                               _null()) == W
    assert lib.lattice_rule_integrate_improved(0, 3, 100, 7, fake, 0, fake, None, fake, 8, _null()) == W
    # precision of the lattice points: the compensated single-precision mode has no
    # lattice kernel; double-float coordinates hold n <= 2^48
    assert lib.lattice_rule_integrate_improved(0, 3, 100, 7, fake, 2, fake, None, fake, 1 << 20, _null()) == U
    assert lib.lattice_rule_integrate_improved(0, 2, (1 << 49) + 2, 3, fake, 3, fake, None, fake, 1 << 20,
                                               _null()) == U
    assert lib.lattice_rule_improved_workspace_size(3, 150, 10, ctypes.byref(b)) == E
    assert lib.lattice_rule_improved_workspace_size(3, 100, 10, ctypes.byref(b)) == _ffi.MDI_OK  # 10^2 | 100: no ghosts
    # double-float plain rule beyond 2^48 points
    z = np.array([1, 3], dtype=np.int64)
    zp = z.ctypes.data_as(ctypes.c_void_p)
    assert lib.lattice_rule_integrate(0, 2, (1 << 48) + 1, zp, fake, 3, fake, fake, 1 << 20, _null()) == U
    assert lib.lattice_rule_integrate_noalloc(0, 2, (1 << 48) + 1, zp, fake, 3, fake, _null()) == U
    # double-float closed state with a >= 2^31
    o = _ffi.MdiOpts()
    o.state = _ffi.STATE["closed"]
    o.precision = 3
    assert lib.mdi_lr_integrate(0, 2, 1 << 31, 4, _null(), fake, ctypes.byref(o), fake, fake, 1 << 30, _null()) == U


def test_empty_batch_is_refused(lib):
    """An empty batch (count 0) or a negative count is refused before any launch,
    as are the planner and the workspace query on it."""
    fake = ctypes.c_void_p(0x1000)
    o = _ffi.MdiOpts()
    for count in (0, -3):
        assert lib.mdi_lr_integrate_batched(fake, fake, count, count, fake, 1 << 20, ctypes.byref(o), fake, fake,
                                            1 << 30, _null()) == _ffi.MDI_EINVAL
        assert lib.mdi_batch_plan(fake, count, 1 << 20, ctypes.byref(o), fake, _null()) == _ffi.MDI_EINVAL
    b = ctypes.c_size_t()
    assert lib.mdi_lr_batched_workspace_size(0, ctypes.byref(o), ctypes.byref(b)) == _ffi.MDI_EINVAL


def test_generating_vector_argument_is_checked_on_the_host(lib):
    """Algorithm 2's z: NULL or Example 2's Korobov vector for (a, n = n_last a^(d-1));
    another vector is refused (MDI_EUNSUPPORTED), and so is any z when n does not
    fit an int64 (MDI_EOVERFLOW) -- before anything is launched."""
    fake = ctypes.c_void_p(0x1000)
    o = _ffi.MdiOpts()
    d, a, nl = 4, 16, 16
    good = mdi.korobov_vector(d, a, nl * a ** (d - 1))
    assert list(good) == [1, 16, 256, 4096]
    for bad in ([1, 16, 256, 4097], [1, 17, 289, 4913], [0, 16, 256, 4096]):
        z = np.asarray(bad, dtype=np.int64)
        zp = z.ctypes.data_as(ctypes.c_void_p)
        assert lib.mdi_lr_integrate(0, d, a, nl, zp, fake, ctypes.byref(o), fake, fake, 1 << 20,
                                    _null()) == _ffi.MDI_EUNSUPPORTED
        assert lib.mdi_lr_grad(0, d, a, nl, zp, fake, ctypes.byref(o), fake, fake, fake, 1 << 20,
                               _null()) == _ffi.MDI_EUNSUPPORTED
    big = np.ones(20, dtype=np.int64)  # n = 16^20 does not fit an int64
    assert lib.mdi_lr_integrate(0, 20, 16, 16, big.ctypes.data_as(ctypes.c_void_p), fake, ctypes.byref(o), fake,
                                fake, 1 << 20, _null()) == _ffi.MDI_EOVERFLOW
    # n_last = 1: z_d = a^(d-1) mod n = 0
    z1 = mdi.korobov_vector(3, 5, 25)
    assert list(z1) == [1, 5, 0]


def test_korobov_vector_entry_point(lib):
    z = np.zeros(5, dtype=np.int64)
    assert lib.lattice_korobov_vector(5, 3, 7, z.ctypes.data_as(ctypes.c_void_p)) == _ffi.MDI_OK
    assert list(z) == [1, 3, 2, 6, 4]
    n = (1 << 63) - 25
    assert lib.lattice_korobov_vector(3, n - 1, n, z.ctypes.data_as(ctypes.c_void_p)) == _ffi.MDI_OK
    assert list(z[:3]) == [1, n - 1, 1]  # (-1)^2 = 1 mod n, exact through 128-bit products
    assert lib.lattice_korobov_vector(0, 3, 7, z.ctypes.data_as(ctypes.c_void_p)) == _ffi.MDI_EINVAL
    assert lib.lattice_korobov_vector(3, 3, 0, z.ctypes.data_as(ctypes.c_void_p)) == _ffi.MDI_EINVAL
    assert lib.lattice_korobov_vector(3, -1, 7, z.ctypes.data_as(ctypes.c_void_p)) == _ffi.MDI_EINVAL
    assert lib.lattice_korobov_vector(3, 3, 7, _null()) == _ffi.MDI_EINVAL


def test_batch_plan_checks_the_parameter_pool(lib):
    """Every descriptor's 2*d parameters must lie inside the pool: an offset one past
    the last admissible one is refused by the planner (the kernel flags it on the
    device, where the host cannot look)."""
    descs = mdi.make_batch_descs(["gauss", "peak"], [3, 4], [8, 9], [8, 9], [0, 6])
    assert sorted(mdi.mdi_batch_plan(descs, 14)[0].tolist()) == [0, 1]
    with pytest.raises(mdi.MdiError):
        mdi.mdi_batch_plan(descs, 13)
    bad = descs.copy()
    bad["param_offset"][1] = 7
    with pytest.raises(mdi.MdiError):
        mdi.mdi_batch_plan(bad, 14)
    o = _ffi.MdiOpts()
    fake = ctypes.c_void_p(0x1000)
    assert lib.mdi_batch_plan(descs.ctypes.data_as(ctypes.c_void_p), 2, -1, ctypes.byref(o), fake,
                              _null()) == _ffi.MDI_EINVAL
    assert lib.mdi_lr_integrate_batched(fake, fake, 2, 2, fake, -1, ctypes.byref(o), fake, fake, 1 << 30,
                                        _null()) == _ffi.MDI_EINVAL
    assert lib.mdi_lr_integrate_batched(fake, fake, 2, -1, fake, 16, ctypes.byref(o), fake, fake, 1 << 30,
                                        _null()) == _ffi.MDI_EINVAL


def test_status_estimate_and_probe_validate_arguments(lib):
    fake = ctypes.c_void_p(0x1000)
    flags = ctypes.c_uint32(0)
    assert lib.mdi_get_device_status(_null(), 1 << 20, 0, ctypes.byref(flags), _null()) == _ffi.MDI_EINVAL
    assert lib.mdi_get_device_status(ctypes.c_void_p(0x1008), 1 << 20, 0, ctypes.byref(flags), _null()) == _ffi.MDI_EINVAL
    assert lib.mdi_get_device_status(fake, 8, 0, ctypes.byref(flags), _null()) == _ffi.MDI_EINVAL
    assert lib.lattice_shifted_estimate(fake, 0, fake, _null()) == _ffi.MDI_EINVAL
    assert lib.lattice_shifted_estimate(fake, 65536, fake, _null()) == _ffi.MDI_EINVAL
    assert lib.lattice_shifted_estimate(_null(), 4, fake, _null()) == _ffi.MDI_EINVAL
    assert lib.mdi_peak_probe(2, 10, fake, _null()) == _ffi.MDI_EINVAL
    assert lib.mdi_peak_probe(0, 0, fake, _null()) == _ffi.MDI_EINVAL
    assert lib.mdi_peak_probe(1, 10, _null(), _null()) == _ffi.MDI_EINVAL
    assert lib.mdi_peak_probe_threads(5) == 0
    assert _ffi.DEV_FLAGS == {"bad_desc": 1, "bad_order": 2, "unprepared": 4, "pool_range": 8}


def test_step_size_limits(lib):
    """Algorithm 1's m > 1 with the node state: FP64 value and gradient, a^m <= 4096;
    the batched call refuses it.  (No call here reaches a launch: each is refused on
    the host.)"""
    fake = ctypes.c_void_p(0x1000)
    b = ctypes.c_size_t()
    o = _ffi.MdiOpts()
    o.state, o.step = _ffi.STATE["nodes"], 2
    assert lib.mdi_lr_workspace_size(2, 10, 64, 64, ctypes.byref(o), ctypes.byref(b)) == _ffi.MDI_OK  # 64^2
    o.step = 3
    assert lib.mdi_lr_workspace_size(2, 10, 17, 17, ctypes.byref(o), ctypes.byref(b)) == _ffi.MDI_EUNSUPPORTED
    assert lib.mdi_lr_workspace_size(2, 10, 16, 16, ctypes.byref(o), ctypes.byref(b)) == _ffi.MDI_OK
    assert lib.mdi_lr_grad_workspace_size(2, 10, 16, 16, ctypes.byref(o), ctypes.byref(b)) == _ffi.MDI_OK
    assert b.value > 0
    assert lib.mdi_lr_grad_workspace_size(2, 10, 17, 17, ctypes.byref(o), ctypes.byref(b)) == _ffi.MDI_EUNSUPPORTED
    assert lib.mdi_lr_grad(2, 10, 17, 17, _null(), fake, ctypes.byref(o), fake, fake, fake, 1 << 30,
                           _null()) == _ffi.MDI_EUNSUPPORTED  # 17^3 > 4096
    o.precision = _ffi.PRECISION["df64"]
    assert lib.mdi_lr_grad(2, 10, 16, 16, _null(), fake, ctypes.byref(o), fake, fake, fake, 1 << 30,
                           _null()) == _ffi.MDI_EUNSUPPORTED  # gradients are FP64
    o.precision = _ffi.PRECISION["fp64"]
    assert lib.mdi_lr_integrate_batched(fake, fake, 4, 4, fake, 1 << 20, ctypes.byref(o), fake, fake, 1 << 30,
                                        _null()) == _ffi.MDI_EUNSUPPORTED
    o.precision = _ffi.PRECISION["df64"]
    assert lib.mdi_lr_integrate(2, 10, 16, 16, _null(), fake, ctypes.byref(o), fake, fake, 1 << 30,
                                _null()) == _ffi.MDI_EUNSUPPORTED


def test_batch_plan_split_rules(lib):
    """The planner's hybrid split: count unless the batch is all real families, with
    64-thread CTAs reading their tables through L1; otherwise within [0, count]."""
    rng = np.random.default_rng(3)
    n = 300
    a = rng.integers(8, 33, n)
    fams = ["gauss", "peak"] * (n // 2)
    descs = mdi.make_batch_descs(fams, rng.integers(6, 21, n), a, a, np.arange(n) * 40)
    _, split = mdi.mdi_batch_plan(descs, 40 * n, block=64, table_in_l1=1)
    assert 0 <= split <= n
    assert mdi.mdi_batch_plan(descs, 40 * n, block=64, table_in_l1=0)[1] == n
    assert mdi.mdi_batch_plan(descs, 40 * n, block=128, table_in_l1=1)[1] == n
    osc = mdi.make_batch_descs(["osc"] + fams[1:], rng.integers(6, 21, n), a, a, np.arange(n) * 40)
    assert mdi.mdi_batch_plan(osc, 40 * n, block=64, table_in_l1=1)[1] == n


def test_batch_plan_hybrid_order_is_longest_modelled_first(lib):
    """With the hybrid schedule's opts (64-thread CTAs, tables through L1) the order
    is a permutation that puts the longest integrals first: for one family with
    n_last = a, the work of a one-warp team grows with the levels and the passes
    per level, ceil(a / 4) (8 node pairs x 4 lanes)."""
    rng = np.random.default_rng(2)
    n = 600
    a = rng.integers(8, 33, n)
    d = rng.integers(6, 21, n)
    descs = mdi.make_batch_descs(["peak"] * n, d, a, a, np.arange(n) * 40)
    order, split = mdi.mdi_batch_plan(descs, 40 * n, block=64, table_in_l1=1, precision="fp64")
    assert sorted(order.tolist()) == list(range(n))
    assert 0 <= split <= n
    work = (descs["d"][order] - 1) * np.ceil(descs["a"][order] / 4)
    head, tail = work[: n // 20], work[-(n // 20):]
    assert head.min() > tail.max()
    assert work[0] == work.max()
