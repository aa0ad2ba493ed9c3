"""Improved lattice rule on the GPU (Definition 3.3): the n Korobov lattice points
plus the n* ghosts completing the transformed grid, against the brute-force
oracle, which builds the ghosts by extending each short line of lattice points
(the kernel instead indexes the completed grid by r = n x_d and recovers each
ghost's line as -r n^{-1} mod a^(d-1))."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as o
import paper_2404_08867_gb300 as mdi
from paper_2404_08867_gb300 import _ffi

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_08867_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def params(fam, d, seed):
    rng = np.random.default_rng(seed)
    if fam == "osc":
        c, w = rng.uniform(0.0, 1.0, d) / np.arange(1, d + 1), np.r_[rng.uniform(), np.zeros(d - 1)]
    else:
        c, w = rng.uniform(0.5, 2.0, d), rng.uniform(0.0, 1.0, d)
    return c, w


@pytest.mark.parametrize("precision,tol", [("fp64", TOL), ("df64", TOL), ("fp32_eval_fp64", 2e-5)])
@pytest.mark.parametrize("fam", ["exp", "osc", "gauss", "peak"])
@pytest.mark.parametrize("d,n,a", [(2, 81, 7), (3, 161, 4), (1, 1000, 7), (4, 2003, 6), (3, 4 * 49, 7),
                                   (6, 100003, 7), (9, 65537, 3), (2, 97, 96), (12, 30011, 2), (40, 20011, 1)])
def test_parity(fam, d, n, a, precision, tol):
    # precision applies to the n lattice points (double-float: the FP64 class of
    # the oracle; float evaluation: a few 1e-7 per factor); the ghosts are FP64.
    c, w = params(fam, d, seed=d * 7919 + n)
    ref, ns_ref = o.improved_rule(fam, d, n, a, c, w)
    got, ns = mdi.lattice_rule_integrate_improved(fam, dev(np.r_[c, w]), d, n, a, precision=precision)
    assert ns == ns_ref
    # |f| <= 1 for OSC: a float evaluation's error is absolute there
    scale = 1.0 if (fam == "osc" and precision == "fp32_eval_fp64") else abs(ref)
    err = abs(got.item() - ref) / scale
    assert err <= tol, (fam, d, n, a, got.item(), ref, err)


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_ghosts_beyond_lattice_at_large_n(precision):
    # n = 1 + 16^7 on z = (1, 16, .., 16^6): n* = 16^6 - 1 ghosts (one per line);
    # in double-float the 2.7e8 lattice coordinates take two 24-bit limbs;
    # f = exp(c x_d) has the closed form (e^{cN/n} - 1) / (N (e^{c/n} - 1)) over the
    # completed last coordinates r/n, r < N.
    d, a = 7, 16
    M = a ** (d - 1)
    n = 1 + a ** d
    N = M * (-(-n // M))
    cd = 0.9
    c = np.zeros(d)
    c[-1] = cd
    got, ns = mdi.lattice_rule_integrate_improved("exp", dev(np.r_[c, np.zeros(d)]), d, n, a, precision=precision)
    assert ns == N - n == M - 1
    expect = math.expm1(cd * N / n) / (N * math.expm1(cd / n))
    assert abs(got.item() - expect) <= 1e-12 * expect


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_wide_ghost_kernel_closed_form(precision):
    # d = 33 (the kernel's widest digit bucket), a = 2, n = 1001: M = 2^32 lines of
    # one position, so the completed grid is r = 0 .. 2^32 - 1 and 2^32 - 1001
    # ghosts carry 32-digit lines; f = exp(c x_d) has the closed form over r/n.
    d, a, n = 33, 2, 1001
    M = a ** (d - 1)
    N = M * (-(-n // M))
    cd = 2e-7  # x_d = r/n reaches N/n = 4.3e6: c N/n = 0.86 keeps the terms in [1, 2.4]
    c = np.zeros(d)
    c[-1] = cd
    got, ns = mdi.lattice_rule_integrate_improved("exp", dev(np.r_[c, np.zeros(d)]), d, n, a, precision=precision)
    assert ns == N - n
    expect = math.expm1(cd * N / n) / (N * math.expm1(cd / n))
    assert abs(got.item() - expect) <= 1e-12 * expect


def test_matches_plain_rule_without_ghosts():
    d, a, nl = 5, 6, 11
    n = nl * a ** (d - 1)
    c, w = params("gauss", d, seed=5)
    p = dev(np.r_[c, w])
    got, ns = mdi.lattice_rule_integrate_improved("gauss", p, d, n, a)
    plain = mdi.lattice_rule_integrate("gauss", p, n, o.korobov_z(d, a, n).astype(np.int64))
    assert ns == 0
    assert got.item() == plain.item()


@pytest.mark.parametrize("d,n,a", [(3, 150, 10), (2, 0, 3), (70, 1000, 2), (41, 1000, 3)])
def test_rejected(d, n, a):
    # gcd(a, n) > 1 with ghosts (M = 100, N = 200); n < 1; d > 64; a^(d-1) = 3^40
    # beyond 2^62.  Every case is refused by the host before any launch.
    p = dev(np.ones(2 * d))
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    st = _ffi.load().lattice_rule_integrate_improved(1, d, n, a, p.data_ptr(), 0, out.data_ptr(), None,
                                                     ws.data_ptr(), ws.numel(), None)
    assert st == _ffi.MDI_EINVAL
