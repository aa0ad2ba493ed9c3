"""Pins of the CPU oracle against things other than itself.

Each test ties one oracle function to a value the paper prints, a closed form,
an identity the paper states, a textbook property, or brute force in Python's
own integers; together they are chosen so that a dropped term, a wrong sign or
index, or a transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.special import fresnel

from oracle import oracle as o

from paper_tables import midpoint_case as _midpoint_case
from paper_tables import one_unit as _one_unit
from paper_tables import rows as _rows


def _fresnel_unit():
    """S = int_0^1 sin(x^2) dx and C = int_0^1 cos(x^2) dx via scipy's Fresnel integrals."""
    s, c = fresnel(math.sqrt(2.0 / math.pi))
    k = math.sqrt(math.pi / 2.0)
    return k * s, k * c


# ----------------------------------------------------------------------------
# Integer lattice arithmetic against Python's arbitrary-precision integers
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("d,a,n", [(4, 12345, 65536), (7, 3, 2**63 - 25), (30, 2**40 + 7, 2**62 + 1),
                                   (1, 5, 1), (5, 16, 16**5)])
def test_korobov_z_matches_python_pow(d, a, n):
    z = o.korobov_z(d, a, n)
    assert [int(v) for v in z] == [pow(a, i, n) for i in range(d)]


@pytest.mark.parametrize("n", [65536, 2**63 - 25, 10**18 + 9, 97])
def test_lattice_indices_match_bigint(n):
    rng = np.random.default_rng(7)
    d = 5
    z = [1] + [int(v) for v in rng.integers(1, min(n, 2**62), size=d - 1)]
    for j0 in (0, n - 3, n // 3):
        r = o.lattice_indices(d, n, z, j0, 3)
        for t in range(3):
            j = (j0 + t) % n
            assert [int(v) for v in r[t]] == [(j * zi) % n for zi in z]


# ----------------------------------------------------------------------------
# Standard lattice rule against the paper's printed SLR errors (Tables 1-1..2-2)
# ----------------------------------------------------------------------------

def _exact(integrand, d):
    if integrand in ("t1", "exp1"):
        return 1.0
    if integrand == "sinsq":
        s, c = _fresnel_unit()
        # sin(2 pi + sum x^2) = Im(prod_i e^{i x_i^2}); int_0^1 e^{i x^2} dx = C + iS
        return ((c + 1j * s) ** d).imag
    if integrand == "gauss":
        return (math.sqrt(math.pi / 2.0) * math.erf(1.0 / math.sqrt(2.0))) ** d
    raise KeyError(integrand)


@pytest.mark.parametrize("row", list(_rows("slr_printed.txt")), ids=lambda r: f"T{r[0]}-{r[1]}-n{r[3]}")
def test_slr_reproduces_printed_errors(row):
    table, integrand, d, n, a, printed = row
    d, n, a = int(d), int(n), int(a)
    z = o.korobov_z(d, a, n)
    if integrand == "t1":
        q = o.slr("t1", d, n, z, None)
    elif integrand == "sinsq":
        q = o.slr("sinsq", d, n, z, None)
    elif integrand == "exp1":
        q = o.slr("exp", d, n, z, np.ones(d)) / (math.e - 1.0) ** 3
    else:
        q = o.slr("gauss", d, n, z, np.full(d, 1.0 / math.sqrt(2.0)), np.zeros(d))
    rel = abs(q - _exact(integrand, d)) / abs(_exact(integrand, d))
    assert abs(rel - float(printed)) <= _one_unit(printed), (rel, printed)


# ----------------------------------------------------------------------------
# Tensor midpoint mode against the printed MDI-LR errors (Tables 2-1..3-3)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("row", list(_rows("midpoint_printed.txt")),
                         ids=lambda r: f"T{r[0]}-{r[1]}-d{r[2]}-N{r[3]}")
def test_midpoint_mode_reproduces_printed_mdi_errors(row):
    table, integrand, d, N, grid, printed = row
    d, N = int(d), int(N)
    Nd = [N] * d if grid == "N" else [N] * (d - 1) + [N + 1]
    fam, c, w = _midpoint_case(integrand, d)
    exact = o.closed_form(fam, d, c, w)
    rel = abs(o.midpoint_product(fam, d, Nd, c, w) - exact) / abs(exact)
    assert abs(rel - float(printed)) <= _one_unit(printed), (rel, printed)


@pytest.mark.parametrize("fam,d,Nd", [("gauss", 3, [3, 4, 5]), ("peak", 2, [7, 3]), ("osc", 3, [2, 3, 4]),
                                      ("exp", 4, [3, 3, 3, 4])])
def test_midpoint_product_equals_grid_bruteforce(fam, d, Nd):
    rng = np.random.default_rng(3)
    c, w = rng.uniform(0.5, 2.0, d), rng.uniform(0, 1, d)
    assert o.midpoint_product(fam, d, Nd, c, w) == pytest.approx(o.midpoint_grid(fam, d, Nd, c, w), rel=1e-14)


# ----------------------------------------------------------------------------
# Grid sizes (eq. 3.5) and the affine map (Theorem 3.1): the paper's examples
# ----------------------------------------------------------------------------

def test_grid_sizes_worked_examples():
    # Fig. 5: 81 points, z = (1, 7): a 7 x 12 grid with n* = 3 added points.
    Nd = o.grid_sizes(2, 81, [1, 7])
    assert list(Nd) == [7, 12] and int(np.prod(Nd)) - 81 == 3
    # Fig. 4: 161 points, z = (1, 4, 16).
    assert list(o.grid_sizes(3, 161, [1, 4, 16])) == [4, 4, 11]
    # Lemma 3.2: a = n^(1/d) gives n_1 = ... = n_d = a.
    assert list(o.grid_sizes(4, 16**4, [1, 16, 256, 4096])) == [16] * 4
    # Section 6.1 (Fig. 8): 100 points in 2-d need 2+50, 20+5 and 10+10 iterations for
    # a = 2, 20, 10; a = 10 is the least.
    its = {a: int(sum(o.grid_sizes(2, 100, [1, a]))) for a in range(2, 100)}
    assert its[2] == 52 and its[20] == 25 and its[10] == 20
    assert min(its.values()) == 20 and [a for a, v in its.items() if v == 20] == [10]


@pytest.mark.parametrize("z,n", [([1, 7], 81), ([1, 4], 81), ([1, 4, 16], 161), ([1, 2, 4], 81), ([1, 7, 49], 81)])
def test_affine_map_gives_cartesian_grid(z, n):
    """Theorem 3.1: y_j = abs(A x_j + b) lie on a Cartesian grid with n_i values on
    axis i (eq. 3.5), all n points distinct, prod n_i - n of the grid points missing."""
    d = len(z)
    y = o.affine_y(d, n, z)
    Nd = o.grid_sizes(d, n, z)
    key = np.round(y * 2**40).astype(np.int64)
    for i in range(d):
        assert len(set(key[:, i])) == int(Nd[i])
    assert len(set(map(tuple, key))) == n
    assert int(np.prod(Nd)) >= n


def test_affine_map_korobov_axis_sets():
    """Lemma 3.2: for z = (1, a, ..., a^(d-1)) and n = a^d the axis sets are
    {s / a^i : s < a} for i < d and {s a^(d-1) / n} on the last axis."""
    d, a = 3, 5
    n = a**d
    y = o.affine_y(d, n, o.korobov_z(d, a, n))
    for i in range(d - 1):
        np.testing.assert_allclose(np.unique(np.round(y[:, i], 12)), np.arange(a) / a ** (i + 1), atol=1e-12)
    np.testing.assert_allclose(np.unique(np.round(y[:, d - 1], 12)), np.arange(a) * a ** (d - 1) / n, atol=1e-12)


# ----------------------------------------------------------------------------
# The text reading: transformed grid = lattice = level sweeps (Lemma 3.2, Alg. 1-2)
# ----------------------------------------------------------------------------

CASES = [(1, 7, 5), (2, 3, 3), (3, 4, 4), (4, 16, 16), (4, 5, 3), (5, 3, 7), (6, 4, 2), (3, 12, 1)]


@pytest.mark.parametrize("fam", ["exp", "osc", "gauss", "peak"])
@pytest.mark.parametrize("d,a,nd", CASES)
def test_grid_exact_sweep_and_lattice_coincide(fam, d, a, nd):
    """For n = nd a^(d-1) the improved rule adds no point (n* = 0), so the
    transformed-grid sum, the exact level sweep and the lattice rule coincide."""
    rng = np.random.default_rng(d * 100 + a)
    c, w = rng.uniform(0.5, 2.0, d), rng.uniform(0, 1, d)
    n = nd * a ** (d - 1)
    slr = o.slr(fam, d, n, o.korobov_z(d, a, n), c, w)
    assert o.grid_korobov(fam, d, a, nd, c, w) == pytest.approx(slr, rel=1e-13, abs=1e-15)
    assert o.mdi_exact(fam, d, a, nd, c, w) == pytest.approx(slr, rel=1e-13, abs=1e-15)
    if fam in ("exp", "osc"):
        assert o.mdi_closed(fam, d, a, nd, c, w) == pytest.approx(slr, rel=1e-13, abs=1e-15)


def test_config_small_lattice_equals_sweep():
    """d = 4, 16 points per axis, f = exp(sum_j x_j / j): the SLR with a = 16 on
    n = 16^4 points and every MDI formulation give the same number."""
    d, a = 4, 16
    c = 1.0 / np.arange(1, d + 1)
    slr = o.slr("exp", d, a**d, o.korobov_z(d, a, a**d), c)
    for q in (o.mdi_exact("exp", d, a, a, c), o.mdi_closed("exp", d, a, a, c), o.mdi_nodes("exp", d, a, a, 16, c)):
        assert q == pytest.approx(slr, rel=1e-14)


def test_sweep_converges_first_order():
    """The rule is a left-endpoint-type lattice rule: the error against the exact
    integral falls like 1/a (doubling a halves it, within 2%)."""
    d = 4
    c = 1.0 / np.arange(1, d + 1)
    exact = o.closed_form("exp", d, c)
    errs = [abs(o.mdi_closed("exp", d, a, a, c) - exact) for a in (256, 512, 1024, 2048)]
    for e0, e1 in zip(errs, errs[1:]):
        assert e0 / e1 == pytest.approx(2.0, rel=0.02)


def test_closed_state_large_d_is_finite_and_converges():
    d = 1000
    c = 1.0 / np.arange(1, d + 1) ** 2
    exact = o.closed_form("exp", d, c)
    e16 = abs(o.mdi_closed("exp", d, 16, 16, c) - exact) / exact
    e64 = abs(o.mdi_closed("exp", d, 64, 64, c) - exact) / exact
    assert 0 < e64 < e16 < 1e-2


# ----------------------------------------------------------------------------
# Node state (S): interpolation properties and agreement with the exact sweep
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("P,a", [(16, 8), (16, 13), (12, 32), (5, 3)])
def test_barycentric_basis_reproduces_polynomials(P, a):
    """The basis of a P-point interpolant sums to one and reproduces every
    polynomial of degree < P exactly (textbook property of Lagrange interpolation)."""
    L = o.bary_matrix(P, a)
    xi = 0.5 * (1.0 + np.cos(np.pi * (2 * np.arange(P) + 1) / (2 * P)))
    u = (np.arange(a)[:, None] + xi[None, :]) / a
    np.testing.assert_allclose(L.sum(axis=2), 1.0, atol=1e-13)
    for m in (1, 2, P - 1):
        np.testing.assert_allclose(L @ xi**m, u**m, atol=1e-11)


@pytest.mark.parametrize("fam", ["gauss", "peak", "exp", "osc"])
@pytest.mark.parametrize("d,a,nd", [(4, 16, 16), (5, 8, 8), (6, 4, 5), (3, 32, 7), (2, 9, 9), (1, 12, 12)])
def test_nodes_state_matches_exact_sweep(fam, d, a, nd):
    rng = np.random.default_rng(11 * d + a)
    c, w = rng.uniform(0.5, 2.0, d), rng.uniform(0, 1, d)
    ex = o.mdi_exact(fam, d, a, nd, c, w)
    assert o.mdi_nodes(fam, d, a, nd, 16, c, w) == pytest.approx(ex, rel=2e-14, abs=1e-15)


def test_nodes_state_error_falls_with_P():
    d, a = 5, 8
    rng = np.random.default_rng(5)
    c, w = rng.uniform(0.5, 2.0, d), rng.uniform(0, 1, d)
    ex = o.mdi_exact("gauss", d, a, a, c, w)
    e = [abs(o.mdi_nodes("gauss", d, a, a, P, c, w) - ex) for P in (4, 6, 8, 12)]
    assert e[0] > e[1] > e[2] and e[3] < 1e-13 * abs(ex)


def test_nodes_state_equals_closed_state_large_d():
    d, a = 200, 16
    c = 1.0 / np.arange(1, d + 1) ** 2
    assert o.mdi_nodes("exp", d, a, a, 16, c) == pytest.approx(o.mdi_closed("exp", d, a, a, c), rel=1e-13)


# ----------------------------------------------------------------------------
# Closed forms against independent quadrature, gradients against differences
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("fam", ["exp", "gauss", "peak", "osc"])
def test_closed_form_matches_quadrature(fam):
    rng = np.random.default_rng(2)
    d = 3
    c, w = rng.uniform(0.3, 2.0, d), rng.uniform(0, 1, d)
    if fam == "osc":
        w = np.array([0.37, 0.0, 0.0])
    quad = 1.0 + 0j
    for j in range(d):
        if fam == "exp":
            quad *= integrate.quad(lambda x: math.exp(c[j] * x), 0, 1, epsabs=1e-15)[0]
        elif fam == "gauss":
            quad *= integrate.quad(lambda x: math.exp(-c[j] ** 2 * (x - w[j]) ** 2), 0, 1, epsabs=1e-15)[0]
        elif fam == "peak":
            quad *= integrate.quad(lambda x: 1.0 / (c[j] ** -2 + (x - w[j]) ** 2), 0, 1, epsabs=1e-15)[0]
        else:
            re = integrate.quad(lambda x: math.cos(c[j] * x), 0, 1, epsabs=1e-15)[0]
            im = integrate.quad(lambda x: math.sin(c[j] * x), 0, 1, epsabs=1e-15)[0]
            quad *= re + 1j * im
    if fam == "osc":
        quad = (np.exp(2j * np.pi * w[0]) * quad).real
    assert o.closed_form(fam, d, c, w) == pytest.approx(quad.real if isinstance(quad, complex) else quad, rel=1e-12)


@pytest.mark.parametrize("fam", ["exp", "gauss", "peak", "osc"])
def test_closed_form_grad_matches_central_difference(fam):
    rng = np.random.default_rng(4)
    d = 4
    c, w = rng.uniform(0.5, 2.0, d), rng.uniform(0, 1, d)
    g = o.closed_form_grad(fam, d, c, w)
    h = 1e-6
    for k in range(2 * d):
        if fam in ("exp", "osc") and k >= d and not (fam == "osc" and k == d):
            assert g[k] == 0.0
            continue
        cp, wp, cm, wm = c.copy(), w.copy(), c.copy(), w.copy()
        if k < d:
            cp[k] += h; cm[k] -= h
        else:
            wp[k - d] += h; wm[k - d] -= h
        fd = (o.closed_form(fam, d, cp, wp) - o.closed_form(fam, d, cm, wm)) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-7, abs=1e-9)


@pytest.mark.parametrize("fam", ["exp", "gauss", "peak", "osc"])
def test_slr_grad_matches_central_difference(fam):
    rng = np.random.default_rng(6)
    d, a = 3, 7
    n = a**d
    z = o.korobov_z(d, a, n)
    c, w = rng.uniform(0.5, 2.0, d), rng.uniform(0, 1, d)
    g = o.slr_grad(fam, d, n, z, c, w)
    h = 1e-6
    for k in range(2 * d):
        cp, wp, cm, wm = c.copy(), w.copy(), c.copy(), w.copy()
        if k < d:
            cp[k] += h; cm[k] -= h
        else:
            wp[k - d] += h; wm[k - d] -= h
        fd = (o.slr(fam, d, n, z, cp, wp) - o.slr(fam, d, n, z, cm, wm)) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-7, abs=1e-9)


@pytest.mark.parametrize("fam", ["gauss", "peak", "exp", "osc"])
@pytest.mark.parametrize("d,a,nd", [(3, 5, 5), (4, 8, 6), (2, 16, 16)])
def test_sweep_gradients_equal_lattice_gradient(fam, d, a, nd):
    """The derivative of the node sweep (and of the closed state) equals the
    derivative of the lattice sum it reproduces."""
    rng = np.random.default_rng(8 * d + a)
    c, w = rng.uniform(0.5, 2.0, d), rng.uniform(0, 1, d)
    n = nd * a ** (d - 1)
    ref = o.slr_grad(fam, d, n, o.korobov_z(d, a, n), c, w)
    scale = np.max(np.abs(ref))
    np.testing.assert_allclose(o.mdi_nodes_grad(fam, d, a, nd, 16, c, w), ref, rtol=1e-11, atol=1e-13 * scale)
    if fam in ("exp", "osc"):
        np.testing.assert_allclose(o.mdi_closed_grad(fam, d, a, nd, c, w), ref, rtol=1e-11, atol=1e-13 * scale)


def test_nodes_grad_large_d_matches_central_difference():
    d, a = 40, 16
    rng = np.random.default_rng(9)
    c, w = rng.uniform(0.2, 1.5, d), rng.uniform(0, 1, d)
    which = np.array([0, 7, d - 1, d, d + 20, 2 * d - 1])
    g = o.mdi_nodes_grad("gauss", d, a, a, 16, c, w, which)
    h = 1e-6
    for t, gv in zip(which, g):
        cp, wp, cm, wm = c.copy(), w.copy(), c.copy(), w.copy()
        if t < d:
            cp[t] += h; cm[t] -= h
        else:
            wp[t - d] += h; wm[t - d] -= h
        fd = (o.mdi_nodes("gauss", d, a, a, 16, cp, wp) - o.mdi_nodes("gauss", d, a, a, 16, cm, wm)) / (2 * h)
        assert gv == pytest.approx(fd, rel=1e-6, abs=1e-10)
