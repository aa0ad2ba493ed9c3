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


# Step size m of Algorithm 1 (eq. 2.14c): m axes per iteration, the state read
# once per m levels.
@pytest.mark.parametrize("fam", ["gauss", "peak", "exp", "osc"])
@pytest.mark.parametrize("d,a,nd", [(4, 16, 16), (5, 8, 8), (6, 4, 5), (7, 3, 4), (3, 12, 7), (2, 9, 9), (1, 5, 5)])
def test_nodes_step_matches_exact_sweep(fam, d, a, nd):
    rng = np.random.default_rng(13 * d + a)
    c, w = rng.uniform(0.5, 2.0, d), rng.uniform(0, 1, d)
    ex = o.mdi_exact(fam, d, a, nd, c, w)
    for m in (2, 3):
        assert o.mdi_nodes_step(fam, d, a, nd, 16, m, c, w) == pytest.approx(ex, rel=2e-14, abs=1e-15)


@pytest.mark.parametrize("fam", ["gauss", "peak", "exp", "osc"])
def test_nodes_step_one_is_the_m1_sweep(fam):
    for d, a, nd in ((6, 8, 8), (4, 6, 9), (9, 5, 3)):
        rng = np.random.default_rng(d + a)
        c, w = rng.uniform(0.5, 2.0, d), rng.uniform(0, 1, d)
        assert o.mdi_nodes_step(fam, d, a, nd, 16, 1, c, w) == o.mdi_nodes(fam, d, a, nd, 16, c, w)


def test_nodes_step_equals_closed_state_large_d():
    """Beyond enumerable sizes: the exponential family's node state with m = 2 and 3
    against the closed state (exact for every m), at d = 61 (m = 3 leaves no
    remainder) and d = 62 (remainders 1 and 2)."""
    for d in (61, 62):
        c = 1.0 / np.arange(1, d + 1)
        ref = o.mdi_closed("exp", d, 8, 8, c)
        for m in (2, 3):
            assert o.mdi_nodes_step("exp", d, 8, 8, 16, m, c) == pytest.approx(ref, rel=1e-13)


def test_nodes_step_converges_in_P():
    """d = 20 Gaussian (no exact sweep at this size): with m = 2 the values for
    P = 12, 16, 24 agree to rounding, and P = 6 is visibly off."""
    d, a = 20, 6
    rng = np.random.default_rng(21)
    c, w = rng.uniform(0.5, 2.0, d), rng.uniform(0, 1, d)
    v = {P: o.mdi_nodes_step("gauss", d, a, a, P, 2, c, w) for P in (6, 12, 16, 24)}
    assert abs(v[16] - v[24]) <= 1e-14 * abs(v[24]) and abs(v[12] - v[24]) <= 1e-12 * abs(v[24])
    assert abs(v[6] - v[24]) > 1e-10 * abs(v[24])


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


@pytest.mark.parametrize("fam", ["gauss", "peak", "exp", "osc"])
@pytest.mark.parametrize("d,a,nd", [(3, 5, 5), (4, 8, 6), (5, 4, 7), (2, 16, 16)])
def test_step_sweep_gradient_equals_lattice_gradient(fam, d, a, nd):
    """The derivative of the step-m node sweep (m = 2, 3) equals the derivative of
    the lattice sum it reproduces, and m = 1 is the m = 1 sweep's derivative."""
    rng = np.random.default_rng(5 * d + a)
    c, w = rng.uniform(0.5, 2.0, d), rng.uniform(0, 1, d)
    if fam == "osc":
        w[0] = 0.3
    n = nd * a ** (d - 1)
    ref = o.slr_grad(fam, d, n, o.korobov_z(d, a, n), c, w)
    scale = np.max(np.abs(ref))
    for m in (2, 3):
        np.testing.assert_allclose(o.mdi_nodes_step_grad(fam, d, a, nd, 16, m, c, w), ref, rtol=1e-11,
                                   atol=1e-13 * scale)
    np.testing.assert_array_equal(o.mdi_nodes_step_grad(fam, d, a, nd, 16, 1, c, w),
                                  o.mdi_nodes_grad(fam, d, a, nd, 16, c, w))


@pytest.mark.parametrize("fam,m", [("gauss", 2), ("peak", 3), ("osc", 2)])
def test_step_sweep_gradient_matches_central_difference(fam, m):
    """Beyond enumerable sizes (d = 14): every parameter's derivative against a
    central difference of the step-m sweep itself, h = 1e-6."""
    d, a = 14, 6
    rng = np.random.default_rng(17 + m)
    c, w = rng.uniform(0.3, 1.5, d), rng.uniform(0, 1, d)
    if fam == "osc":
        w[0] = 0.3
    g = o.mdi_nodes_step_grad(fam, d, a, a, 16, m, c, w)
    h = 1e-6
    scale = np.max(np.abs(g))
    for t in range(2 * d):
        cp, wp, cm, wm = c.copy(), w.copy(), c.copy(), w.copy()
        if t < d:
            cp[t] += h; cm[t] -= h
        else:
            wp[t - d] += h; wm[t - d] -= h
        fd = (o.mdi_nodes_step(fam, d, a, a, 16, m, cp, wp) - o.mdi_nodes_step(fam, d, a, a, 16, m, cm, wm)) / (2 * h)
        assert g[t] == pytest.approx(fd, rel=1e-6, abs=1e-9 * scale), (t, g[t], fd)


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


# ----------------------------------------------------------------------------
# Generating-vector criteria of Section 2.2: P_alpha (eq. 2.4) and the
# shift-averaged worst-case error (eq. 2.12), the Korobov search (Example 2) and
# the CBC construction (Example 3)
# ----------------------------------------------------------------------------
ZETA = {2: math.pi ** 2 / 6.0, 4: math.pi ** 4 / 90.0}


@pytest.mark.parametrize("alpha", [2, 4])
@pytest.mark.parametrize("n", [1, 2, 7, 64, 1001])
def test_p_alpha_one_dimension_closed_form(alpha, n):
    """d = 1, z = (1): the dual lattice is nZ, so the defining sum is 2 zeta(alpha) / n^alpha."""
    assert o.p_alpha(alpha, 1, n, [1]) == pytest.approx(2.0 * ZETA[alpha] / n ** alpha, rel=1e-12)


@pytest.mark.parametrize("alpha", [2, 4])
def test_p_alpha_degenerate_second_component(alpha):
    """z = (1, 0): h . z = h_1, so the dual lattice is nZ x Z and the defining sum
    factorises to (1 + 2 zeta / n^alpha)(1 + 2 zeta) - 1."""
    n = 13
    expect = (1.0 + 2.0 * ZETA[alpha] / n ** alpha) * (1.0 + 2.0 * ZETA[alpha]) - 1.0
    assert o.p_alpha(alpha, 2, n, [1, 0]) == pytest.approx(expect, rel=1e-12)


@pytest.mark.parametrize("n,z", [(5, [1, 2]), (7, [1, 3]), (11, [1, 4])])
def test_p_alpha_equals_its_dual_lattice_definition(n, z):
    """The finite form of eq. (2.4) against the definition, the sum of
    1/(hbar_1 hbar_2)^4 over the nonzero h with h . z = 0 (mod n), taken over
    |h_i| <= 300 (the omitted tail is below 2e-7)."""
    H = 300
    h = np.arange(-H, H + 1)
    hb = np.maximum(1, np.abs(h)).astype(np.float64) ** -4
    h1, h2 = np.meshgrid(h, h, indexing="ij")
    mask = ((h1 * z[0] + h2 * z[1]) % n == 0) & ~((h1 == 0) & (h2 == 0))
    brute = float((np.outer(hb, hb) * mask).sum())
    assert abs(o.p_alpha(4, 2, n, z) - brute) < 5e-7


def test_korobov_search_symmetries_and_argmin():
    """P_alpha(z(a)) = P_alpha(z(n - a)) (B_alpha(1 - x) = B_alpha(x)) and
    = P_alpha(z(a^-1 mod n)) (the same points with the coordinates reversed);
    inadmissible a (gcd(a, n) > 1) are +inf; best_a attains the minimum."""
    n, d = 210, 4
    vals, best = o.korobov_search(2, d, n, 1, n - 1)
    for a in range(1, n):
        v = vals[a - 1]
        if math.gcd(a, n) != 1:
            assert v == math.inf
            continue
        assert v == pytest.approx(vals[n - a - 1], rel=1e-12, abs=1e-15)
        assert v == pytest.approx(vals[pow(a, -1, n) - 1], rel=1e-12, abs=1e-15)
    assert vals[best - 1] == vals[np.isfinite(vals)].min()


@pytest.mark.parametrize("beta", [0.0, 1.0 / 12.0])
def test_wce2_one_dimension_closed_form(beta):
    """d = 1, z = (1): sum_{k<n} B_2(k/n) = 1/(6n), so [E^(sh)]^2 = gamma / (6 n^2) for
    any beta (beta cancels against the leading product)."""
    for n in (1, 3, 50, 997):
        assert o.wce2_shift(1, n, [1], [0.7], beta) == pytest.approx(0.7 / (6.0 * n * n), rel=1e-11)


@pytest.mark.parametrize("beta", [0.0, 0.25 - 0.5 + 1.0 / 3.0])
def test_wce2_product_form_equals_subset_form(beta):
    """The two sides of eq. (2.12): the sum over nonempty subsets nu of
    gamma_nu ((1/n) sum_k prod_{j in nu} [B_2({k z_j/n}) + beta] - beta^|nu|), with
    product weights gamma_nu = prod_{j in nu} gamma_j, equals the product form."""
    n, z, gamma = 31, [1, 12, 7], [0.9, 0.6, 0.3]
    k = np.arange(n)
    x = [((k * zj) % n) / n for zj in z]
    b2 = [xi * xi - xi + 1.0 / 6.0 for xi in x]
    total = 0.0
    for mask in range(1, 8):
        nu = [j for j in range(3) if mask >> j & 1]
        g = np.prod([gamma[j] for j in nu])
        total += g * (np.mean(np.prod([b2[j] + beta for j in nu], axis=0)) - beta ** len(nu))
    assert o.wce2_shift(3, n, z, gamma, beta) == pytest.approx(total, rel=1e-12)


def test_cbc_components_minimise_against_exhaustive_subset_form():
    """Each CBC component attains the minimum of the s-dimensional error over all
    admissible z, evaluated here with the subset form of eq. (2.12); e2 holds those
    minima; the error of the mirrored choice n - z_s is the same."""
    n, d, beta = 53, 4, 0.0
    gamma = [0.8 ** j for j in range(d)]
    z, e2 = o.cbc(d, n, gamma, beta)
    assert z[0] == 1
    k = np.arange(n)
    for s in range(1, d):
        best = math.inf
        for c in range(1, n):
            zz = [int(v) for v in z[:s]] + [c]
            x = [((k * zj) % n) / n for zj in zz]
            b2 = [xi * xi - xi + 1.0 / 6.0 for xi in x]
            tot = 0.0
            for mask in range(1, 1 << (s + 1)):
                nu = [j for j in range(s + 1) if mask >> j & 1]
                tot += np.prod([gamma[j] for j in nu]) * np.mean(np.prod([b2[j] for j in nu], axis=0))
            best = min(best, tot)
        assert e2[s] == pytest.approx(best, rel=1e-10)
        mirrored = [int(v) for v in z[:s]] + [n - int(z[s])]
        assert o.wce2_shift(s + 1, n, mirrored, gamma, beta) == pytest.approx(e2[s], rel=1e-12)


# ----------------------------------------------------------------------------
# Randomly shifted lattice rule (Section 2.1)
# ----------------------------------------------------------------------------
def test_shifted_rule_with_zero_shift_is_the_lattice_rule():
    n, d = 1009, 3
    z = o.korobov_z(d, 76, n)
    c, w = np.array([0.7, -1.1, 0.4]), np.zeros(d)
    assert o.slr_shifted("exp", d, n, z, c, w, np.zeros(d)) == o.slr("exp", d, n, z, c, w)


def test_shifted_rule_on_characters():
    """For f = cos(2 pi (u + h . x)) (the OSC family with c = 2 pi h) the shifted rule
    is exactly cos(2 pi (u + h . Delta)) when h . z = 0 (mod n) and 0 otherwise (the
    character sum over the lattice, eq. 2.3 with one Fourier mode)."""
    n, z = 31, [1, 12]
    rng = np.random.default_rng(4)
    delta = rng.uniform(0, 1, 2)
    for h in ([1, 18], [2, 5], [31, 0], [0, 1], [1, 1]):  # the first three are in the dual lattice
        c = 2.0 * math.pi * np.array(h, dtype=float)
        w = np.array([0.3, 0.0])
        dual = (h[0] * z[0] + h[1] * z[1]) % n == 0
        expect = math.cos(2.0 * math.pi * (0.3 + float(np.dot(h, delta)))) if dual else 0.0
        assert o.slr_shifted("osc", 2, n, z, c, w, delta) == pytest.approx(expect, abs=1e-12)


def test_shift_by_a_lattice_point_permutes_the_points():
    """Delta = {k0 z / n} maps the lattice onto itself: the rule is unchanged (a
    periodic integrand, so the wrap at 1 is invisible)."""
    n, z, k0 = 101, [1, 37, 56], 29
    c = 2.0 * math.pi * np.array([1.0, 2.0, -1.0])
    w = np.array([0.1, 0.0, 0.0])
    delta = np.array([(k0 * zi % n) / n for zi in z])
    assert o.slr_shifted("osc", 3, n, z, c, w, delta) == pytest.approx(o.slr("osc", 3, n, z, c, w), abs=1e-13)


# ----------------------------------------------------------------------------
# Ridge integrand of Test 7 in the paper-table mode: histogram state
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("d,N,nl", [(1, 7, 7), (2, 5, 6), (3, 4, 5), (4, 3, 4), (5, 3, 3)])
def test_midpoint_ridge_equals_grid_bruteforce(d, N, nl):
    """f_6 = (1 + sum x_i)^-(d+1): the histogram recursion equals the brute-force sum
    over the whole grid (the oracle's independent point-by-point rule)."""
    assert o.midpoint_ridge(d, N, nl) == pytest.approx(o.midpoint_grid("ridge", d, [N] * (d - 1) + [nl]), rel=1e-13)


@pytest.mark.parametrize("d", [2, 4, 6])
def test_midpoint_ridge_converges_to_the_exact_integral(d):
    """The integral of (1 + sum x_i)^-(d+1) over [0,1]^d is 1/(d+1)! (d integrations,
    each lowering the power by one, and sum_j (-1)^j C(d,j)/(1+j) = 1/(d+1)); the
    midpoint rule's error falls by 4 when N doubles."""
    exact = 1.0 / math.factorial(d + 1)
    e1 = o.midpoint_ridge(d, 12, 12) - exact
    e2 = o.midpoint_ridge(d, 24, 24) - exact
    assert abs(e2) < abs(e1)
    assert 3.6 < e1 / e2 < 4.4


def test_midpoint_ridge_general_power_against_numpy():
    """c0 = 0.5, p = 2.5, d = 2: the direct double sum in numpy."""
    N, nl = 6, 7
    x = (np.arange(N) + 0.5) / N
    y = (np.arange(nl) + 0.5) / nl
    direct = float(np.mean((0.5 + x[:, None] + y[None, :]) ** -2.5))
    assert o.midpoint_ridge(2, N, nl, 0.5, 2.5) == pytest.approx(direct, rel=1e-13)
