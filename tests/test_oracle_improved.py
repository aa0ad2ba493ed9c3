"""Pins of the oracle's improved lattice rule (Definition 3.3, Section 2.2.2) on
the Korobov lattice z = (1, a, .., a^(d-1)) for general n.

The ghost convention (each short line of the transformed grid continued by one
lattice step z/n, not reduced mod 1) is a reading; these tests pin what the paper
and the mathematics fix: the paper's n* = 3 for n = 81, z = (1, 7); n* as the
tensor-grid size of eq. (3.5) less the n distinct transformed points of eq. (3.1);
no ghosts and the plain rule when a^(d-1) divides n (Lemma 3.2); the ghost
positions of the paper's example worked by hand; and a closed form for an
integrand of the last coordinate alone, which fixes where the ghosts sit."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "improved_rule_example.txt")


def _rows():
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            yield [int(v) for v in line.split()]


def test_paper_example_nstar():
    # Definition 3.3's example (Figure 5's text): 3 added points.
    for n, z1, z2, nstar in _rows():
        assert z1 == 1
        _, ns = o.improved_rule("exp", 2, n, z2, [0.3, 0.7])
        assert ns == nstar


def test_paper_example_ghosts_by_hand():
    # n = 81, z = (1, 7): lines L = floor(7 j / 81) = 2, 4, 6 hold 11 of n_d = 12
    # points; their last points j = 34, 57, 80 are (34, 76)/81, (57, 75)/81,
    # (80, 74)/81, continued by (1, 7)/81 to (35, 83)/81, (58, 82)/81, (81, 81)/81.
    c = np.array([0.3, -0.45])
    ghosts = np.array([[35, 83], [58, 82], [81, 81]]) / 81.0
    lattice = 81 * o.slr("exp", 2, 81, [1, 7], c)
    expect = (lattice + np.exp(ghosts @ c).sum()) / 84
    got, ns = o.improved_rule("exp", 2, 81, 7, c)
    assert ns == 3
    assert abs(got - expect) <= 1e-15 * abs(expect)


@pytest.mark.parametrize("d,n,a", [(2, 81, 7), (3, 161, 4), (3, 1009, 10), (4, 2003, 6), (5, 3001, 5), (2, 97, 96)])
def test_nstar_is_grid_size_less_points(d, n, a):
    # eq. (3.5): n_i = a (i < d), n_d = ceil(n / a^(d-1)); the n transformed points
    # of eq. (3.1) are distinct grid points, so n* = prod n_i - n.
    z = o.korobov_z(d, a, n)
    sizes = o.grid_sizes(d, n, z)
    y = o.affine_y(d, n, z)
    assert len({tuple(np.round(r * 1e9).astype(np.int64)) for r in y}) == n
    _, ns = o.improved_rule("gauss", d, n, a, np.full(d, 0.8), np.full(d, 0.4))
    assert ns == int(np.prod(sizes.astype(np.float64))) - n


@pytest.mark.parametrize("fam", ["exp", "osc", "gauss", "peak"])
@pytest.mark.parametrize("d,a,nl", [(2, 7, 5), (3, 4, 6), (4, 3, 2), (1, 5, 37)])
def test_no_ghosts_when_grid_is_complete(fam, d, a, nl):
    # a^(d-1) | n: the lattice already is the tensor grid (Lemma 3.2), n* = 0.
    n = nl * a ** (d - 1)
    rng = np.random.default_rng(d * 100 + a)
    c, w = rng.uniform(0.3, 1.5, d), rng.uniform(0.0, 1.0, d)
    got, ns = o.improved_rule(fam, d, n, a, c, w)
    assert ns == 0
    ref = o.slr(fam, d, n, o.korobov_z(d, a, n), c, w)
    assert abs(got - ref) <= 1e-14 * abs(ref)


@pytest.mark.parametrize("d,n,a", [(2, 81, 7), (3, 161, 4), (4, 2003, 6), (3, 10007, 13)])
def test_last_coordinate_closed_form(d, n, a):
    # With gcd(a, n) = 1 the completed grid's last coordinates are r/n, r = 0..N-1,
    # each once (N = a^(d-1) ceil(n / a^(d-1))), so for f = exp(c x_d):
    #     Q = (1/N) sum_{r<N} e^{c r/n} = (e^{c N/n} - 1) / (N (e^{c/n} - 1)).
    # A ghost reduced mod 1 would sit at (r - n)/n instead and fail this.
    assert math.gcd(a, n) == 1
    cd = 1.3
    c = np.zeros(d)
    c[-1] = cd
    M = a ** (d - 1)
    N = M * (-(-n // M))
    expect = math.expm1(cd * N / n) / (N * math.expm1(cd / n))
    got, ns = o.improved_rule("exp", d, n, a, c)
    assert ns == N - n
    assert abs(got - expect) <= 1e-13 * expect
