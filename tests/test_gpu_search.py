"""Generating-vector construction on the GPU (Section 2.2) against the oracle.

Korobov search (Example 2): every candidate's P_alpha (eq. 2.4) element by element.
CBC (Example 3): the squared shift-averaged worst-case errors (eq. 2.12) after each
component.  The criteria have exact ties (a and n - a, a and a^-1 mod n; z and
n - z), so the chosen indices are not unique: each one the GPU returns must be
admissible and attain the oracle's minimum."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as o
import paper_2404_08867_gb300 as mdi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_08867_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _close_p(got, ref):
    """P_alpha = -1 + mean of products: the rounding of the mean is relative to it."""
    inf = np.isinf(ref)
    assert np.array_equal(np.isinf(got), inf)
    err = np.abs(got[~inf] - ref[~inf]) / (1.0 + np.abs(ref[~inf]))
    assert err.max(initial=0.0) <= 1e-12, err.max()


@pytest.mark.parametrize("alpha,n,d", [(2, 1009, 3), (2, 210, 4), (4, 997, 5), (2, 2, 3), (2, 1, 2), (4, 64, 9),
                                       (2, 101, 17)])
def test_korobov_values_match_oracle(alpha, n, d):
    count = n + 2  # also a = n and a = n + 1: not admissible
    vals, best = mdi.lattice_korobov_search(n, d, alpha=alpha, a_first=1, count=count)
    ref, ref_best = o.korobov_search(alpha, d, n, 1, count)
    got = vals.cpu().numpy()
    _close_p(got, ref)
    b = int(best.item())
    if ref_best == 0:
        assert b == 0
    else:
        assert math.gcd(b, n) == 1 and 1 <= b < n
        assert ref[b - 1] <= ref[ref_best - 1] + 1e-12 * (1.0 + abs(ref[ref_best - 1]))


def test_korobov_search_at_the_small_workload_size():
    """n = 65536 = 16^4, d = 4 (the small workload's lattice size): all 65535
    candidates on the GPU, 48 of them (and the winner) by the oracle."""
    n, d = 65536, 4
    vals, best = mdi.lattice_korobov_search(n, d)
    got = vals.cpu().numpy()
    rng = np.random.default_rng(0)
    picks = list(rng.choice(np.arange(1, n, 2), 48, replace=False)) + [int(best.item()), 12345, 2, 16]
    for a in picks:
        ref, _ = o.korobov_search(2, d, n, int(a), 1)
        _close_p(got[a - 1:a], ref)
    b = int(best.item())
    assert got[b - 1] == np.min(got)
    assert b % 2 == 1


@pytest.mark.parametrize("n,d,beta,gamma_kind", [(53, 4, 0.0, "geo"), (1024, 5, 0.0, "geo"),
                                                 (4093, 6, 1.0 / 12.0, "inv_sq"), (2, 3, 0.0, "geo"),
                                                 (97, 8, 0.25, "inv_sq")])
def test_cbc_steps_match_oracle(n, d, beta, gamma_kind):
    """Every CBC step the GPU takes is a correct step of Example 3: given the GPU's
    own earlier components, its e2[s] is the oracle's minimum of the (s+1)-dimensional
    error over all admissible z, and its z_s attains it.  (Exactly tied candidates --
    here z_2 in {35, 36, 61, 62} for n = 97 -- make the later components depend on
    which one is taken, so the GPU's vector is not compared with the oracle's own.)"""
    gamma = np.array([0.8 ** j for j in range(d)]) if gamma_kind == "geo" else 1.0 / np.arange(1, d + 1) ** 2
    z, e2 = mdi.lattice_cbc(n, torch.as_tensor(gamma).cuda(), beta)
    z, e2 = z.cpu().numpy().astype(np.uint64), e2.cpu().numpy()
    assert z[0] == 1
    # [E^(sh)]^2 = (mean of products) - prod_j (1 + gamma_j beta): its rounding is
    # relative to the mean of the products, not to the (small) difference
    scale = np.cumprod(1.0 + gamma * beta) + np.abs(e2)
    assert abs(e2[0] - o.wce2_shift(1, n, z[:1], gamma, beta)) <= 1e-12 * scale[0]
    for s in range(1, d):
        assert math.gcd(int(z[s]), n) == 1 and 1 <= z[s] <= max(1, n // 2)
        cand = np.concatenate([z[:s], [0]]).astype(np.uint64)
        best = math.inf
        for c in range(1, n):
            if math.gcd(c, n) != 1:
                continue
            cand[s] = c
            best = min(best, o.wce2_shift(s + 1, n, cand, gamma, beta))
        assert abs(e2[s] - best) <= 1e-12 * scale[s], (s, e2[s], best)
        assert abs(o.wce2_shift(s + 1, n, z[:s + 1], gamma, beta) - best) <= 1e-12 * scale[s]
