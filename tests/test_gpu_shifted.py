"""Randomly shifted lattice rule on the GPU (Section 2.1) against the oracle: R
replicates (1/n) sum_j f({j z/n + Delta_r}) in one call."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as o
import paper_2404_08867_gb300 as mdi
from paper_2404_08867_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_08867_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).cuda()


@pytest.mark.parametrize("fam", ["exp", "osc", "gauss", "peak"])
@pytest.mark.parametrize("d,n,a,R", [(1, 1, 1, 2), (3, 1009, 76, 5), (9, 65536, 12345, 3), (40, 20011, 5, 2),
                                     (2, 100003, 1234, 7)])
def test_shifted_replicates_match_oracle(fam, d, n, a, R):
    params = inputs.random_product(fam, d, seed=d + R, c_range=(0.2, 0.8) if d >= 40 else (0.5, 2.0))
    if fam == "osc":
        params[d] = 0.61
    z = o.korobov_z(d, a, n)
    shifts = np.random.default_rng(n + d).uniform(0.0, 1.0, (R, d))
    got = mdi.lattice_rule_integrate_shifted(fam, dev(params), n, z.astype(np.int64), dev(shifts)).cpu().numpy()
    for r in range(R):
        ref = o.slr_shifted(fam, d, n, z, params[:d], params[d:], shifts[r])
        scale = max(abs(ref), 1.0) if fam == "osc" else abs(ref)
        assert abs(got[r] - ref) <= TOL * scale, (r, got[r], ref)


@pytest.mark.parametrize("fam", ["exp", "osc", "gauss", "peak"])
@pytest.mark.parametrize("d,n,a,R", [(1, 1, 1, 2), (3, 1009, 76, 5), (9, 65536, 12345, 3), (40, 20011, 5, 2),
                                     (3, (1 << 25) + 3, 76543, 2)])
def test_shifted_df64_matches_oracle(fam, d, n, a, R):
    # Double-float replicates (the shifted coordinate as a float pair, wrapped by an
    # exact subtraction of 1); n > 2^24 takes the two-limb coordinate; OSC in FP64.
    params = inputs.random_product(fam, d, seed=d + R + 1, c_range=(0.2, 0.8) if d >= 40 else (0.5, 2.0))
    if fam == "osc":
        params[d] = 0.61
    z = o.korobov_z(d, a, n)
    shifts = np.random.default_rng(n + d + 1).uniform(0.0, 1.0, (R, d))
    got = mdi.lattice_rule_integrate_shifted(fam, dev(params), n, z.astype(np.int64), dev(shifts),
                                             precision="df64").cpu().numpy()
    for r in range(R):
        ref = o.slr_shifted(fam, d, n, z, params[:d], params[d:], shifts[r])
        scale = max(abs(ref), 1.0) if fam == "osc" else abs(ref)
        assert abs(got[r] - ref) <= TOL * scale, (r, got[r], ref)


@pytest.mark.parametrize("fam", ["exp", "gauss", "peak"])
def test_zero_shift_df64_is_the_df64_lattice_rule(fam):
    d, n = 4, 65536
    params = inputs.random_product(fam, d, seed=3)
    z = o.korobov_z(d, 12345, n).astype(np.int64)
    one = mdi.lattice_rule_integrate_shifted(fam, dev(params), n, z, dev(np.zeros((1, d))), precision="df64").item()
    plain = mdi.lattice_rule_integrate(fam, dev(params), n, z, precision="df64").item()
    assert abs(one - plain) <= 1e-15 * abs(plain)


@pytest.mark.parametrize("fam", ["exp", "osc", "gauss"])
def test_zero_shift_is_the_lattice_rule_bitwise(fam):
    d, n = 4, 65536
    params = inputs.random_product(fam, d, seed=3)
    z = o.korobov_z(d, 12345, n).astype(np.int64)
    one = mdi.lattice_rule_integrate_shifted(fam, dev(params), n, z, dev(np.zeros((1, d)))).item()
    assert one == mdi.lattice_rule_integrate(fam, dev(params), n, z).item()


def test_shifted_rule_on_characters_is_exact():
    """cos(2 pi (u + h . x)): cos(2 pi (u + h . Delta)) for h in the dual lattice, 0 otherwise."""
    n, d, a = 1009, 3, 76
    z = o.korobov_z(d, a, n)
    shifts = np.random.default_rng(7).uniform(0.0, 1.0, (4, d))
    h_dual = np.array([-int(z[1]) % n, 1, 0])  # h . z = -z_1 + z_1 = 0 (mod n)
    for h in (h_dual, np.array([1, 1, 1])):
        params = np.concatenate([2.0 * math.pi * h, [0.2, 0.0, 0.0]])
        got = mdi.lattice_rule_integrate_shifted("osc", dev(params), n, z.astype(np.int64), dev(shifts)).cpu().numpy()
        dual = int(np.dot(h, z.astype(np.int64))) % n == 0
        for r in range(4):
            expect = math.cos(2.0 * math.pi * (0.2 + float(np.dot(h, shifts[r])))) if dual else 0.0
            assert abs(got[r] - expect) <= 1e-11, (h, r, got[r], expect)


def test_shift_average_estimates_the_integral_and_its_error():
    """64 uniform shifts (fixed seed): the mean is within four standard errors of the
    exact integral, and the standard error is far below the unshifted rule's error
    scale for this smooth integrand."""
    d, n = 5, 4099
    params = inputs.random_product("gauss", d, seed=11)
    z = o.korobov_z(d, 1234, n).astype(np.int64)
    shifts = np.random.default_rng(12).uniform(0.0, 1.0, (64, d))
    vals = mdi.lattice_rule_integrate_shifted("gauss", dev(params), n, z, dev(shifts))
    mean, se = mdi.shifted_estimate(vals)
    exact = o.closed_form("gauss", d, params[:d], params[d:])
    assert abs(mean.item() - exact) <= 4.0 * se.item() + 1e-15
    assert se.item() < 1e-3 * abs(exact)


@pytest.mark.parametrize("R", [1, 2, 17, 64, 1000, 65535])
def test_shifted_estimate_kernel_matches_its_definition(R):
    """The device estimate of Section 2.1 (mean of the replicates and its standard
    error, sqrt(sum (v - mean)^2 / (R (R - 1)))) against the same formulas in numpy
    on the same values, including a large common offset (the two-pass variance
    keeps the spread that a one-pass formula would cancel)."""
    vals = 3.0e6 + np.random.default_rng(R).normal(0.0, 1e-3, R)
    mean, se = mdi.shifted_estimate(dev(vals))
    ref_mean = float(np.mean(vals))
    ref_se = float(np.std(vals, ddof=1) / math.sqrt(R)) if R > 1 else 0.0
    assert abs(mean.item() - ref_mean) <= 1e-14 * abs(ref_mean)
    assert abs(se.item() - ref_se) <= 1e-9 * max(ref_se, 1e-300) if R > 1 else se.item() == 0.0
