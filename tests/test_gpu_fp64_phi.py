"""The FP64 batched sweep's own exp (Tang's table-driven method) and reciprocal
(float seed, one cubic Newton-Raphson step) against CUDA's exp and IEEE division
on the same device: within one unit in the last place over the arguments the
sweep meets (the Gaussian's -t^2, the exponential family's c u, the peak's
t^2 + 1/c^2) and far beyond them, including the fallbacks' edges."""
import numpy as np
import pytest
import torch

import paper_2404_08867_gb300 as mdi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_08867_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def ulps(got, ref):
    """|got - ref| in units of the last place of ref (doubles)."""
    spacing = np.spacing(np.abs(ref))
    return np.abs(got - ref) / spacing


def _args(kind):
    rng = np.random.default_rng(7 if kind == "exp" else 8)
    if kind == "exp":
        parts = [rng.uniform(-16.0, 0.0, 400000), rng.uniform(-4.0, 4.0, 400000), rng.uniform(-699.9, 699.9, 200000),
                 np.linspace(-1e-3, 1e-3, 20001), rng.uniform(-745.2, -700.0, 20000), rng.uniform(700.0, 709.78, 20000),
                 np.array([0.0, -0.0, 1e-300, -1e-300, 699.99, -699.99, 700.0, -700.0, -744.0, 709.0, 1e-10, -1e-10,
                           -708.4, -708.39, -745.13, -745.14, -745.15, -746.0, -1e4, 710.0, 745.2, 1e4])]
    else:
        parts = [rng.uniform(0.25, 5.0, 400000), 10.0 ** rng.uniform(-36.0, 36.0, 400000),
                 10.0 ** rng.uniform(-307.0, 307.0, 100000),
                 np.array([1.0, 2.0, 0.5, 2.0 ** -120, 2.0 ** 120, 2.0 ** -121, 2.0 ** 121, 1e-300, 1e300, 3.0,
                           5e-324, 1e-310, 2.0 ** -1022, 1.7e308, 0.0, np.inf, np.nan])]
    return np.concatenate(parts)


@pytest.mark.parametrize("kind", ["exp", "rcp"])
def test_fp64_phi_within_one_ulp_of_cuda(kind):
    xa = _args(kind)
    if kind == "exp":
        xa = np.concatenate([xa, [np.inf, -np.inf, np.nan]])
    x = torch.as_tensor(xa).cuda()
    got = mdi.mdi_debug_fp64_phi(kind, x).cpu().numpy()
    ref = (torch.exp(x) if kind == "exp" else 1.0 / x).cpu().numpy()
    same_special = (got == ref) | (np.isnan(got) & np.isnan(ref))
    fin = np.isfinite(ref)  # a zero ref counts in units of the least subnormal
    assert np.all(same_special[~fin]), x.cpu().numpy()[~fin][~same_special[~fin]]
    err = ulps(got[fin], ref[fin])
    assert err.max() <= 1.0, (kind, err.max(), x.cpu().numpy()[fin][np.argmax(err)])
    # and no systematic bias: most results are the correctly rounded ones
    assert np.mean(err == 0) > 0.5, np.mean(err == 0)
