"""Step size m of Algorithm 1 on the GPU (mdi_lr_integrate with the node state and
opts step = 2, 3): every value against the oracle's step-m sweep, which is pinned
to the exact sweep and the closed state, within 1e-12 relative (absolute for the
oscillatory family)."""
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


def close(got, ref, fam, tol=TOL):
    if fam == "osc":
        assert abs(got - ref) <= tol, (got, ref)
    else:
        assert abs(got - ref) <= tol * abs(ref), (got, ref, abs(got - ref) / abs(ref))


@pytest.mark.parametrize("fam", ["gauss", "peak", "exp", "osc"])
@pytest.mark.parametrize("m", [2, 3])
@pytest.mark.parametrize("d,a,nd,P", [(1, 7, 7, 16), (2, 9, 5, 16), (3, 16, 16, 16), (6, 8, 8, 16), (7, 5, 9, 8),
                                      (12, 6, 6, 12), (20, 16, 16, 16), (31, 3, 4, 32), (40, 1, 6, 16)])
def test_step_matches_oracle(fam, m, d, a, nd, P):
    params = inputs.random_product(fam, d, seed=7 * d + a + m)
    if fam == "osc":
        params[d] = 0.37
    got = mdi.mdi_lr_integrate(fam, dev(params), d, a, nd, state="nodes", nodes=P, step=m).item()
    close(got, o.mdi_nodes_step(fam, d, a, nd, P, m, params[:d], params[d:]), fam)


@pytest.mark.parametrize("m,C", [(2, 0), (2, 1), (2, 7), (3, 0), (3, 40)])
def test_step_differentiation_config(m, C):
    """d = 100, N = 16 Gaussian (the differentiation workload's integrand), every
    checkpoint grouping of the step operators."""
    w = inputs.gaussian(100, 16, seed=0)
    got = mdi.mdi_lr_integrate("gauss", dev(w.params), 100, 16, state="nodes", step=m, checkpoint=C).item()
    close(got, o.mdi_nodes_step("gauss", 100, 16, 16, 16, m, w.c, w.w), "gauss")


def test_step_one_is_the_default_sweep():
    w = inputs.gaussian(30, 16, seed=4)
    v0 = mdi.mdi_lr_integrate("gauss", dev(w.params), 30, 16, state="nodes").item()
    v1 = mdi.mdi_lr_integrate("gauss", dev(w.params), 30, 16, state="nodes", step=1).item()
    assert v0 == v1


def test_step_closed_and_exact_states_ignore_m():
    """With the exact and closed states every m gives the same sum."""
    p = inputs.random_product("exp", 5, seed=2)
    for state in ("closed", "exact"):
        v1 = mdi.mdi_lr_integrate("exp", dev(p), 5, 8, state=state).item()
        v2 = mdi.mdi_lr_integrate("exp", dev(p), 5, 8, state=state, step=2).item()
        assert v1 == v2


def assert_grad_close(got, ref, fam, tol=TOL, floor=1e-15):
    """Per component: |g_i - ref_i| <= tol |ref_i| + floor M, M = max|ref| (2 pi for
    the oscillatory family, the bound of |df/du|), as the m = 1 adjoint's tests."""
    got, ref = np.asarray(got), np.asarray(ref)
    scale = max(np.max(np.abs(ref)), 2 * np.pi if fam == "osc" else 0.0, 1e-300)
    bad = np.flatnonzero(np.abs(got - ref) > tol * np.abs(ref) + floor * scale)
    assert bad.size == 0, (bad[:5].tolist(), got[bad[:5]].tolist(), ref[bad[:5]].tolist())


@pytest.mark.parametrize("fam", ["gauss", "peak", "exp", "osc"])
@pytest.mark.parametrize("m", [2, 3])
@pytest.mark.parametrize("d,a,nd,P,C", [(1, 7, 7, 16, 0), (2, 9, 5, 16, 0), (4, 16, 16, 16, 1), (7, 5, 9, 8, 0),
                                        (12, 6, 6, 12, 2), (20, 8, 16, 16, 0), (31, 3, 4, 32, 5)])
def test_step_grad_matches_oracle(fam, m, d, a, nd, P, C):
    """The adjoint over the step-m operators against the oracle's forward-mode
    derivative of the step-m sweep, every component."""
    params = inputs.random_product(fam, d, seed=11 * d + a + m)
    if fam == "osc":
        params[d] = 0.37
    val, g = mdi.mdi_lr_grad(fam, dev(params), d, a, nd, state="nodes", nodes=P, step=m, checkpoint=C)
    ref = o.mdi_nodes_step_grad(fam, d, a, nd, P, m, params[:d], params[d:])
    assert_grad_close(g.cpu().numpy(), ref, fam)
    close(val.item(), o.mdi_nodes_step(fam, d, a, nd, P, m, params[:d], params[d:]), fam)


@pytest.mark.parametrize("m,C", [(2, 0), (3, 7)])
def test_step_grad_differentiation_config(m, C):
    """d = 100, N = 16 Gaussian, 200 parameters: sampled components (first, last
    and interior axes, c and w) against the oracle, which takes one forward-mode
    pass per parameter, and every component against the m = 1 adjoint (both are
    derivatives of rules exact to rounding at P = 16)."""
    w = inputs.gaussian(100, 16, seed=0)
    _, g = mdi.mdi_lr_grad("gauss", dev(w.params), 100, 16, state="nodes", step=m, checkpoint=C)
    g = g.cpu().numpy()
    which = np.array([0, 1, 2, 3, 50, 97, 98, 99, 100, 101, 102, 150, 198, 199])
    ref = o.mdi_nodes_step_grad("gauss", 100, 16, 16, 16, m, w.c, w.w, which)
    assert_grad_close(g[which], ref, "gauss")
    _, g1 = mdi.mdi_lr_grad("gauss", dev(w.params), 100, 16, state="nodes")
    assert_grad_close(g, g1.cpu().numpy(), "gauss", tol=1e-11, floor=1e-14)
