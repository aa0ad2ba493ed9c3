"""Adjoint sweep on the GPU (mdi_lr_grad and the autograd Function) against the
oracle's forward-mode derivative of the same rule, central differences and the
closed-form gradient.  Gradients are compared component by component: every
|g_i - ref_i| <= 1e-12 |ref_i| + 1e-15 M (the absolute floor, three orders below
the relative bound of the largest component, only matters for components at
rounding level, e.g. dQ/dw_j of a factor centred at w_j = 1/2), and in the max
norm as well.  M = max_k |ref_k| for the real families.  For the oscillatory
family M = 2 pi, the bound of |df/du| (|df/dc_j| <= 1): its cluster sums add
unit-modulus terms that can cancel to far below them, so a component is only
determined to rounding relative to those terms -- the same reason its forward
values are held to an absolute tolerance."""
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


def assert_grad_close(got, ref, tol=TOL, floor=1e-15, fam=None):
    got, ref = np.asarray(got), np.asarray(ref)
    scale = max(np.max(np.abs(ref)), 2 * np.pi if fam == "osc" else 0.0, 1e-300)
    err = np.abs(got - ref)
    bound = tol * np.abs(ref) + floor * scale
    bad = np.flatnonzero(err > bound)
    assert bad.size == 0, (f"{bad.size} components outside |g - ref| <= {tol:g}|ref| + {floor:g} max|ref|; first "
                           f"{bad[:5].tolist()}: got {got[bad[:5]].tolist()} ref {ref[bad[:5]].tolist()}")
    assert np.max(err) / scale <= tol, f"normwise relative error {np.max(err) / scale:.3e}"


@pytest.mark.parametrize("fam", ["gauss", "peak", "exp", "osc"])
@pytest.mark.parametrize("d,a,nd,P,C", [(1, 9, 9, 16, 0), (2, 5, 7, 16, 0), (6, 16, 16, 16, 0), (9, 8, 8, 8, 1),
                                        (13, 20, 11, 16, 13), (25, 32, 32, 16, 4), (40, 3, 5, 12, 7)])
def test_nodes_grad_matches_oracle(fam, d, a, nd, P, C):
    params = inputs.random_product(fam, d, seed=5 * d + a)
    if fam == "osc":
        params[d] = 0.41
    val, g = mdi.mdi_lr_grad(fam, dev(params), d, a, nd, state="nodes", nodes=P, checkpoint=C)
    ref = o.mdi_nodes_grad(fam, d, a, nd, P, params[:d], params[d:])
    assert_grad_close(g.cpu().numpy(), ref, fam=fam)
    fwd = o.mdi_nodes(fam, d, a, nd, P, params[:d], params[d:])
    assert abs(val.item() - fwd) <= TOL * max(abs(fwd), 1.0 if fam == "osc" else 0.0)


@pytest.mark.parametrize("fam", ["gauss", "peak"])
@pytest.mark.parametrize("d,a,nd,P,C", [(300, 16, 16, 16, 0), (300, 24, 11, 16, 5), (300, 16, 16, 12, 0),
                                        (520, 16, 16, 16, 40), (520, 9, 13, 16, 0), (300, 8, 8, 32, 0),
                                        (20, 6, 6, 32, 3), (12, 4, 5, 2, 2), (15, 9, 9, 4, 0)])
def test_nodes_grad_deep_matches_oracle(fam, d, a, nd, P, C):
    """Depths where the adjoint takes several levels per CTA (one recompute of each
    chain for all of them) and the group products run in two stages (C >= 8), with
    more cluster points per level than threads (a = 24), P = 12 and P = 32 (four
    lanes and eight entries per operator row), and shallow cases with P = 2, 4, 32:
    every component against the oracle."""
    params = inputs.random_product(fam, d, seed=3 * d + a)
    val, g = mdi.mdi_lr_grad(fam, dev(params), d, a, nd, state="nodes", nodes=P, checkpoint=C)
    ref = o.mdi_nodes_grad(fam, d, a, nd, P, params[:d], params[d:])
    assert_grad_close(g.cpu().numpy(), ref, fam=fam)
    fwd = o.mdi_nodes(fam, d, a, nd, P, params[:d], params[d:])
    assert abs(val.item() - fwd) <= TOL * abs(fwd)


@pytest.mark.parametrize("fam", ["exp", "osc"])
@pytest.mark.parametrize("d,a,nd", [(1, 7, 7), (4, 16, 16), (50, 32, 32), (300, 16, 16), (1500, 2, 3), (64, 1, 9)])
def test_closed_grad_matches_oracle(fam, d, a, nd):
    params = inputs.random_product(fam, d, seed=d + a, c_range=(0.05, 1.0))
    if fam == "osc":
        params[d] = 0.29
    val, g = mdi.mdi_lr_grad(fam, dev(params), d, a, nd, state="closed")
    assert_grad_close(g.cpu().numpy(), o.mdi_closed_grad(fam, d, a, nd, params[:d], params[d:]), fam=fam)
    fwd = o.mdi_closed(fam, d, a, nd, params[:d], params[d:])
    assert abs(val.item() - fwd) <= TOL * (1.0 if fam == "osc" else abs(fwd))


def test_grads_equal_lattice_gradient_small():
    """On an enumerable lattice the node-state and closed-state gradients equal the
    derivative of the lattice sum itself."""
    d, a = 4, 8
    n = a**d
    z = o.korobov_z(d, a, n)
    for fam, state in (("gauss", "nodes"), ("peak", "nodes"), ("exp", "closed"), ("osc", "closed")):
        params = inputs.random_product(fam, d, seed=17)
        _, g = mdi.mdi_lr_grad(fam, dev(params), d, a, a, state=state)
        assert_grad_close(g.cpu().numpy(), o.slr_grad(fam, d, n, z, params[:d], params[d:]), tol=2e-12, fam=fam)


def test_differentiation_workload():
    """d = 100, N = 16 Gaussian, 200 parameters, checkpoints every 10 levels: the
    adjoint against the oracle, against central differences (h = 1e-6) of the
    oracle's forward value, and against the exact integral's gradient (which
    differs by the rule's discretisation error)."""
    w = inputs.gaussian(100, 16, seed=0)
    val, g = mdi.mdi_lr_grad("gauss", dev(w.params), 100, 16, 16, state="nodes", checkpoint=10)
    g = g.cpu().numpy()
    assert_grad_close(g, o.mdi_nodes_grad("gauss", 100, 16, 16, 16, w.c, w.w))
    h = 1e-6
    for t in (0, 37, 99, 100, 150, 199):
        pp, pm = w.params.copy(), w.params.copy()
        pp[t] += h
        pm[t] -= h
        fd = (o.mdi_nodes("gauss", 100, 16, 16, 16, pp[:100], pp[100:]) -
              o.mdi_nodes("gauss", 100, 16, 16, 16, pm[:100], pm[100:])) / (2 * h)
        assert abs(g[t] - fd) <= 1e-6 * np.max(np.abs(g)), (t, g[t], fd)
    exact = o.closed_form_grad("gauss", 100, w.c, w.w)
    assert np.max(np.abs(g - exact)) / np.max(np.abs(exact)) < 0.05


@pytest.mark.parametrize("C", [1, 3, 10, 99, 200])
def test_checkpoint_interval_does_not_change_the_gradient(C):
    w = inputs.gaussian(100, 16, seed=1)
    _, g0 = mdi.mdi_lr_grad("gauss", dev(w.params), 100, 16, 16, state="nodes", checkpoint=10)
    _, g1 = mdi.mdi_lr_grad("gauss", dev(w.params), 100, 16, 16, state="nodes", checkpoint=C)
    assert_grad_close(g1.cpu().numpy(), g0.cpu().numpy(), tol=1e-14, floor=1e-16)


def test_scale_workload_gradient():
    """d = 1000, N = 16, f = exp(sum x_j / j^2): closed-state adjoint vs the oracle on
    every parameter, node-state adjoint vs the closed one."""
    w = inputs.scale_exp(1000, 16)
    _, gc = mdi.mdi_lr_grad("exp", dev(w.params), 1000, 16, 16, state="closed")
    gc = gc.cpu().numpy()
    assert_grad_close(gc, o.mdi_closed_grad("exp", 1000, 16, 16, w.c, w.w))
    _, gn = mdi.mdi_lr_grad("exp", dev(w.params), 1000, 16, 16, state="nodes")
    assert_grad_close(gn.cpu().numpy(), gc, tol=1e-12)


def test_autograd_function_backward_runs_the_adjoint():
    w = inputs.gaussian(30, 16, seed=2)
    p = dev(w.params).requires_grad_(True)
    q = mdi.mdi_lr("gauss", p, 30, 16, state="nodes")
    (3.0 * q).backward()
    _, g = mdi.mdi_lr_grad("gauss", dev(w.params), 30, 16, 16, state="nodes")
    torch.testing.assert_close(p.grad, 3.0 * g, rtol=0, atol=0)
    assert abs(q.item() - o.mdi_nodes("gauss", 30, 16, 16, 16, w.c, w.w)) <= TOL * abs(q.item())


def test_autograd_fused_forward_and_the_two_call_path_agree():
    """With a gradient needed (FP64) the forward pass runs the adjoint call once and
    keeps its gradient; without one, or in another precision, the forward pass is
    the plain sweep and the backward pass runs the adjoint call.  Both give the
    same value (to the parity tolerance) and the adjoint's gradient."""
    w = inputs.gaussian(12, 16, seed=5)
    _, g_ref = mdi.mdi_lr_grad("gauss", dev(w.params), 12, 16, 16, state="nodes")
    p = dev(w.params).requires_grad_(True)
    q_fused = mdi.mdi_lr("gauss", p, 12, 16, state="nodes")
    q_fused.backward()
    torch.testing.assert_close(p.grad, g_ref, rtol=0, atol=0)
    q_plain = mdi.mdi_lr("gauss", dev(w.params), 12, 16, state="nodes")  # no gradient needed
    assert abs(q_fused.item() - q_plain.item()) <= TOL * abs(q_plain.item())
    p2 = dev(w.params).requires_grad_(True)
    q_df = mdi.mdi_lr("gauss", p2, 12, 16, state="nodes", precision="df64")  # backward: the FP64 adjoint
    q_df.backward()
    torch.testing.assert_close(p2.grad, g_ref, rtol=0, atol=0)
    assert abs(q_df.item() - q_plain.item()) <= TOL * abs(q_plain.item())


def test_autograd_matches_device_central_differences():
    w = inputs.oscillatory(20, 16, seed=3)
    p = dev(w.params).requires_grad_(True)
    (g,) = torch.autograd.grad(mdi.mdi_lr("osc", p, 20, 16, state="closed"), p)
    h = 1e-6
    for t in (0, 7, 19, 20):
        pp, pm = w.params.copy(), w.params.copy()
        pp[t] += h
        pm[t] -= h
        fd = (mdi.mdi_lr_integrate("osc", dev(pp), 20, 16, state="closed").item() -
              mdi.mdi_lr_integrate("osc", dev(pm), 20, 16, state="closed").item()) / (2 * h)
        assert abs(g[t].item() - fd) <= 1e-7, (t, g[t].item(), fd)
