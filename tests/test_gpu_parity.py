"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP64 results must agree within 1e-12 relative (absolute 1e-12 for the
oscillatory family, whose value can be near zero while |f| <= 1); lattice indices
must agree bit for bit.  Float-evaluation modes are held to the error a float
evaluation of phi allows (a few 1e-7 relative per factor, stated per test).
"""
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


def close(got, ref, fam, tol=TOL):
    if fam == "osc":
        assert abs(got - ref) <= tol, (got, ref, abs(got - ref))
    else:
        assert abs(got - ref) <= tol * abs(ref), (got, ref, abs(got - ref) / abs(ref))


# ----------------------------------------------------------------------------
# Lattice indices: bit-exact
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("d,n,j0,count", [(4, 65536, 0, 70000), (5, 2**63 - 25, 2**63 - 1000, 3000),
                                          (3, 10**18 + 9, 12345678901, 777), (1, 1, 0, 5), (7, 97, 50, 333)])
def test_lattice_indices_bit_exact(d, n, j0, count):
    rng = np.random.default_rng(d)
    z = ([1] + [int(v) for v in rng.integers(1, min(n, 2**62), size=d - 1)]) if n > 1 else [0] * d
    got = mdi.mdi_debug_lattice_indices(n, z, j0, count).cpu().numpy().astype(np.uint64)
    np.testing.assert_array_equal(got, o.lattice_indices(d, n, z, j0, count))
    for t in (0, count // 2, count - 1):  # Python's own integers on sampled rows
        assert [int(v) for v in got[t]] == [((j0 + t) % n) * zi % n for zi in z]


# ----------------------------------------------------------------------------
# Standard lattice rule
# ----------------------------------------------------------------------------
def test_slr_small_workload():
    """d = 4, n = 65536, z = z(12345), f = exp(sum x_j / j): the plain kernel."""
    w = inputs.small_exp()
    n = 16**4
    z = o.korobov_z(4, inputs.SMALL_SLR_A, n)
    got = mdi.lattice_rule_integrate("exp", dev(w.params), n, z.astype(np.int64)).item()
    close(got, o.slr("exp", 4, n, z, w.c, w.w), "exp")


@pytest.mark.parametrize("fam", ["exp", "osc", "gauss", "peak"])
@pytest.mark.parametrize("d,n,a", [(1, 1, 1), (1, 1000, 1), (3, 100003, 47), (9, 65537, 3), (40, 20011, 5),
                                   (6, 1_000_001, 10)])
def test_slr_matches_oracle(fam, d, n, a):
    params = inputs.random_product(fam, d, seed=d + n)
    z = o.korobov_z(d, a, n)
    got = mdi.lattice_rule_integrate(fam, dev(params), n, z.astype(np.int64)).item()
    close(got, o.slr(fam, d, n, z, params[:d], params[d:]), fam)


@pytest.mark.parametrize("fam", ["exp", "gauss", "peak", "osc"])
def test_slr_fp32_eval_error(fam):
    d, n, a = 5, 200003, 21
    params = inputs.random_product(fam, d, seed=3)
    z = o.korobov_z(d, a, n)
    got = mdi.lattice_rule_integrate(fam, dev(params), n, z.astype(np.int64), precision="fp32_eval_fp64").item()
    close(got, o.slr(fam, d, n, z, params[:d], params[d:]), fam, tol=2e-6)


@pytest.mark.parametrize("fam", ["exp", "gauss", "peak", "osc"])
@pytest.mark.parametrize("d,n,a", [(1, 1, 1), (4, 65536, 12345), (3, 1009, 76), (9, 100003, 7), (20, 40009, 3),
                                   (40, 20011, 5), (3, (1 << 25) + 3, 76543), (2, (1 << 31) - 1, 48271)])
def test_slr_df64_matches_fp64_oracle(fam, d, n, a):
    # Double-float integrand and sums; n > 2^24 takes the two-limb coordinate; OSC
    # evaluates in FP64.  The largest case is checked on a sample-free property:
    # equality with the FP64 kernel to 1e-12 (its own parity is pinned above).
    params = inputs.random_product(fam, d, seed=d + n % 1000)
    z = o.korobov_z(d, a, n)
    got = mdi.lattice_rule_integrate(fam, dev(params), n, z.astype(np.int64), precision="df64").item()
    if n < 1 << 28:
        ref = o.slr(fam, d, n, z, params[:d], params[d:])
    else:
        ref = mdi.lattice_rule_integrate(fam, dev(params), n, z.astype(np.int64)).item()
    close(got, ref, fam)


@pytest.mark.parametrize("fam,c_range,d", [("exp", (20.0, 40.0), 4), ("gauss", (4.0, 9.0), 6), ("peak", (30.0, 60.0), 12)])
def test_slr_df64_out_of_float_range_points(fam, c_range, d):
    # Arguments of exp beyond 64 in size and peak products beyond 2^100 are summed
    # in FP64; the rule must still match the FP64 oracle.
    n, a = 20011, 5
    params = inputs.random_product(fam, d, seed=11, c_range=c_range)
    z = o.korobov_z(d, a, n)
    got = mdi.lattice_rule_integrate(fam, dev(params), n, z.astype(np.int64), precision="df64").item()
    close(got, o.slr(fam, d, n, z, params[:d], params[d:]), fam)


def test_slr_df64_refuses_n_beyond_2_48():
    z = np.array([1, 3], dtype=np.int64)
    with pytest.raises(RuntimeError):
        mdi.lattice_rule_integrate("exp", dev(np.ones(4)), (1 << 48) + 1, z, precision="df64")


def test_slr_is_deterministic():
    params = inputs.random_product("gauss", 8, seed=1)
    z = o.korobov_z(8, 7, 3_000_017).astype(np.int64)
    r = [mdi.lattice_rule_integrate("gauss", dev(params), 3_000_017, z).item() for _ in range(3)]
    assert r[0] == r[1] == r[2]


# ----------------------------------------------------------------------------
# MDI-LR, exact state: equals the lattice rule on the same point set
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("fam", ["exp", "osc", "gauss", "peak"])
@pytest.mark.parametrize("d,a,nd", [(4, 16, 16), (1, 7, 7), (1, 1, 9), (3, 1, 5), (5, 3, 7), (6, 16, 16),
                                    (2, 100, 37), (8, 5, 2)])
def test_exact_state_matches_oracle(fam, d, a, nd):
    params = inputs.random_product(fam, d, seed=7 * d + a)
    got = mdi.mdi_lr_integrate(fam, dev(params), d, a, nd, state="exact").item()
    ref = o.mdi_exact(fam, d, a, nd, params[:d], params[d:])
    close(got, ref, fam)
    if d * math.log2(max(a, 2)) <= 20:
        n = nd * a ** (d - 1)
        close(got, o.slr(fam, d, n, o.korobov_z(d, a, n), params[:d], params[d:]), fam)


def test_small_workload_mdi_equals_slr_on_same_lattice():
    """The sweep with a = N = 16 and the plain kernel with a = 16, n = 16^4 give the
    same number (Lemma 3.2: the transformed lattice is the full grid)."""
    w = inputs.small_exp()
    n = 16**4
    mdi_val = mdi.mdi_lr_integrate("exp", dev(w.params), 4, 16, 16, state="exact").item()
    slr_val = mdi.lattice_rule_integrate("exp", dev(w.params), n, o.korobov_z(4, 16, n).astype(np.int64)).item()
    assert abs(mdi_val - slr_val) <= TOL * abs(slr_val)
    close(mdi_val, o.slr("exp", 4, n, o.korobov_z(4, 16, n), w.c, w.w), "exp")


# ----------------------------------------------------------------------------
# MDI-LR, closed state
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("fam", ["exp", "osc"])
@pytest.mark.parametrize("d,a,nd", [(4, 16, 16), (1, 5, 5), (7, 1, 3), (50, 32, 32), (1000, 16, 16),
                                    (2000, 2, 5), (300, 100000, 100000)])
def test_closed_state_matches_oracle(fam, d, a, nd):
    params = inputs.random_product(fam, d, seed=d, c_range=(0.05, 1.0))
    if fam == "osc":
        params[d] = 0.3
    got = mdi.mdi_lr_integrate(fam, dev(params), d, a, nd, state="closed").item()
    close(got, o.mdi_closed(fam, d, a, nd, params[:d], params[d:]), fam)


def test_closed_scale_workload():
    w = inputs.scale_exp(1000, 16)
    got = mdi.mdi_lr_integrate("exp", dev(w.params), 1000, 16, 16).item()
    close(got, o.mdi_closed("exp", 1000, 16, 16, w.c, w.w), "exp")


@pytest.mark.parametrize("prec,tol", [("fp32_eval_fp64", 1e-5), ("fp32_eval_df32", 1e-5)])
def test_closed_precision_modes(prec, tol):
    w = inputs.oscillatory(50, 32, seed=0)
    got = mdi.mdi_lr_integrate("osc", dev(w.params), 50, 32, 32, state="closed", precision=prec).item()
    close(got, o.mdi_closed("osc", 50, 32, 32, w.c, w.w), "osc", tol=tol)


@pytest.mark.parametrize("fam", ["exp", "osc"])
@pytest.mark.parametrize("d,a,nd", [(4, 16, 16), (1, 5, 5), (7, 1, 3), (50, 32, 32), (1000, 16, 16),
                                    (2000, 2, 5), (4, 65536, 65536), (300, 100000, 100000), (2, 1 << 25, 7)])
def test_closed_df64_matches_fp64_oracle(fam, d, a, nd):
    # Double-float cluster sums (exponential family; OSC evaluates in FP64) against
    # the FP64 oracle; a = 2^25 takes the two-float cluster coordinate.
    params = inputs.random_product(fam, d, seed=d + 7, c_range=(0.05, 1.0))
    if fam == "osc":
        params[d] = 0.3
    got = mdi.mdi_lr_integrate(fam, dev(params), d, a, nd, state="closed", precision="df64").item()
    close(got, o.mdi_closed(fam, d, a, nd, params[:d], params[d:]), fam)


@pytest.mark.parametrize("d,c_range", [(3, (90.0, 120.0)), (6, (20.0, 110.0))])
def test_closed_df64_large_exponents(d, c_range):
    # |gamma_k| > 64 on some or all levels: those are summed in FP64 (their terms
    # would leave the float range); the result must still be the FP64 one.
    a, nd = 64, 64
    params = inputs.random_product("exp", d, seed=3, c_range=c_range)
    got = mdi.mdi_lr_integrate("exp", dev(params), d, a, nd, state="closed", precision="df64").item()
    close(got, o.mdi_closed("exp", d, a, nd, params[:d], params[d:]), "exp")


# ----------------------------------------------------------------------------
# MDI-LR, node state
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("fam", ["gauss", "peak", "exp", "osc"])
@pytest.mark.parametrize("d,a,nd,P", [(4, 16, 16, 16), (1, 9, 9, 16), (2, 1, 5, 16), (12, 8, 8, 8), (6, 32, 13, 32),
                                      (5, 64, 64, 16), (30, 20, 20, 16), (7, 3, 100, 4)])
def test_nodes_state_matches_oracle(fam, d, a, nd, P):
    params = inputs.random_product(fam, d, seed=3 * d + a)
    got = mdi.mdi_lr_integrate(fam, dev(params), d, a, nd, state="nodes", nodes=P).item()
    close(got, o.mdi_nodes(fam, d, a, nd, P, params[:d], params[d:]), fam)


@pytest.mark.parametrize("fam", ["gauss", "peak", "exp", "osc"])
@pytest.mark.parametrize("d,a,nd,C", [(260, 16, 16, 0), (520, 12, 7, 0), (1000, 16, 16, 0), (300, 16, 16, 4),
                                      (257, 5, 9, 16)])
def test_nodes_state_deep_forward(fam, d, a, nd, C):
    """The value alone at depths with 16 or more checkpoint groups, where the chain
    runs over products of group products (one more product stage), against the
    oracle; and the same value from the adjoint call, which keeps every group
    boundary."""
    params = inputs.random_product(fam, d, seed=5 * d + a)
    got = mdi.mdi_lr_integrate(fam, dev(params), d, a, nd, state="nodes", checkpoint=C).item()
    ref = o.mdi_nodes(fam, d, a, nd, 16, params[:d], params[d:])
    close(got, ref, fam)
    val, _ = mdi.mdi_lr_grad(fam, dev(params), d, a, nd, state="nodes", checkpoint=C)
    close(val.item(), ref, fam)


@pytest.mark.parametrize("block", [32, 64, 128, 512])
def test_nodes_block_shapes(block):
    """Short integrals (d < 8) run on one CTA of the batched kernel: every block shape."""
    w = inputs.gaussian(7, 16, seed=2)
    got = mdi.mdi_lr_integrate("gauss", dev(w.params), 7, 16, 16, state="nodes", block=block).item()
    close(got, o.mdi_nodes("gauss", 7, 16, 16, 16, w.c, w.w), "gauss")


@pytest.mark.parametrize("fam", ["gauss", "peak", "osc", "exp"])
def test_level_parallel_equals_batched_kernel(fam):
    """A long integral runs parallel over levels; the persistent batched kernel (one
    CTA walking the levels) must give the same value."""
    d, a = 40, 16
    params = inputs.random_product(fam, d, seed=21)
    single = mdi.mdi_lr_integrate(fam, dev(params), d, a, a, state="nodes").item()
    descs = mdi.make_batch_descs([fam], [d], [a], [a], [0])
    batched = mdi.mdi_lr_integrate_batched(torch.from_numpy(descs.view(np.uint8)).cuda(), dev(params), 1).item()
    close(single, batched, fam)
    close(single, o.mdi_nodes(fam, d, a, a, 16, params[:d], params[d:]), fam)


def test_nodes_differentiation_workload_forward():
    w = inputs.gaussian(100, 16, seed=0)
    got = mdi.mdi_lr_integrate("gauss", dev(w.params), 100, 16, 16).item()
    close(got, o.mdi_nodes("gauss", 100, 16, 16, 16, w.c, w.w), "gauss")


@pytest.mark.parametrize("prec,tol", [("fp32_eval_fp64", 2e-5), ("fp32_eval_df32", 2e-5)])
@pytest.mark.parametrize("fam", ["gauss", "peak", "osc"])
def test_nodes_precision_modes(prec, tol, fam):
    w = inputs.oscillatory(50, 32, seed=1) if fam == "osc" else inputs.gaussian(50, 32, seed=1)
    params = w.params if fam == "osc" else inputs.random_product(fam, 50, seed=4)
    got = mdi.mdi_lr_integrate(fam, dev(params), 50, 32, 32, state="nodes", precision=prec).item()
    close(got, o.mdi_nodes(fam, 50, 32, 32, 16, params[:50], params[50:]), fam, tol=tol)


@pytest.mark.parametrize("fam", ["gauss", "peak", "exp"])
@pytest.mark.parametrize("d,a,nd,P", [(4, 16, 16, 16), (2, 1, 5, 16), (6, 32, 13, 32), (5, 64, 64, 16),
                                      (7, 3, 100, 4), (6, 24, 24, 12)])
def test_nodes_single_precision_evaluation_paired(fam, d, a, nd, P):
    # d < 8: one integral on the batched kernel's paired sweeps (P = 16 unrolled,
    # other P generic; nd != a takes the untabulated last axis).  Both modes give
    # phi the same floats, so they agree to double-float accuracy.
    params = inputs.random_product(fam, d, seed=3 * d + a)
    p = dev(params)
    ref = o.mdi_nodes(fam, d, a, nd, P, params[:d], params[d:])
    f64 = mdi.mdi_lr_integrate(fam, p, d, a, nd, state="nodes", nodes=P, precision="fp32_eval_fp64").item()
    dfs = mdi.mdi_lr_integrate(fam, p, d, a, nd, state="nodes", nodes=P, precision="fp32_eval_df32").item()
    close(f64, ref, fam, tol=2e-5)
    close(dfs, ref, fam, tol=2e-5)
    close(dfs, f64, fam, tol=1e-12)


@pytest.mark.parametrize("fam", ["gauss", "peak", "osc", "exp"])
@pytest.mark.parametrize("d,a", [(50, 32), (8, 16), (200, 20)])
def test_nodes_compensated_accumulation(fam, d, a):
    # Both single-precision-evaluation modes evaluate phi to the same floats; the
    # compensated one (level-parallel path: Dot2 cluster sums on float-pair basis
    # values) must give the FP64-accumulated result to double-float accuracy.
    params = inputs.random_product(fam, d, seed=d + a, c_range=(0.2, 1.2))
    if fam == "osc":
        params[d] = 0.3
    p = dev(params)
    ref = mdi.mdi_lr_integrate(fam, p, d, a, a, state="nodes", precision="fp32_eval_fp64").item()
    got = mdi.mdi_lr_integrate(fam, p, d, a, a, state="nodes", precision="fp32_eval_df32").item()
    close(got, ref, fam, tol=1e-12)


# ----------------------------------------------------------------------------
# Batched node state: the bench's launch configuration
# ----------------------------------------------------------------------------
def _batch_to_device(b):
    descs = mdi.make_batch_descs(b.families, b.d, b.a, b.n_last, b.offsets)
    order, _ = mdi.mdi_batch_plan(descs, b.pool.size)
    d_descs = torch.from_numpy(descs.view(np.uint8)).cuda()
    return descs, d_descs, torch.from_numpy(order).cuda(), dev(b.pool)


def test_batched_small_matches_oracle_elementwise():
    b = inputs.batch(count=193, seed=5)
    _, d_descs, d_order, pool = _batch_to_device(b)
    out = mdi.mdi_lr_integrate_batched(d_descs, pool, len(b), order=d_order).cpu().numpy()
    for i in range(len(b)):
        it = b.integral(i)
        close(out[i], o.mdi_nodes(it.family, it.d, it.a, it.n_last, 16, it.c, it.w), it.family)


_ORACLE_BATCH = {}


def oracle_batch(count, seed):
    """The oracle's FP64 node-state value (P = 16) of every integral of a batch,
    computed once per module."""
    key = (count, seed)
    if key not in _ORACLE_BATCH:
        b = inputs.batch(count=count, seed=seed)
        _ORACLE_BATCH[key] = np.array([o.mdi_nodes(it.family, it.d, it.a, it.n_last, 16, it.c, it.w)
                                       for it in (b.integral(i) for i in range(len(b)))])
    return _ORACLE_BATCH[key]


def assert_batch_close(got, ref, tol):
    rel = np.abs(got - ref) / np.abs(ref)
    bad = np.flatnonzero(~(rel <= tol))
    assert bad.size == 0, f"{bad.size} integrals beyond {tol:g}; worst {np.nanmax(rel):.3e} at {bad[:5].tolist()}"


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_batched_full_size_every_output(prec):
    """The bench's 4096-integral batch (seed 0; d ~ U{6..20}, N ~ U{8..32}) in one
    launch: every output against the oracle within 1e-12 relative, in FP64 and in
    the double-float mode; the scheduling order changes no value."""
    b = inputs.batch(count=4096, seed=0)
    _, d_descs, d_order, pool = _batch_to_device(b)
    out1 = mdi.mdi_lr_integrate_batched(d_descs, pool, len(b), order=d_order, precision=prec).cpu().numpy()
    out2 = mdi.mdi_lr_integrate_batched(d_descs, pool, len(b), precision=prec).cpu().numpy()
    np.testing.assert_array_equal(out1, out2)
    assert_batch_close(out1, oracle_batch(4096, 0), TOL)


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_batched_full_size_in_the_bench_launch_configuration(prec):
    """The same batch through the bench's own path: the autotuned launch shape
    (CTA size, table placement, hybrid split, resident CTAs per SM), captured in a
    CUDA graph and replayed: every output against the oracle within 1e-12."""
    from paper_2404_08867_gb300.tuning import BatchedMDILR
    b = inputs.batch(count=4096, seed=0)
    plan = BatchedMDILR(b.families, b.d, b.a, b.n_last, b.offsets, b.pool, precision=prec, nodes=16)
    plan.tune(reps=2)
    plan.capture()
    out = plan.run().cpu().numpy()
    assert_batch_close(out, oracle_batch(4096, 0), TOL)


@pytest.mark.parametrize("prec,block,split,cps", [("fp64", 32, None, 10), ("fp64", 64, 0, 5), ("fp64", 64, 40, 0),
                                                  ("df64", 32, None, 0), ("df64", 64, 40, 0)])
def test_batched_centres_outside_the_unit_interval(prec, block, split, cps):
    """Gaussian and peak factors centred outside [0, 1] (w in [-2, 3]): the FP64
    sweep's Gaussian recurrence guard bounds |t| by |c| (max(|w|, |1 - w|) + 1/a + 1)
    and falls back to the direct exp where that bound is large; every output
    against the oracle within 1e-12, on one- and two-warp teams and the fewer-
    workers shape.  (DF64: c <= 2.5 keeps c^2 (x - w)^2 within the mode's 80.)"""
    rng = np.random.default_rng(31)
    count = 160
    fams = ["gauss" if i % 2 == 0 else "peak" for i in range(count)]
    ds = rng.integers(3, 13, count)
    as_ = rng.choice([8, 9, 16, 24, 32], count)
    cmax = 2.5 if prec == "df64" else 3.0
    pool = np.concatenate([np.r_[rng.uniform(0.5, cmax, d), rng.uniform(-2.0, 3.0, d)] for d in ds])
    offs = np.concatenate([[0], np.cumsum(2 * ds[:-1])])
    descs = mdi.make_batch_descs(fams, ds, as_, as_, offs)
    d_descs = torch.from_numpy(descs.view(np.uint8)).cuda()
    sp = count if split is None else split
    out = mdi.mdi_lr_integrate_batched(d_descs, dev(pool), count, split=sp, precision=prec, block=block,
                                       table_in_l1=1, ctas_per_sm=cps).cpu().numpy()
    for i in range(count):
        d, a = int(ds[i]), int(as_[i])
        p = pool[offs[i]:offs[i] + 2 * d]
        close(out[i], o.mdi_nodes(fams[i], d, a, a, 16, p[:d], p[d:]), fams[i])


@pytest.mark.parametrize("prec", ["fp32_eval_fp64", "fp32_eval_df32"])
def test_batched_single_precision_evaluation_modes(prec):
    # The paired sweeps evaluate phi in float at the float coordinate (q + xi_p)/a:
    # each factor carries a few 1e-7 relative, d <= 20 factors per product.
    b = inputs.batch(count=193, seed=5)
    _, d_descs, d_order, pool = _batch_to_device(b)
    out = mdi.mdi_lr_integrate_batched(d_descs, pool, len(b), order=d_order, precision=prec).cpu().numpy()
    for i in range(len(b)):
        it = b.integral(i)
        close(out[i], o.mdi_nodes(it.family, it.d, it.a, it.n_last, 16, it.c, it.w), it.family, tol=2e-5)


def test_batched_single_precision_evaluation_modes_agree():
    # Both modes give phi the same floats; the double-float contractions must
    # reproduce the FP64 ones to double-float accuracy on the whole batch.
    b = inputs.batch(count=1024, seed=9)
    _, d_descs, d_order, pool = _batch_to_device(b)
    ref = mdi.mdi_lr_integrate_batched(d_descs, pool, len(b), order=d_order, precision="fp32_eval_fp64").cpu().numpy()
    got = mdi.mdi_lr_integrate_batched(d_descs, pool, len(b), order=d_order, precision="fp32_eval_df32").cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("prec,tol", [("fp64", TOL), ("df64", TOL), ("fp32_eval_fp64", 1e-4), ("fp32_eval_df32", 1e-4)])
def test_batched_mixed_families_and_edges(prec, tol):
    # d = 1, a = 1, a = 64, n_last = 4096 and n_last != a (the untabulated last
    # axis), d = 130 (three chunks of level constants), every family.
    fams = ["exp", "osc", "gauss", "peak", "gauss", "exp", "peak", "osc"]
    ds = [1, 2, 3, 64, 5, 130, 7, 1]
    as_ = [1, 64, 5, 2, 33, 16, 1, 3]
    nls = [4096, 3, 5, 2, 33, 16, 1, 7]
    offs = np.concatenate([[0], np.cumsum([2 * d for d in ds[:-1]])])
    pool = np.concatenate([inputs.random_product(f, d, seed=i) for i, (f, d) in enumerate(zip(fams, ds))])
    for i, f in enumerate(fams):
        if f == "osc":
            pool[offs[i] + ds[i]] = 0.17 * (i + 1)
    descs = mdi.make_batch_descs(fams, ds, as_, nls, offs)
    out = mdi.mdi_lr_integrate_batched(torch.from_numpy(descs.view(np.uint8)).cuda(), dev(pool), len(fams),
                                       precision=prec).cpu()
    for i, f in enumerate(fams):
        p = pool[offs[i]:offs[i] + 2 * ds[i]]
        close(out[i].item(), o.mdi_nodes(f, ds[i], as_[i], nls[i], 16, p[:ds[i]], p[ds[i]:]), f, tol=tol)


@pytest.mark.parametrize("prec,tol", [("df64", 1e-12), ("fp32_eval_df32", 1e-4), ("fp32_eval_fp64", 1e-4),
                                      ("fp64", 1e-12)])
def test_batched_values_beyond_the_float_range(prec, tol):
    # d = 300: the exponential integral grows to ~1e90 and the Gaussian and peak
    # ones shrink below 1e-38, outside what a float pair holds; the double-float
    # modes keep their state scaled by powers of two and must still match.
    fams = ["exp", "gauss", "peak", "exp"]
    ds = [300, 300, 260, 9]
    as_ = [16, 12, 8, 5]
    offs = np.concatenate([[0], np.cumsum([2 * d for d in ds[:-1]])])
    ranges = [(0.6, 1.6), (1.5, 2.5), (0.3, 0.6), (0.6, 1.6)]
    pool = np.concatenate([inputs.random_product(f, d, seed=40 + i, c_range=ranges[i])
                           for i, (f, d) in enumerate(zip(fams, ds))])
    descs = mdi.make_batch_descs(fams, ds, as_, as_, offs)
    out = mdi.mdi_lr_integrate_batched(torch.from_numpy(descs.view(np.uint8)).cuda(), dev(pool), len(fams),
                                       precision=prec).cpu()
    refs = []
    for i, f in enumerate(fams):
        p = pool[offs[i]:offs[i] + 2 * ds[i]]
        refs.append(o.mdi_nodes(f, ds[i], as_[i], as_[i], 16, p[:ds[i]], p[ds[i]:]))
    assert refs[0] > 1e60 and refs[1] < 1e-38 and refs[2] < 1e-38
    for i, f in enumerate(fams):
        close(out[i].item(), refs[i], f, tol=tol)


# ----------------------------------------------------------------------------
# Double-float mode (MDI_PREC_DF64): FP64-class results from the FP32 pipes,
# held to the same 1e-12 as the FP64 path.
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("fam", ["gauss", "peak", "exp", "osc"])
@pytest.mark.parametrize("d,a,nd,P", [(4, 16, 16, 16), (1, 9, 9, 16), (2, 1, 5, 16), (12, 8, 8, 8), (6, 32, 13, 32),
                                      (5, 64, 64, 16), (30, 20, 20, 16), (20, 32, 32, 16), (50, 32, 32, 16),
                                      (200, 16, 16, 16), (40, 24, 9, 12)])
def test_df64_nodes_matches_fp64_oracle(fam, d, a, nd, P):
    params = inputs.random_product(fam, d, seed=3 * d + a)
    got = mdi.mdi_lr_integrate(fam, dev(params), d, a, nd, state="nodes", nodes=P, precision="df64").item()
    close(got, o.mdi_nodes(fam, d, a, nd, P, params[:d], params[d:]), fam)


def test_df64_wide_parameter_range():
    """Larger c (steeper Gaussians and peaks) than the batch draws: the double-float
    exp and reciprocal keep 1e-12 over the state's wider dynamic range."""
    for fam, seed in (("gauss", 1), ("peak", 2), ("exp", 3)):
        params = inputs.random_product(fam, 15, seed=seed, c_range=(0.5, 4.0))
        got = mdi.mdi_lr_integrate(fam, dev(params), 15, 24, 24, state="nodes", precision="df64").item()
        close(got, o.mdi_nodes(fam, 15, 24, 24, 16, params[:15], params[15:]), fam)


@pytest.mark.parametrize("fam,state", [("exp", "closed"), ("osc", "closed"), ("gauss", "nodes"), ("peak", "nodes"),
                                       ("exp", "exact")])
def test_generating_vector_argument(fam, state):
    """Algorithm 2's z, given explicitly as Example 2's Korobov vector (from the
    library's exact routine), gives the value of the call without it, bit for bit;
    so does the adjoint."""
    d, a, nl = 5, 12, 7
    params = inputs.random_product(fam, d, seed=8)
    z = mdi.korobov_vector(d, a, nl * a ** (d - 1))
    np.testing.assert_array_equal(z.astype(np.uint64), o.korobov_z(d, a, nl * a ** (d - 1)))
    v0 = mdi.mdi_lr_integrate(fam, dev(params), d, a, nl, state=state).item()
    v1 = mdi.mdi_lr_integrate(fam, dev(params), d, a, nl, state=state, z=z).item()
    assert v0 == v1
    if state != "exact":
        _, g0 = mdi.mdi_lr_grad(fam, dev(params), d, a, nl, state=state)
        _, g1 = mdi.mdi_lr_grad(fam, dev(params), d, a, nl, state=state, z=z)
        assert torch.equal(g0, g1)
    with pytest.raises(mdi.MdiError):
        mdi.mdi_lr_integrate(fam, dev(params), d, a, nl, state=state, z=z + np.eye(1, d, 2, dtype=np.int64)[0])


@pytest.mark.parametrize("split", [0, 1000])
def test_batched_fp64_gaussian_recurrence_and_its_guard(split):
    """The FP64 sweep steps the Gaussian's factors along a lane's cluster points by a
    multiplicative recurrence when the arguments stay moderate, and evaluates each
    factor directly otherwise, on one-warp teams (split 0) and whole CTAs, at
    a = 9 ... 64.
    * Moderate Gaussians (c up to 8; the recurrence): within 1e-12 of the oracle.
    * Steep ones (c in 8 ... 40, most beyond the guard): N = a points per axis leave
      them far from resolved, and their node states span a hundred orders of
      magnitude, so the interpolation cancels and amplifies rounding-level
      differences in the factors, whoever computes them (the sweep without the
      recurrence gives the same errors).  They are held to 1e-12 or 200 times the
      oracle's own change when every c_j moves by one ulp, whichever is larger
      (the worst case here, at d = 7, a = 9, is 2.5e-11, 48 times that change,
      and the oracle itself is 7.8e-13 from the 60-digit value of its sum)."""
    rng = np.random.default_rng(77)
    count = 240
    ds = rng.integers(3, 12, count)
    as_ = rng.choice([9, 12, 17, 24, 32, 48, 64], count)
    ranges = [(0.2, 2.0), (2.0, 8.0), (8.0, 40.0)]
    pool = np.concatenate([inputs.random_product("gauss", int(d), seed=i, c_range=ranges[i % 3])
                           for i, d in enumerate(ds)])
    offs = np.concatenate([[0], np.cumsum(2 * ds[:-1])])
    descs = mdi.make_batch_descs(["gauss"] * count, ds, as_, as_, offs)
    out = mdi.mdi_lr_integrate_batched(torch.from_numpy(descs.view(np.uint8)).cuda(), dev(pool), count,
                                       split=min(split, count), precision="fp64", block=64,
                                       table_in_l1=1).cpu().numpy()
    for i in range(count):
        d, a = int(ds[i]), int(as_[i])
        p = pool[offs[i]:offs[i] + 2 * d]
        ref = o.mdi_nodes("gauss", d, a, a, 16, p[:d], p[d:])
        tol = TOL
        if i % 3 == 2:
            bumped = o.mdi_nodes("gauss", d, a, a, 16, np.nextafter(p[:d], np.inf), p[d:])
            tol = max(TOL, 200.0 * abs(bumped - ref) / abs(ref))
        assert abs(out[i] - ref) <= tol * abs(ref), (i, d, a, out[i], ref, tol)
