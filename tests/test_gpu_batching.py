"""Batched launch machinery on the GPU: the autotuner's choice, CUDA-graph
capture and replay, and the launch shapes the tuner may pick."""
import numpy as np
import pytest
import torch

from oracle import oracle as o
from paper_2404_08867_gb300 import inputs
from paper_2404_08867_gb300.tuning import CANDIDATE_BLOCKS, BatchedMDILR

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2404_08867_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _plan(b, precision):
    return BatchedMDILR(b.families, b.d, b.a, b.n_last, b.offsets, b.pool, precision=precision)


def _check_sample(b, out, k=48, seed=0, tol=TOL):
    for i in np.random.default_rng(seed).choice(len(b), k, replace=False):
        it = b.integral(int(i))
        ref = o.mdi_nodes(it.family, it.d, it.a, it.n_last, 16, it.c, it.w)
        assert abs(out[i] - ref) <= tol * abs(ref), (i, out[i], ref)


@pytest.mark.parametrize("precision", ["df64", "fp64"])
def test_tuned_graph_replay_matches_oracle_and_direct_launch(precision):
    b = inputs.batch(count=1024, seed=3)
    plan = _plan(b, precision)
    t = plan.tune(reps=2)
    assert t["block"] in CANDIDATE_BLOCKS and t["table_in_l1"] in (0, 1)
    direct = plan.launch().clone()
    plan.capture()
    r1 = plan.run().clone()
    r2 = plan.run().clone()
    torch.cuda.synchronize()
    assert torch.equal(direct, r1) and torch.equal(r1, r2)
    _check_sample(b, r1.cpu().numpy())


@pytest.mark.parametrize("precision,tol", [("df64", TOL), ("fp64", TOL), ("fp32_eval_df32", 2e-5),
                                           ("fp32_eval_fp64", 2e-5)])
@pytest.mark.parametrize("block", [32, 64, 128, 256, 512])
@pytest.mark.parametrize("table_in_l1", [0, 1])
def test_every_launch_shape_gives_the_same_values(block, table_in_l1, precision, tol):
    # Every CTA size (1..16 warps per integral, 1..16 lanes per node pair) and
    # table placement, in every precision's paired sweep.
    b = inputs.batch(count=256, seed=4)
    plan = _plan(b, precision)
    out = plan.launch(block=block, table_in_l1=table_in_l1).cpu().numpy()
    _check_sample(b, out, k=32, seed=block, tol=tol)


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_fewer_resident_ctas_give_the_same_values(precision):
    """The tuner's fewer-workers shapes (ctas_per_sm below the occupancy, one- and
    two-warp CTAs, the hybrid split for that worker count): the worker count only
    changes which CTA takes an integral, so each shape equals the default launch of
    the same CTA size and split bit for bit, and every output is within 1e-12 of
    the oracle."""
    import paper_2404_08867_gb300 as mdi
    b = inputs.batch(count=512, seed=8)
    plan = _plan(b, precision)
    ref = np.array([o.mdi_nodes(it.family, it.d, it.a, it.n_last, 16, it.c, it.w)
                    for it in (b.integral(i) for i in range(len(b)))])
    for block, cps in ((32, 8), (32, 1), (64, 4), (64, 5)):
        sp = len(b)
        if block == 64:
            _, sp = mdi.mdi_batch_plan(plan.descs_host, plan.pool_len, nodes=16, precision=precision, block=64,
                                       table_in_l1=1, ctas_per_sm=cps)
        got = plan.launch(block=block, table_in_l1=1, split=sp, ctas_per_sm=cps).clone()
        dflt = plan.launch(block=block, table_in_l1=1, split=sp).clone()
        assert torch.equal(got, dflt), (block, cps)
        g = got.cpu().numpy()
        assert np.all(np.abs(g - ref) <= TOL * np.abs(ref)), (block, cps, np.max(np.abs(g - ref) / np.abs(ref)))


def test_graph_replays_after_input_update():
    """A captured graph reads the parameter pool at replay time: new parameters
    copied into the same device buffer give new results without re-capture."""
    b = inputs.batch(count=128, seed=5)
    plan = _plan(b, "df64")
    plan.capture()
    plan.run()
    b2 = inputs.batch(count=128, seed=5)
    b2.pool = b2.pool * 0.97
    plan.pool.copy_(torch.from_numpy(b2.pool))
    out = plan.run().cpu().numpy()
    _check_sample(b2, out, k=24, seed=1)


def test_packed_host_inputs_in_one_copy():
    """A new batch of the same shape written into the plan's pinned packed host
    layout and copied in one transfer gives the same results as a plan built on it."""
    b = inputs.batch(count=256, seed=6)
    plan = _plan(b, "df64")
    plan.capture()
    plan.run()
    b2 = inputs.batch(count=256, seed=6)
    b2.pool = b2.pool * 1.03
    h = plan.host_inputs(pinned=True)
    hd, ho, hp = plan.host_views(h)
    hp.copy_(torch.from_numpy(b2.pool))
    plan.inputs.copy_(h, non_blocking=True)
    out = plan.run().cpu()
    fresh = _plan(b2, "df64")
    fresh.opts.update(plan.opts)
    assert torch.equal(out, fresh.launch().cpu())
    _check_sample(b2, out.numpy(), k=16, seed=2)


def test_bench_batch_in_the_bench_launch_configuration():
    """The bench's own workload (4096 integrals, seed 0, DF64) through the bench's
    path -- autotuned shape, CUDA-graph capture, replay -- with 96 sampled outputs
    against the oracle, and the replay equal to a direct launch of the same shape."""
    b = inputs.batch(count=4096, seed=0)
    plan = _plan(b, "df64")
    plan.tune(reps=2)
    direct = plan.launch().clone()
    plan.capture()
    replay = plan.run().clone()
    torch.cuda.synchronize()
    assert torch.equal(direct, replay)
    _check_sample(b, replay.cpu().numpy(), k=96, seed=7)


def _descs_dev(descs):
    return torch.from_numpy(descs.view(np.uint8).copy()).cuda()


@pytest.mark.parametrize("precision", ["df64", "fp64"])
def test_injected_faults_are_reported_not_run(precision):
    """Host-side fault injection: descriptors outside the limits, and one whose
    parameters run one double past the end of the pool, give NaN in their own
    output only; a zeroed (unprepared) workspace and one prepared for another node
    count (whose tag differs) give NaN everywhere; order entries outside the batch
    are skipped.  Each is rejected before the kernel touches memory for that entry,
    and each sets its flag in the workspace's device status word, which
    mdi_get_device_status reads (and clears)."""
    import paper_2404_08867_gb300 as mdi
    F = mdi._ffi.DEV_FLAGS
    b = inputs.batch(count=16, seed=2)
    descs = mdi.make_batch_descs(b.families, b.d, b.a, b.n_last, b.offsets)
    pool = torch.as_tensor(b.pool).cuda()
    ws = mdi.mdi_lr_batched_prepare(nodes=16, precision=precision)

    def run(dd, **kw):
        kw.setdefault("workspace", ws)
        return mdi.mdi_lr_integrate_batched(_descs_dev(dd), pool, 16, precision=precision, **kw)

    good = run(descs).cpu().numpy()
    assert mdi.mdi_get_device_status(ws) == 0
    bad = descs.copy()
    bad["a"][3], bad["d"][5], bad["family"][7], bad["n_last"][9], bad["param_offset"][11] = 65, 0, 9, 5000, -8
    out = run(bad).cpu().numpy()
    hit = [3, 5, 7, 9, 11]
    assert np.all(np.isnan(out[hit]))
    keep = [i for i in range(16) if i not in hit]
    np.testing.assert_array_equal(out[keep], good[keep])
    assert mdi.mdi_get_device_status(ws, clear=True) == F["bad_desc"]
    assert mdi.mdi_get_device_status(ws) == 0  # cleared
    # The last integral's 2d parameters moved one double past the pool's end.
    past = descs.copy()
    past["param_offset"][15] = pool.numel() - 2 * int(descs["d"][15]) + 1
    out = run(past).cpu().numpy()
    assert np.isnan(out[15]) and np.array_equal(out[:15], good[:15])
    assert mdi.mdi_get_device_status(ws, clear=True) == F["pool_range"]
    # At the pool's end exactly: accepted (the parameters are those of another
    # integral, so only the status is checked).
    edge = descs.copy()
    edge["param_offset"][15] = pool.numel() - 2 * int(descs["d"][15])
    assert np.all(np.isfinite(run(edge).cpu().numpy()))
    assert mdi.mdi_get_device_status(ws) == 0
    nbytes = mdi.mdi_lr_batched_workspace_size(16, nodes=16, precision=precision)
    zeroed = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    assert torch.isnan(run(descs, workspace=zeroed)).all()
    assert mdi.mdi_get_device_status(zeroed) == F["unprepared"]
    # prepared for P = 18: large enough, but its tag names another node count
    other = mdi.mdi_lr_batched_prepare(nodes=18, precision=precision)
    assert other.numel() >= nbytes
    assert torch.isnan(run(descs, workspace=other)).all()
    assert mdi.mdi_get_device_status(other) == F["unprepared"]
    order = torch.as_tensor(np.array([-1] + list(range(15)), dtype=np.int32)).cuda()
    filled = torch.full((16,), 7.0, dtype=torch.float64, device="cuda")
    out = run(descs, order=order, out=filled).cpu().numpy()
    assert out[15] == 7.0
    np.testing.assert_array_equal(out[:15], good[:15])
    assert mdi.mdi_get_device_status(ws, clear=True) == F["bad_order"]


def _oracle_values(b):
    return np.array([o.mdi_nodes(it.family, it.d, it.a, it.n_last, 16, it.c, it.w)
                     for it in (b.integral(i) for i in range(len(b)))])


@pytest.mark.parametrize("precision,tol", [("fp64", TOL), ("df64", TOL), ("fp32_eval_df32", 2e-5),
                                           ("fp32_eval_fp64", 2e-5)])
def test_hybrid_schedule_every_split(precision, tol):
    """The hybrid schedule (two-warp CTAs, tables through L1): the order's first
    `split` integrals on whole CTAs, the rest one per warp with a state of its own,
    in every precision's paired sweep.  Every split -- none, the planner's, a third,
    all -- gives every output within the mode's tolerance of the oracle; the
    one-warp and two-warp sweeps add their cluster sums in different orders, so
    values agree to rounding, not bit for bit."""
    import paper_2404_08867_gb300 as mdi
    b = inputs.batch(count=1500, seed=11)
    plan = _plan(b, precision)
    ref = _oracle_values(b)
    assert 0 <= plan.hybrid_split <= len(b)
    for split in sorted({0, plan.hybrid_split, len(b) // 3, len(b)}):
        out = plan.launch(block=64, table_in_l1=1, split=split).cpu().numpy()
        rel = np.abs(out - ref) / np.abs(ref)
        assert rel.max() <= tol, (split, rel.max())
    assert mdi.mdi_get_device_status(plan.workspace) == 0


def test_hybrid_graph_replay_and_bench_batch():
    """The bench's batch (4096, seed 0) with the planner's split, captured and
    replayed: equal to a direct launch, every output within 1e-12 of the oracle."""
    b = inputs.batch(count=4096, seed=0)
    plan = _plan(b, "fp64")
    plan.opts.update(block=64, table_in_l1=1, split=plan.hybrid_split)
    direct = plan.launch().clone()
    plan.capture()
    replay = plan.run().clone()
    torch.cuda.synchronize()
    assert torch.equal(direct, replay)
    ref = _oracle_values(b)
    assert (np.abs(replay.cpu().numpy() - ref) / np.abs(ref)).max() <= TOL


def test_hybrid_rejects_what_a_warp_cannot_run():
    """A one-warp team runs the FP64 paired sweep only: an oscillatory integral past
    the split (which the planner never produces) is rejected with NaN and a flag,
    and the others are unaffected."""
    import paper_2404_08867_gb300 as mdi
    F = mdi._ffi.DEV_FLAGS
    b = inputs.batch(count=64, seed=12)
    fams = list(b.families)
    fams[-1] = "osc"
    descs = mdi.make_batch_descs(fams, b.d, b.a, b.n_last, b.offsets)
    pool = torch.as_tensor(b.pool).cuda()
    ws = mdi.mdi_lr_batched_prepare(nodes=16, precision="fp64", block=64, table_in_l1=1)
    out = mdi.mdi_lr_integrate_batched(_descs_dev(descs), pool, 64, split=0, workspace=ws, precision="fp64",
                                       block=64, table_in_l1=1).cpu().numpy()
    assert np.isnan(out[-1]) and np.all(np.isfinite(out[:-1]))
    assert mdi.mdi_get_device_status(ws, clear=True) == F["bad_desc"]
    whole = mdi.mdi_lr_integrate_batched(_descs_dev(descs), pool, 64, workspace=ws, precision="fp64", block=64,
                                         table_in_l1=1).cpu().numpy()
    assert np.all(np.isfinite(whole)) and mdi.mdi_get_device_status(ws) == 0


@pytest.mark.parametrize("P", [8, 12, 32])
def test_hybrid_schedule_other_node_counts(P):
    """The one-warp teams of the hybrid schedule with node counts other than the
    unrolled P = 16 (8, 12 and 32 nodes: 4, 6 and 16 node pairs over 32 lanes)."""
    import paper_2404_08867_gb300 as mdi
    b = inputs.batch(count=300, seed=13)
    descs = mdi.make_batch_descs(b.families, b.d, b.a, b.n_last, b.offsets)
    order, split = mdi.mdi_batch_plan(descs, b.pool.size, nodes=P, precision="fp64", block=64, table_in_l1=1)
    pool = torch.as_tensor(b.pool).cuda()
    ws = mdi.mdi_lr_batched_prepare(nodes=P, precision="fp64", block=64, table_in_l1=1)
    for sp in sorted({0, split, 150}):
        out = mdi.mdi_lr_integrate_batched(_descs_dev(descs), pool, len(b), order=torch.from_numpy(order).cuda(),
                                           split=sp, workspace=ws, nodes=P, precision="fp64", block=64,
                                           table_in_l1=1).cpu().numpy()
        for i in range(0, len(b), 7):
            it = b.integral(i)
            ref = o.mdi_nodes(it.family, it.d, it.a, it.n_last, P, it.c, it.w)
            assert abs(out[i] - ref) <= TOL * abs(ref), (P, sp, i, out[i], ref)
    assert mdi.mdi_get_device_status(ws) == 0


@pytest.mark.parametrize("precision,big_tol", [("fp64", 1e-11), ("df64", 5e-10)])
def test_batched_maximum_dimension(precision, big_tol):
    """The batched kernel's largest dimension, d = 65536 (65535 cluster levels in one
    CTA), next to small integrals, on whole CTAs and on the hybrid schedule's warps.
    Rounding accumulates over the levels, at most about d u relative with u the
    arithmetic's unit roundoff, so this case is held to 1e-11 in FP64 (d 2^-53 =
    7.3e-12) and 5e-10 in double-float (d 2^-47 = 4.7e-10); the small ones to the
    usual 1e-12."""
    import paper_2404_08867_gb300 as mdi
    dmax = 65536
    big = inputs.random_product("gauss", dmax, seed=3, c_range=(0.05, 0.3))
    small = inputs.random_product("peak", 7, seed=4)
    pool = np.concatenate([big, small, small])
    descs = mdi.make_batch_descs(["gauss", "peak", "peak"], [dmax, 7, 7], [2, 9, 9], [3, 9, 9],
                                 [0, 2 * dmax, 2 * dmax + 14])
    ref_big = o.mdi_nodes("gauss", dmax, 2, 3, 16, big[:dmax], big[dmax:])
    ref_small = o.mdi_nodes("peak", 7, 9, 9, 16, small[:7], small[7:])
    for split in (3, 1, 0):
        out = mdi.mdi_lr_integrate_batched(_descs_dev(descs), torch.as_tensor(pool).cuda(), 3, split=split,
                                           precision=precision, block=64, table_in_l1=1).cpu().numpy()
        assert abs(out[0] - ref_big) <= big_tol * abs(ref_big), (split, out[0], ref_big)
        for v in out[1:]:
            assert abs(v - ref_small) <= TOL * abs(ref_small), (split, v, ref_small)
