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


def _check_sample(b, out, k=48, seed=0):
    for i in np.random.default_rng(seed).choice(len(b), k, replace=False):
        it = b.integral(int(i))
        ref = o.mdi_nodes(it.family, it.d, it.a, it.n_last, 16, it.c, it.w)
        assert abs(out[i] - ref) <= TOL * abs(ref), (i, out[i], ref)


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


@pytest.mark.parametrize("block", [32, 64, 128, 256, 512])
@pytest.mark.parametrize("table_in_l1", [0, 1])
def test_every_launch_shape_gives_the_same_values(block, table_in_l1):
    b = inputs.batch(count=256, seed=4)
    plan = _plan(b, "df64")
    out = plan.launch(block=block, table_in_l1=table_in_l1).cpu().numpy()
    _check_sample(b, out, k=32, seed=block)


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
