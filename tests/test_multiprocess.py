"""The N > 1 path on the CPU: two gloo ranks (127.0.0.1) run bench.py's rank
aggregation -- every rank sweeps its own batch (weak scaling), the job time is
the slowest rank's, no collective touches the data -- and the per-rank batches
the bench draws differ by seed.  The sharded computation itself is exercised with
the CPU oracle standing in for each rank's GPU: every rank integrates its own
seed's batch, and rank 0 gathers the results (for the check only) and compares
them element by element with one process integrating the concatenated batches.
Multi-GPU runs are unmeasured on hardware: every GPU call of this build gets one
GPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2404_08867_gb300 import inputs
    local_ms = [12.0, 30.0][rank]  # the slower rank sets the job time
    value, total = bench.combine_ranks(local_ms, 4096, 10, world, dist, "cpu")
    b = inputs.batch(count=64, seed=rank)
    out[rank] = (value, total, float(b.pool.sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_weak_scaling_aggregation():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    v0, t0, s0 = out[0]
    v1, t1, s1 = out[1]
    assert t0 == t1 == 30.0
    assert v0 == v1 == pytest.approx(4096 * 2 * 10 / 0.030)
    assert s0 != s1  # each rank integrates its own batch


def _oracle_rank(rank, world, port, count, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as o
    from paper_2404_08867_gb300 import inputs
    b = inputs.batch(count=count, seed=rank)  # the bench's per-rank batch
    vals = torch.tensor([o.mdi_nodes(it.family, it.d, it.a, it.n_last, 16, it.c, it.w)
                         for it in (b.integral(i) for i in range(count))], dtype=torch.float64)
    gathered = [torch.empty(count, dtype=torch.float64) for _ in range(world)] if rank == 0 else None
    dist.gather(vals, gathered, dst=0)
    if rank == 0:
        out["vals"] = torch.cat(gathered).numpy().tolist()
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_integrals_match_one_process():
    from oracle import oracle as o
    from paper_2404_08867_gb300 import inputs
    o.build()
    count, world = 24, 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_oracle_rank, args=(world, port, count, out), nprocs=world, start_method="spawn", join=True)
    got = np.array(out["vals"])
    ref = []
    for seed in range(world):
        b = inputs.batch(count=count, seed=seed)
        ref += [o.mdi_nodes(it.family, it.d, it.a, it.n_last, 16, it.c, it.w)
                for it in (b.integral(i) for i in range(count))]
    np.testing.assert_array_equal(got, np.array(ref))


def test_single_rank_needs_no_process_group():
    import bench
    value, total = bench.combine_ranks(20.0, 4096, 5, 1)
    assert total == 20.0 and value == pytest.approx(4096 * 5 / 0.020)
