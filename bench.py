"""Benchmark of the MDI-LR hot path on GB300.

Workload (one "step"): one batched MDI-LR call over 4096 synthetic integrals of
uneven size -- d ~ U{6..20}, N ~ U{8..32} points per transformed axis (a = n_last
= N), product-peak and Gaussian integrands alternating, c_j ~ U(0.5, 2),
w_j ~ U(0, 1), node state with P = 16, FP64.  Every level of every integral runs
in one persistent kernel launch.

Printed (rank 0, one JSON line): integrals/s over the timed steps (device time,
inputs resident in HBM, L2 flushed between steps), the same metric end to end
through the C ABI from pinned host buffers, the roofline of the batched kernel,
the CPU oracle's throughput on a bounded sample, the small-workload comparison of
MDI-LR and the plain lattice kernel, and SM clocks sampled during the timed
region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank sweeps its own batch (weak scaling, no collective on
the data path); the barrier and the max over ranks bracket the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "integrals/s"
BASELINE_METRIC = "time to 1e-6 rel err, MDI-LR vs plain lattice kernel; integrals/s; % FP64 peak"
COUNT = 4096
P_NODES = 16
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
# FP64 peak derived from unit counts and clocks: 152 SMs x 2 DFMA/clk (4 flop) x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--count", type=int, default=COUNT)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_eval_fp64", "fp32_eval_df32", "df64"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="budget of the CPU oracle sample")
    ap.add_argument("--no-extras", action="store_true", help="skip the small-workload comparison")
    return ap.parse_args()


def workload_config(count, precision):
    return {"workload": f"batch of {count} MDI-LR integrals, d~U{{6..20}}, N~U{{8..32}} per transformed axis, "
                        f"product-peak/Gaussian alternating, node state P={P_NODES}",
            "count": count, "d_range": [6, 20], "N_range": [8, 32], "nodes_P": P_NODES, "precision": precision,
            "state": "nodes", "l2": "flushed between timed steps (256 MiB write)", "seed": "rank"}


def algorithmic_flops(b, P=P_NODES):
    """FP64 operations the sweep formula itself needs, counting exp and division as
    one each: per cluster point of level k >= 2: P multiply-adds of the
    interpolation (2P), u = (q + xi)/a (2), phi (4), product and sum (2); level 1:
    no interpolation; last level per point: P weights (2P: subtract, divide), the
    weighted sums (4P), normalisation (2), phi (4), product and sum (2)."""
    d = b.d.astype(np.float64)
    a = b.a.astype(np.float64)
    nl = b.n_last.astype(np.float64)
    pts_interp = np.maximum(d - 2, 0) * a * P
    pts_first = np.where(d >= 2, a * P, 0)
    return float((pts_interp * (2 * P + 8) + pts_first * 8 + nl * (6 * P + 8)).sum())


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9 and f[1].replace(".", "").isdigit():
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()),
                "reasons": sorted(reasons)}


def cpu_oracle_sample(b, budget_s, P=P_NODES, limit=None):
    """Times the FP64 CPU oracle (node state) on consecutive integrals of the batch
    until `budget_s` seconds of work are done; returns (integrals/s, how many)."""
    from oracle import oracle as o
    o.build()
    t0 = time.perf_counter()
    done = 0
    i = 0
    while True:
        it = b.integral(i % len(b))
        o.mdi_nodes(it.family, it.d, it.a, it.n_last, P, it.c, it.w)
        done += 1
        i += 1
        el = time.perf_counter() - t0
        if (limit is None and el >= budget_s) or (limit is not None and done >= limit):
            return done / el, done, el


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    from paper_2404_08867_gb300 import inputs
    b = inputs.batch(count=args.count, seed=0)
    per_step = 48
    for _ in range(args.warmup):
        cpu_oracle_sample(b, 0, limit=per_step)
    times = []
    done = 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, n, _ = cpu_oracle_sample(b, 0, limit=per_step)
        times.append(time.perf_counter() - t0)
        done += n
    value = done / sum(times)
    line = {"metric": METRIC, "value": value, "unit": "integrals/s", "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.count, "fp64"),
            "cpu_baseline": {"value": value, "unit": "integrals/s", "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} integrals of the batch per step (node state, P=16)"},
            "e2e": {"value": value, "unit": "integrals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def small_workload_extras(torch, mdi, o, inputs):
    """d = 4, N = 16, f = exp(sum x_j / j): MDI-LR and the plain lattice kernel on the
    GPU, their relative errors against the closed form, and the time each needs to
    reach 1e-6 (MDI-LR: closed state with a growing a; plain kernel: Korobov a = 12345,
    n = 2^m), measured here with CUDA events."""
    w = inputs.small_exp()
    c = torch.as_tensor(w.params).cuda()
    exact = o.closed_form("exp", 4, w.c, w.w)

    def timed(fn, reps=20):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            r = fn()
        e1.record()
        torch.cuda.synchronize()
        return r.item(), e0.elapsed_time(e1) / reps

    n = 16**4
    z = o.korobov_z(4, inputs.SMALL_SLR_A, n).astype(np.int64)
    slr_val, slr_ms = timed(lambda: mdi.lattice_rule_integrate("exp", c, n, z))
    mdi_val, mdi_ms = timed(lambda: mdi.mdi_lr_integrate("exp", c, 4, 16, 16, state="exact"))
    res = {"workload": "d=4, N=16, f=exp(sum x_j/j)", "slr_a12345_n65536": {"rel_err": abs(slr_val - exact) / exact,
                                                                         "ms": slr_ms},
           "mdi_lr_exact_N16": {"rel_err": abs(mdi_val - exact) / exact, "ms": mdi_ms}}
    # time to 1e-6 relative error
    a = 16
    while True:
        v, ms = timed(lambda: mdi.mdi_lr_integrate("exp", c, 4, a, a, state="closed"))
        if abs(v - exact) / exact <= 1e-6 or a > 1 << 24:
            res["mdi_lr_to_1e-6"] = {"a": a, "rel_err": abs(v - exact) / exact, "ms": ms}
            break
        a *= 2
    reached = None
    for m in range(16, 31):
        n = 1 << m
        z = o.korobov_z(4, inputs.SMALL_SLR_A, n).astype(np.int64)
        v, ms = timed(lambda: mdi.lattice_rule_integrate("exp", c, n, z), reps=3)
        if abs(v - exact) / exact <= 1e-6:
            reached = {"n": n, "a": inputs.SMALL_SLR_A, "rel_err": abs(v - exact) / exact, "ms": ms}
            break
        last = {"n": n, "rel_err": abs(v - exact) / exact, "ms": ms}
    res["slr_to_1e-6"] = reached if reached else {"reached": False, "largest_tried": last}
    return res


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    import paper_2404_08867_gb300 as mdi
    from paper_2404_08867_gb300 import inputs

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    b = inputs.batch(count=args.count, seed=rank)
    descs = mdi.make_batch_descs(b.families, b.d, b.a, b.n_last, b.offsets)
    order = mdi.mdi_batch_plan(descs, nodes=P_NODES)
    opts = dict(nodes=P_NODES, precision=args.precision)

    # Device-resident inputs.
    d_descs = torch.from_numpy(descs.view(np.uint8).copy()).cuda()
    d_order = torch.from_numpy(order).cuda()
    d_pool = torch.from_numpy(b.pool.copy()).cuda()
    d_out = torch.empty(len(b), dtype=torch.float64, device="cuda")
    ws = mdi.mdi_lr_batched_prepare(device="cuda", **opts)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        mdi.mdi_lr_integrate_batched(d_descs, d_pool, len(b), order=d_order, out=d_out, workspace=ws, **opts)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # evict L2 between timed steps (outside the events)
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = t.item()
    value = len(b) * world * args.steps / (total_ms / 1e3)

    # End to end through the C ABI from pinned host buffers: H2D inputs, kernel, D2H results.
    h_descs = torch.from_numpy(descs.view(np.uint8).copy()).pin_memory()
    h_order = torch.from_numpy(order.copy()).pin_memory()
    h_pool = torch.from_numpy(b.pool.copy()).pin_memory()
    h_out = torch.empty(len(b), dtype=torch.float64).pin_memory()
    e_descs, e_order, e_pool = torch.empty_like(d_descs), torch.empty_like(d_order), torch.empty_like(d_pool)
    e_out = torch.empty_like(d_out)

    def e2e_step():
        e_descs.copy_(h_descs, non_blocking=True)
        e_order.copy_(h_order, non_blocking=True)
        e_pool.copy_(h_pool, non_blocking=True)
        mdi.mdi_lr_integrate_batched(e_descs, e_pool, len(b), order=e_order, out=e_out, workspace=ws, **opts)
        h_out.copy_(e_out, non_blocking=True)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms.append(e0.elapsed_time(e1))
    e2e_total = sum(e_ms)
    if world > 1:
        t = torch.tensor([e2e_total], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_total = t.item()
    e2e_value = len(b) * world * args.steps / (e2e_total / 1e3)
    assert np.allclose(h_out.numpy(), d_out.cpu().numpy(), rtol=0, atol=0), "e2e result differs from device run"

    if rank == 0:
        flops = algorithmic_flops(b)
        kernel_ms = statistics.mean(step_ms)
        achieved = flops / (kernel_ms / 1e3) / 1e12
        line = {"metric": METRIC, "value": value, "unit": "integrals/s", "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else args.precision,
                "data": "synthetic", "config": workload_config(len(b), args.precision),
                "baseline_metric": BASELINE_METRIC, "gpu_launches": args.steps,
                "e2e": {"value": e2e_value, "unit": "integrals/s",
                        "h2d_bytes_per_step": int(h_descs.numel() + 4 * h_order.numel() + 8 * h_pool.numel()),
                        "d2h_bytes_per_step": int(8 * h_out.numel())},
                "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                             "kernel": "nodes_batched_kernel", "peak_source": "derived: 152 SMs x 4 FP64 flop/clk "
                             "x 2.07 GHz", "flops_per_launch": flops, "kernel_ms": kernel_ms},
                "clocks": clocks, "wall_s_timed_region": wall}
        if not args.no_extras:
            from oracle import oracle as o
            line["small_workload"] = small_workload_extras(torch, mdi, o, inputs)
        rate, n_done, secs = cpu_oracle_sample(b, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": "integrals/s", "cores": 1, "kind": "oracle",
                                "sample": f"first {n_done} integrals of the batch, {secs:.1f} s single-threaded"}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
