"""Benchmark of the MDI-LR hot path on GB300.

Workload (one "step"): one batched MDI-LR launch over 4096 synthetic integrals of
uneven size -- d ~ U{6..20}, N ~ U{8..32} points per transformed axis (a = n_last
= N), product-peak and Gaussian integrands alternating, c_j ~ U(0.5, 2),
w_j ~ U(0, 1), node state with P = 16.  Every level of every integral runs in one
persistent kernel launch, autotuned (CTA size, table placement) and replayed from
a CUDA graph.  The headline arithmetic is FP64 (the paper's); the double-float
and single-precision-evaluation modes are timed on the same batch as secondary
entries, each with its largest error against the FP64 oracle over the whole batch.

Printed (rank 0, one JSON line): integrals/s over the timed steps (device time,
inputs resident in HBM, L2 flushed between steps), the same metric end to end
(pinned host inputs copied in and results copied out inside the timed region),
the roofline of the batched kernel against FMA peaks measured in the same run,
the CPU oracle on all host cores (and on one), SM clocks sampled during the timed
region, and (unless --no-extras) the other workloads: the d = 4 comparison of
MDI-LR with the plain lattice kernel including time to 1e-6 (with a Korobov
parameter from the GPU's P_2 search, and 16 random shifts), the precision modes on
the oscillatory d = 50 integral, the adjoint on the d = 100 Gaussian, the
cost-vs-d sweep, the paper's printed MDI-LR errors recomputed in the paper-table
mode (and Test 7's ridge integrand), and the Korobov search and CBC construction
at n = 65536.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --case NAME [--repeats R]     (one workload, for profilers)
Under torchrun every rank sweeps its own batch (weak scaling, no collective on
the data path); the barrier and the max over ranks bracket the timed region.
"""
from __future__ import annotations

import argparse
import json
import math
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
# Peaks from unit counts and the maximum SM clock (2.07 GHz, 152 SMs), context
# beside the peaks the run measures with the library's FMA probe:
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12    # 2 DFMA lanes per SM per clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # 128 FFMA lanes per SM per clock
# Algorithmic flops of one node-state integral:
# d N (P C_phi + P^2) -- per level and cluster point, P evaluations of phi at
# C_phi flops each and the P^2 terms of interpolating the state.  C_phi counts an
# exp or a division as 20 flops plus the affine argument, its square and the
# scaling (Gaussian: exp(-(c (u - w))^2); peak: 1/(c^-2 + (u - w)^2)).
C_PHI = {"gauss": 25, "peak": 25, "exp": 25, "osc": 50}

# Float operations (an FMA counts 2) of the double-float primitives, by construction.
DF_FLOPS = {"u": 28, "dot_term": 15, "dot_value": 6, "acc": 15, "combine": 22,
            "phi": {"gauss": 122, "peak": 83, "exp": 93, "osc": 0}}
# The single-precision-evaluation mode with double-float sums: the coordinate is
# one float FMA, phi the float formula with exp or the reciprocal counted as one
# operation (gauss: subtract, multiply, square, exp; peak: subtract, FMA,
# reciprocal; exp: multiply, exp), the accumulation a float-by-pair Dot2 step.
F32_FLOPS = {"u": 2, "acc": 13, "phi": {"gauss": 4, "peak": 4, "exp": 2, "osc": 0}}


def exact_integral(family, d, c, w=None):
    """Closed forms of the product-form integrals over [0,1]^d (textbook
    antiderivatives of each factor), the targets of the bench's error columns:
      exp    prod_j (e^{c_j} - 1) / c_j
      gauss  prod_j sqrt(pi)/(2 c_j) (erf(c_j (1 - w_j)) + erf(c_j w_j))
      peak   prod_j c_j (atan(c_j (1 - w_j)) + atan(c_j w_j))
      osc    Re(e^{2 pi i u} prod_j (e^{i c_j} - 1)/(i c_j)),  u = w_1."""
    c = np.asarray(c, dtype=np.float64)[:d]
    w = np.zeros(d) if w is None else np.asarray(w, dtype=np.float64)[:d]
    if family == "exp":
        return float(np.prod([math.expm1(x) / x if x != 0.0 else 1.0 for x in c]))
    if family == "gauss":
        return float(np.prod([math.sqrt(math.pi) / (2 * x) * (math.erf(x * (1 - y)) + math.erf(x * y))
                              for x, y in zip(c, w)]))
    if family == "peak":
        return float(np.prod([x * (math.atan(x * (1 - y)) + math.atan(x * y)) for x, y in zip(c, w)]))
    if family == "osc":
        p = complex(math.cos(2 * math.pi * w[0]), math.sin(2 * math.pi * w[0]))
        for x in c:
            p *= (complex(math.cos(x), math.sin(x)) - 1) / complex(0.0, x) if x != 0.0 else 1.0
        return p.real
    raise ValueError(family)


def exact_gauss_grad(d, c, w):
    """Gradient of the Gaussian closed form, (dI/dc_j, dI/dw_j): with
    g_j = sqrt(pi)/(2 c_j) (erf(c_j (1 - w_j)) + erf(c_j w_j)),
      dg/dc = -g/c + ((1 - w) e^{-c^2 (1-w)^2} + w e^{-c^2 w^2}) / c,
      dg/dw = e^{-c^2 w^2} - e^{-c^2 (1-w)^2}."""
    c = np.asarray(c, dtype=np.float64)[:d]
    w = np.asarray(w, dtype=np.float64)[:d]
    g = np.sqrt(np.pi) / (2 * c) * (np.array([math.erf(x) for x in c * (1 - w)]) +
                                    np.array([math.erf(x) for x in c * w]))
    e1, e0 = np.exp(-(c * (1 - w)) ** 2), np.exp(-(c * w) ** 2)
    dgc = -g / c + ((1 - w) * e1 + w * e0) / c
    dgw = e0 - e1
    total = float(np.prod(g))
    return np.concatenate([total / g * dgc, total / g * dgw])


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--count", type=int, default=COUNT)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "df64", "fp32_eval_fp64", "fp32_eval_df32"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="budget of the CPU oracle sample (all cores)")
    ap.add_argument("--case", default=None, help="run one named workload --repeats times and exit (profiling)")
    ap.add_argument("--repeats", type=int, default=5)
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads")
    ap.add_argument("--no-tune", action="store_true", help="fixed launch shape (--block, --table-in-l1), no autotuning")
    ap.add_argument("--block", type=int, default=128, help="CTA size with --no-tune")
    ap.add_argument("--table-in-l1", type=int, default=1, choices=[0, 1], help="table placement with --no-tune")
    return ap.parse_args()


def combine_ranks(total_ms, units_per_rank, steps, world, dist=None, device="cpu"):
    """Whole-job throughput under weak scaling: every rank processes its own
    `units_per_rank` per step; the job's time is the slowest rank's (max over
    ranks, no data-path collective).  Returns (units per second, max ms)."""
    if world > 1:
        import torch
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = t.item()
    return units_per_rank * world * steps / (total_ms / 1e3), total_ms


def workload_config(count, precision):
    return {"workload": f"batch of {count} MDI-LR integrals, d~U{{6..20}}, N~U{{8..32}} per transformed axis, "
                        f"product-peak/Gaussian alternating, node state P={P_NODES}",
            "count": count, "d_range": [6, 20], "N_range": [8, 32], "nodes_P": P_NODES, "precision": precision,
            "state": "nodes", "l2": "flushed between timed steps (256 MiB write)", "seed": "rank"}


def fp64_flops(b, P=P_NODES, paired=True):
    """FP64 operations the sweep formula needs (exp and division count one): per
    cluster point of level k >= 2: interpolation 2P (paired: P, the P/2 sums and
    P/2 differences of table values shared by two mirrored points, plus one add),
    u 2, phi 4, product and sum 2; level 1 without interpolation; last level per
    point: 2P (tabulated basis) + 8."""
    d, a, nl = (x.astype(np.float64) for x in (b.d, b.a, b.n_last))
    interp = np.maximum(d - 2, 0) * a * P
    first = np.where(d >= 2, a * P, 0)
    per_point = (P + 1 if paired else 2 * P) + 8
    return float((interp * per_point + first * 8 + nl * (2 * P + 8)).sum())


def df_flops(b, P=P_NODES, paired=True, float_phi=False):
    """Float operations of the double-float formulation (FMA = 2), by construction:
    per cluster point of level k >= 2: coordinate, phi, the interpolation and the
    accumulation; level 1 without interpolation; last axis with a P-term Dot2 per
    point.  Paired (DF64, real families): one pass of P Dot2 terms (P/2 for the
    sums of the table values, P/2 for their differences) interpolates two mirrored
    points, plus per point one Dot2 value, a double-float add and a halving;
    otherwise P Dot2 terms and one value per point.  float_phi: the cluster points'
    coordinate, phi and accumulation as F32_FLOPS counts them."""
    total = 0.0
    interp_one = P * DF_FLOPS["dot_term"] + DF_FLOPS["dot_value"]
    interp_paired = P * DF_FLOPS["dot_term"] / 2 + DF_FLOPS["dot_value"] + DF_FLOPS["combine"]
    for i, fam in enumerate(b.families):
        d, a, nl = int(b.d[i]), int(b.a[i]), int(b.n_last[i])
        phi = DF_FLOPS["phi"][fam]
        pt = DF_FLOPS["u"] + phi + DF_FLOPS["acc"]
        pc = (F32_FLOPS["u"] + F32_FLOPS["phi"][fam] + F32_FLOPS["acc"]) if (float_phi and fam != "osc") else pt
        interp = interp_paired if (paired and fam != "osc") else interp_one
        total += max(d - 2, 0) * a * P * (pc + interp) + (a * P * pc if d >= 2 else 0) + nl * (pt + interp_one)
    return total


def alg_flops(b, P=P_NODES, phi=True):
    """Algorithmic flops of a batch: sum over integrals of d N (P C_phi + P^2)
    (a = n_last = N), whatever arithmetic the kernel uses to get there; without
    phi, the interpolation and contraction part d N P^2 alone."""
    d, a = b.d.astype(np.float64), b.a.astype(np.float64)
    cphi = np.array([C_PHI[f] for f in b.families], dtype=np.float64) if phi else np.zeros(len(b.d))
    return float((d * a * (P * cphi + P * P)).sum())


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
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
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


def host_cores():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


_CPU_BATCH = {}


def cpu_oracle_chunk(task):
    """Worker of the CPU oracle legs: the FP64 oracle's node-state value (P = 16) of
    integrals lo..hi-1 of the seeded batch (count, seed), which every worker draws
    itself from the seeded generator."""
    from oracle import oracle as o
    from paper_2404_08867_gb300 import inputs
    count, seed, lo, hi = task
    if (count, seed) not in _CPU_BATCH:
        _CPU_BATCH[(count, seed)] = inputs.batch(count=count, seed=seed)
    b = _CPU_BATCH[(count, seed)]
    out = []
    for i in range(lo, hi):
        it = b.integral(i)
        out.append(o.mdi_nodes(it.family, it.d, it.a, it.n_last, P_NODES, it.c, it.w))
    return lo, out


def cpu_oracle_pool(cores):
    """A pool of `cores` oracle workers, started by spawn (not fork: the parent may
    already hold a CUDA context)."""
    import multiprocessing as mp
    from oracle import oracle as o
    o.build()
    return mp.get_context("spawn").Pool(processes=cores)


def cpu_oracle_batch_pass(pool, count, seed, cores):
    """One pass of the oracle over the whole batch on the pool; returns the values."""
    step = max(1, count // (cores * 8))
    tasks = [(count, seed, lo, min(count, lo + step)) for lo in range(0, count, step)]
    vals = np.empty(count)
    for lo, out in pool.imap_unordered(cpu_oracle_chunk, tasks):
        vals[lo:lo + len(out)] = out
    return vals


def cpu_baseline_all_cores(count, seed, budget_s):
    """CPU baseline on every host core: whole passes of the FP64 oracle over the
    batch until `budget_s` seconds, after one untimed pass (pool start-up).
    Returns (oracle values of the batch, integrals/s, cores, passes, seconds)."""
    cores = host_cores()
    with cpu_oracle_pool(cores) as pool:
        vals = cpu_oracle_batch_pass(pool, count, seed, cores)
        t0 = time.perf_counter()
        passes = 0
        while True:
            cpu_oracle_batch_pass(pool, count, seed, cores)
            passes += 1
            el = time.perf_counter() - t0
            if el >= budget_s:
                break
    return vals, passes * count / el, cores, passes, el


def cpu_baseline_one_core(b, budget_s, P=P_NODES):
    """The FP64 oracle (node state) on one core, on consecutive integrals of the
    batch until `budget_s` seconds."""
    from oracle import oracle as o
    o.build()
    t0 = time.perf_counter()
    done = 0
    while True:
        it = b.integral(done % len(b))
        o.mdi_nodes(it.family, it.d, it.a, it.n_last, P, it.c, it.w)
        done += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            return done / el, done, el


def cpu_baseline_korobov_search(d, n, budget_s):
    """CPU baseline of the Korobov search: the oracle's P_2 criterion for consecutive
    candidates a = 1, 3, 5, ... on one host core for `budget_s` seconds."""
    from oracle import oracle as o
    o.build()
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < budget_s:
        o.korobov_search(2, d, n, 1 + 2 * k, 1)
        k += 1
    el = time.perf_counter() - t0
    return {"value": k / el, "unit": "candidates/s", "cores": 1, "kind": "oracle",
            "sample": f"{k} candidates of the n = {n}, d = {d} search in {el:.1f} s"}


def cpu_reference_arm(args, rank, world):
    """Reference arm: the CPU oracle, as it stands, on every host core; one step is
    one pass over the same 4096-integral batch (seed 0) as our arm's step."""
    if rank != 0:
        return
    cores = host_cores()
    with cpu_oracle_pool(cores) as pool:
        for _ in range(max(1, args.warmup)):
            cpu_oracle_batch_pass(pool, args.count, 0, cores)
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            cpu_oracle_batch_pass(pool, args.count, 0, cores)
            times.append(time.perf_counter() - t0)
    value = args.count * args.steps / sum(times)
    line = {"metric": METRIC, "value": value, "unit": "integrals/s", "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.count, "fp64"),  # the same workload as our arm
            "reference_arithmetic": "f64 (the oracle computes every integral in double)",
            "cpu_baseline": {"value": value, "unit": "integrals/s", "cores": cores, "kind": "oracle",
                             "sample": f"the whole {args.count}-integral batch per step on {cores} host cores "
                                       f"(node state, P=16)"},
            "e2e": {"value": value, "unit": "integrals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def event_ms(torch, fn, reps=5):
    """Device time of fn: its launches are captured once into a CUDA graph and the
    graph is replayed between CUDA events (median), so host-side marshalling of
    the Python binding is not counted for microsecond-scale calls."""
    fn()
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        r = fn()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return r, statistics.median(ts)


def extra_small_workload(torch, mdi, inputs):
    """d = 4, N = 16, f = exp(sum x_j/j): MDI-LR and the plain lattice kernel on the
    GPU, and the time each needs to reach 1e-6 relative error against the closed
    form (MDI-LR: closed state, a doubling; plain kernel: a = 12345, n = 2^m)."""
    w = inputs.small_exp()
    c = torch.as_tensor(w.params).cuda()
    exact = exact_integral("exp", 4, w.c, w.w)
    n = 16**4
    z = mdi.korobov_vector(4, inputs.SMALL_SLR_A, n).astype(np.int64)
    slr, slr_ms = event_ms(torch, lambda: mdi.lattice_rule_integrate("exp", c, n, z))
    mv, m_ms = event_ms(torch, lambda: mdi.mdi_lr_integrate("exp", c, 4, 16, 16, state="exact"))
    res = {"workload": "d=4, N=16, f=exp(sum x_j/j)",
           "slr_a12345_n65536": {"rel_err": abs(slr.item() - exact) / exact, "ms": slr_ms},
           "mdi_lr_exact_N16": {"rel_err": abs(mv.item() - exact) / exact, "ms": m_ms}}
    for key, prec in (("mdi_lr_to_1e-6", "fp64"), ("mdi_lr_df64_to_1e-6", "df64")):
        a = 16
        while True:
            v, ms = event_ms(torch, lambda: mdi.mdi_lr_integrate("exp", c, 4, a, a, state="closed", precision=prec))
            if abs(v.item() - exact) / exact <= 1e-6 or a > 1 << 24:
                res[key] = {"a": a, "rel_err": abs(v.item() - exact) / exact, "ms": ms}
                break
            a *= 2
    reached, last = None, None
    for m in range(16, 31):
        nn = 1 << m
        zz = mdi.korobov_vector(4, inputs.SMALL_SLR_A, nn).astype(np.int64)
        v, ms = event_ms(torch, lambda: mdi.lattice_rule_integrate("exp", c, nn, zz), reps=2)
        last = {"n": nn, "a": inputs.SMALL_SLR_A, "rel_err": abs(v.item() - exact) / exact, "ms": ms}
        if last["rel_err"] <= 1e-6:
            reached = last
            break
    res["slr_a12345_to_1e-6"] = reached if reached else {"reached": False, "largest_tried": last}
    # The plain kernel with a searched generating vector: for n = 2^m, 64 seeded odd
    # Korobov parameters (and 12345) are tried on the GPU (search untimed, reported
    # separately); the first n whose best parameter reaches 1e-6 is timed.
    rng = np.random.default_rng(2024)
    found, search_s = None, 0.0
    for m in range(16, 27):
        nn = 1 << m
        cands = [inputs.SMALL_SLR_A % nn] + [int(x) | 1 for x in rng.integers(3, nn, 64)]
        t0 = time.perf_counter()
        errs = []
        for a_c in cands:
            zz = mdi.korobov_vector(4, a_c, nn).astype(np.int64)
            errs.append(abs(mdi.lattice_rule_integrate("exp", c, nn, zz).item() - exact) / exact)
        search_s += time.perf_counter() - t0
        best = int(np.argmin(errs))
        if errs[best] <= 1e-6:
            zz = mdi.korobov_vector(4, cands[best], nn).astype(np.int64)
            _, ms = event_ms(torch, lambda: mdi.lattice_rule_integrate("exp", c, nn, zz), reps=5)
            _, ms_df = event_ms(torch, lambda: mdi.lattice_rule_integrate("exp", c, nn, zz, precision="df64"),
                                reps=5)
            found = {"n": nn, "a": cands[best], "rel_err": errs[best], "ms": ms, "ms_df64": ms_df}
            break
    res["slr_searched_a_to_1e-6"] = found if found else {"reached": False, "n_max": 1 << 26}
    res["slr_a_search_s_untimed"] = search_s
    if found:
        res["time_to_1e-6_ratio_slr_over_mdi"] = found["ms"] / res["mdi_lr_to_1e-6"]["ms"]
        res["time_to_1e-6_ratio_slr_over_mdi_df64"] = found["ms_df64"] / res["mdi_lr_df64_to_1e-6"]["ms"]
    # The same protocol with the paper's own criterion: for n = 2^m the Korobov
    # parameter minimising P_2 (eq. 2.4) over every a in 1..n/2, searched on the GPU
    # (device time reported separately), then the plain kernel with it.
    p2 = None
    p2_search_ms = 0.0
    for m in range(16, 19):
        nn = 1 << m
        (vals, best), sms = event_ms(torch, lambda: mdi.lattice_korobov_search(nn, 4, a_first=1, count=nn // 2), reps=1)
        p2_search_ms += sms
        a_best = int(best.item())
        zz = mdi.korobov_vector(4, a_best, nn).astype(np.int64)
        v, ms = event_ms(torch, lambda: mdi.lattice_rule_integrate("exp", c, nn, zz), reps=5)
        p2 = {"n": nn, "a": a_best, "p2": float(vals[a_best - 1].item()),
              "rel_err": abs(v.item() - exact) / exact, "ms": ms, "search_ms": sms}
        if p2["rel_err"] <= 1e-6:
            break
    res["slr_p2_searched_a"] = p2
    res["slr_p2_search_ms_total"] = p2_search_ms
    # Randomly shifted rule (Section 2.1): 16 uniform shifts of the a = 12345
    # lattice at n = 65536 in one call; the mean estimates the integral and the
    # replicates' spread its error.
    shifts = torch.as_tensor(np.random.default_rng(16).uniform(0.0, 1.0, (16, 4))).cuda()
    z16 = mdi.korobov_vector(4, inputs.SMALL_SLR_A, n).astype(np.int64)
    vals, sh_ms = event_ms(torch, lambda: mdi.lattice_rule_integrate_shifted("exp", c, n, z16, shifts))
    _, sh_df_ms = event_ms(torch, lambda: mdi.lattice_rule_integrate_shifted("exp", c, n, z16, shifts,
                                                                             precision="df64"))
    mean, se = mdi.shifted_estimate(vals)
    res["slr_shifted_R16_n65536"] = {"rel_err_of_mean": abs(mean.item() - exact) / exact,
                                     "rel_std_error": se.item() / exact, "ms": sh_ms, "ms_df64": sh_df_ms}
    return res


def extra_time_to_1e6_vs_d(torch, mdi, inputs, dims=(4, 6, 8, 10, 12, 16, 20, 24)):
    """Time to 1e-6 relative error against the closed form, f = exp(sum x_j / j),
    as d grows.  MDI-LR: closed state, a = N doubling from 16.  Plain kernel: for
    n = 2^m (m = 16..28) the best of 33 Korobov parameters (12345 and 32 seeded odd
    ones) by an error scan against the closed form (untimed, reported separately);
    the first n whose best parameter reaches 1e-6 is timed.  Both are timed in FP64
    and in the double-float mode, and each ratio compares like with like."""
    rows = []
    for d in dims:
        w = inputs.small_exp(d)
        c = torch.as_tensor(w.params).cuda()
        exact = exact_integral("exp", d, w.c, w.w)
        row = {"d": d}
        for key, prec in (("mdi_lr", "fp64"), ("mdi_lr_df64", "df64")):
            a = 16
            while a <= 1 << 24:
                v, ms = event_ms(torch, lambda: mdi.mdi_lr_integrate("exp", c, d, a, a, state="closed", precision=prec),
                                 reps=3)
                err = abs(v.item() - exact) / exact
                if err <= 1e-6:
                    row[key] = {"a": a, "rel_err": err, "ms": ms}
                    break
                a *= 2
        rng = np.random.default_rng(1000 + d)
        search_s, found, best_seen = 0.0, None, None
        for m in range(16, 29):
            nn = 1 << m
            cands = [inputs.SMALL_SLR_A % nn] + [int(x) | 1 for x in rng.integers(3, nn, 32)]
            t0 = time.perf_counter()
            errs = []
            for a_c in cands:
                zz = mdi.korobov_vector(d, a_c, nn).astype(np.int64)
                errs.append(abs(mdi.lattice_rule_integrate("exp", c, nn, zz).item() - exact) / exact)
            search_s += time.perf_counter() - t0
            b = int(np.argmin(errs))
            best_seen = {"n": nn, "a": cands[b], "rel_err": errs[b]}
            if errs[b] <= 1e-6:
                zz = mdi.korobov_vector(d, cands[b], nn).astype(np.int64)
                _, ms = event_ms(torch, lambda: mdi.lattice_rule_integrate("exp", c, nn, zz), reps=3)
                v64, ms_df = event_ms(torch, lambda: mdi.lattice_rule_integrate("exp", c, nn, zz, precision="df64"),
                                      reps=3)
                found = dict(best_seen, ms=ms, ms_df64=ms_df, rel_err_df64=abs(v64.item() - exact) / exact)
                break
        row["plain_searched_a"] = found if found else {"reached": False, "best_at_2^28": best_seen}
        row["plain_search_s_untimed"] = search_s
        if found and "mdi_lr" in row:
            row["ratio_plain_over_mdi"] = found["ms"] / row["mdi_lr"]["ms"]
        if found and "mdi_lr_df64" in row:
            row["ratio_plain_over_mdi_df64"] = found["ms_df64"] / row["mdi_lr_df64"]["ms"]
        rows.append(row)
    return {"workload": "f = exp(sum_j x_j / j), d in " + str(list(dims)), "rows": rows}


# DRAM bytes per launch of the batched kernel from the ncu captures summarised in
# profiles/ (dram__bytes_read.sum + dram__bytes_write.sum), valid only for the kernel
# sources they were taken on (SHA-256 prefix of the files below, comments
# removed): after any change to their code the bench reports null until the capture
# is repeated.
TRAFFIC_SOURCES = ["paper_2404_08867_gb300/csrc/mdi_nodes.cu", "paper_2404_08867_gb300/csrc/mdi_nodes.cuh",
                   "paper_2404_08867_gb300/csrc/mdi_common.cuh", "paper_2404_08867_gb300/csrc/mdi_fp64.cuh"]
PROFILED_TRAFFIC = {"fp64": ("06e548c0a4bc3142", 1703680), "df64": ("06e548c0a4bc3142", 1753856)}
# The same captures' pipe utilisation (fractions of peak over the SMs' active
# cycles, or the elapsed time where stated), under the same key: the FP64 mode is
# bound by the FP64 pipe, the double-float mode by instruction issue.
PROFILED_PIPE = {
    "fp64": ("06e548c0a4bc3142", {"fp64_pipe_active": 0.912, "fp64_pipe_elapsed": 0.882,
                                  "metric": "sm__inst_executed_pipe_fp64"}),
    "df64": ("06e548c0a4bc3142", {"issue_active": 0.637, "fma_pipe_active": 0.533,
                                  "metric": "smsp__issue_active, sm__pipe_fma_cycles_active"}),
}


def kernel_sources_key() -> str:
    """SHA-256 prefix of TRAFFIC_SOURCES with comments and blank lines removed, so
    that editing a comment does not invalidate a capture."""
    import hashlib
    h = hashlib.sha256()
    root = os.path.dirname(os.path.abspath(__file__))
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(root, f)) as fh:
            for line in fh:
                code = line.split("//", 1)[0].strip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic(precision: str):
    entry = PROFILED_TRAFFIC.get(precision)
    return entry[1] if entry is not None and kernel_sources_key() == entry[0] else None


def profiled_pipe(precision: str):
    """The capture's pipe utilisation for this mode, or None once the kernel
    sources have changed since it was taken."""
    entry = PROFILED_PIPE.get(precision)
    if entry is None or kernel_sources_key() != entry[0]:
        return None
    return dict(entry[1], source="ncu capture summarised in profiles/")


def extra_batch_vs_plain(torch, mdi, inputs):
    """The batch's integrals whose full point set is small enough for the plain
    lattice kernel (n = N^d <= 2^27): the plain kernel on the Korobov lattice with
    a = N and n = N^d -- by Lemma 3.2 the same sum as MDI-LR's text reading --
    one call per integral, beside one batched MDI-LR launch (DF64) over the same
    integrals; their values agree to the node state's approximation."""
    from paper_2404_08867_gb300.tuning import BatchedMDILR
    b = inputs.batch(count=COUNT, seed=0)
    idx = [i for i in range(len(b)) if float(b.a[i]) ** int(b.d[i]) <= 2.0 ** 27]
    fams = [b.families[i] for i in idx]
    ds, as_ = b.d[idx], b.a[idx]
    offs = np.concatenate([[0], np.cumsum(2 * ds[:-1])]).astype(np.int64)
    pool = np.concatenate([b.pool[b.offsets[i]:b.offsets[i] + 2 * b.d[i]] for i in idx])
    plan = BatchedMDILR(fams, ds, as_, as_, offs, pool, precision="df64", nodes=P_NODES)
    plan.tune()
    mv, mdi_ms = event_ms(torch, lambda: plan.launch(), reps=3)
    mv = mv.cpu().numpy()
    slr_ms, worst = 0.0, 0.0
    for j, i in enumerate(idx):
        d, a = int(b.d[i]), int(b.a[i])
        n = a ** d
        p = torch.as_tensor(pool[offs[j]:offs[j] + 2 * d]).cuda()
        z = mdi.korobov_vector(d, a, n).astype(np.int64)
        v, ms = event_ms(torch, lambda: mdi.lattice_rule_integrate(fams[j], p, n, z), reps=1)
        slr_ms += ms
        worst = max(worst, abs(v.item() - mv[j]) / abs(mv[j]))
    return {"workload": f"{len(idx)} integrals of the batch with N^d <= 2^27 "
                        f"(points per integral up to {int(max(float(as_[k]) ** int(ds[k]) for k in range(len(idx))))})",
            "mdi_lr_batched_ms": mdi_ms, "plain_kernel_ms_total": slr_ms, "ratio_plain_over_mdi": slr_ms / mdi_ms,
            "max_rel_diff_plain_vs_mdi": worst}


def extra_improved_rule(torch, mdi):
    """Improved lattice rule (Definition 3.3) at the paper's kind of size n = 1 + a^d
    (d = 7, a = 16: n = 2.7e8 lattice points, n* = a^(d-1) - 1 ghosts), beside the
    plain rule on the same n points; f = exp(sum x_j / j), whose integral is
    prod_j j (e^{1/j} - 1)."""
    d, a = 7, 16
    n = 1 + a ** d
    c = 1.0 / np.arange(1, d + 1)
    p = torch.as_tensor(np.r_[c, np.zeros(d)]).cuda()
    exact = float(np.prod(np.arange(1, d + 1) * np.expm1(c)))
    ws = torch.empty(mdi.lattice_rule_improved_workspace_size(d, n, a), dtype=torch.uint8, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    nstar = mdi.lattice_rule_integrate_improved("exp", p, d, n, a, out=out, workspace=ws)[1]
    v, ms = event_ms(torch, lambda: mdi.lattice_rule_integrate_improved("exp", p, d, n, a, out=out, workspace=ws)[0],
                     reps=3)
    vd, ms_d = event_ms(torch, lambda: mdi.lattice_rule_integrate_improved("exp", p, d, n, a, precision="df64",
                                                                             out=out, workspace=ws)[0], reps=3)
    z = mdi.korobov_vector(d, a, n).astype(np.int64)
    vp, ms_p = event_ms(torch, lambda: mdi.lattice_rule_integrate("exp", p, n, z), reps=3)
    vpd, ms_pd = event_ms(torch, lambda: mdi.lattice_rule_integrate("exp", p, n, z, precision="df64"), reps=3)
    return {"workload": f"d={d}, z=(1,{a},..,{a}^{d - 1}), n=1+{a}^{d}={n}, f=exp(sum x_j/j)",
            "n_ghost": nstar, "improved_ms": ms, "improved_points_per_s": (n + nstar) / (ms * 1e-3),
            "improved_rel_err": abs(v.item() - exact) / exact,
            "improved_df64_ms": ms_d, "improved_df64_vs_fp64": abs(vd.item() - v.item()) / abs(v.item()),
            "plain_ms": ms_p, "plain_rel_err": abs(vp.item() - exact) / exact, "plain_df64_ms": ms_pd}


def extra_batch_size_sweep(torch, mdi, inputs, precision, counts=(4096, 16384, 65536)):
    """The batched launch on larger batches of the same distribution (seed 0):
    integrals/s as the persistent launch's tail (its largest integrals finishing
    alone) weighs less.  Context beside the configured 4096-integral step."""
    from paper_2404_08867_gb300.tuning import BatchedMDILR
    rows = []
    for count in counts:
        b = inputs.batch(count=count, seed=0)
        plan = BatchedMDILR(b.families, b.d, b.a, b.n_last, b.offsets, b.pool, precision=precision, nodes=P_NODES)
        plan.tune()
        _, ms = event_ms(torch, lambda: plan.launch(), reps=5)
        rows.append({"count": count, "ms": ms, "integrals_per_s": count / (ms * 1e-3),
                     "block": plan.opts.get("block"), "split": plan.opts.get("split"),
                     "ctas_per_sm": plan.opts.get("ctas_per_sm")})
    return {"workload": f"batches of the configured distribution, {precision}, tuned shape", "rows": rows}


def extra_paper_context(torch, mdi):
    """The paper's own MDI-LR CPU times (Matlab on an Intel Xeon Gold 6226R at
    2.90 GHz, one process, Section 4) beside this GPU's time for the nearest
    workloads, context only: the paper's printed columns use the midpoint point set
    (reading R1) where this path computes the text's transformed-lattice sum, on
    the same integrand, d and N."""
    import math
    hw = "Matlab, Intel Xeon Gold 6226R @ 2.90 GHz, 32 GB (Section 4)"
    cases = [
        ("exp(sum (-1)^(i+1) x_i), d=1000, a=N=8", "exp", 1000, 8,
         np.array([(-1.0) ** i for i in range(1000)]), np.zeros(1000), 69992.0, "Table 2-3"),
        ("prod 1/(0.9^2 + (x_i - 0.6)^2), d=1000, a=N=20", "peak", 1000, 20, np.full(1000, 1.0 / 0.9),
         np.full(1000, 0.6), 189.13, "Table 2-3"),
        ("(2 pi)^(-1/2) exp(-|x|^2/2), d=12, N=10", "gauss", 12, 10, np.full(12, 1.0 / math.sqrt(2.0)),
         np.zeros(12), 4.592, "Table 2-1"),
    ]
    out = {"hardware_of_paper": hw, "cases": []}
    for name, fam, d, a, c, w, paper_s, table in cases:
        p = torch.as_tensor(np.concatenate([c, w])).cuda()
        v, ms = event_ms(torch, lambda: mdi.mdi_lr_integrate(fam, p, d, a, a), reps=3)
        exact = exact_integral(fam, d, c, w)
        out["cases"].append({"workload": name, "gpu_ms": ms, "gpu_rel_err_vs_exact": abs(v.item() - exact) / abs(exact),
                             "paper_cpu_s": paper_s, "paper_source": table, "ratio_paper_over_gpu": paper_s * 1e3 / ms})
    return out


PAPER_ROWS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "midpoint_printed.txt")


def extra_paper_tables(torch, mdi):
    """Paper-table mode: the MDI-LR relative errors printed in Section 5 (Tables 2-1
    to 3-3, the golden rows) recomputed by the GPU's tensor midpoint rule on the
    grid of eq. (3.5); the count reproduced to one unit in the last printed digit,
    and the device time of the largest case (d = 1000)."""
    def case(integrand, d):
        if integrand == "gauss":
            return "gauss", np.full(d, 1.0 / math.sqrt(2.0)), np.zeros(d)
        if integrand == "expalt":
            return "exp", np.array([(-1.0) ** i for i in range(d)]), np.zeros(d)
        if integrand == "peak":
            return "peak", np.full(d, 1.0 / 0.9), np.full(d, 0.6)
        w = np.zeros(d)
        w[0] = 1.0
        return "osc", np.full(d, 2.0), w

    rows, ok, worst = 0, 0, None
    for line in open(PAPER_ROWS):
        line = line.split("#", 1)[0].split()
        if not line:
            continue
        table, integrand, d, N, grid, printed = line
        d, N = int(d), int(N)
        fam, cc, ww = case(integrand, d)
        p = torch.as_tensor(np.concatenate([cc, ww])).cuda()
        nl = N if grid == "N" else N + 1
        v, ms = event_ms(torch, lambda: mdi.mdi_midpoint_integrate(fam, p, d, N, nl), reps=3)
        exact = exact_integral(fam, d, cc, ww)
        rel = abs(v.item() - exact) / abs(exact)
        mant, ex = printed.lower().split("e")
        unit = 10.0 ** (int(ex) - (len(mant.split(".")[1]) if "." in mant else 0))
        rows += 1
        ok += abs(rel - float(printed)) <= unit
        if worst is None or d > worst["d"]:
            worst = {"table": table, "integrand": integrand, "d": d, "N": N, "printed": printed, "gpu_rel_err": rel,
                     "ms": ms}
    # Test 7's ridge integrand f_6 = (1 + sum x_i)^-(d+1) by the histogram state:
    # device time against d at N = 16 (the paper fits its CPU time against d,
    # Table 4-2) and the error against the exact 1/(d+1)!.
    ds, ts = [25, 50, 100, 150], []
    for d in ds:
        v, ms = event_ms(torch, lambda: mdi.mdi_midpoint_ridge(d, 16, 16), reps=3)
        ts.append(ms)
        if d == 50:
            ridge50 = abs(v.item() * math.factorial(51) - 1.0)
    ridge = {"N": 16, "d": ds, "ms": ts, "beta": float(np.polyfit(np.log(ds), np.log(ts), 1)[0]),
             "d50_rel_err_vs_exact": ridge50}
    return {"workload": "Section 5 MDI-LR columns (tensor midpoint rule on the eq. 3.5 grid)", "rows": rows,
            "reproduced": ok, "largest": worst, "ridge_f6": ridge}


def extra_lattice_search(torch, mdi):
    """Generating-vector construction (Section 2.2) on the GPU: the Korobov search
    of Example 2 (P_2 of eq. 2.4 for every a in 1..n/2) and the CBC construction of
    Example 3 (eq. 2.12, product weights 1/j^2, unanchored), n = 65536, d = 4; the
    oracle's rate on a bounded sample beside them (one host core)."""
    n, d = 65536, 4
    res = {"workload": "n=65536, d=4: Korobov P_2 search over a in 1..n/2; CBC, gamma_j = 1/j^2, beta = 0"}
    (vals, best), ms = event_ms(torch, lambda: mdi.lattice_korobov_search(n, d, a_first=1, count=n // 2), reps=3)
    cand = n // 2
    res["korobov"] = {"ms": ms, "best_a": int(best.item()), "p2_best": float(vals[int(best.item()) - 1].item()),
                      "candidates_per_s": cand / (ms / 1e3),
                      "fp64_flops": 5.0 * d * cand * (n // 2) / (ms / 1e3)}
    res["korobov"]["cpu_baseline"] = cpu_baseline_korobov_search(d, n, 2.0)
    gamma = torch.as_tensor(1.0 / np.arange(1, d + 1) ** 2).cuda()
    (z, e2), cms = event_ms(torch, lambda: mdi.lattice_cbc(n, gamma, 0.0), reps=3)
    res["cbc"] = {"ms": cms, "z": [int(x) for x in z.cpu().numpy()], "e2": [float(x) for x in e2.cpu().numpy()],
                  "candidate_evals_per_s": (d - 1) * (n // 2) / (cms / 1e3)}
    return res


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "oracle_workloads.json")


def golden_oracle():
    """The oracle's FP64 values of the fixed extra workloads, stored by
    tests/golden/make_oracle_workloads.py (which calls only the oracle)."""
    with open(GOLDEN) as f:
        return json.load(f)


def extra_precision(torch, mdi, inputs):
    """d = 50, N = 32, f = cos(2 pi u + sum a_j x_j): every precision mode, closed and
    node state, its error against the FP64 oracle's value of the same state and
    against the exact integral (|f| <= 1: absolute errors)."""
    w = inputs.oscillatory(50, 32, seed=0)
    p = torch.as_tensor(w.params).cuda()
    exact = exact_integral("osc", 50, w.c, w.w)
    ref = golden_oracle()["precision"]
    res = {"workload": "d=50, N=32, cos(2 pi u + sum a_j x_j)", "exact": exact, "oracle": ref}
    for state in ("closed", "nodes"):
        for prec in ("fp64", "fp32_eval_fp64", "fp32_eval_df32", "df64"):
            v, ms = event_ms(torch, lambda: mdi.mdi_lr_integrate("osc", p, 50, 32, state=state, precision=prec))
            res[f"{state}/{prec}"] = {"abs_err_vs_oracle": abs(v.item() - ref[state]),
                                      "abs_err_vs_exact": abs(v.item() - exact), "ms": ms}
    return res


def extra_differentiation(torch, mdi, inputs):
    """d = 100, N = 16 Gaussian: value and 200-parameter gradient by the adjoint
    sweep (checkpoints every 10 levels) against the FP64 oracle's derivative of the
    same rule (component by component), against central differences of the GPU's
    FP64 forward sweep (h = 1e-6, 400 forward calls) and the exact gradient."""
    w = inputs.gaussian(100, 16, seed=0)
    p = torch.as_tensor(w.params).cuda()
    (val, g), ms = event_ms(torch, lambda: mdi.mdi_lr_grad("gauss", p, 100, 16, 16, state="nodes", checkpoint=10))
    _, fwd_ms = event_ms(torch, lambda: mdi.mdi_lr_integrate("gauss", p, 100, 16, state="nodes"))
    g = g.cpu().numpy()
    ref = golden_oracle()["differentiation"]
    gref = np.array(ref["grad"])
    h, base = 1e-6, w.params.copy()
    fd = np.empty(2 * 100)
    for i in range(2 * 100):
        up, dn = base.copy(), base.copy()
        up[i] += h
        dn[i] -= h
        fu = mdi.mdi_lr_integrate("gauss", torch.as_tensor(up).cuda(), 100, 16, state="nodes").item()
        fdn = mdi.mdi_lr_integrate("gauss", torch.as_tensor(dn).cuda(), 100, 16, state="nodes").item()
        fd[i] = (fu - fdn) / (2 * h)
    exact = exact_gauss_grad(100, w.c, w.w)
    # The torch.autograd path a user takes: value and backward through the MDILR
    # Function (its forward runs the adjoint call once), CUDA events around eager
    # calls, so the host's Python and launch overhead is included.
    pa = p.clone().requires_grad_(True)
    for _ in range(3):
        mdi.mdi_lr("gauss", pa, 100, 16, state="nodes", checkpoint=10).backward()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record()
    for _ in range(reps):
        pa.grad = None
        mdi.mdi_lr("gauss", pa, 100, 16, state="nodes", checkpoint=10).backward()
    e1.record()
    torch.cuda.synchronize()
    auto_ms = e0.elapsed_time(e1) / reps
    auto_err = float(np.max(np.abs(pa.grad.cpu().numpy() - gref) / np.abs(gref)))
    return {"workload": "d=100, N=16 Gaussian, 200 parameters, checkpoint 10", "adjoint_ms": ms, "forward_ms": fwd_ms,
            "autograd_forward_backward_ms_eager": auto_ms, "autograd_grad_max_componentwise_rel_err_vs_oracle": auto_err,
            "grad_max_componentwise_rel_err_vs_oracle": float(np.max(np.abs(g - gref) / np.abs(gref))),
            "value_rel_err_vs_oracle": abs(val.item() - ref["value"]) / abs(ref["value"]),
            "grad_err_vs_central_fd_normwise": float(np.max(np.abs(g - fd)) / np.max(np.abs(fd))),
            "grad_diff_vs_exact_normwise": float(np.max(np.abs(g - exact)) / np.max(np.abs(exact))),
            "value_rel_err_vs_exact": abs(val.item() - exact_integral("gauss", 100, w.c, w.w)) /
            exact_integral("gauss", 100, w.c, w.w)}


def extra_scale(torch, mdi, inputs):
    """d in {100, 250, 500, 1000}, N = 16, f = exp(sum x_j/j^2): forward and adjoint
    in the closed and node states; fitted exponent of time ~ d^beta; each forward
    value's error against the FP64 oracle's."""
    res = {"workload": "N=16, f=exp(sum x_j/j^2)"}
    ref = golden_oracle()["scale"]
    for state in ("closed", "nodes"):
        ds, fw, ad, err = [], [], [], []
        for d in (100, 250, 500, 1000):
            w = inputs.scale_exp(d, 16)
            p = torch.as_tensor(w.params).cuda()
            v, f_ms = event_ms(torch, lambda: mdi.mdi_lr_integrate("exp", p, d, 16, state=state))
            _, a_ms = event_ms(torch, lambda: mdi.mdi_lr_grad("exp", p, d, 16, 16, state=state))
            ds.append(d)
            fw.append(f_ms)
            ad.append(a_ms)
            err.append(abs(v.item() / ref[str(d)][state] - 1.0))
            if d == 1000:
                exact = exact_integral("exp", d, w.c, w.w)
                res[f"{state}/d1000_rel_err_vs_exact"] = abs(v.item() - exact) / exact
        beta = lambda t: float(np.polyfit(np.log(ds), np.log(t), 1)[0])
        res[state] = {"d": ds, "forward_ms": fw, "adjoint_ms": ad, "forward_beta": beta(fw), "adjoint_beta": beta(ad),
                      "forward_rel_err_vs_oracle": err}
    return res


def extra_step_size(torch, mdi, inputs):
    """Algorithm 1's step size m = 1, 2, 3 with the node state (P = 16 unless stated):
    the state is read once per m levels, at the price of a^m cluster tuples per
    operator instead of a.  d = 100, N = 16: time and value for the Gaussian of the
    differentiation workload and for exp(sum x_j/j^2), each against the oracle's
    step-m value, the exponential one also against its closed state (the exact
    rule, so that difference is the node state's own error), and the adjoint's
    time and its gradient against m = 1's; and on an enumerable case (d = 6,
    a = 8, P = 8) each m's error against the exact sweep."""
    ref = golden_oracle()["step"]
    res = {"workload": "node state, step m = 1, 2, 3"}
    g = inputs.gaussian(100, 16, seed=0)
    e = inputs.scale_exp(100, 16)
    for name, fam, w in (("gauss_d100", "gauss", g), ("exp_d100", "exp", e)):
        p = torch.as_tensor(w.params).cuda()
        rows = {}
        g1 = None
        for m in (1, 2, 3):
            v, ms = event_ms(torch, lambda: mdi.mdi_lr_integrate(fam, p, 100, 16, state="nodes", step=m), reps=3)
            row = {"ms": ms, "value": v.item(), "rel_err_vs_oracle": abs(v.item() / ref[fam][str(m)] - 1.0)}
            if fam == "exp":
                row["rel_err_vs_exact_rule"] = abs(v.item() / ref["exp_closed"] - 1.0)
            # the adjoint over the step-m operators: time, and its gradient against m = 1's
            (_, gm), gms = event_ms(torch, lambda: mdi.mdi_lr_grad(fam, p, 100, 16, state="nodes", step=m), reps=3)
            gm = gm.cpu().numpy()
            g1 = gm if m == 1 else g1
            row["adjoint_ms"] = gms
            if m > 1:
                row["grad_max_rel_diff_vs_m1"] = float(np.max(np.abs(gm - g1)) / np.max(np.abs(g1)))
            rows[f"m{m}"] = row
        res[name] = rows
    small = {}
    for fam in ("gauss", "peak"):
        p = torch.as_tensor(inputs.random_product(fam, 6, seed=19)).cuda()
        ex = mdi.mdi_lr_integrate(fam, p, 6, 8, state="exact").item()
        small[fam] = {f"m{m}": abs(mdi.mdi_lr_integrate(fam, p, 6, 8, state="nodes", nodes=8, step=m).item() / ex - 1.0)
                      for m in (1, 2, 3)}
    res["d6_a8_P8_rel_err_vs_exact_sweep"] = small
    return res


def measure_peaks(torch, mdi, reps=3):
    """FMA throughput of this GPU at its current clock, from the library's probe
    kernel (16 independent FMA chains per thread, several CTAs per SM): the best
    of `reps` launches, timed with CUDA events.  TFLOP/s, an FMA counting 2."""
    out = {}
    for kind, iters in (("fp64", 2048), ("fp32", 65536)):
        threads = mdi.mdi_peak_probe_threads(kind)
        sink = torch.zeros(1, dtype=torch.float64, device="cuda")
        mdi.mdi_peak_probe(kind, 64, sink)
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            mdi.mdi_peak_probe(kind, iters, sink)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        out[kind] = {"tflops": threads * 32.0 * iters / (best * 1e-3) / 1e12, "ms": best, "threads": threads,
                     "fma_per_thread": 16 * iters}
    return out


def time_plan(torch, plan, flush, stream, steps):
    """CUDA-event times (ms) of `steps` graph replays of a batched plan, L2 flushed
    before each."""
    ts = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.run()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return ts


def roofline_entry(b, precision, kernel_ms, peaks, traffic=None):
    """Roofline of one batched launch: the algorithmic flops (d N (P C_phi + P^2)
    per integral) over the launch's time, against the measured
    FMA peak of the pipe the mode runs on (FP64 for the FP64 mode, FP32 for the
    double-float and single-precision-evaluation modes); impl_flops is what the
    kernel's own formulation executes (the paired interpolation, and double-float
    primitives counted in float operations).  With phi in float and the rest in
    FP64 (fp32_eval_fp64) only the interpolation and contraction, d N P^2, run on
    the FP64 pipe, so only they are counted against its peak."""
    flops = alg_flops(b, phi=precision != "fp32_eval_fp64")
    achieved = flops / (kernel_ms / 1e3) / 1e12
    fp64 = precision in ("fp64", "fp32_eval_fp64")
    peak = peaks["fp64" if fp64 else "fp32"]["tflops"]
    impl = fp64_flops(b) if fp64 else df_flops(b, paired=True, float_phi=precision == "fp32_eval_df32")
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_unit": "DRAM bytes per launch (ncu)", "kernel": "nodes_batched_kernel",
            "pipe": "FP64" if fp64 else "FP32 (double-float arithmetic)",
            "peak_source": "measured in this run: mdi_peak_probe (" + ("DFMA" if fp64 else "FFMA") + "), of measured",
            "peak_from_unit_counts": FP64_PEAK_TFLOPS if fp64 else FP32_PEAK_TFLOPS,
            "flops_per_launch": flops,
            "flops_formula": ("sum_i d_i N_i P^2 (phi in float, off the FP64 pipe), P = 16"
                              if precision == "fp32_eval_fp64" else "sum_i d_i N_i (P C_phi + P^2), P = 16"),
            "c_phi": {f: C_PHI[f] for f in sorted(set(b.families))}, "kernel_ms": kernel_ms,
            "impl_flops_per_launch": impl, "impl_tflops": impl / (kernel_ms / 1e3) / 1e12}


def max_rel_err(got, ref):
    return float(np.max(np.abs(np.asarray(got) - ref) / np.abs(ref)))


# ---------------------------------------------------------------------------
# Named workloads for profilers (``python bench.py --case NAME --repeats R``): each
# runs R times through the public API on the seeded synthetic inputs.
# ---------------------------------------------------------------------------
def _case_batch(precision, block, hybrid=False, ctas_per_sm=0, split=None):
    from paper_2404_08867_gb300 import inputs
    from paper_2404_08867_gb300.tuning import BatchedMDILR
    b = inputs.batch(count=COUNT, seed=0)
    plan = BatchedMDILR(b.families, b.d, b.a, b.n_last, b.offsets, b.pool, precision=precision, nodes=P_NODES)
    if split is None:
        split = plan.hybrid_split if hybrid else plan.count
    plan.opts.update(block=block, table_in_l1=1, split=split, ctas_per_sm=ctas_per_sm)
    return plan.launch


def build_case(name):
    """The launch function of a named workload:
      batch-fp64      4096-integral batch, FP64 node state (block 64, table via L1)
      batch-fp64-hybrid  the same with the planner's hybrid schedule
      batch-fp64-w10  the same on 5 two-warp CTAs per SM (10 warps), one warp per
                      integral (the tuner's choice for this batch)
      batch-df64      the same batch, double-float node state (block 32, table via L1)
      batch-df64-w12  the same on 6 two-warp CTAs per SM, the 102 largest integrals on
                      whole CTAs (the tuner's choice for this batch)
      batch-f32df     the same batch, phi in float, double-float sums (block 32)
      levels-d100     one integral, node state parallel over levels, the differentiation
                      workload (d = 100, N = 16 Gaussian, checkpoint 10): forward and adjoint
      levels-d1000    one integral, node state parallel over levels, d = 1000, N = 16:
                      forward and adjoint
      korobov         P_2 Korobov search, n = 65536, d = 4, every a in 1..n/2
      cbc             CBC, n = 65536, d = 4, gamma_j = 1/j^2, unanchored
      midpoint-d1000  paper-table mode, d = 1000, N = 20, n_last = 21 (Gaussian)
      closed-d4       closed state forward, f = exp(sum x_j / j), d = 4, a = N = 65536,
                      double-float cluster sums (time to 1e-6 of the small workload)
      closed-d4-fp64  the same in FP64
      closed-d1000    closed state forward, exp(sum x_j / j^2), d = 1000, N = 16, FP64
      slr-d4          plain lattice rule, f = exp(sum x_j / j), d = 4, n = 65536,
                      Korobov a = 11119 (the small workload's error-scanned parameter)
      slr-d7          plain lattice rule in FP64, f = exp(sum x_j / j), d = 7, n = 2^24,
                      Korobov a = 12345
      slr-df-d7       plain lattice rule in double-float, f = exp(sum x_j / j), d = 7,
                      n = 2^24, Korobov a = 12345
      improved-d7     improved lattice rule, d = 7, z = (1, 16, .., 16^6), n = 1 + 16^7
                      (16^6 - 1 ghosts), f = exp(sum x_j / j)
      improved-d7-df64  the same with the lattice points in double-float"""
    import torch
    import paper_2404_08867_gb300 as mdi
    from paper_2404_08867_gb300 import inputs
    if name == "batch-fp64":
        return _case_batch("fp64", 64)
    if name == "batch-fp64-hybrid":
        return _case_batch("fp64", 64, hybrid=True)
    if name == "batch-fp64-w10":
        return _case_batch("fp64", 64, ctas_per_sm=5, split=0)
    if name == "batch-df64":
        return _case_batch("df64", 32)
    if name == "batch-df64-w12":
        return _case_batch("df64", 64, ctas_per_sm=6, split=102)
    if name == "batch-f32df":
        return _case_batch("fp32_eval_df32", 32)
    if name == "levels-d100":
        w = inputs.gaussian(100, 16, seed=0)
        p = torch.as_tensor(w.params).cuda()
        return lambda: (mdi.mdi_lr_integrate("gauss", p, 100, 16, state="nodes"),
                        mdi.mdi_lr_grad("gauss", p, 100, 16, state="nodes", checkpoint=10))
    if name == "levels-d1000":
        w = inputs.scale_exp(1000, 16)
        p = torch.as_tensor(w.params).cuda()
        return lambda: (mdi.mdi_lr_integrate("exp", p, 1000, 16, state="nodes"),
                        mdi.mdi_lr_grad("exp", p, 1000, 16, 16, state="nodes"))
    if name == "korobov":
        vals = torch.empty(32768, dtype=torch.float64, device="cuda")
        return lambda: mdi.lattice_korobov_search(65536, 4, a_first=1, count=32768, values=vals)
    if name == "cbc":
        g = torch.as_tensor(1.0 / np.arange(1, 5) ** 2).cuda()
        ws = torch.empty(mdi.lattice_cbc_workspace_size(65536), dtype=torch.uint8, device="cuda")
        return lambda: mdi.lattice_cbc(65536, g, 0.0, workspace=ws)
    if name == "midpoint-d1000":
        w = inputs.gaussian(1000, 20, seed=0)
        p = torch.as_tensor(w.params).cuda()
        return lambda: mdi.mdi_midpoint_integrate("gauss", p, 1000, 20, 21)
    if name in ("closed-d4", "closed-d4-fp64"):
        p = torch.as_tensor(inputs.small_exp(4).params).cuda()
        prec = "fp64" if name.endswith("fp64") else "df64"
        return lambda: mdi.mdi_lr_integrate("exp", p, 4, 65536, 65536, state="closed", precision=prec)
    if name == "closed-d1000":
        p = torch.as_tensor(inputs.scale_exp(1000, 16).params).cuda()
        return lambda: mdi.mdi_lr_integrate("exp", p, 1000, 16, 16, state="closed")
    if name == "slr-d4":
        p = torch.as_tensor(inputs.small_exp(4).params).cuda()
        z = mdi.korobov_vector(4, 11119, 65536)
        return lambda: mdi.lattice_rule_integrate("exp", p, 65536, z)
    if name == "slr-d7":
        p = torch.as_tensor(inputs.small_exp(7).params).cuda()
        z = mdi.korobov_vector(7, 12345, 1 << 24)
        return lambda: mdi.lattice_rule_integrate("exp", p, 1 << 24, z)
    if name == "slr-df-d7":
        p = torch.as_tensor(inputs.small_exp(7).params).cuda()
        z = mdi.korobov_vector(7, 12345, 1 << 24)
        return lambda: mdi.lattice_rule_integrate("exp", p, 1 << 24, z, precision="df64")
    if name in ("improved-d7", "improved-d7-df64"):
        d, a = 7, 16
        prec = "df64" if name.endswith("df64") else "fp64"
        p = torch.as_tensor(np.r_[1.0 / np.arange(1, d + 1), np.zeros(d)]).cuda()
        ws = torch.empty(mdi.lattice_rule_improved_workspace_size(d, 1 + a ** d, a), dtype=torch.uint8,
                         device="cuda")
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        return lambda: mdi.lattice_rule_integrate_improved("exp", p, d, 1 + a ** d, a, precision=prec, out=out,
                                                           workspace=ws)
    raise SystemExit(f"unknown case {name!r}; see build_case")


def run_case(name, repeats):
    import torch
    run = build_case(name)
    for _ in range(repeats):
        run()
    torch.cuda.synchronize()
    print(f"{name}: {repeats} runs ok")


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return cpu_reference_arm(args, rank, world)
    if args.case:
        return run_case(args.case, args.repeats)

    import torch
    import torch.distributed as dist
    import paper_2404_08867_gb300 as mdi
    from paper_2404_08867_gb300 import inputs
    from paper_2404_08867_gb300.tuning import BatchedMDILR

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    b = inputs.batch(count=args.count, seed=rank)
    plan = BatchedMDILR(b.families, b.d, b.a, b.n_last, b.offsets, b.pool, precision=args.precision, nodes=P_NODES)
    tuning = {"block": args.block, "table_in_l1": args.table_in_l1} if args.no_tune else plan.tune()
    if args.no_tune:
        plan.opts.update(block=args.block, table_in_l1=args.table_in_l1)
    plan.capture()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    for _ in range(max(3, args.warmup)):
        plan.run()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.4)
    # FMA peaks at this clock, inside the sampled window, before the timed steps.
    peaks = measure_peaks(torch, mdi)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # evict L2 between timed steps (outside the events)
        starts[k].record(stream)
        plan.run()
        ends[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    value, total_ms = combine_ranks(sum(step_ms), len(b), args.steps, world, dist, "cuda")
    device_out = plan.out.clone()

    # End to end: pinned host inputs -> device, the launch, results -> pinned host.
    # The step's inputs (descriptors, order, parameters) in the plan's packed
    # layout, pinned: one host-to-device copy per step, one copy of the results back.
    h_in = plan.host_inputs(pinned=True)
    h_out = torch.empty(len(b), dtype=torch.float64).pin_memory()

    def e2e_step():
        plan.inputs.copy_(h_in, non_blocking=True)
        plan.run()
        h_out.copy_(plan.out, non_blocking=True)

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
    e2e_value, e2e_total = combine_ranks(sum(e_ms), len(b), args.steps, world, dist, "cuda")
    assert torch.equal(h_out, device_out.cpu()), "end-to-end result differs from the device-timed run"

    if rank == 0:
        kernel_ms = statistics.mean(step_ms)
        roof = roofline_entry(b, args.precision, kernel_ms, peaks, profiled_traffic(args.precision))
        pipe = profiled_pipe(args.precision)
        if pipe is not None:
            roof["pipe_busy_ncu"] = pipe
        dtype = {"df64": "f32x2 (double-float, FP64-class)", "fp64": "f64", "fp32_eval_fp64": "f32 eval + f64",
                 "fp32_eval_df32": "f32 eval + f32x2"}[args.precision]
        line = {"metric": METRIC, "value": value, "unit": "integrals/s", "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
                "config": workload_config(len(b), args.precision), "baseline_metric": BASELINE_METRIC,
                "gpu_launches": args.steps, "launch": {"cuda_graph": True, **{k: v for k, v in tuning.items()
                                                                              if k != "candidates"}},
                "e2e": {"value": e2e_value, "unit": "integrals/s",
                        "h2d_bytes_per_step": int(h_in.numel()),
                        "d2h_bytes_per_step": int(8 * h_out.numel())},
                "roofline": roof, "measured_peaks": peaks, "clocks": clocks, "wall_s_timed_region": wall}
        # The other arithmetic modes on the same batch (secondary entries).
        modes_out = {}
        if not args.no_extras:
            modes = {}
            for prec in ("fp64", "df64", "fp32_eval_df32", "fp32_eval_fp64"):
                if prec == args.precision:
                    continue
                mp_ = BatchedMDILR(b.families, b.d, b.a, b.n_last, b.offsets, b.pool, precision=prec, nodes=P_NODES)
                mt = mp_.tune()
                mp_.capture()
                ms = statistics.median(time_plan(torch, mp_, flush, stream, 10))
                modes_out[prec] = mp_.out.cpu().numpy()
                modes[prec] = {"ms_per_step": ms, "integrals_per_s": len(b) / (ms / 1e3), "block": mt["block"],
                               "table_in_l1": mt["table_in_l1"], "split": mt["split"],
                               "ctas_per_sm": mt["ctas_per_sm"],
                               "roofline": {k: v for k, v in roofline_entry(b, prec, ms, peaks,
                                                                           profiled_traffic(prec)).items()
                                            if k in ("achieved", "peak", "frac", "pipe", "impl_tflops",
                                                     "flops_formula", "traffic")}}
                if profiled_pipe(prec) is not None:
                    modes[prec]["roofline"]["pipe_busy_ncu"] = profiled_pipe(prec)
            line["modes"] = modes
            line["small_workload"] = extra_small_workload(torch, mdi, inputs)
            line["precision_workload"] = extra_precision(torch, mdi, inputs)
            line["differentiation_workload"] = extra_differentiation(torch, mdi, inputs)
            line["scale_workload"] = extra_scale(torch, mdi, inputs)
            line["step_size_workload"] = extra_step_size(torch, mdi, inputs)
            line["paper_table_workload"] = extra_paper_tables(torch, mdi)
            line["lattice_search_workload"] = extra_lattice_search(torch, mdi)
            line["paper_context"] = extra_paper_context(torch, mdi)
            line["batch_vs_plain_kernel"] = extra_batch_vs_plain(torch, mdi, inputs)
            line["improved_rule"] = extra_improved_rule(torch, mdi)
            line["time_to_1e-6_vs_d"] = extra_time_to_1e6_vs_d(torch, mdi, inputs)
            line["batch_size_sweep"] = extra_batch_size_sweep(torch, mdi, inputs, args.precision)
        # CPU baseline: the FP64 oracle on every host core (whole passes over this
        # batch), and on one core; the all-core pass also gives the oracle's value of
        # every integral, against which each mode's largest error is stated.
        ref, rate, cores, passes, secs = cpu_baseline_all_cores(len(b), rank, args.cpu_seconds)
        rate1, n1, secs1 = cpu_baseline_one_core(b, min(3.0, args.cpu_seconds))
        line["cpu_baseline"] = {"value": rate, "unit": "integrals/s", "cores": cores, "kind": "oracle",
                                "sample": f"{passes} passes over the {len(b)}-integral batch on {cores} host cores "
                                          f"in {secs:.1f} s",
                                "one_core": {"value": rate1, "unit": "integrals/s", "cores": 1,
                                             "sample": f"first {n1} integrals of the batch, {secs1:.1f} s"}}
        line["max_rel_err_vs_oracle"] = max_rel_err(device_out.cpu().numpy(), ref)
        for prec, out in modes_out.items():
            line["modes"][prec]["max_rel_err_vs_oracle"] = max_rel_err(out, ref)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
