"""Named workloads, each run a fixed number of times through the public API, for
profiling one kernel at a time (``python -m paper_2404_08867_gb300.cases NAME
[REPEATS]``).  Inputs are the seeded synthetic ones of ``inputs``; nothing here
computes: every launch goes through the C ABI.

  batch-df64      4096-integral batch, double-float node state (block 32, table via L1)
  batch-fp64      the same batch in FP64 (block 64, table via L1)
  batch-f32df     the same batch, phi in float, double-float sums (block 32, table via L1)
  levels-d1000    one integral, node state parallel over levels, d = 1000, N = 16:
                  forward and adjoint
  korobov         P_2 Korobov search, n = 65536, d = 4, every a in 1..n/2
  cbc             CBC, n = 65536, d = 4, gamma_j = 1/j^2, unanchored
  midpoint-d1000  paper-table mode, d = 1000, N = 20, n_last = 21 (Gaussian)
  closed-d4       closed state forward, f = exp(sum x_j / j), d = 4, a = N = 65536,
                  double-float cluster sums (time to 1e-6 of the small workload)
  closed-d1000    closed state forward, exp(sum x_j / j^2), d = 1000, N = 16, FP64
  slr-d4          plain lattice rule, f = exp(sum x_j / j), d = 4, n = 65536, Korobov
                  a = 11119 (the small workload's error-scanned parameter)
  slr-df-d7       plain lattice rule in double-float, f = exp(sum x_j / j), d = 7,
                  n = 2^24, Korobov a = 12345
  improved-d7     improved lattice rule, d = 7, z = (1, 16, .., 16^6), n = 1 + 16^7
                  (16^6 - 1 ghosts), f = exp(sum x_j / j)
  improved-d7-df64  the same with the lattice points in double-float
"""
from __future__ import annotations

import sys

import numpy as np
import torch

import paper_2404_08867_gb300 as mdi
from paper_2404_08867_gb300 import inputs


def _batch(precision: str, block: int):
    from paper_2404_08867_gb300.tuning import BatchedMDILR
    b = inputs.batch(count=4096, seed=0)
    plan = BatchedMDILR(b.families, b.d, b.a, b.n_last, b.offsets, b.pool, precision=precision, nodes=16)
    plan.opts.update(block=block, table_in_l1=1)
    return plan.launch


def build_case(name: str):
    if name == "batch-df64":
        return _batch("df64", 32)
    if name == "batch-fp64":
        return _batch("fp64", 64)
    if name == "batch-f32df":
        return _batch("fp32_eval_df32", 32)
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
    if name == "closed-d4":
        p = torch.as_tensor(inputs.small_exp(4).params).cuda()
        return lambda: mdi.mdi_lr_integrate("exp", p, 4, 65536, 65536, state="closed", precision="df64")
    if name == "closed-d1000":
        p = torch.as_tensor(inputs.scale_exp(1000, 16).params).cuda()
        return lambda: mdi.mdi_lr_integrate("exp", p, 1000, 16, 16, state="closed")
    if name == "slr-d4":
        p = torch.as_tensor(inputs.small_exp(4).params).cuda()
        z = mdi.korobov_vector(4, 11119, 65536)
        return lambda: mdi.lattice_rule_integrate("exp", p, 65536, z)
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
    raise SystemExit(f"unknown case {name!r}; see the module docstring")


def main(argv):
    if len(argv) < 2:
        raise SystemExit(__doc__)
    run = build_case(argv[1])
    repeats = int(argv[2]) if len(argv) > 2 else 5
    for _ in range(repeats):
        run()
    torch.cuda.synchronize()
    print(f"{argv[1]}: {repeats} runs ok")


if __name__ == "__main__":
    main(sys.argv)
