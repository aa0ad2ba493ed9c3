"""Writes oracle_workloads.json: the CPU oracle's FP64 values for the bench's
small fixed workloads, so that the bench can state each GPU result's error
against the oracle without running the oracle outside its CPU-baseline leg.
Calls only the oracle (and the seeded input generator); rerun it after any change
to either:

    python tests/golden/make_oracle_workloads.py

Contents (the node state with P = 16 everywhere):
  precision        d = 50, N = 32, cos(2 pi u + sum a_j x_j) (seed 0): closed and
                   node-state values
  differentiation  d = 100, N = 16 Gaussian (seed 0): node-state value and its 200
                   derivatives (c_1..c_100, w_1..w_100)
  scale            N = 16, exp(sum x_j / j^2), d in {100, 250, 500, 1000}: closed
                   and node-state values
  step             Algorithm 1's step size m = 1, 2, 3 with the node state at d = 100,
                   N = 16: the Gaussian of the differentiation workload, and
                   exp(sum x_j / j^2) beside its closed state (the exact rule)
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as o  # noqa: E402
from paper_2404_08867_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "oracle_workloads.json")
SCALE_DS = (100, 250, 500, 1000)


def compute():
    w = inputs.oscillatory(50, 32, seed=0)
    precision = {"closed": o.mdi_closed("osc", 50, 32, 32, w.c, w.w),
                 "nodes": o.mdi_nodes("osc", 50, 32, 32, 16, w.c, w.w)}
    g = inputs.gaussian(100, 16, seed=0)
    differentiation = {"value": o.mdi_nodes("gauss", 100, 16, 16, 16, g.c, g.w),
                       "grad": [float(x) for x in o.mdi_nodes_grad("gauss", 100, 16, 16, 16, g.c, g.w)]}
    scale = {}
    for d in SCALE_DS:
        s = inputs.scale_exp(d, 16)
        scale[str(d)] = {"closed": o.mdi_closed("exp", d, 16, 16, s.c, s.w),
                         "nodes": o.mdi_nodes("exp", d, 16, 16, 16, s.c, s.w)}
    s100 = inputs.scale_exp(100, 16)
    step = {"gauss": {str(m): o.mdi_nodes_step("gauss", 100, 16, 16, 16, m, g.c, g.w) for m in (1, 2, 3)},
            "exp": {str(m): o.mdi_nodes_step("exp", 100, 16, 16, 16, m, s100.c, s100.w) for m in (1, 2, 3)},
            "exp_closed": o.mdi_closed("exp", 100, 16, 16, s100.c, s100.w)}
    return {"precision": precision, "differentiation": differentiation, "scale": scale, "step": step}


if __name__ == "__main__":
    with open(OUT, "w") as f:
        json.dump(compute(), f, indent=1)
        f.write("\n")
    print(OUT)
