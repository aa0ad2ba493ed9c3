"""Host helpers outside the oracle, pinned against it: the bench's closed forms
(its error columns' targets), the package's Korobov generating vector, and the
boundary rule that only the bench's CPU-baseline legs and reference arm, and no
module of the package, import the oracle."""
import ast
import os

import numpy as np
import pytest

import bench
import paper_2404_08867_gb300 as mdi
from oracle import oracle as o

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("fam", ["exp", "gauss", "peak", "osc"])
@pytest.mark.parametrize("d,seed", [(1, 0), (7, 1), (50, 2)])
def test_exact_integral_matches_oracle(fam, d, seed):
    rng = np.random.default_rng(seed)
    c, w = rng.uniform(0.2, 2.0, d), rng.uniform(0.0, 1.0, d)
    ref = o.closed_form(fam, d, c, w)
    got = bench.exact_integral(fam, d, c, w)
    assert abs(got - ref) <= 1e-13 * max(abs(ref), 1e-3)


def test_exact_gauss_grad_matches_oracle():
    rng = np.random.default_rng(5)
    c, w = rng.uniform(0.2, 1.5, 100), rng.uniform(0.0, 1.0, 100)
    ref = o.closed_form_grad("gauss", 100, c, w)
    assert np.max(np.abs(bench.exact_gauss_grad(100, c, w) - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("d,a,n", [(4, 12345, 65536), (20, 3, (1 << 63) - 25), (9, (1 << 62) + 7, (1 << 63) - 25),
                                   (1, 5, 7), (6, 16, 1 + 16 ** 7)])
def test_korobov_vector_matches_oracle(d, a, n):
    assert np.array_equal(mdi.korobov_vector(d, a, n).astype(np.uint64), o.korobov_z(d, a, n))


def _oracle_importers(path):
    tree = ast.parse(open(path).read())
    found = []

    class V(ast.NodeVisitor):
        def __init__(self):
            self.stack = []

        def visit_FunctionDef(self, node):
            self.stack.append(node.name)
            self.generic_visit(node)
            self.stack.pop()

        def visit_ImportFrom(self, node):
            if node.module and node.module.split(".")[0] == "oracle":
                found.append(self.stack[0] if self.stack else "<module>")

        def visit_Import(self, node):
            if any(a.name.split(".")[0] == "oracle" for a in node.names):
                found.append(self.stack[0] if self.stack else "<module>")

    V().visit(tree)
    return found


def test_oracle_only_in_cpu_baseline_and_reference_legs():
    users = _oracle_importers(os.path.join(ROOT, "bench.py"))
    assert users, "the CPU baseline must still time the oracle"
    assert all(u.startswith("cpu_") for u in users), users
    pkg = os.path.join(ROOT, "paper_2404_08867_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            assert not _oracle_importers(os.path.join(pkg, f)), f


def test_flop_counts_of_the_batched_formulations():
    # By construction: one cluster point of an unpaired level costs the coordinate,
    # phi, the accumulation and a P-term Dot2; pairing halves the Dot2 terms; the
    # float-phi mode replaces the coordinate, phi and accumulation counts.
    from types import SimpleNamespace
    P = bench.P_NODES
    one = SimpleNamespace(families=["gauss"], d=np.array([3]), a=np.array([5]), n_last=np.array([5]))
    F = bench.DF_FLOPS
    pt = F["u"] + F["phi"]["gauss"] + F["acc"]
    full = P * F["dot_term"] + F["dot_value"]
    half = P * F["dot_term"] / 2 + F["dot_value"] + F["combine"]
    last = 5 * (pt + full)
    assert bench.df_flops(one, paired=False) == 5 * P * (pt + full) + 5 * P * pt + last
    assert bench.df_flops(one) == 5 * P * (pt + half) + 5 * P * pt + last
    pf = bench.F32_FLOPS["u"] + bench.F32_FLOPS["phi"]["gauss"] + bench.F32_FLOPS["acc"]
    assert bench.df_flops(one, float_phi=True) == 5 * P * (pf + half) + 5 * P * pf + last
    osc = SimpleNamespace(families=["osc"], d=np.array([3]), a=np.array([5]), n_last=np.array([5]))
    assert bench.df_flops(osc, float_phi=True) == bench.df_flops(osc, paired=False)  # OSC: unpaired, FP64 phi


def test_algorithmic_flop_count():
    """The algorithmic count for the batch: d N (P C_phi + P^2) per integral (a = N)."""
    from types import SimpleNamespace
    P = bench.P_NODES
    b = SimpleNamespace(families=["gauss", "peak"], d=np.array([3, 7]), a=np.array([5, 20]), n_last=np.array([5, 20]))
    expect = 3 * 5 * (P * bench.C_PHI["gauss"] + P * P) + 7 * 20 * (P * bench.C_PHI["peak"] + P * P)
    assert bench.alg_flops(b) == expect
    assert bench.C_PHI["gauss"] == bench.C_PHI["peak"] == 25


def test_reference_arm_prints_one_line():
    """bench.py --impl reference: the CPU oracle on the host cores (spawned pool),
    one pass over the batch per step, one JSON line with the contract's keys."""
    import json
    import subprocess
    import sys
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--count", "48"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr
    line = json.loads(res.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "integrals/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["steps"] == 2 and line["dtype"] == "f64"
