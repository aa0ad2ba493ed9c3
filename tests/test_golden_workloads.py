"""The stored oracle values of the bench's fixed workloads
(tests/golden/oracle_workloads.json) are the oracle's: recomputed here and
compared within rounding (the host's libm may differ by an ulp between
machines)."""
import importlib.util
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _module():
    spec = importlib.util.spec_from_file_location("make_oracle_workloads",
                                                  os.path.join(HERE, "golden", "make_oracle_workloads.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_stored_values_are_the_oracles():
    m = _module()
    stored = json.load(open(m.OUT))
    fresh = m.compute()
    assert stored.keys() == fresh.keys()
    for k in ("closed", "nodes"):
        assert abs(stored["precision"][k] - fresh["precision"][k]) <= 1e-14
    assert abs(stored["differentiation"]["value"] / fresh["differentiation"]["value"] - 1) <= 1e-14
    g0, g1 = np.array(stored["differentiation"]["grad"]), np.array(fresh["differentiation"]["grad"])
    assert g0.shape == (200,)
    assert np.all(np.abs(g0 - g1) <= 1e-14 * np.abs(g1) + 1e-17 * np.max(np.abs(g1)))
    for d in map(str, m.SCALE_DS):
        for k in ("closed", "nodes"):
            assert abs(stored["scale"][d][k] / fresh["scale"][d][k] - 1) <= 1e-14
    for fam in ("gauss", "exp"):
        for k in ("1", "2", "3"):
            assert abs(stored["step"][fam][k] / fresh["step"][fam][k] - 1) <= 1e-14
    assert abs(stored["step"]["exp_closed"] / fresh["step"]["exp_closed"] - 1) <= 1e-14
