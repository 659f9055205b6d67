"""The oracle still reproduces its frozen outputs (tests/golden/oracle_regression.json)."""
import json
import os

import pytest

from paper_1412_3655_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_regression.json")


def _cases():
    with open(GOLDEN) as f:
        return list(json.load(f)["cases"].items())


@pytest.mark.parametrize("name,case", _cases())
def test_oracle_regression(orc, name, case):
    L, nc = tuple(case["dims"]), case["nc"]
    U = synth.gauge_config(L, nc, case["eps"], case["seed"])
    th0, F0 = orc.theta(U, L, nc)
    assert th0 == pytest.approx(case["theta0"], rel=1e-13)
    assert F0 == pytest.approx(case["F0"], rel=1e-13)
    assert orc.plaquette(U, L, nc) == pytest.approx(case["plaquette0"], rel=1e-13)
    orc.sweep(U, L, nc, case["omega"], 1)
    th1, F1 = orc.theta(U, L, nc)
    assert th1 == pytest.approx(case["theta1"], rel=1e-12)
    assert F1 == pytest.approx(case["F1"], rel=1e-13)
    for i, mu, re, im in case["links_after_one_sweep"]:
        assert U[i, mu, 0, 1] == pytest.approx(complex(re, im), abs=1e-14)
    U = synth.gauge_config(L, nc, case["eps"], case["seed"])
    r = orc.landau_fix(U, L, nc, case["omega"], 1e-12, 3000, 1, 0)
    assert r["sweeps"] == case["fix_sweeps"]
    assert r["F"] == pytest.approx(case["fix_F"], rel=1e-12)
