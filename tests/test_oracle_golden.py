"""The oracle still reproduces its frozen outputs (tests/golden/oracle_regression.json)."""
import json
import os

import numpy as np
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


def _extensions():
    with open(GOLDEN) as f:
        return list(json.load(f)["extensions"].items())


@pytest.mark.parametrize("group,case", _extensions())
def test_oracle_regression_extensions(orc, group, case):
    """Annealing (Landau, MAG, Coulomb) and the maximally Abelian gauge still
    give their frozen outputs."""
    nc = int(group[2:])
    L = (4, 4, 4, 4)
    U = synth.gauge_config(L, nc, 0.3, 1)
    orc.heatbath_sweep(U, L, nc, 0.5, 77, 3)
    re, im, F = case["heatbath_sweep_T0.5_seed77_word3"]
    assert U[5, 1, 0, 1] == pytest.approx(complex(re, im), abs=1e-14)
    assert orc.theta(U, L, nc)[1] == pytest.approx(F, rel=1e-13)
    U = synth.gauge_config(L, nc, 0.5, 1)
    orc.anneal(U, L, nc, 0.6, 0.05, 10, 2, 78, reunit_every=20)
    r = orc.landau_fix(U, L, nc, 1.7, 1e-12, 5000, 5, 50)
    assert r["sweeps"] == case["anneal_then_landau_fix"]["sweeps"]
    assert r["F"] == pytest.approx(case["anneal_then_landau_fix"]["F"], rel=1e-12)
    U = synth.gauge_config(L, nc, 0.3, 1)
    orc.mag_sweep(U, L, nc, 1.7, 1)
    th, F = orc.mag_theta(U, L, nc)
    assert th == pytest.approx(case["mag_one_sweep_theta_F"][0], rel=1e-12)
    assert F == pytest.approx(case["mag_one_sweep_theta_F"][1], rel=1e-13)
    U = synth.gauge_config(L, nc, 0.3, 1)
    r = orc.mag_fix(U, L, nc, 1.7, 1e-12, 5000, 5, 50)
    assert r["sweeps"] == case["mag_fix"]["sweeps"] and r["F"] == pytest.approx(case["mag_fix"]["F"], rel=1e-12)
    U = synth.gauge_config(L, nc, 0.5, 1)
    orc.mag_anneal(U, L, nc, 0.6, 0.05, 10, 2, 79, reunit_every=20)
    r = orc.mag_fix(U, L, nc, 1.7, 1e-12, 5000, 5, 50)
    assert r["sweeps"] == case["mag_anneal_then_fix"]["sweeps"]
    assert r["F"] == pytest.approx(case["mag_anneal_then_fix"]["F"], rel=1e-12)
    Lc = (4, 4, 4, 2)
    U = synth.gauge_config(Lc, nc, 0.5, 6)
    rc = orc.coulomb_fix_anneal(U, Lc, nc, 0.6, 0.05, 10, 2, 80, 1.7, 1e-12, 5000, 5, 25)
    assert list(rc["sweeps"]) == case["coulomb_anneal"]["sweeps"]
    assert np.allclose(rc["F"], case["coulomb_anneal"]["F"], rtol=1e-12, atol=0)
