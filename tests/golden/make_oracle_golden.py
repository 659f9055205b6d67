"""Write oracle_regression.json from the CPU oracle alone (no CUDA code).

Run from the repository root:  python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1412_3655_gb300 import synth  # noqa: E402

CASES = [
    # (name, dims, nc, eps, seed, omega)
    ("su3_4x4x4x4_seed1", (4, 4, 4, 4), 3, 0.3, 1, 1.7),
    ("su2_4x4x4x4_seed1", (4, 4, 4, 4), 2, 0.3, 1, 1.7),
    ("su3_2x4x2x6_seed7", (2, 4, 2, 6), 3, 0.5, 7, 1.5),
]


def main():
    out = {"source": "oracle/culgt_oracle.c via tests/golden/make_oracle_golden.py", "cases": {}}
    for name, L, nc, eps, seed, omega in CASES:
        U = synth.gauge_config(L, nc, eps, seed)
        th0, F0 = oracle.theta(U, L, nc)
        P0 = oracle.plaquette(U, L, nc)
        oracle.sweep(U, L, nc, omega, 1)
        th1, F1 = oracle.theta(U, L, nc)
        sample = [[int(i), int(mu), float(U[i, mu, 0, 1].real), float(U[i, mu, 0, 1].imag)]
                  for i, mu in [(0, 0), (5, 1), (len(U) - 1, 3)]]
        U = synth.gauge_config(L, nc, eps, seed)
        r = oracle.landau_fix(U, L, nc, omega, 1e-12, 3000, 1, 0)
        out["cases"][name] = {
            "dims": list(L), "nc": nc, "eps": eps, "seed": seed, "omega": omega,
            "theta0": th0, "F0": F0, "plaquette0": P0,
            "theta1": th1, "F1": F1, "links_after_one_sweep": sample,
            "fix_sweeps": r["sweeps"], "fix_theta": r["theta"], "fix_F": r["F"],
        }
    # the extensions: simulated annealing (Landau, MAG, Coulomb) and the
    # maximally Abelian gauge, on the 4^4 SU(3) and SU(2) fields
    ext = {}
    for nc in (3, 2):
        L = (4, 4, 4, 4)
        U = synth.gauge_config(L, nc, 0.3, 1)
        oracle.heatbath_sweep(U, L, nc, 0.5, 77, 3)
        hb = [float(U[5, 1, 0, 1].real), float(U[5, 1, 0, 1].imag), oracle.theta(U, L, nc)[1]]
        U = synth.gauge_config(L, nc, 0.5, 1)
        oracle.anneal(U, L, nc, 0.6, 0.05, 10, 2, 78, reunit_every=20)
        r = oracle.landau_fix(U, L, nc, 1.7, 1e-12, 5000, 5, 50)
        U = synth.gauge_config(L, nc, 0.3, 1)
        oracle.mag_sweep(U, L, nc, 1.7, 1)
        mag1 = list(oracle.mag_theta(U, L, nc))
        U = synth.gauge_config(L, nc, 0.3, 1)
        rm = oracle.mag_fix(U, L, nc, 1.7, 1e-12, 5000, 5, 50)
        U = synth.gauge_config(L, nc, 0.5, 1)
        oracle.mag_anneal(U, L, nc, 0.6, 0.05, 10, 2, 79, reunit_every=20)
        ra = oracle.mag_fix(U, L, nc, 1.7, 1e-12, 5000, 5, 50)
        Lc = (4, 4, 4, 2)
        U = synth.gauge_config(Lc, nc, 0.5, 6)
        rc = oracle.coulomb_fix_anneal(U, Lc, nc, 0.6, 0.05, 10, 2, 80, 1.7, 1e-12, 5000, 5, 25)
        ext[f"su{nc}"] = {
            "heatbath_sweep_T0.5_seed77_word3": hb,
            "anneal_then_landau_fix": {"sweeps": r["sweeps"], "F": r["F"]},
            "mag_one_sweep_theta_F": mag1,
            "mag_fix": {"sweeps": rm["sweeps"], "F": rm["F"]},
            "mag_anneal_then_fix": {"sweeps": ra["sweeps"], "F": ra["F"]},
            "coulomb_anneal": {"sweeps": [int(x) for x in rc["sweeps"]], "F": [float(x) for x in rc["F"]]},
        }
    out["extensions"] = ext
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
