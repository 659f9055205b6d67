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
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
