"""Writes tests/golden/thc20_oracle.json from the FP64 oracle only.

The 20-AO workload (n=20, N=60, 32 Gauss-Legendre tau points, beta=100) is
drawn by workloads.synth; every stored value comes from oracle.thc_oracle.
Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import thc_oracle as o  # noqa: E402
from workloads import synth  # noqa: E402


def main():
    case = synth.make_workload("thc20")
    Sd = o.sigma_thc(case.X, case.V, case.G_tau, case.G_bmt, terms="direct")
    Sx = o.sigma_thc(case.X, case.V, case.G_tau, case.G_bmt, terms="sox")
    rng = np.random.default_rng(0)
    idx = [(int(k), int(i), int(j)) for k, i, j in zip(rng.integers(0, case.n_tau, 24),
                                                       rng.integers(0, case.n, 24),
                                                       rng.integers(0, case.n, 24))]
    out = {
        "workload": "thc20", "n": case.n, "N": case.N, "n_tau": case.n_tau, "beta": case.beta,
        "E_dyn_direct": o.energy_dyn_tau(case.G_bmt, Sd, case.tau_w),
        "E_dyn_sox": o.energy_dyn_tau(case.G_bmt, Sx, case.tau_w),
        "sigma_fro_per_tau": [float(np.linalg.norm(Sd[k] + Sx[k])) for k in range(case.n_tau)],
        "samples": [[k, i, j, float(Sd[k, i, j]), float(Sx[k, i, j])] for k, i, j in idx],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "thc20_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
