"""Writes the oracle's values for the full-size workloads, from the FP64 oracle only.

For each workload named on the command line (default: thc200 thc500) it draws the
inputs with workloads.synth, evaluates Sigma(tau_k) = Sigma^dir + Sigma^SOX at every
tau point with oracle.thc_oracle (SOX through ``sigma_sox_thc_rows``, the scheme's
steps on slices of P, so that the N x N x n intermediates fit in host memory) and
stores in tests/golden/<name>_oracle.json:

* E_dyn of both terms together and of each term (Eq. E2b with the workload's own
  Gauss-Legendre weights), and the per-tau traces Tr[G(beta - tau_k) Sigma(tau_k)];
* at three tau points (the first, the middle and the last) the diagonal of Sigma,
  a seeded sample of off-diagonal elements, max|Sigma| and its Frobenius norm.

At 500 AOs and 2500 THC points this takes about 45 minutes on 8 x86 cores; partial
results are kept in <name>_oracle.partial.npz beside the output and reused.
Run: python tests/golden/make_golden_large.py [thc200] [thc500]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import thc_oracle as o  # noqa: E402
from workloads import synth  # noqa: E402

N_OFFDIAG = 1500  # sampled off-diagonal elements per stored tau point


def sample_points(n_tau: int) -> list[int]:
    return sorted({0, n_tau // 2, n_tau - 1})


def offdiag_sample(n: int, seed: int) -> list[tuple[int, int]]:
    rng = np.random.default_rng(seed)
    i = rng.integers(0, n, 3 * N_OFFDIAG)
    j = rng.integers(0, n, 3 * N_OFFDIAG)
    keep = [(int(a), int(b)) for a, b in zip(i, j) if a != b]
    return keep[:N_OFFDIAG]


def run(name: str) -> None:
    case = synth.make_workload(name)
    out_path = os.path.join(HERE, f"{name}_oracle.json")
    part_path = os.path.join(HERE, f"{name}_oracle.partial.npz")
    nt = case.n_tau
    tr_dir = np.full(nt, np.nan)
    tr_sox = np.full(nt, np.nan)
    if os.path.exists(part_path):
        p = np.load(part_path)
        tr_dir, tr_sox = p["tr_dir"], p["tr_sox"]
    stored = sample_points(nt)
    pairs = offdiag_sample(case.n, seed=case.n)
    samples = {}
    t_start = time.time()
    U = o.thc_U(case.X, case.V)
    for k in range(nt):
        need_sample = k in stored
        if np.isfinite(tr_dir[k]) and np.isfinite(tr_sox[k]) and not need_sample:
            continue
        G = case.G_tau[k]
        Gm = o.g_minus_tau(case.G_bmt[k])
        Sd = o.sigma_direct_thc(case.X, case.V, G, Gm)
        Sx = o.sigma_sox_thc_rows(case.X, U, G, Gm)
        tr_dir[k] = np.trace(case.G_bmt[k] @ Sd)
        tr_sox[k] = np.trace(case.G_bmt[k] @ Sx)
        if need_sample:
            S = Sd + Sx
            samples[str(k)] = {
                "tau": float(case.tau[k]),
                "max_abs": float(np.abs(S).max()),
                "fro": float(np.linalg.norm(S)),
                "diag": [float(x) for x in np.diag(S)],
                "offdiag": [[i, j, float(S[i, j])] for i, j in pairs],
            }
        np.savez(part_path, tr_dir=tr_dir, tr_sox=tr_sox)
        print(f"{name}: tau {k + 1}/{nt} done, {time.time() - t_start:.0f} s", flush=True)
    w = case.tau_w
    out = {
        "workload": name, "n": case.n, "N": case.N, "n_tau": nt, "beta": case.beta,
        "source": "oracle.thc_oracle (sigma_direct_thc, sigma_sox_thc_rows, energy as -sum_k w_k tr_k)",
        "E_dyn": float(-np.dot(w, tr_dir + tr_sox)),
        "E_dyn_direct": float(-np.dot(w, tr_dir)),
        "E_dyn_sox": float(-np.dot(w, tr_sox)),
        "trace_per_tau": [float(x) for x in tr_dir + tr_sox],
        "samples": samples,
    }
    with open(out_path, "w") as f:
        json.dump(out, f, indent=0)
    os.remove(part_path)
    print("wrote", out_path)


if __name__ == "__main__":
    for nm in (sys.argv[1:] or ["thc200", "thc500"]):
        run(nm)
