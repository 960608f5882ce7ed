"""Seeded batches of molecules of uneven size for the batched evaluation.

The batched workload draws n_ao uniformly in [n_lo, n_hi], N_THC = alpha
n_ao, and per molecule the single-evaluation recipe of workloads.synth
(gapped orbital energies with a quarter of the levels occupied, S = I,
Gauss-Legendre tau grid shared by all molecules).
"""
from __future__ import annotations

import numpy as np

from . import synth


def make_batch(n_mol: int, n_lo: int, n_hi: int, n_tau: int, beta: float, seed: int, alpha: int = 5):
    rng = synth.rng_for(seed)
    sizes = rng.integers(n_lo, n_hi + 1, size=n_mol)
    cases = []
    for i, n in enumerate(sizes):
        n = int(n)
        cases.append(synth.make_sigma_case(n, alpha * n, n_tau, beta, seed * 1000 + i, n_occ=max(1, n // 4)))
    return cases
