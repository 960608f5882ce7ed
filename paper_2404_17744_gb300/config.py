"""Run configuration of the self-consistent loop (host side).

`LoopConfig` collects the knobs of a run: the precision of the Sigma evaluation, the
method (GF2, or scGWSOX with the screened direct term), the mixing (damping, residual
DIIS or commutator DIIS, Sec. III.A), the stopping rule, the learned proposals, the
autotuner cache and the checkpoint / metrics paths.  It round-trips through JSON, and
`run_loop` runs one loop from it.  The arrays (THC factors, F, S, the IR grid and, for
scGWSOX, the bosonic transforms) are passed separately.
"""
from __future__ import annotations

import dataclasses
import json
import os

from . import thc

PRECISIONS = {"fp64": thc.THC_FP64, "bf16x3": thc.THC_BF16X3}
METHODS = ("gf2", "gwsox")
MIXINGS = ("diis", "cdiis", "damp")


@dataclasses.dataclass
class LoopConfig:
    precision: str = "fp64"          # "fp64" or "bf16x3"
    method: str = "gf2"              # "gf2" (direct + SOX) or "gwsox" (screened direct + SOX)
    mixing: str = "diis"             # "diis", "cdiis" or "damp"
    damping: float = 0.5
    n_damp: int = 2                  # damped iterations before DIIS starts
    diis_size: int = 6
    tol: float = 1e-8                # |E_k - E_(k-1)| < tol ends the run
    max_iter: int = 60
    learned_proposals: int = 0       # online-trained learned proposals per run (0: none)
    autotune_cache: str | None = None  # tile table loaded before and saved after the run
    checkpoint: str | None = None      # loop state written after every iteration
    metrics: str | None = None         # one JSON line per iteration

    def __post_init__(self):
        if self.precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
        if self.method not in METHODS:
            raise ValueError(f"method must be one of {METHODS}")
        if self.mixing not in MIXINGS:
            raise ValueError(f"mixing must be one of {MIXINGS}")
        if not (0.0 < self.damping <= 1.0):
            raise ValueError("damping must lie in (0, 1]")
        if self.n_damp < 0 or not (1 <= self.diis_size <= 16) or self.max_iter < 1 or self.tol < 0:
            raise ValueError("need n_damp >= 0, 1 <= diis_size <= 16, max_iter >= 1 and tol >= 0")
        if self.learned_proposals < 0:
            raise ValueError("learned_proposals must be >= 0")

    def to_json(self) -> str:
        return json.dumps(dataclasses.asdict(self), sort_keys=True)

    @classmethod
    def from_json(cls, text: str) -> "LoopConfig":
        return cls(**json.loads(text))


def run_loop(X, V, F, S, grid, n_elec, config: LoopConfig, bosonic=None, device="cuda:0", stream=None,
             resume=False):
    """One self-consistent run as `config` describes; returns (converged, records).

    bosonic: the grid's bosonic transforms (to_iw, to_tau), required for method "gwsox".
    resume: continue from config.checkpoint when that file exists."""
    from . import scf
    if config.method == "gwsox" and bosonic is None:
        raise ValueError("method 'gwsox' needs the bosonic transforms of the grid")
    if config.autotune_cache and os.path.exists(config.autotune_cache):
        thc.thc_autotune_load(config.autotune_cache)
    L = scf.GF2Loop(X, V, F, S, grid, n_elec, precision=PRECISIONS[config.precision], device=device, stream=stream,
                    damping=config.damping, n_damp=config.n_damp, diis_size=config.diis_size, mixing=config.mixing,
                    bosonic=bosonic if config.method == "gwsox" else None)
    P = scf.LearnedProposer(L, max_proposals=config.learned_proposals) if config.learned_proposals else None
    try:
        if resume and config.checkpoint and os.path.exists(config.checkpoint):
            L.resume(config.checkpoint, P)
        conv = L.run(tol=config.tol, max_iter=config.max_iter, proposer=P, metrics=config.metrics,
                     checkpoint=config.checkpoint)
        records = list(L.records)
    finally:
        if P is not None:
            P.close()
        L.close()
    if config.autotune_cache:
        thc.thc_autotune_save(config.autotune_cache)
    return conv, records
