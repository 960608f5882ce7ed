"""Self-consistent GF2 loop on the GPU (Sec. II.A of arXiv:2404.17744).

Each iteration: Sigma[G] with thc_sigma_eval (FP64 or 3 x BF16 tensor
cores), the Galitskii-Migdal energy, damping then DIIS on the self-energy,
and the Dyson step with the chemical potential re-optimised at fixed
electron count (thc_dyson_solve).  Every array operation runs in the
library's kernels; this module holds the host-side control: the iteration,
the convergence test and the small DIIS system (at most 16 x 16).

Monitor energy with a fixed one-body matrix F:  E = 2 Tr[gamma F] + E_dyn.

Auxiliary parts: `run(metrics=...)` writes one JSON line per iteration (energy,
its change, mu, electron count, residual, proposal label, and the per-kernel-class
GPU time of the iteration when the library profiler is on); `run(checkpoint=...)`
saves the loop state after every iteration and `GF2Loop.resume(path)` restores
it, so that an interrupted run continues from the iteration it had completed.
"""
from __future__ import annotations

import dataclasses
import json
import os
import time

import numpy as np

from . import thc


@dataclasses.dataclass
class IterationRecord:
    iter: int
    E: float
    E_dyn: float
    mu: float
    n_per_spin: float
    residual: float
    seconds: float
    sigma_seconds: float
    dyson_evals: int
    proposal: str = ""


class GF2Loop:
    """Fully self-consistent GF2 (or, with `bosonic` transforms, scGWSOX) with THC
    self-energies on one GPU.

    grid: an object with tau, iw, U_tau, fit_tau, U_iw, fit_iw, u_beta, u_zero
    and basis.beta / basis.L (workloads.ir.LoopGrid); the tau points must be
    mirror-symmetric.  X, V, F, S are numpy FP64 arrays.
    """

    def __init__(self, X, V, F, S, grid, n_elec, precision=thc.THC_FP64, device="cuda:0", stream=None,
                 damping=0.5, n_damp=2, diis_size=6, mixing="diis", bosonic=None):
        import torch
        self.torch = torch
        self.dev = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.dev)
        self.n, self.N = X.shape
        self.grid = grid
        self.n_tau = len(grid.tau)
        self.n_elec = float(n_elec)
        self.damping, self.n_damp, self.diis_size = damping, n_damp, min(diis_size, 16)
        if mixing not in ("diis", "cdiis", "damp"):
            raise ValueError("mixing must be 'diis', 'cdiis' or 'damp'")
        self.mixing = mixing
        with torch.cuda.stream(self.stream):
            self.X = torch.from_numpy(np.ascontiguousarray(X)).to(self.dev)
            self.V = torch.from_numpy(np.ascontiguousarray(V)).to(self.dev)
            self.F = torch.from_numpy(np.ascontiguousarray(F)).to(self.dev)
            self.S = torch.from_numpy(np.ascontiguousarray(S)).to(self.dev)
            shape = (self.n_tau, self.n, self.n)
            self.G = torch.empty(shape, dtype=torch.float64, device=self.dev)
            self.Sig_out = torch.empty_like(self.G)
            self.Sig_in = torch.zeros_like(self.G)
            self.scratch = torch.empty(512, dtype=torch.float64, device=self.dev)
        s = self.stream.cuda_stream
        # bosonic: transforms (to_iw, to_tau) of the grid for the screened direct term, i.e. the
        # scGWSOX loop (Sigma = Sigma^GW + Sigma^SOX); None: the GF2 loop (direct + SOX)
        terms = (thc.THC_GW | thc.THC_SOX) if bosonic is not None else (thc.THC_DIRECT | thc.THC_SOX)
        self.ctx = thc.thc_sigma_init(self.n, self.N, self.n_tau, grid.basis.beta, self.X, self.V,
                                      np.ascontiguousarray(grid.tau), precision, terms, s)
        if bosonic is not None:
            thc.thc_sigma_set_bosonic(self.ctx, bosonic.to_iw, bosonic.to_tau)
        self.dy = thc.thc_dyson_init(self.n, self.n_tau, len(grid.iw), grid.basis.L, grid.basis.beta, self.S, self.F,
                                     grid.U_tau, grid.fit_tau, grid.U_iw, grid.fit_iw, grid.iw, grid.u_beta,
                                     grid.u_zero, s)
        self.mu = 0.0
        self.history: list[tuple] = []   # (Sigma_out, residual) device tensors for DIIS
        self.records: list[IterationRecord] = []
        self.iteration = 0               # iterations completed (mixing and Dyson step included)
        self.E_prev = None
        self._kernel_ms: dict[str, float] = {}

    def close(self):
        if self.ctx is not None:
            thc.thc_destroy(self.ctx)
            self.ctx = None
        if self.dy is not None:
            thc.thc_dyson_destroy(self.dy)
            self.dy = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ pieces
    def _len(self):
        return self.n_tau * self.n * self.n

    def _dot(self, a, b):
        return thc.thc_vec_dot(a.numel(), a, b, self.scratch, self.stream.cuda_stream)

    def _lincomb(self, coeffs, vecs, out):
        thc.thc_vec_lincomb(coeffs, vecs, self._len(), out, self.stream.cuda_stream)

    def dyson(self, sigma=None):
        self.mu = thc.thc_dyson_solve(self.dy, sigma, self.n_elec, self.mu, 1e-11, self.G)
        return thc.thc_dyson_evals(self.dy)

    def sigma(self):
        thc.thc_sigma_eval(self.ctx, self.G, None, self.Sig_out)
        thc.thc_sync(self.ctx)

    def energy(self):
        e_dyn, trgf, n = thc.thc_dyson_energy(self.dy, self.G, self.Sig_out)
        return 2.0 * trgf + e_dyn, e_dyn, n

    def mix(self, it):
        """Next input self-energy from the history: damping, then DIIS on the residual
        Sigma_out - Sigma_in ("diis"), on the frequency-dependent commutator residual
        H G S - S G H of thc_dyson_commutator ("cdiis", Sec. III.A), or damping only
        ("damp").  The returned residual norm is that of Sigma_out - Sigma_in in every mode."""
        torch = self.torch
        with torch.cuda.stream(self.stream):
            r = torch.empty_like(self.G)
        self._lincomb([1.0, -1.0], [self.Sig_out, self.Sig_in], r)
        res = float(np.sqrt(self._dot(r, r)))
        if self.mixing == "cdiis":
            with torch.cuda.stream(self.stream):
                e = torch.empty((len(self.grid.iw), self.n, self.n, 2), dtype=torch.float64, device=self.dev)
            thc.thc_dyson_commutator(self.dy, self.Sig_out, e)
            r = e
        out = self.Sig_out.clone()
        self.history.append((out, r))
        self.history = self.history[-self.diis_size:]
        if it <= self.n_damp or self.mixing == "damp":
            a = self.damping
            self._lincomb([a, 1.0 - a], [self.Sig_out, self.Sig_in], self.Sig_in)
            return res
        k = len(self.history)
        B = np.empty((k + 1, k + 1))
        for i in range(k):
            for j in range(i, k):
                B[i, j] = B[j, i] = self._dot(self.history[i][1], self.history[j][1])
        B[k, :k] = B[:k, k] = -1.0
        B[k, k] = 0.0
        rhs = np.zeros(k + 1)
        rhs[k] = -1.0
        c = np.linalg.lstsq(B, rhs, rcond=None)[0][:k]
        self._lincomb(list(c), [h[0] for h in self.history], self.Sig_in)
        return res

    # --------------------------------------------------------------- run
    def run(self, tol=1e-8, max_iter=60, proposer=None, log=None, metrics=None, checkpoint=None):
        """Iterates until |E_k - E_{k-1}| < tol.  proposer(loop, it, residual) may replace
        Sig_in before the Dyson step and returns a label (learned proposals); it is judged
        by the exact Sigma of the next iteration like any other input.

        metrics: a path (appended to) or a writable text file for one JSON line per
        iteration.  checkpoint: a path; after every iteration that does not end the run
        the loop state (and the proposer's, when given) is written there, replacing the
        previous one.  After resume() the run continues with the next iteration."""
        out, own = None, False
        if metrics is not None:
            out, own = (open(metrics, "a"), True) if isinstance(metrics, (str, os.PathLike)) else (metrics, False)
        try:
            if self.iteration == 0:
                self.dyson(None)
                self.E_prev = None
            converged = False
            for it in range(self.iteration + 1, max_iter + 1):
                t0 = time.perf_counter()
                self.sigma()
                t_sig = time.perf_counter() - t0
                E, E_dyn, n = self.energy()
                done = self.E_prev is not None and abs(E - self.E_prev) < tol
                res = 0.0 if done else self.mix(it)
                label = ""
                if not done and proposer is not None:
                    label = proposer(self, it, res) or ""
                evals = 0 if done else self.dyson(self.Sig_in)
                rec = IterationRecord(it, E, E_dyn, self.mu, n, res, time.perf_counter() - t0, t_sig, evals, label)
                self.records.append(rec)
                if log:
                    log(rec)
                if out is not None:
                    self._write_metrics(out, rec)
                if done:
                    converged = True
                    break
                self.E_prev = E
                self.iteration = it
                if checkpoint is not None:
                    self.save(checkpoint, proposer)
            return converged
        finally:
            if own:
                out.close()

    # ---------------------------------------------------- metrics, checkpoints
    def _kernel_times(self):
        """Per-kernel-class GPU milliseconds since the last call (library profiler on), else {}."""
        now, k = {}, 0
        while True:
            r = thc.thc_profile_get(self.ctx, k)
            if r is None:
                break
            name, launches, ms, _ = r
            if launches:
                now[name] = ms
            k += 1
        delta = {name: ms - self._kernel_ms.get(name, 0.0) for name, ms in now.items()}
        self._kernel_ms = now
        return {name: round(ms, 4) for name, ms in delta.items() if ms > 0}

    def _write_metrics(self, out, rec):
        d = dataclasses.asdict(rec)
        d["dE"] = None if len(self.records) < 2 else rec.E - self.records[-2].E
        d["kernel_ms"] = self._kernel_times()
        out.write(json.dumps(d) + "\n")
        out.flush()

    def save(self, path, proposer=None):
        """Writes the loop state after a completed iteration to `path` (.npz): Sigma_in, G,
        mu, the iteration count, the last energy, the DIIS history, the records and, when
        given, the proposer's state.  U_Pqs and the Dyson workspace are rebuilt on resume."""
        h = [(o.cpu().numpy(), r.cpu().numpy()) for o, r in self.history]
        state = dict(
            version=np.array(1), n=np.array(self.n), N=np.array(self.N), n_tau=np.array(self.n_tau),
            tau=np.asarray(self.grid.tau), mixing=np.array(self.mixing), iteration=np.array(self.iteration),
            mu=np.array(self.mu), E_prev=np.array(np.nan if self.E_prev is None else self.E_prev),
            Sig_in=self.Sig_in.cpu().numpy(), G=self.G.cpu().numpy(), n_hist=np.array(len(h)),
            records=np.array(json.dumps([dataclasses.asdict(r) for r in self.records])))
        for i, (o, r) in enumerate(h):
            state[f"hist_out_{i}"] = o
            state[f"hist_res_{i}"] = r
        if proposer is not None:
            state.update(proposer.state())
        tmp = str(path) + ".tmp.npz"
        np.savez(tmp, **state)
        os.replace(tmp, path)

    def resume(self, path, proposer=None):
        """Restores a state written by save() into this loop (same sizes, tau grid and mixing)."""
        torch = self.torch
        z = np.load(path, allow_pickle=False)
        if (int(z["n"]), int(z["N"]), int(z["n_tau"])) != (self.n, self.N, self.n_tau) or \
                not np.array_equal(z["tau"], np.asarray(self.grid.tau)) or str(z["mixing"]) != self.mixing:
            raise ValueError("checkpoint does not match this loop (sizes, tau grid or mixing)")
        with torch.cuda.stream(self.stream):
            self.Sig_in.copy_(torch.from_numpy(z["Sig_in"]))
            self.G.copy_(torch.from_numpy(z["G"]))
            self.history = [(torch.from_numpy(z[f"hist_out_{i}"]).to(self.dev),
                             torch.from_numpy(z[f"hist_res_{i}"]).to(self.dev)) for i in range(int(z["n_hist"]))]
        self.stream.synchronize()
        self.mu = float(z["mu"])
        self.iteration = int(z["iteration"])
        e = float(z["E_prev"])
        self.E_prev = None if np.isnan(e) else e
        self.records = [IterationRecord(**r) for r in json.loads(str(z["records"]))]
        if proposer is not None:
            proposer.load_state(z)


class LearnedProposer:
    """Learned Sigma proposals for GF2Loop.run (include/thc_learned.h).

    Two ways of use:

    * online (default): every iteration the exact Sigma_out is observed; from
      the third iterate on, while the residual is above `active_above`, the
      network is retrained on the trajectory and its proposal replaces the DIIS
      input;
    * transfer: `record=True` only observes a first run; `fit()` trains the
      network on that trajectory (pairs from every iterate to the converged
      one); `start_transfer()` forgets the trajectory and makes the network,
      unchanged, propose from the second iterate of the next run (same sizes,
      a related system).

    A proposal replaces the input of one iteration; at most `max_proposals`
    are made per run (default one: a jump-start in place of a damping step,
    after which DIIS, which extrapolates better once it has a few pairs, is left
    alone).  A proposal is judged by the next iteration's exact residual: if that
    is not below the residual the proposal was made at, it counts as rejected;
    either way the loop continues from DIIS, which keeps the evaluated pair in
    its history.
    """

    def __init__(self, loop, hidden=512, max_hist=8, steps=150, batch=8192, lr=2e-3, seed=17744,
                 active_above=1e-5, cooldown=2, record=False, max_proposals=1):
        g = loop.grid
        L = g.basis.L
        rng = np.random.default_rng(seed)
        # He initialisation; the last layer starts small, so early proposals stay near the latest iterate
        self.W1 = (rng.standard_normal((hidden, 2 * L)) * np.sqrt(2.0 / (2 * L))).astype(np.float32)
        self.b1 = np.zeros(hidden, np.float32)
        self.W2 = (rng.standard_normal((L, hidden)) * np.sqrt(1.0 / hidden) * 0.1).astype(np.float32)
        self.b2 = np.zeros(L, np.float32)
        self.p = thc.thc_proposer_init(loop.n, loop.n_tau, L, g.U_tau, g.fit_tau, hidden, max_hist, self.W1, self.b1,
                                       self.W2, self.b2, loop.stream.cuda_stream)
        self.steps, self.batch, self.lr = steps, batch, lr
        self.active_above, self.cooldown = active_above, cooldown
        self.record = record           # observe only
        self.transfer = False          # propose with the fitted network, no retraining
        self.pending = None            # residual at which the last proposal was made
        self.pause = 0
        self.max_proposals = max_proposals
        self.proposed = 0
        self.accepted = self.rejected = 0
        self.losses = []

    def close(self):
        if self.p is not None:
            thc.thc_proposer_destroy(self.p)
            self.p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def state(self) -> dict:
        """Host arrays of the proposer's state (network, Adam moments, observed window, counters)."""
        return {"prop_state": thc.thc_proposer_save_state(self.p),
                "prop_counters": np.array([self.proposed, self.accepted, self.rejected, self.pause,
                                           -1.0 if self.pending is None else self.pending,
                                           float(self.record), float(self.transfer)])}

    def load_state(self, z):
        thc.thc_proposer_load_state(self.p, z["prop_state"])
        c = z["prop_counters"]
        self.proposed, self.accepted, self.rejected, self.pause = int(c[0]), int(c[1]), int(c[2]), int(c[3])
        self.pending = None if c[4] < 0 else float(c[4])
        self.record, self.transfer = bool(c[5]), bool(c[6])

    def fit(self, steps=None, lr=None):
        """Train on the recorded trajectory: inputs from each iterate, targets towards the last."""
        self.losses.append(thc.thc_proposer_train(self.p, steps or self.steps, self.batch, lr or self.lr))
        return self.losses[-1]

    def start_transfer(self):
        thc.thc_proposer_reset(self.p)
        self.record, self.transfer = False, True
        self.pending, self.pause, self.proposed = None, 0, 0

    def __call__(self, loop, it, residual):
        thc.thc_proposer_observe(self.p, loop.Sig_out)
        if self.record:
            return "recorded"
        label = ""
        if self.pending is not None:
            if residual < self.pending:
                self.accepted += 1
                label = "accepted; "
            else:
                self.rejected += 1
                self.pause = self.cooldown
                label = "rejected; "
            self.pending = None
        if self.pause > 0:
            self.pause -= 1
            return label + "paused"
        count = thc.thc_proposer_count(self.p)
        if residual < self.active_above or count < (2 if self.transfer else 3) or self.proposed >= self.max_proposals:
            return label.rstrip("; ")
        if not self.transfer:
            self.losses.append(thc.thc_proposer_train(self.p, self.steps, self.batch, self.lr))
        thc.thc_proposer_propose(self.p, loop.Sig_in)
        self.pending = residual
        self.proposed += 1
        return label + "proposed"
