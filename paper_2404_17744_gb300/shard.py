"""Partition of the tau points over independent workers (host logic only).

Sigma(tau_k) depends on G at tau_k and beta - tau_k only, so the tau points of
one evaluation split into independent shards; the paper instead distributes the
THC index P over MPI ranks (Sec. II.C).  This library runs the whole grid on one
GPU; the helpers below state how a replica-per-GPU deployment would shard and
merge, and are exercised on CPU ranks only.
"""
from __future__ import annotations


def tau_shard(n_tau: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [start, stop) range of tau points owned by `rank` of `world`:
    sizes differ by at most one, earlier ranks take the extra point."""
    if world < 1 or not 0 <= rank < world or n_tau < 0:
        raise ValueError("need world >= 1, 0 <= rank < world and n_tau >= 0")
    base, extra = divmod(n_tau, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def mirror_partners(start: int, stop: int, n_tau: int) -> list[int]:
    """Tau indices whose G a shard reads for G(beta - tau_k) on a mirror-symmetric grid."""
    return [n_tau - 1 - k for k in range(start, stop)]
