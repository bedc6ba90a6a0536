"""Sharding of independent systems across ranks (one GPU per rank).

The batched workload -- many crystals of uneven size, each its own BSE problem -- partitions
with no exchange between ranks: every rank assembles its own subset (through
bse_batch_assemble on its GPU) and nothing crosses ranks on the data path.  Every rank computes
the same assignment from the systems' sizes, so no collective is needed to agree on it.

The assignment is Graham's longest-processing-time-first rule (1969): systems in decreasing
estimated work, each to the rank with the least work so far (lowest rank on ties); its
largest rank load is within 4/3 of the best possible.  The work estimate is that of the batch
graph's ordering: the direct term's M_vv W(q) GEMM and second contraction over all pairs plus
the exchange over the full square.
"""
from __future__ import annotations

__all__ = ["assembly_work", "assign_systems"]


def assembly_work(nk: int, naux: int, nv: int, nc: int) -> float:
    """Relative assembly work of one system (flops up to a common factor)."""
    dim = float(nk) * nv * nc
    return float(nk) * nk * nv * nv * (float(naux) ** 2 + nc * nc * naux) + dim * dim * naux


def assign_systems(works, world: int):
    """Per-rank lists of system indices (LPT); each list in increasing work, the order in which
    the rank's batch graph runs them."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(works)), key=lambda i: (-works[i], i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += works[i]
    return [sorted(lst, key=lambda i: (works[i], i)) for lst in out]
