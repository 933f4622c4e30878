"""Host-side helpers for running the featurizer on several GPUs of a node.

Centers (and whole structures) are independent given all positions, so a
batch shards across ranks with no collective on the data path: each rank
featurizes its own structures (or its own replica of a workload); the only
collectives are the timing reduction (max over ranks) and, for reporting,
the sum of the work done.  A single structure shards by centers: features
need no exchange, and the VJP one sum of the [N, 3] partial gradients.
"""
from __future__ import annotations

import numpy as np


def shard_structures(atom_off, rank: int, world: int):
    """Contiguous structure range [s0, s1) of `rank` with roughly equal atom
    counts (greedy split of the cumulative atom counts)."""
    off = np.asarray(atom_off, np.int64)
    S = off.size - 1
    if world <= 1:
        return 0, S
    total = off[-1]
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        s = int(np.searchsorted(off, target, side="left"))
        s = min(max(s, bounds[-1]), S)
        bounds.append(s)
    bounds.append(S)
    return bounds[rank], bounds[rank + 1]


def slice_workload(w, s0: int, s1: int):
    """The sub-batch of structures [s0, s1) of a synth.Workload."""
    a0, a1 = int(w.atom_off[s0]), int(w.atom_off[s1])
    return w.replace(positions=w.positions[a0:a1], species=w.species[a0:a1],
                     atom_off=(w.atom_off[s0:s1 + 1] - a0).astype(np.int64),
                     cells=w.cells[s0:s1], pbc=w.pbc[s0:s1])


def shard_centers(n: int, rank: int, world: int):
    """Contiguous center range [c0, c1) of `rank` (as equal as possible)."""
    c0 = (n * rank) // world
    c1 = (n * (rank + 1)) // world
    return c0, c1


def allreduce_sum_(t):
    """In-place sum of a tensor over ranks (the one exchange a center-sharded
    VJP of a single structure needs: every rank holds partial gradients of
    all atoms from its own centers); identity without a process group."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def reduce_timing(ms: float, units: float, device=None):
    """(max ms over ranks, sum of units over ranks); identity without an
    initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(ms), float(units)
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
