"""Row sharding across processes (one GPU each).

After dimensional splitting every row of a RAM step is an independent periodic
problem (Sec. 3.5: the azimuthal sweep of each ring needs nothing from the other
rings), so a batch of rows shards across ranks with no data exchange: each rank
takes a contiguous range of rows, balanced by cell count, builds its own plan
and steps its rows.  The only cross-rank operations are host-side scalar
reductions: the global mass (Eq. 10: conserved per row, so the sum over ranks is
conserved) and the step time (the max over ranks).
"""
from __future__ import annotations

import dataclasses
from typing import List, Tuple

import numpy as np

from .workloads import Workload


def partition_rows(row_offset: np.ndarray, world: int) -> List[Tuple[int, int]]:
    """Contiguous row ranges [r0, r1), one per rank, splitting the cells as evenly
    as whole rows allow: rank k's range starts at the first row whose start is at
    or past k/world of the cells.  Every row belongs to exactly one range; a rank
    may get an empty range when there are fewer rows than ranks."""
    row_offset = np.asarray(row_offset, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    n_rows = row_offset.size - 1
    total = int(row_offset[-1])
    bounds = [0]
    for k in range(1, world):
        target = (total * k + world - 1) // world
        r = int(np.searchsorted(row_offset[:-1], target, side="left"))
        bounds.append(min(max(r, bounds[-1]), n_rows))
    bounds.append(n_rows)
    return [(bounds[k], bounds[k + 1]) for k in range(world)]


def shard_workload(w: Workload, rank: int, world: int) -> Workload:
    """The rows of `w` that rank `rank` of `world` owns, as a workload of its own
    (offsets rebased to zero; per-row meshes, shifts, orders and sub-step counts
    carried along)."""
    r0, r1 = partition_rows(w.row_offset, world)[rank]
    c0, c1 = int(w.row_offset[r0]), int(w.row_offset[r1])
    ro = w.row_offset[r0:r1 + 1] - c0
    if w.shared_mesh:
        nodes = w.nodes
    else:
        nodes = w.nodes[c0 + r0: c1 + r1]
    return dataclasses.replace(
        w, name="%s[rank %d/%d]" % (w.name, rank, world), row_offset=ro.astype(np.int64),
        nodes=nodes, order=w.order[r0:r1], q0=w.q0[c0:c1], v0=w.v0[r0:r1],
        dv=None if w.dv is None else w.dv[c0:c1], nsub=w.nsub[r0:r1])


def _reduce(value: float, op_name: str, group=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    # NCCL reduces device tensors, gloo host tensors
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name), group=group)
    return float(t.item())


def global_sum(value: float, group=None) -> float:
    """Sum of a host scalar over the ranks (FP64): the global mass."""
    return _reduce(value, "SUM", group)


def global_max(value: float, group=None) -> float:
    """Max of a host scalar over the ranks: the step time of a weak-scaled run."""
    return _reduce(value, "MAX", group)
