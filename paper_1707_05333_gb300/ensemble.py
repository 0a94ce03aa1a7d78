"""Multi-GPU split of an ensemble of independent periodic boxes.

The boxes of a batch share nothing: each has its own generators, bins, faces
and timestep, so the natural way to spread a batch over several GPUs is to
give every GPU (one process, one rank) a subset of whole boxes and run
``mm_step_batched`` on that subset, with no exchange on the data path.  Only
the per-box results a caller reads afterwards (each box's timestep and
conserved totals) are gathered, once, at the end.  This is the GPU analogue of
the paper's over-decomposition of the domain into pieces that are processed
independently (Sec. 1, Sec. 3: each cell is constructed locally).

The cost of stepping a box grows like N_b log N_b in its cell count N_b (the
neighbour search and sort terms on top of the per-cell work), so boxes are
assigned by greedy longest-processing-time list scheduling on that cost: the
costliest box first, each to the rank with the smallest load so far.  Graham's
bound for list scheduling holds for any order: the largest load is at most the
mean load plus the largest single box cost.

Host logic only: the stepping itself is the library's.
"""
from __future__ import annotations

import math

import numpy as np


def box_cost(n_cells: int) -> float:
    """Relative cost of one step of a box of n_cells cells."""
    n = float(n_cells)
    return n * max(1.0, math.log2(n))


def partition_boxes(sizes, world: int) -> list[np.ndarray]:
    """Box indices of each rank (ascending), every box on exactly one rank.

    Greedy longest-processing-time assignment on box_cost; ties are broken by
    box index and rank index, so every rank computes the same partition."""
    if world < 1:
        raise ValueError("world must be >= 1")
    sizes = np.asarray(sizes, dtype=np.int64)
    cost = np.array([box_cost(int(n)) for n in sizes])
    order = sorted(range(len(sizes)), key=lambda b: (-cost[b], b))
    load = [0.0] * world
    owned: list[list[int]] = [[] for _ in range(world)]
    for b in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owned[r].append(b)
        load[r] += cost[b]
    return [np.array(sorted(o), dtype=np.int64) for o in owned]


def rank_loads(sizes, parts) -> np.ndarray:
    sizes = np.asarray(sizes, dtype=np.int64)
    return np.array([sum(box_cost(int(sizes[b])) for b in p) for p in parts])


def graham_bound(sizes, world: int) -> float:
    """Upper bound on the largest rank load of any list schedule: the mean
    load plus the largest single box cost."""
    cost = np.array([box_cost(int(n)) for n in np.asarray(sizes, dtype=np.int64)])
    return cost.sum() / world + cost.max()


def offsets(sizes) -> np.ndarray:
    """box_off of a batch: box b holds cells [off[b], off[b+1])."""
    return np.concatenate([[0], np.cumsum(np.asarray(sizes, dtype=np.int64))]).astype(np.int64)


def gather_box_results(nboxes: int, mine, per_box, group=None):
    """Combine per-box result rows computed on each rank into the full table
    on every rank.

    mine: the global indices of this rank's boxes; per_box: a float64 array
    (len(mine), k) of their rows (for example the timestep and the five
    conserved totals).  Every box belongs to exactly one rank, so a sum over
    ranks of tables that are zero elsewhere is exact (x + 0 = x).  One
    all-reduce on the process group's device (CPU for gloo); a single
    process returns its own table."""
    import torch
    import torch.distributed as dist

    mine = np.asarray(mine, dtype=np.int64)
    per_box = np.asarray(per_box, dtype=np.float64)
    k = per_box.shape[1] if per_box.ndim == 2 else 1
    table = np.zeros((nboxes, k))
    table[mine] = per_box.reshape(len(mine), k)
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return table
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor(table, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


def check_partition(parts, nboxes: int) -> None:
    """Every box on exactly one rank."""
    allb = np.concatenate([np.asarray(p, dtype=np.int64) for p in parts]) if parts else np.zeros(0, np.int64)
    if len(allb) != nboxes or not np.array_equal(np.sort(allb), np.arange(nboxes)):
        raise ValueError("the partition does not cover every box exactly once")
