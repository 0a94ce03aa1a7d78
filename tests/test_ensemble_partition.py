"""Multi-GPU split of the batched ensemble (whole boxes per rank, results
gathered once at the end), checked on the CPU: the partition itself, and two
gloo ranks stepping their own boxes with the oracle as a host stand-in for
the library's batched step, against one process stepping every box."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1707_05333_gb300 import ensemble as E
from paper_1707_05333_gb300 import workloads as WL


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_partition_covers_every_box_once_and_balances_cost(world):
    sizes = WL.ensemble_sizes(512)
    parts = E.partition_boxes(sizes, world)
    assert len(parts) == world
    E.check_partition(parts, len(sizes))
    loads = E.rank_loads(sizes, parts)
    assert loads.max() <= E.graham_bound(sizes, world)
    # on this ensemble (512 boxes of 2^10..2^16 cells) greedy longest-first
    # scheduling balances the estimated cost to within 1 % of the mean
    assert loads.max() <= 1.01 * loads.mean(), loads / loads.mean()
    # deterministic: every rank computes the same partition
    again = E.partition_boxes(sizes, world)
    assert all(np.array_equal(a, b) for a, b in zip(parts, again))


def test_partition_edge_cases():
    # fewer boxes than ranks: some ranks get none, none twice
    parts = E.partition_boxes([100, 5000], 4)
    E.check_partition(parts, 2)
    assert sum(len(p) for p in parts) == 2
    # one box far costlier than the rest gets a rank of its own
    parts = E.partition_boxes([2 ** 20] + [1000] * 12, 2)
    big = [p for p in parts if 0 in p][0]
    assert list(big) == [0]
    with pytest.raises(ValueError):
        E.check_partition([np.array([0, 1]), np.array([1])], 3)
    with pytest.raises(ValueError):
        E.partition_boxes([10], 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


SIZES = [40, 90, 27, 64, 120, 33, 75]


def _oracle_box_results(boxes):
    """The host stand-in for a batched step: the oracle's step on each box,
    returning per box (dt, five conserved totals after the step)."""
    from oracle import oracle as O
    rows = []
    for b in boxes:
        w = WL.ensemble_box(int(b), SIZES[int(b)])
        T = O.tessellate(w.pos, w.box, 0)
        U = O.charges_from_prims(T["volume"], w.rho, w.vel, w.pres, w.gamma)
        cfg = O.make_cfg(gamma=w.gamma, cfl=w.cfl, limiter=1)
        S = O.step(w.pos, U, w.box, cfg, tess=T)
        rows.append(np.concatenate([[S["dt"]], S["U"].sum(axis=0)]))
    return np.array(rows).reshape(len(boxes), 6)


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    parts = E.partition_boxes(SIZES, world)
    mine = parts[rank]
    rows = _oracle_box_results(mine)
    table = E.gather_box_results(len(SIZES), mine, rows)
    out[rank] = (list(mine), table.tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_the_single_process_results(oracle):
    world, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    whole = _oracle_box_results(range(len(SIZES)))
    mine0, t0 = out[0]
    mine1, t1 = out[1]
    # the two ranks stepped disjoint subsets that cover every box
    assert sorted(mine0 + mine1) == list(range(len(SIZES))) and mine0 and mine1
    # every rank holds the full table, equal to the single-process run bit for bit
    np.testing.assert_array_equal(np.array(t0), whole)
    np.testing.assert_array_equal(np.array(t1), whole)


def test_single_process_gather_is_the_local_table():
    rows = np.arange(12, dtype=float).reshape(2, 6)
    table = E.gather_box_results(4, [3, 1], rows)
    np.testing.assert_array_equal(table[3], rows[0])
    np.testing.assert_array_equal(table[1], rows[1])
    assert not table[0].any() and not table[2].any()
