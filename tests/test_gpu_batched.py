"""mm_step_batched: independent periodic boxes in one captured CUDA graph must
give exactly what mm_step gives on each box alone."""
import numpy as np
import pytest

from paper_1707_05333_gb300 import workloads as WL
from tests import helpers as H

pytestmark = pytest.mark.gpu


def make_batch():
    boxes, parts = [], []
    specs = [(WL.random_points(700, box=(1.0, 1.0, 1.0), seed=21), (1.0, 1.0, 1.0)),
             (WL.random_points(1500, box=(2.0, 1.0, 1.0), seed=22), (2.0, 1.0, 1.0)),
             (WL.smooth_wave(8).pos, (1.0, 1.0, 1.0)),
             (WL.random_points(7, box=(0.5, 0.7, 1.3), seed=23), (0.5, 0.7, 1.3)),
             (WL.random_points(333, box=(0.5, 0.7, 1.3), seed=24), (0.5, 0.7, 1.3))]
    for k, (pos, box) in enumerate(specs):
        rho, vel, pres = WL.random_state(len(pos), seed=30 + k, v_sigma=0.2)
        parts.append((pos, rho, vel, pres))
        boxes.append(box)
    return parts, np.array(boxes)


def charges(oracle, pos, box, rho, vel, pres, gamma):
    T = oracle.tessellate(pos, box, 1)
    return oracle.charges_from_prims(T["volume"], rho, vel, pres, gamma)


@pytest.mark.parametrize("precision,integrator", [(0, 0), (1, 0), (0, 1)])
def test_batched_step_equals_per_box_steps(oracle, precision, integrator):
    import torch
    from paper_1707_05333_gb300 import binding
    parts, boxes = make_batch()
    gamma = 5.0 / 3.0
    Us = [charges(oracle, p, b, r, v, P, gamma) for (p, r, v, P), b in zip(parts, boxes)]
    off = np.concatenate([[0], np.cumsum([len(p[0]) for p in parts])]).astype(np.int64)
    pos_all = np.concatenate([p[0] for p in parts])
    U_all = np.concatenate(Us)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = binding.Context(stream=stream, limiter=2, regularize=1, precision=precision, integrator=integrator)
        pos = H.to_dev(torch, pos_all.T)
        U = H.to_dev(torch, U_all.T)
        dt = torch.empty(len(parts), dtype=torch.float64, device="cuda")
        outs = []
        for _ in range(2):  # first call captures, second replays the graph
            ctx.mm_step_batched(pos, U, off, boxes, dt_out=dt)
            ctx.mm_sync_status()
            outs.append((pos.cpu().numpy().copy(), U.cpu().numpy().copy(), dt.cpu().numpy().copy()))
        ref = binding.Context(stream=stream, limiter=2, regularize=1, precision=precision, integrator=integrator)
        for b, ((p, r, v, P), box) in enumerate(zip(parts, boxes)):
            pb = H.to_dev(torch, p.T)
            Ub = H.to_dev(torch, Us[b].T)
            d1 = torch.empty(1, dtype=torch.float64, device="cuda")
            for step in range(2):
                ref.mm_step(pb, Ub, box, dt_out=d1)
                got_pos, got_U, got_dt = outs[step]
                sl = slice(off[b], off[b + 1])
                np.testing.assert_array_equal(got_U[:, sl], Ub.cpu().numpy(), err_msg=f"box {b} step {step}")
                np.testing.assert_array_equal(got_pos[:, sl], pb.cpu().numpy(), err_msg=f"box {b} step {step}")
                assert got_dt[b] == float(d1.item())
        ctx.close()
        ref.close()


def test_batched_mesh_is_the_union_of_the_boxes(oracle):
    import torch
    from paper_1707_05333_gb300 import binding
    parts, boxes = make_batch()
    off = np.concatenate([[0], np.cumsum([len(p[0]) for p in parts])]).astype(np.int64)
    pos_all = np.concatenate([p[0] for p in parts])
    gamma = 5.0 / 3.0
    U_all = np.concatenate([charges(oracle, p, b, r, v, P, gamma) for (p, r, v, P), b in zip(parts, boxes)])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = binding.Context(stream=stream)
        pos = H.to_dev(torch, pos_all.T)
        U = H.to_dev(torch, U_all.T)
        ctx.mm_step_batched(pos, U, off, boxes)
        ctx.mm_sync_status()
        G = {k: v.cpu().numpy() for k, v in ctx.mm_current_mesh().to_torch().items()}
        ctx.close()
    # every box tiles its own volume, and no face crosses boxes
    for b in range(len(parts)):
        sl = slice(off[b], off[b + 1])
        assert abs(G["cell_volume"][sl].sum() - np.prod(boxes[b])) <= 1e-11 * np.prod(boxes[b])
    bi = np.searchsorted(off, G["face_i"], side="right") - 1
    bj = np.searchsorted(off, G["face_j"], side="right") - 1
    assert np.array_equal(bi, bj)
    H.check_incidence(G)


def test_ensemble_split_across_ranks_equals_one_batch():
    """The multi-GPU split of an ensemble (whole boxes per rank, chosen by
    cost; paper_1707_05333_gb300/ensemble.py), run here as one batch per
    "rank" on the same GPU one after the other: every box's charges,
    positions and timestep equal those of one batch over all boxes, bit for
    bit, and the gathered per-box table matches."""
    import torch
    from paper_1707_05333_gb300 import binding
    from paper_1707_05333_gb300 import ensemble as E
    sizes = [300, 1200, 450, 2048, 64, 777, 1500]
    boxes = [WL.ensemble_box(b, n) for b, n in enumerate(sizes)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = binding.Context(stream=stream, gamma=5.0 / 3.0, cfl=0.3, limiter=1, precision=1)
        Us = []
        for wb in boxes:
            pb = torch.tensor(wb.pos.T.copy(), dtype=torch.float64, device="cuda")
            mb = ctx.mm_tessellate(pb, wb.box)
            Us.append(ctx.mm_prims_to_charges(mb, torch.tensor(wb.rho, device="cuda"),
                                              torch.tensor(wb.vel.T.copy(), device="cuda"),
                                              torch.tensor(wb.pres, device="cuda")))

        def batch(ids):
            c = binding.Context(stream=stream, gamma=5.0 / 3.0, cfl=0.3, limiter=1, precision=1)
            pos = torch.tensor(np.concatenate([boxes[b].pos for b in ids]).T.copy(), dtype=torch.float64,
                               device="cuda")
            U = torch.cat([Us[b] for b in ids], dim=1).contiguous()
            off = E.offsets([sizes[b] for b in ids])
            dt = torch.empty(len(ids), dtype=torch.float64, device="cuda")
            for _ in range(2):
                c.mm_step_batched(pos, U, off, np.ones((len(ids), 3)), dt_out=dt)
            c.mm_sync_status()
            out = {}
            for k, b in enumerate(ids):
                lo, hi = off[k], off[k + 1]
                out[b] = (pos[:, lo:hi].clone(), U[:, lo:hi].clone(), float(dt[k].item()))
            c.close()
            return out

        whole = batch(list(range(len(sizes))))
        parts = E.partition_boxes(sizes, 3)
        E.check_partition(parts, len(sizes))
        split = {}
        for p in parts:
            split.update(batch([int(b) for b in p]))
        ctx.close()
    for b in range(len(sizes)):
        assert torch.equal(whole[b][0], split[b][0]) and torch.equal(whole[b][1], split[b][1]), b
        assert whole[b][2] == split[b][2], b
    # the gathered table (one process here) is the per-box rows in box order
    rows = np.array([[split[b][2]] + split[b][1].sum(dim=1).cpu().tolist() for b in range(len(sizes))])
    table = E.gather_box_results(len(sizes), np.arange(len(sizes)), rows)
    np.testing.assert_array_equal(table, rows)
