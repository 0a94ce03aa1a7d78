"""The benchmark's multi-rank path (one replica per rank, slowest rank's time,
whole-job throughput) with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank 1 is slower: the job time is its time
    value, ms = bench.aggregate(100.0 * (rank + 1), cells_per_rank=1000, steps=5, world=world)
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_uses_slowest_rank():
    world, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        value, ms = out[r]
        assert ms == pytest.approx(200.0)
        assert value == pytest.approx(2 * 1000 * 5 / 0.2)


def test_single_rank_aggregation():
    import bench
    value, ms = bench.aggregate(50.0, cells_per_rank=10, steps=2, world=1)
    assert ms == 50.0 and value == pytest.approx(400.0)


def test_clip_traffic_is_scaled_from_the_capture_of_the_same_clipper(monkeypatch):
    """roofline.traffic is the DRAM bytes per cell of the 64^3 k_clip capture
    times the cells of the launch, and null once the clipper's sources differ
    from those the capture was taken on, or for the direct FP64 clipper."""
    import bench
    digest = bench.clip_sources_digest()
    monkeypatch.setitem(bench.CLIP_TRAFFIC, "bytes_per_cell", 900.0)
    monkeypatch.setitem(bench.CLIP_TRAFFIC, "sha256_16", digest)
    assert bench.clip_traffic(256 ** 3, 1) == int(900.0 * 256 ** 3)
    assert bench.clip_traffic(64 ** 3, 1) == int(900.0 * 64 ** 3)
    assert bench.clip_traffic(256 ** 3, 0) is None
    monkeypatch.setitem(bench.CLIP_TRAFFIC, "sha256_16", "0" * 16)
    assert bench.clip_traffic(256 ** 3, 1) is None


def test_committed_clip_traffic_matches_the_current_clipper_or_is_absent():
    import bench
    if bench.CLIP_TRAFFIC["bytes_per_cell"] is not None:
        # a stale figure is withheld at run time; this flags it in review
        assert bench.CLIP_TRAFFIC["sha256_16"] == bench.clip_sources_digest()
        assert 64 <= bench.CLIP_TRAFFIC["bytes_per_cell"] <= 4000


def test_window_counts_average_every_step_of_the_window():
    """The method's work of the clipper is counted on every step of the timed
    window (the window replayed from its start state): counters averaged over
    the steps, maxima kept as maxima, the direct clipper used for the counts
    and the caller's clipper restored for the steps."""
    import bench

    class FakeCtx:
        def __init__(self):
            self.cfg = {}
            self.k = 0
            self.steps = 0
            self.tess_filters = []

        def set_config(self, **kw):
            self.cfg.update(kw)

        def mm_tessellate(self, pos, box):
            self.tess_filters.append(self.cfg.get("clip_filter"))

        def mm_tess_stats(self):
            self.k += 1
            return {"cuts": 10 * self.k, "fp64_plane_tests": 100.0 * self.k, "max_vertices": 30 + self.k}

        def mm_step(self, pos, U, box):
            assert self.cfg.get("collect_stats") == 0 and self.cfg.get("clip_filter") == 1
            self.steps += 1

    ctx = FakeCtx()
    out = bench.window_direct_counts(ctx, None, None, None, 4, 1)
    assert ctx.steps == 4 and ctx.tess_filters == [0, 0, 0, 0]
    assert out["cuts"] == pytest.approx((10 + 20 + 30 + 40) / 4)
    assert out["fp64_plane_tests"] == pytest.approx(250.0)
    assert out["max_vertices"] == 34
