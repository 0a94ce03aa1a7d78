#!/usr/bin/env python
"""Throughput of the moving-mesh hot path on GB300: cell-updates per second.

One step = one pass of the whole path on the resident state (pos, U):
bin generators, clip every Voronoi cell, compact faces, mesh velocity and CFL
timestep, limited gradient + half step, limited half-step gradient, face-frame
HLLC fluxes, conservative update, drift (mm_step).

Default workload: the 3-D shear layer with 256^3 jittered-lattice generators
in the periodic unit box (inputs far larger than L2).  With N GPUs every rank
advances its own copy of the box (independent replicas, weak scaling); value
is the cells all ranks updated divided by the slowest rank's time.

--impl reference times the FP64 CPU oracle instead (a bounded sample of the
same workload recipe per step, on the host cores), printing the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per GB300 (tessellate+MUSCL flux), plain FP64 vs mixed/batched"
UNIT = "cell-updates/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    # the shear layer is specified as a 20-step run; steps 11-15 are its slow phase (bins and lattice
    # half a spacing apart), so the default times 20 steps after 5 warm-up steps
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n-side", type=int, default=256, help="shear layer generators per axis")
    p.add_argument("--precision", choices=["fp64", "mixed"], default=None,
                   help="default: fp64 for the shear layer, mixed for the ensemble")
    p.add_argument("--clip-filter", type=int, choices=[0, 1], default=1,
                   help="1: FP32-filtered clipping with exact FP64 fallback (same mesh bit for bit)")
    p.add_argument("--cpu-sample-side", type=int, default=24)
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-variants", action="store_true",
                   help="skip the variant measurements (mixed precision, direct FP64 clipping, entropy "
                        "switch, Heun integration, batched ensemble)")
    p.add_argument("--ensemble-boxes", type=int, default=512)
    p.add_argument("--workload", choices=["shear_layer", "ensemble"], default="shear_layer",
                   help="shear_layer: one 256^3 box per rank (replicas, weak scaling); ensemble: the batch of "
                        "independent boxes split across ranks by cost (strong scaling)")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the default clipper settings instead of tuning them first")
    return p.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# --------------------------------------------------------------------------- clocks
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def clocks_start(gpu_index):
    f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    try:
        proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={CLOCK_Q}",
                                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=f,
                                stderr=subprocess.DEVNULL)
    except (OSError, ValueError):
        proc = None
    return proc, f.name


def clocks_stop(proc, path):
    if proc is not None:
        proc.terminate()
        try:
            proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            proc.kill()
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower() == "active":
                    reasons.add(nm)
    finally:
        try:
            os.unlink(path)
        except OSError:
            pass
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- peaks
# GB300 FP64 ALU peak from unit counts and the maximum SM clock: 152 SMs x 2
# FP64 FMA lanes per SM per clock x 2 flops x 2.07 GHz (an FMA-chain probe on
# this pool measured 1.19 TFLOP/s at 1.995 GHz, consistent with 2 lanes/SM).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12

# Algorithmic flops per unit of clipping work: a plane test q.v > o
# (2 FMA + 1 MUL -> 5 flops), a three-plane solve (3 cross products, the
# determinant, the reciprocal and the scaled numerators -> 51 flops), and a
# face-fan term of the area/centroid sums in the face's own plane (two
# offsets, a 2-D cross product, three weighted sums -> 12 flops).
FLOPS_PLANE_TEST, FLOPS_SOLVE, FLOPS_FAN = 5, 51, 12
# FP32 lanes: 128 per SM per clock, so one FP32 flop costs 1/64 of an FP64
# flop of issue time on GB300.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# FP64 flops per unit of the hydro stages (the method's arithmetic, FMA = 2):
# a gradient pass ~60 per face, the face flux (reconstruction of both sides,
# floors, boosts, rotation, HLLC) ~400 per face, the update 10 per incidence.
FLOPS_GRADIENT_FACE, FLOPS_FLUX_FACE, FLOPS_UPDATE_INCIDENCE = 60, 400, 10


def clip_method_flops(direct):
    """The method's FP64 work in one tessellation (Sec. 3): every plane test
    and vertex solve of clipping with FP64 vertices (the counters of the
    direct clipper, clip_filter = 0), and the face fans of the final
    geometry.  Independent of how the kernel filters its tests."""
    return (FLOPS_PLANE_TEST * direct["fp64_plane_tests"] + FLOPS_SOLVE * direct["fp64_vertex_solves"] +
            FLOPS_FAN * direct["fp64_fan_terms"])


def window_direct_counts(ctx, pos, U, box, steps, clip_filter):
    """The direct FP64 clipper's counters (the method's tests, solves and
    fans, Sec. 3) averaged over the timed window: the window's steps are
    replayed from its start state (bitwise the same trajectory, outside the
    timed region) and every step's positions are tessellated once more with
    clip_filter = 0 and the counters on.  The work per cell changes along
    the shear layer's run (steps 11-15 test more candidates), so one count
    at the start would misstate the window's average."""
    tot = {}
    for _ in range(steps):
        ctx.set_config(collect_stats=1, clip_filter=0)
        ctx.mm_tessellate(pos, box)
        st = ctx.mm_tess_stats()
        ctx.set_config(collect_stats=0, clip_filter=clip_filter)
        for k, v in st.items():
            tot[k] = max(tot.get(k, 0), v) if k.startswith("max") else tot.get(k, 0) + v
        ctx.mm_step(pos, U, box)
    return {k: (v if k.startswith("max") else v / steps) for k, v in tot.items()}


def clip_roofline(direct, filtered, ms, n, clip_filter):
    """FP64 ALU roofline of the clipping kernel: the method's FP64 work
    (clip_method_flops) per launch over the launch's event time, against the
    FP64 peak.  The FP64-equivalent count of what the filtered kernel itself
    executes (FP32 tests and solves weighted by the FP64/FP32 peak ratio,
    plus its FP64 fallbacks, final solves and fans) is kept as an extra key."""
    f_method = clip_method_flops(direct)
    ach = f_method / (ms / 1e3) / 1e12
    out = {"kernel": "k_clip", "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
           "unit": "TFLOP/s (FP64)", "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
           "peak_source": "derived: 152 SMs x 2 FP64 FMA lanes/clk x 2 flops x 2.07 GHz",
           "fp64_flops_per_launch": f_method, "fp64_flops_per_cell": f_method / n, "launch_ms": ms}
    if clip_filter:
        f32 = FLOPS_PLANE_TEST * direct["fp64_plane_tests"] + FLOPS_SOLVE * direct["fp64_vertex_solves"]
        f64 = (FLOPS_PLANE_TEST * filtered["fp64_plane_tests"] + FLOPS_SOLVE * filtered["fp64_vertex_solves"] +
               FLOPS_FAN * filtered["fp64_fan_terms"])
        eq = f64 + f32 * FP64_PEAK_TFLOPS / FP32_PEAK_TFLOPS
        out["executed_fp64_equivalent"] = {
            "fp64_flops_per_launch": f64, "fp32_flops_per_launch": f32, "fp64_equiv_flops_per_cell": eq / n,
            "frac": eq / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
            "note": "FP32 flops weighted 1/64 (the FP64/FP32 lane ratio): the work the filtered kernel executes"}
    return out


# DRAM traffic of one k_clip launch, from an ncu capture of one launch on the
# 128^3 shear layer (dram__bytes_read.sum + dram__bytes_write.sum = 459,768,320
# + 1,439,416,576 bytes over 2,097,152 cells; filtered clipping, two warps per
# block), per cell; it scales with the cells of the launch.  Valid only for the
# clipper source it was taken on: the digest of the clipping kernel's sources
# must match, else the figure is withheld.
CLIP_TRAFFIC = {"sources": ("csrc/mm_clip.cu", "csrc/mm_internal.cuh"), "sha256_16": "ed02d4137c2d00bd",
                "bytes_per_cell": 1908677632 / 2097152, "cells_captured": 2097152}


def clip_sources_digest():
    import hashlib
    h = hashlib.sha256()
    for rel in CLIP_TRAFFIC["sources"]:
        with open(os.path.join(ROOT, "paper_1707_05333_gb300", rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def clip_traffic(n, clip_filter):
    """DRAM bytes of one k_clip launch on n cells, scaled from the 128^3
    capture by cell count; None when the capture does not cover the current
    clipper source or clipper variant."""
    if not clip_filter or CLIP_TRAFFIC["bytes_per_cell"] is None:
        return None
    if clip_sources_digest() != CLIP_TRAFFIC["sha256_16"]:
        return None
    return int(round(CLIP_TRAFFIC["bytes_per_cell"] * n))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# --------------------------------------------------------------------------- oracle timing
def oracle_rate(n_side, seconds, gamma_cfg=None):
    """Cells per second of the oracle's whole step (tessellation + hydro) on
    the shear-layer recipe at n_side^3 generators; one thread."""
    from oracle import oracle as O
    from paper_1707_05333_gb300 import workloads as WL
    O.build()
    w = WL.shear_layer(n_side)
    cfg = O.make_cfg(gamma=w.gamma, cfl=w.cfl, limiter=1)
    T = O.tessellate(w.pos, w.box, 1)
    U = O.charges_from_prims(T["volume"], w.rho, w.vel, w.pres, w.gamma)
    pos = w.pos
    cells, t0 = 0, time.perf_counter()
    steps = 0
    while True:
        S = O.step(pos, U, w.box, cfg, mode=1)
        pos, U = S["pos"], S["U"]
        cells += w.n
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return cells / el, steps, el, w.n


def _oracle_worker(job):
    n_side, seconds = job
    rate, steps, el, _ = oracle_rate(n_side, seconds)
    return rate, steps, el


def oracle_rate_all_cores(n_side, seconds, procs=None):
    """The oracle as it stands on every host core: `procs` independent
    replicas of the same sample run at once (one thread each, processes
    started with spawn, since this process may already hold a CUDA context);
    the rate is their sum."""
    import multiprocessing as mp
    from oracle import oracle as O
    O.build()
    procs = procs or os.cpu_count() or 1
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_oracle_worker, [(n_side, seconds)] * procs)
    return sum(r[0] for r in res), procs, sum(r[1] for r in res)


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state beyond the first build
    from oracle import oracle as O
    O.build()
    side = args.cpu_sample_side
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps))
    rates, procs = [], 1
    for _ in range(args.steps):
        rate, procs, _ = oracle_rate_all_cores(side, per_step)
        rates.append(rate)
    value = statistics.mean(rates)
    sample = (f"shear-layer recipe at {side}^3 generators, whole oracle step, {procs} concurrent replicas "
              f"(one thread each), {args.steps} x ~{per_step:.0f} s; the per-cell rate stands for the "
              f"{args.n_side}^3 box (same recipe, the oracle's work per cell does not depend on the box size)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * (side ** 3) / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"shear_layer_{args.n_side}^3", "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- our path
# Algorithmic HBM bytes per launch of each stage, from the data layout
# (struct of arrays): n cells, F unique faces, I = 2F incidences.  Every array
# is counted once per producer and once per consuming stage; gathers of a
# neighbour's cell data are counted once per cell and shared face records once
# per face.
def algorithmic_bytes(stage, n, F):
    I = 2 * F
    if stage == "gradient_half_step":
        # states W = U / V (read U, V; write W); face geometry (read i, j, image, A, n and the
        # centroids; write A n and d); predictor pass (read W, the CSR, the other cell and the
        # geometry of each face; write W_half and M^-1)
        states = n * (5 * 8 + 8) + n * 5 * 8
        geom = F * (12 + 8 + 24) + n * 24 + F * 48
        pred = n * 5 * 8 + n * 4 + I * 4 + F * (8 + 48) + n * 4 + n * (5 + 9) * 8
        return states + geom + pred
    if stage == "gradient":
        # read W_half, M^-1, the CSR, the other cell and the geometry; write the 15 gradient rows
        return n * (5 + 9) * 8 + n * 4 + I * 4 + F * (8 + 48) + n * 15 * 8
    if stage == "face_flux":
        return F * (12 + 8 + 24 + 24) + n * (5 + 15 + 3 + 3 + 3) * 8 + F * 5 * 8
    if stage == "update":
        return n * 4 + I * 4 + F * 5 * 8 + n * (8 + 2 * 5 * 8)
    if stage == "clip":
        # compulsory: sorted generators in, volume + centroid + face slots out
        return n * 32 + n * 32 + F * 2 * (4 + 1 + 8 + 24)
    if stage == "faces":
        # slots in (neighbour, image, area, centroid per directed face), unique faces and the
        # incident CSR out (i, j, image, A, normal, centroid; inc_off, inc_face), cells' moments
        return I * (4 + 1 + 8 + 24) + F * (12 + 8 + 24 + 24) + n * 4 + I * 4 + n * 2 * 32
    if stage == "bin":
        # positions in, binned FP64 and FP32 copies out, bin counts and offsets
        return n * 24 + n * (32 + 16) + n * 3 * 4
    if stage == "mesh_velocity":
        return n * (5 * 8 + 8 + 24) + n * 24
    if stage == "drift":
        return n * (24 + 24 + 4) + n * 24
    return None


def algorithmic_bytes_mixed(stage, n, F):
    """The same for the mixed-precision stages (FP32 face and cell records of
    16-byte vectors, FP64 charges)."""
    I = 2 * F
    if stage == "gradient_half_step":
        faces32 = F * (12 + 8 + 24 + 24) + n * 28 + F * 48       # face records out
        pack = n * (40 + 8 + 24 + 24 + 24) + n * 48               # W^n and c - r, w out
        pred = n * (32 + 4) + I * 4 + F * 40 + n * 32              # W^(n+1/2) out
        return faces32 + pack + pred
    if stage == "gradient":
        return n * (32 + 4) + I * 4 + F * 40 + n * 64
    if stage == "face_flux":
        return F * 48 + n * (32 + 64 + 16) + F * 32
    if stage == "update":
        return n * (4 + 4 + 8 + 2 * 40) + I * 4 + F * 32
    return algorithmic_bytes(stage, n, F)


def hydro_method_flops(n, F):
    """The method's FP64 work in the hydro stages of one step."""
    return F * (2 * FLOPS_GRADIENT_FACE + FLOPS_FLUX_FACE) + 2 * F * FLOPS_UPDATE_INCIDENCE


def stage_rooflines(stage_ms, n, F, mixed, hbm_peak, peak_kind):
    """HBM roofline of every stage from its algorithmic bytes and its live
    event time."""
    out = {}
    for k, ms in stage_ms.items():
        byts = (algorithmic_bytes_mixed if mixed else algorithmic_bytes)(k, n, F)
        if byts is None or not ms:
            continue
        ach = byts / (ms / 1e3) / 1e9
        out[k] = {"bound": "hbm", "algorithmic_bytes": int(byts), "bytes_per_cell": byts / n, "ms": ms,
                  "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                  "peak_source": peak_kind}
    return out


def step_roofline(step_ms, stage_ms, n, F, clip_flops, mixed, hbm_peak, peak_kind):
    """The whole step against both ceilings: the method's FP64 flops per cell
    (clipping + hydro; in the mixed path the hydro flops run in FP32 and are
    left out) over the FP64 peak, and the algorithmic bytes per cell summed
    over the stages over the measured HBM bandwidth."""
    f64 = clip_flops + (0 if mixed else hydro_method_flops(n, F))
    byts = sum((algorithmic_bytes_mixed if mixed else algorithmic_bytes)(k, n, F) or 0 for k in stage_ms)
    sec = step_ms / 1e3
    return {"fp64_flops_per_cell": f64 / n, "bytes_per_cell": byts / n,
            "fp64": {"achieved": f64 / sec / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": f64 / sec / 1e12 / FP64_PEAK_TFLOPS, "peak_source": "derived"},
            "hbm": {"achieved": byts / sec / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "frac": byts / sec / 1e9 / hbm_peak, "peak_source": peak_kind},
            "ms_per_step": step_ms}


def aggregate(ms, cells_per_rank, steps, world):
    """Whole-job throughput across ranks: every rank advanced its own replica,
    so value = world * cells * steps / (slowest rank's time).  Returns
    (value, slowest ms); the maximum is an all-reduce when world > 1."""
    if world > 1:
        import torch
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * cells_per_rank * steps / (ms / 1e3), ms


def time_steps(torch, stream, fn, steps):
    """Device time of `steps` calls of fn on `stream`, in ms (CUDA events)."""
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    stream.synchronize()
    return e0.elapsed_time(e1)


def tune_clipper(args, pos_np, box, reps=3):
    """mm_autotune on a sample of the workload (untimed): the clipper's warps
    per block, candidate batch and bin width, each setting timed over `reps`
    tessellations after a warm-up."""
    import torch
    from paper_1707_05333_gb300 import binding as BD
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = BD.Context(stream=stream)
        pos = torch.tensor(pos_np.T.copy(), dtype=torch.float64, device="cuda")
        res = ctx.mm_autotune(pos, box, reps=reps)
        ctx.close()
    return res


DEFAULT_CLIPPER = {"clip_warps": 2, "cand_cap": 64, "bin_scale": 1.0, "clip_sort": 0}


def confirm_clipper(w, tuned, reps=2, **cfg):
    """The tuned and the default clipper settings, each timed on `reps`
    tessellations of the full workload (after one warm-up, untimed by the
    bench): the faster is kept, since a setting tuned on a sample need not
    carry over."""
    import torch
    from paper_1707_05333_gb300 import binding as BD
    stream = torch.cuda.Stream()
    times = {}
    with torch.cuda.stream(stream):
        ctx = BD.Context(stream=stream, **cfg)
        pos = torch.tensor(w.pos.T.copy(), dtype=torch.float64, device="cuda")
        for name, st in (("tuned", tuned), ("default", DEFAULT_CLIPPER)):
            ctx.set_config(**st)
            ctx.mm_tessellate(pos, w.box)
            ms = time_steps(torch, stream, lambda: ctx.mm_tessellate(pos, w.box), reps)
            times[name] = ms / reps
        ctx.close()
    pick = "tuned" if times["tuned"] <= times["default"] else "default"
    return (tuned if pick == "tuned" else dict(DEFAULT_CLIPPER)), {"tessellate_ms_full_size": times, "kept": pick}


def measure_variant(args, w, steps, dtype, note, stages=False, **cfg):
    """One configuration of the step on the same workload and protocol
    (warm-up steps, then `steps` timed steps with CUDA events); with stages,
    also the per-stage event times of the timed steps."""
    import torch
    from paper_1707_05333_gb300 import binding as BD
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = BD.Context(stream=stream, gamma=w.gamma, cfl=w.cfl, limiter=1, **args.tuned, **cfg)
        pos = torch.tensor(w.pos.T.copy(), dtype=torch.float64, device="cuda")
        mesh = ctx.mm_tessellate(pos, w.box)
        U = ctx.mm_prims_to_charges(mesh, torch.tensor(w.rho, device="cuda"), torch.tensor(w.vel.T.copy(), device="cuda"),
                                    torch.tensor(w.pres, device="cuda"))
        for _ in range(args.warmup):
            ctx.mm_step(pos, U, w.box)
        if stages:
            ctx.mm_set_timing(True)
        ms = time_steps(torch, stream, lambda: ctx.mm_step(pos, U, w.box), steps)
        st = ctx.mm_stage_times() if stages else None
        nf = ctx.mm_tessellate(pos, w.box).nfaces if stages else None
        ctx.close()
    out = {"value": w.n * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
           "dtype": dtype, "note": note}
    if stages:
        out["stage_ms"] = {k: v[0] / max(1, v[1]) for k, v in st.items()}
        out["faces"] = nf
    return out


def measure_variants(args, w, clip_flops):
    half = max(2, args.steps // 2)
    peak, peak_kind = measured_peaks()
    mixed = measure_variant(args, w, args.steps, "f64+f32", "FP32 gradients/half step/fluxes, FP64 clipping "
                            "decisions, geometry and update", stages=True, precision=1)
    mixed["stage_roofline"] = stage_rooflines(mixed["stage_ms"], w.n, mixed["faces"], True, peak, peak_kind)
    mixed["roofline_step"] = step_roofline(mixed["ms_per_step"], mixed["stage_ms"], w.n, mixed["faces"],
                                           clip_flops + 2 * mixed["faces"] * FLOPS_UPDATE_INCIDENCE, True, peak,
                                           peak_kind)
    return {
        "mixed_same_workload": mixed,
        "direct_fp64_clip_same_workload": measure_variant(
            args, w, half, "f64", "clip_filter=0: every clipping vertex solved and tested in FP64 as it appears",
            clip_filter=0),
        "entropy_switch_same_workload": measure_variant(
            args, w, half, "f64", "sixth state column rho A and the energy/entropy switch at Mach 1.1",
            entropy=1, mach_th=1.1),
        "heun_same_workload": measure_variant(
            args, w, half, "f64", "Heun time integration: two flux stages, second tessellation per step",
            integrator=1),
        "batched_ensemble": measure_ensemble(args, precision=1),
        "batched_ensemble_fp64": measure_ensemble(args, precision=0, per_box=False),
    }


def measure_ensemble(args, precision=1, per_box=True):
    """Batched ensemble of independent periodic boxes (log-uniform sizes,
    lognormal GRF density): one CUDA-graph replay per step for all boxes,
    against one mm_step per box (per_box).  precision 1 mixed, 0 FP64."""
    import numpy as np
    import torch
    from paper_1707_05333_gb300 import binding as BD
    from paper_1707_05333_gb300 import workloads as WL
    sizes = WL.ensemble_sizes(args.ensemble_boxes)
    boxes = [WL.ensemble_box(b, int(nb)) for b, nb in enumerate(sizes)]
    # the clipper tuned on the largest box of the ensemble (once for both precisions)
    if not hasattr(args, "ensemble_tuned"):
        big = boxes[int(np.argmax(sizes))]
        args.ensemble_tuned = {} if args.no_autotune else tune_clipper(args, big.pos, big.box)
    tuned = args.ensemble_tuned
    tunables = {k: tuned[k] for k in ("clip_warps", "cand_cap", "bin_scale", "clip_sort")} if tuned else {}
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    L = np.ones((len(boxes), 3))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = BD.Context(stream=stream, gamma=5.0 / 3.0, cfl=0.3, limiter=1, precision=precision, **tunables)
        # charges from each box's own tessellation
        Us = []
        for wb in boxes:
            pb = torch.tensor(wb.pos.T.copy(), dtype=torch.float64, device="cuda")
            mb = ctx.mm_tessellate(pb, wb.box)
            Us.append(ctx.mm_prims_to_charges(mb, torch.tensor(wb.rho, device="cuda"),
                                              torch.tensor(wb.vel.T.copy(), device="cuda"),
                                              torch.tensor(wb.pres, device="cuda")))
        pos0 = torch.tensor(np.concatenate([wb.pos for wb in boxes]).T.copy(), dtype=torch.float64, device="cuda")
        U0 = torch.cat(Us, dim=1).contiguous()
        pos, U = pos0.clone(), U0.clone()
        for _ in range(max(2, args.warmup)):
            ctx.mm_step_batched(pos, U, off, L)
        ctx.mm_sync_status()
        l0 = ctx.mm_kernel_launches()
        ms_graph = time_steps(torch, stream, lambda: ctx.mm_step_batched(pos, U, off, L), args.steps)
        launches = (ctx.mm_kernel_launches() - l0) // max(1, args.steps)
        ctx.mm_sync_status()
        ms_box = None
        if per_box:
            # one launch sequence per box (each box its own arrays)
            pb = [pos0[:, off[b]:off[b + 1]].contiguous() for b in range(len(boxes))]
            ub = [U0[:, off[b]:off[b + 1]].contiguous() for b in range(len(boxes))]

            def per_box_step():
                for b in range(len(boxes)):
                    ctx.mm_step(pb[b], ub[b], L[b])
            per_box_step()
            ms_box = time_steps(torch, stream, per_box_step, 1)
        ctx.close()
    graph = n * args.steps / (ms_graph / 1e3)
    out = {"workload": f"ensemble of {len(boxes)} periodic unit boxes, {n} cells (2^10..2^16 per box)",
           "precision": "mixed" if precision else "fp64", "graph_cells_per_s": graph,
           "graph_ms_per_step": ms_graph / args.steps, "kernels_per_step": launches,
           "clipper_settings": tuned or "defaults"}
    if ms_box is not None:
        out.update(per_box_cells_per_s=n / (ms_box / 1e3), per_box_ms_per_step=ms_box,
                   speedup=graph / (n / (ms_box / 1e3)))
    return out


def run_ensemble(args, world, rank, local):
    """The batched ensemble split across ranks: whole boxes per rank by cost
    (greedy longest-first on N_b log N_b), each rank one mm_step_batched
    graph replay per step over its own boxes, no exchange on the data path;
    per-box timesteps and conserved totals gathered once at the end.  value =
    all ranks' cells per step / the slowest rank's time (strong scaling: the
    batch is fixed).  Mixed precision unless --precision fp64."""
    args.precision = args.precision or "mixed"
    import numpy as np
    import torch
    from paper_1707_05333_gb300 import build as B
    from paper_1707_05333_gb300 import binding as BD
    from paper_1707_05333_gb300 import ensemble as E
    from paper_1707_05333_gb300 import workloads as WL

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    B.build()
    sizes = WL.ensemble_sizes(args.ensemble_boxes)
    parts = E.partition_boxes(sizes, world)
    mine = parts[rank]
    loads = E.rank_loads(sizes, parts)
    boxes = [WL.ensemble_box(int(b), int(sizes[b])) for b in mine]
    msz = [int(sizes[b]) for b in mine]
    off = E.offsets(msz)
    n_mine = int(off[-1])
    n_all = int(np.sum(sizes))
    L = np.ones((len(boxes), 3))
    prec = 0 if args.precision == "fp64" else 1
    tuned = {}
    if not args.no_autotune:
        big = boxes[int(np.argmax(msz))]
        t = tune_clipper(args, big.pos, big.box)
        tuned = {k: t[k] for k in ("clip_warps", "cand_cap", "bin_scale", "clip_sort")}
    stream = torch.cuda.Stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    with torch.cuda.stream(stream):
        ctx = BD.Context(stream=stream, gamma=5.0 / 3.0, cfl=0.3, limiter=1, precision=prec, **tuned)
        Us = []
        for wb in boxes:
            pb = torch.tensor(wb.pos.T.copy(), dtype=torch.float64, device="cuda")
            mb = ctx.mm_tessellate(pb, wb.box)
            Us.append(ctx.mm_prims_to_charges(mb, torch.tensor(wb.rho, device="cuda"),
                                              torch.tensor(wb.vel.T.copy(), device="cuda"),
                                              torch.tensor(wb.pres, device="cuda")))
        pos0 = torch.tensor(np.concatenate([wb.pos for wb in boxes]).T.copy(), dtype=torch.float64, device="cuda")
        U0 = torch.cat(Us, dim=1).contiguous()
        del Us
        pos, U = pos0.clone(), U0.clone()
        dt = torch.empty((len(boxes),), dtype=torch.float64, device="cuda")
        for _ in range(max(3, args.warmup)):
            ctx.mm_step_batched(pos, U, off, L, dt_out=dt)
        ctx.mm_sync_status()
        l0 = ctx.mm_kernel_launches()
        barrier()
        torch.cuda.synchronize()
        proc, cpath = clocks_start(local)
        time.sleep(0.3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            ctx.mm_step_batched(pos, U, off, L, dt_out=dt)
        e1.record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        barrier()
        clocks = clocks_stop(proc, cpath)
        ms = e0.elapsed_time(e1)
        launches = ctx.mm_kernel_launches() - l0
        ctx.mm_sync_status()
        _, ms = aggregate(ms, n_mine, args.steps, world)
        value = n_all * args.steps / (ms / 1e3)
        # per-box results, gathered once (outside the timed region): dt and the five totals
        cb = torch.repeat_interleave(torch.arange(len(boxes), device="cuda"),
                                     torch.as_tensor(np.diff(off), device="cuda"))
        tot = torch.zeros((len(boxes), 5), dtype=torch.float64, device="cuda")
        tot.index_add_(0, cb, U.T.contiguous())
        rows = torch.cat([dt[:, None], tot], dim=1).cpu().numpy()
        table = E.gather_box_results(len(sizes), mine, rows)

        # ---- end to end: inputs from pinned host buffers, results back, every step
        pos_h = pos0.cpu().pin_memory()
        U_h = U0.cpu().pin_memory()
        barrier()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            pos.copy_(pos_h, non_blocking=True)
            U.copy_(U_h, non_blocking=True)
            ctx.mm_step_batched(pos, U, off, L, dt_out=dt)
            pos_h.copy_(pos, non_blocking=True)
            U_h.copy_(U, non_blocking=True)
        f1.record(stream)
        stream.synchronize()
        e2e_ms = f0.elapsed_time(f1)
        _, e2e_ms = aggregate(e2e_ms, n_mine, args.steps, world)
        ctx.close()
    if rank == 0:
        nbytes = int(pos0.numel() * 8 + U0.numel() * 8)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f64" if prec == 0 else "f64+f32",
                "data": "synthetic",
                "config": {"workload": f"ensemble of {len(sizes)} periodic unit boxes, {n_all} cells",
                           "cells": n_all, "precision": args.precision,
                           "parallelism": f"boxes split over {world} ranks by cost N_b log N_b",
                           "rank_cost_imbalance": float(loads.max() / loads.mean()),
                           "clipper_settings": tuned or "defaults",
                           "l2": "state + meshes larger than L2, no flush"},
                "roofline": None,
                "roofline_note": "per-kernel times are not separable inside the captured graph; the ncu launch "
                                 "list of this mode gives each kernel's share",
                "cpu_baseline": None,
                "e2e": {"value": n_all * args.steps / (e2e_ms / 1e3), "unit": UNIT,
                        "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                        "note": "rank 0's share of the bytes"},
                "gpu_launches": launches, "clocks": clocks,
                "box_results": {"min_dt": float(table[:, 0].min()), "max_dt": float(table[:, 0].max()),
                                "total_mass": float(table[:, 1].sum()), "total_energy": float(table[:, 5].sum())}}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_ours(args, world, rank, local):
    import torch
    from paper_1707_05333_gb300 import build as B
    from paper_1707_05333_gb300 import binding as BD
    from paper_1707_05333_gb300 import workloads as WL

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    B.build()
    args.precision = args.precision or "fp64"
    w = WL.shear_layer(args.n_side)
    prec = 0 if args.precision == "fp64" else 1
    # clipper settings tuned on the same recipe at half the side (untimed)
    args.tuned, tune_info = {}, None
    if not args.no_autotune:
        ws = WL.shear_layer(max(32, args.n_side // 2))
        tune_info = tune_clipper(args, ws.pos, ws.box)
        tune_info["sample"] = f"shear_layer_{max(32, args.n_side // 2)}^3, 3 timed tessellations per setting"
        del ws
        tuned = {k: tune_info[k] for k in ("clip_warps", "cand_cap", "bin_scale", "clip_sort")}
        args.tuned, check = confirm_clipper(w, tuned, clip_filter=args.clip_filter)
        tune_info.update(check)
        tune_info["used"] = dict(args.tuned)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = BD.Context(stream=stream, gamma=w.gamma, cfl=w.cfl, limiter=1, precision=prec,
                         clip_filter=args.clip_filter, **args.tuned)
        pos0 = torch.tensor(w.pos.T.copy(), dtype=torch.float64, device="cuda")
        mesh = ctx.mm_tessellate(pos0, w.box)
        U0 = ctx.mm_prims_to_charges(mesh, torch.tensor(w.rho, device="cuda"),
                                     torch.tensor(w.vel.T.copy(), device="cuda"),
                                     torch.tensor(w.pres, device="cuda"))
        pos, U = pos0.clone(), U0.clone()
        for _ in range(args.warmup):
            ctx.mm_step(pos, U, w.box)
        # counters of what the filtered clipper executes, on the state the
        # timed window starts from (outside the timed region); the method's
        # work is counted over the whole window after it (window_direct_counts)
        ctx.set_config(collect_stats=1, clip_filter=args.clip_filter)
        ctx.mm_tessellate(pos, w.box)
        tstats = ctx.mm_tess_stats()
        ctx.set_config(collect_stats=0)
        pos_w0, U_w0 = pos.clone(), U.clone()
        stream.synchronize()

        def barrier():
            if world > 1:
                import torch.distributed as dist
                dist.barrier()

        # ---- device-resident timed region
        ctx.mm_set_timing(True)
        launches0 = ctx.mm_kernel_launches()
        barrier()
        torch.cuda.synchronize()
        proc, cpath = clocks_start(local)
        time.sleep(0.3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            ctx.mm_step(pos, U, w.box)
        e1.record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        barrier()
        clocks = clocks_stop(proc, cpath)
        launches = ctx.mm_kernel_launches() - launches0
        ms = e0.elapsed_time(e1)
        stages = ctx.mm_stage_times()
        ctx.mm_set_timing(False)
        nf = ctx.mm_tessellate(pos, w.box).nfaces  # faces of the current mesh, for the byte counts
        n = w.n
        value, ms = aggregate(ms, n, args.steps, world)

        # ---- end to end through the ABI with host buffers: mm_step_host copies
        # the step's inputs up and its results back (page-locked memory, the
        # copies overlapped with the step inside the library)
        # the same steps as the timed window: from its start state, args.steps steps
        pos_h = torch.empty_like(pos, device="cpu").pin_memory()
        U_h = torch.empty_like(U, device="cpu").pin_memory()
        pos_h.copy_(pos0.cpu())
        U_h.copy_(U0.cpu())
        ctx.mm_step_host(pos_h, U_h, w.box)  # untimed: the context's device copies are allocated here
        pos_h.copy_(pos_w0.cpu())
        U_h.copy_(U_w0.cpu())
        barrier()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            ctx.mm_step_host(pos_h, U_h, w.box)
        f1.record(stream)
        stream.synchronize()
        e2e_ms = f0.elapsed_time(f1)
        e2e_value, e2e_ms = aggregate(e2e_ms, n, args.steps, world)
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": int(pos.numel() * 8 + U.numel() * 8),
               "d2h_bytes_per_step": int(pos.numel() * 8 + U.numel() * 8)}
        tdirect = window_direct_counts(ctx, pos_w0, U_w0, w.box, args.steps, args.clip_filter)
        del pos_w0, U_w0

    # ---- roofline of the dominant kernel, from the live stage times
    stage_ms = {k: v[0] / max(1, v[1]) for k, v in stages.items()}
    dom = max(stages, key=lambda k: stages[k][0])
    dom_ms = stage_ms[dom]
    peak, peak_kind = measured_peaks()
    clip_flops = clip_method_flops(tdirect)
    roofline = None
    if dom == "clip":
        roofline = clip_roofline(tdirect, tstats, dom_ms, n, args.clip_filter)
        roofline["traffic"] = clip_traffic(n, args.clip_filter)
        if roofline["traffic"] is not None:
            roofline["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_clip launch "
                                          "at 128^3, scaled by cells")
    else:
        byts = algorithmic_bytes(dom, n, nf)
        if byts is not None:
            ach = byts / (dom_ms / 1e3) / 1e9
            roofline = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                        "frac": ach / peak, "traffic": None, "peak_source": peak_kind,
                        "algorithmic_bytes_per_launch": byts, "launch_ms": dom_ms}
    roofline_step = step_roofline(ms / args.steps, stage_ms, n, nf, clip_flops, prec == 1, peak, peak_kind)
    stage_roofline = stage_rooflines(stage_ms, n, nf, prec == 1, peak, peak_kind)

    variants = None
    if rank == 0 and not args.no_variants:
        variants = measure_variants(args, w, clip_flops)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        r1, steps1, el1, _ = oracle_rate(args.cpu_sample_side, args.cpu_seconds / 2)
        rate, procs, steps = oracle_rate_all_cores(args.cpu_sample_side, args.cpu_seconds / 2)
        cpu = {"value": rate, "unit": UNIT, "cores": procs, "kind": "oracle",
               "sample": f"shear-layer recipe at {args.cpu_sample_side}^3 generators, whole oracle steps: "
                         f"{procs} concurrent replicas (one thread each, {steps} steps in about "
                         f"{args.cpu_seconds / 2:.0f} s); the per-cell rate stands for the "
                         f"{args.n_side}^3 box (same recipe and spacing statistics, the oracle's work per "
                         f"cell does not depend on the box size)",
               "single_thread": {"value": r1, "steps": steps1, "seconds": round(el1, 1)}}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == 0 else "f64+f32",
                "data": "synthetic",
                "config": {"workload": f"shear_layer_{args.n_side}^3", "cells": n, "faces": nf,
                           "precision": args.precision, "clip_filter": args.clip_filter,
                           "clipper_settings": tune_info or "defaults",
                           "parallelism": f"replicas x{world}",
                           "l2": "inputs larger than L2 (state + mesh >> 129 MB), no flush"},
                "roofline": roofline, "roofline_step": roofline_step, "stage_ms": stage_ms,
                "stage_roofline": stage_roofline,
                "tess_stats_per_cell": {k: v / n for k, v in tstats.items() if not k.startswith("max")},
                "tess_stats_direct_per_cell": {k: v / n for k, v in tdirect.items() if not k.startswith("max")},
                "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks, "variants": variants}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.workload == "ensemble":
        return run_ensemble(args, world, rank, local)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
