"""Shared test helpers: run the CUDA path through the binding and compare it
with the oracle on identical seeded inputs."""
import numpy as np


def gpu_context(**cfg):
    import torch
    from paper_1707_05333_gb300 import binding
    binding.load()
    return binding.Context(**cfg), torch


def to_dev(torch, a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def gpu_tessellate(ctx, torch, pos, box):
    """pos (n,3) numpy -> dict of numpy arrays in the oracle's conventions."""
    P = to_dev(torch, pos.T)
    mesh = ctx.mm_tessellate(P, box)
    d = {k: v.cpu().numpy() for k, v in mesh.to_torch().items()}
    return mesh, P, d


def face_key_map(i, j, code):
    return {(int(a), int(b), int(c)): k for k, (a, b, c) in enumerate(zip(i, j, code))}


AREA_REL = 1e-10    # the face threshold of the library and the oracle: area <= AREA_REL (V_box/n)^(2/3)
GEOM_RTOL = 1e-9    # geometry: per face relative to its own area (and its own size for centroids)


def compare_tessellations(oracle, T, G, pos, box, geom_rtol=GEOM_RTOL, area_rel=AREA_REL, label=""):
    """Topology exact except faces at or below the drop threshold
    area_rel (V_box/n)^(2/3) (a face within the geometry tolerance of the
    threshold may fall on either side of it); every common face's area within
    geom_rtol of its own area, its centroid within geom_rtol times its own
    size sqrt(A_f), its normal to 1e-12; cell volumes to geom_rtol relative and
    cell centroids to geom_rtol times the mean spacing.  Prints how many faces
    fall in the band (1e-10, 1e-8] of the scale, which an earlier, looser
    reading of the threshold excused.  Returns the number of common faces."""
    n = len(pos)
    scale = (np.prod(box) / n) ** (2.0 / 3.0)
    h = np.sqrt(scale)
    thr = area_rel * scale
    excuse = thr * (1.0 + geom_rtol)
    F = oracle.unique_faces(T)
    ocode = oracle.shift_code(F["shift"])
    om = face_key_map(F["i"], F["j"], ocode)
    gm = face_key_map(G["face_i"], G["face_j"], G["face_shift"])
    only_o = [k for key, k in om.items() if key not in gm]
    only_g = [k for key, k in gm.items() if key not in om]
    band = int(np.count_nonzero((F["area"] > thr) & (F["area"] <= 1e-8 * scale)))
    print(f"[tessellation parity {label}] faces {len(om)} oracle / {len(gm)} GPU; in the band "
          f"(1e-10, 1e-8] of (V/n)^(2/3): {band}; missing on the GPU: {len(only_o)}, only on the GPU: "
          f"{len(only_g)} (each must be within the tolerance of the threshold)")
    for k in only_o:
        assert F["area"][k] <= excuse, (
            f"face {F['i'][k], F['j'][k], ocode[k]} (area {F['area'][k] / scale:.3e} of the scale) missing on the GPU")
    for k in only_g:
        assert G["face_area"][k] <= excuse, (
            f"face {G['face_i'][k], G['face_j'][k], G['face_shift'][k]} (area "
            f"{G['face_area'][k] / scale:.3e} of the scale) only on the GPU")
    common = [(om[key], gm[key]) for key in om if key in gm]
    oi = np.array([a for a, _ in common], dtype=np.int64)
    gi = np.array([b for _, b in common], dtype=np.int64)
    A_o = F["area"][oi]
    dA = np.abs(G["face_area"][gi] - A_o)
    worst = int(np.argmax(dA / A_o)) if len(oi) else 0
    assert np.all(dA <= geom_rtol * A_o), (
        f"face area off by {dA[worst] / A_o[worst]:.3e} of itself (area {A_o[worst] / scale:.3e} of the scale)")
    np.testing.assert_allclose(G["face_normal"][:, gi].T, F["normal"][oi], rtol=0, atol=1e-12)
    dc = np.abs(G["face_centroid"][:, gi].T - F["centroid"][oi]).max(axis=1)
    size = np.sqrt(A_o)
    worst = int(np.argmax(dc / size)) if len(oi) else 0
    assert np.all(dc <= geom_rtol * size), (
        f"face centroid off by {dc[worst] / size[worst]:.3e} of the face's size (area {A_o[worst] / scale:.3e})")
    np.testing.assert_allclose(G["cell_volume"], T["volume"], rtol=geom_rtol)
    np.testing.assert_allclose(G["cell_centroid"].T, T["centroid"], rtol=0, atol=geom_rtol * h)
    return len(common)


def check_incidence(G):
    """Every unique face appears exactly once in each of its two cells' lists."""
    n = len(G["cell_volume"])
    off, inc = G["inc_off"], G["inc_face"]
    assert off[0] == 0 and off[-1] == len(inc)
    nf = len(G["face_area"])
    seen_i = np.zeros(nf, int)
    seen_j = np.zeros(nf, int)
    cell_of = np.repeat(np.arange(n), np.diff(off))
    fwd = inc >= 0
    seen_i_idx = inc[fwd]
    seen_j_idx = ~inc[~fwd]
    np.add.at(seen_i, seen_i_idx, 1)
    np.add.at(seen_j, seen_j_idx, 1)
    assert np.all(seen_i == 1) and np.all(seen_j == 1)
    assert np.all(G["face_i"][seen_i_idx] == cell_of[fwd])
    assert np.all(G["face_j"][seen_j_idx] == cell_of[~fwd])


def oracle_local_step(oracle, pos, U, box, cfg, cells, dt):
    """The oracle's one-step result (Sec. 2) on a few cells of a large box,
    without tessellating all of it.  A cell's new charges depend on its own
    faces' fluxes, which read the half-step states and limited gradients of
    the cell and its neighbours (ring 1); those gradients read the half-step
    states of ring 2, which need the first gradients of ring 2 (from the
    states of ring 3).  So the oracle tessellates rings 0..3 (every generator
    stays a candidate), keeps the faces among them, and steps that
    sub-problem with the given dt: rings 0..2 have all their faces, and
    whatever ring 3's incomplete face lists give never reaches ring 0.
    Returns (new charges, new positions, mesh velocities) of `cells`, in
    their order, and the number of cells the oracle tessellated."""
    cells = np.asarray(cells, dtype=np.int64)
    have = set()
    parts = []
    ring = np.unique(cells)
    for depth in range(4):
        T = oracle.tessellate(pos, box, cells=ring)
        parts.append(T)
        have.update(int(c) for c in ring)
        if depth == 3:
            break
        nxt = np.unique(T["nb"])
        ring = np.array([c for c in nxt if int(c) not in have], dtype=np.int64)
    idx = np.array(sorted(have), dtype=np.int64)
    loc = {int(g): k for k, g in enumerate(idx)}
    m = len(idx)
    vol = np.zeros(m)
    cen = np.zeros((m, 3))
    keys = ("cell", "nb", "shift", "area", "normal", "fcentroid")
    acc = {k: [] for k in keys}
    for T in parts:
        own = np.unique(T["cell"])
        for g in own:
            vol[loc[int(g)]] = T["volume"][g]
            cen[loc[int(g)]] = T["centroid"][g]
        inside = np.array([int(j) in loc for j in T["nb"]], dtype=bool)
        for k in keys:
            acc[k].append(T[k][inside])
    sub = {k: np.concatenate(v) for k, v in acc.items()}
    sub["cell"] = np.array([loc[int(g)] for g in sub["cell"]], dtype=np.int32)
    sub["nb"] = np.array([loc[int(g)] for g in sub["nb"]], dtype=np.int32)
    sub["shift"] = sub["shift"].astype(np.int32)
    sub.update(volume=vol, centroid=cen, box=np.asarray(box, dtype=float).copy(), n=m)
    S = oracle.step(pos[idx], U[idx], box, cfg, dt=dt, tess=sub)
    li = np.array([loc[int(c)] for c in cells], dtype=np.int64)
    return S["U"][li], S["pos"][li], S["w"][li], m
