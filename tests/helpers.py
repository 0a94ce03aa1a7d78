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


def compare_tessellations(oracle, T, G, pos, box, geom_rtol=1e-9, tiny_rel=1e-8):
    """Topology exact for faces above tiny_rel * mean cell area; geometry to geom_rtol."""
    n = len(pos)
    scale = (np.prod(box) / n) ** (2.0 / 3.0)
    h = np.sqrt(scale)
    F = oracle.unique_faces(T)
    ocode = oracle.shift_code(F["shift"])
    om = face_key_map(F["i"], F["j"], ocode)
    gm = face_key_map(G["face_i"], G["face_j"], G["face_shift"])
    for key, k in om.items():
        if key not in gm:
            assert F["area"][k] <= tiny_rel * scale, f"face {key} (area {F['area'][k]:.3e}) missing on GPU"
    for key, k in gm.items():
        if key not in om:
            assert G["face_area"][k] <= tiny_rel * scale, f"face {key} (area {G['face_area'][k]:.3e}) only on GPU"
    common = [(om[key], gm[key]) for key in om if key in gm]
    oi = np.array([a for a, _ in common])
    gi = np.array([b for _, b in common])
    np.testing.assert_allclose(G["face_area"][gi], F["area"][oi], rtol=0, atol=geom_rtol * scale)
    np.testing.assert_allclose(G["face_normal"][:, gi].T, F["normal"][oi], rtol=0, atol=1e-12)
    np.testing.assert_allclose(G["face_centroid"][:, gi].T, F["centroid"][oi], rtol=0, atol=geom_rtol * h)
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
