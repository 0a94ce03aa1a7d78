"""Cells beyond the clipper's per-cell lists, and inputs with no Voronoi
tessellation: the tessellation either succeeds through the large-capacity
clipper (and then matches the oracle) or returns a status; the context stays
usable either way."""
import numpy as np
import pytest

from paper_1707_05333_gb300 import workloads as WL
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c, torch = H.gpu_context()
    yield c, torch
    c.close()


def sphere_points(m, radius, centre, rng):
    """m points on a sphere (Fibonacci spiral) with 1 % radial jitter."""
    k = np.arange(m) + 0.5
    z = 1.0 - 2.0 * k / m
    phi = np.pi * (1.0 + 5.0 ** 0.5) * k
    rr = np.sqrt(1.0 - z * z)
    d = np.stack([rr * np.cos(phi), rr * np.sin(phi), z], axis=1)
    return centre + radius * d * (1.0 + 0.01 * rng.uniform(-1.0, 1.0, size=(m, 1)))


def hubs(centres, m, radius, background, seed):
    """Generators at `centres`, each ringed by m points on a sphere (its cell
    has m faces), plus uniform background points away from the spheres."""
    rng = np.random.default_rng(seed)
    pts = [np.asarray(centres)]
    for c in centres:
        pts.append(sphere_points(m, radius, c, rng))
    bg = rng.uniform(0.0, 1.0, size=(background, 3))
    d = np.min(np.linalg.norm(bg[:, None, :] - np.asarray(centres)[None, :, :], axis=2), axis=1)
    pts.append(bg[d > 2.0 * radius])
    return np.concatenate(pts) % 1.0


def test_cell_with_80_faces_is_reclipped_and_matches_oracle(oracle, ctx):
    """One generator ringed by 80 others: its cell has 80 faces and 156
    vertices, beyond the main clipper's 48 faces, 64 planes and 128 vertices.
    The large clipper clips it again and the mesh equals the oracle's."""
    c, torch = ctx
    pos = hubs([[0.5, 0.5, 0.5]], 80, 0.08, 400, seed=1)
    box = np.ones(3)
    T = oracle.tessellate(pos, box, 0)
    counts = np.bincount(T["cell"], minlength=len(pos))
    assert counts[0] == 80
    c.set_config(collect_stats=1)
    try:
        mesh, P, G = H.gpu_tessellate(c, torch, pos, box)
        st = c.mm_tess_stats()
    finally:
        c.set_config(collect_stats=0)
    # the hub is the only cell over 48 faces; over a list of the main clipper
    assert 1 <= st["retried_cells"] <= 3
    H.compare_tessellations(oracle, T, G, pos, box, label="80-face cell")
    H.check_incidence(G)
    assert np.diff(G["inc_off"])[0] == 80
    assert abs(G["cell_volume"].sum() - 1.0) <= 1e-12
    # the filtered and the direct FP64 clippers agree bit for bit here too
    c.set_config(clip_filter=0)
    try:
        _, _, D = H.gpu_tessellate(c, torch, pos, box)
    finally:
        c.set_config(clip_filter=1)
    for k in D:
        np.testing.assert_array_equal(D[k], G[k], err_msg=k)


def test_more_overflowing_cells_than_overflow_rows(oracle, ctx):
    """343 hub cells of 60 faces each (and background cells beside them over
    48 faces): more than the 256 overflow rows a
    context starts with.  mm_tessellate grows the rows to the count it reads
    and re-clips the list; the mesh equals the oracle's.  A captured batch
    keeps its fixed rows and reports the excess as MM_ECAPACITY through
    mm_sync_status, and the context keeps working."""
    import torch as T_
    from paper_1707_05333_gb300 import binding
    c, torch = ctx
    g = (np.arange(7) + 0.5) / 7.0
    centres = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    pos = hubs(centres, 60, 0.03, 3000, seed=2)
    box = np.ones(3)
    T = oracle.tessellate(pos, box, 1)
    counts = np.bincount(T["cell"], minlength=len(pos))
    assert np.all(counts[:343] == 60)
    over = int(np.count_nonzero(counts > 48))  # the hubs and some background cells beside the spheres
    c.set_config(collect_stats=1)
    try:
        mesh, P, G = H.gpu_tessellate(c, torch, pos, box)
        st = c.mm_tess_stats()
    finally:
        c.set_config(collect_stats=0)
    assert over <= st["retried_cells"] <= int(np.count_nonzero(counts > 40))
    H.compare_tessellations(oracle, T, G, pos, box, label="343 hubs")
    H.check_incidence(G)
    # the same input as a captured one-box batch: over 256 retried cells, more than its rows
    stream = T_.cuda.Stream()
    with T_.cuda.stream(stream):
        b = binding.Context(stream=stream)
        Pd = H.to_dev(torch, pos.T)
        U = torch.zeros((5, len(pos)), dtype=torch.float64, device="cuda")
        U[0] = 1.0
        U[4] = 1.0
        b.mm_step_batched(Pd, U, np.array([0, len(pos)]), np.ones((1, 3)))
        with pytest.raises(binding.MMError) as e:
            b.mm_sync_status()
        assert e.value.status == 3 and "overflow rows" in str(e.value)
        b.close()
    # the context still tessellates
    _, _, G2 = H.gpu_tessellate(c, torch, WL.random_points(500, seed=3), box)
    assert abs(G2["cell_volume"].sum() - 1.0) <= 1e-12


def test_batched_step_with_a_reclipped_cell_equals_per_box_steps(oracle, ctx):
    """A captured batch of two boxes, one with an 80-face cell: the step
    equals mm_step on each box alone, bit for bit."""
    import torch as T_
    from paper_1707_05333_gb300 import binding
    c, torch = ctx
    a = hubs([[0.5, 0.5, 0.5]], 80, 0.08, 400, seed=1)
    bpos = WL.random_points(600, seed=5)
    sizes = [len(a), len(bpos)]
    allpos = np.concatenate([a, bpos])
    rho, vel, pres = WL.random_state(len(allpos), seed=4)
    stream = T_.cuda.Stream()
    with T_.cuda.stream(stream):
        b = binding.Context(stream=stream, gamma=5.0 / 3.0, limiter=1)
        Us, per = [], []
        for k, p in enumerate((a, bpos)):
            lo, hi = sum(sizes[:k]), sum(sizes[:k + 1])
            Pd = H.to_dev(torch, p.T)
            m = b.mm_tessellate(Pd, np.ones(3))
            U = b.mm_prims_to_charges(m, H.to_dev(torch, rho[lo:hi]), H.to_dev(torch, vel[lo:hi].T),
                                      H.to_dev(torch, pres[lo:hi]))
            Us.append(U.clone())
            b.mm_step(Pd, U, np.ones(3))
            per.append((Pd.clone(), U.clone()))
        Pall = H.to_dev(torch, allpos.T)
        Uall = torch.cat(Us, dim=1).contiguous()
        b.mm_step_batched(Pall, Uall, np.array([0, sizes[0], sum(sizes)]), np.ones((2, 3)))
        b.mm_sync_status()
        assert torch.equal(Uall[:, :sizes[0]], per[0][1]) and torch.equal(Uall[:, sizes[0]:], per[1][1])
        assert torch.equal(Pall[:, :sizes[0]], per[0][0]) and torch.equal(Pall[:, sizes[0]:], per[1][0])
        b.close()


def test_coincident_generators_are_degenerate(ctx):
    """Two generators at the same position have no Voronoi tessellation (the
    clipper meets a candidate at distance 0): MM_EDEGENERATE, and the
    context stays usable."""
    from paper_1707_05333_gb300.binding import MMError
    c, torch = ctx
    pos = WL.random_points(200, seed=6)
    pos[17] = pos[3]
    with pytest.raises(MMError) as e:
        H.gpu_tessellate(c, torch, pos, np.ones(3))
    assert e.value.status == 4
    _, _, G = H.gpu_tessellate(c, torch, WL.random_points(200, seed=6), np.ones(3))
    assert abs(G["cell_volume"].sum() - 1.0) <= 1e-12


@pytest.mark.parametrize("case", ["pairs_1e-10_apart", "cubic_24_jitter_1e-12", "cubic_12_jitter_1e-11"])
def test_near_degenerate_inputs_succeed_exactly_or_are_reported(ctx, case):
    """Generators in pairs 1e-10 apart, cubic lattices perturbed by 1e-12 and
    1e-11 of a spacing: cuts that are inconsistent under the tie margin are
    clipped again with the strict rule, and two cells that disagree on a face
    far above the area threshold are reported.  So the call either succeeds
    with volumes that sum to the box and a consistent incidence structure, or
    fails with MM_EDEGENERATE: never a mesh with a face missing.  The context
    keeps working either way."""
    from paper_1707_05333_gb300.binding import MMError
    c, torch = ctx
    rng = np.random.default_rng(31)
    if case == "pairs_1e-10_apart":
        base = rng.uniform(0.0, 1.0, size=(1000, 3))
        pos = np.concatenate([base, (base + 1e-10) % 1.0])
    else:
        m = 24 if case == "cubic_24_jitter_1e-12" else 12
        jit = 1e-12 if m == 24 else 1e-11
        g = np.arange(m) / m
        lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
        pos = (lat + jit / m * rng.standard_normal(lat.shape)) % 1.0
    pos = np.where(pos >= 1.0, 0.0, pos)
    try:
        mesh, P, G = H.gpu_tessellate(c, torch, pos, np.ones(3))
    except MMError as e:
        assert e.status == 4, e
    else:
        H.check_incidence(G)
        assert np.all(G["cell_volume"] > 0)
        assert abs(G["cell_volume"].sum() - 1.0) <= 1e-9
    _, _, G2 = H.gpu_tessellate(c, torch, WL.random_points(300, seed=8), np.ones(3))
    assert abs(G2["cell_volume"].sum() - 1.0) <= 1e-12
