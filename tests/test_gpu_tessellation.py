"""GPU tessellation (mm_tessellate) against the oracle, element by element."""
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


def lattice(kind, m):
    s = 1.0 / m
    basis = {"sc": [(0, 0, 0)], "bcc": [(0, 0, 0), (0.5, 0.5, 0.5)],
             "fcc": [(0, 0, 0), (0.5, 0.5, 0), (0.5, 0, 0.5), (0, 0.5, 0.5)]}[kind]
    pts = [((i + b[0] + 0.25) * s, (j + b[1] + 0.25) * s, (k + b[2] + 0.25) * s)
           for k in range(m) for j in range(m) for i in range(m) for b in basis]
    return np.array(pts)


CASES = {
    "smooth_wave_16^3": lambda: (WL.smooth_wave(16).pos, np.ones(3)),
    "jittered_13^3_ragged": lambda: (WL.smooth_wave(13).pos, np.ones(3)),
    "random_1001": lambda: (WL.random_points(1001, seed=4), np.ones(3)),
    "random_box_2x1x0.5": lambda: (WL.random_points(777, box=(2.0, 1.0, 0.5), seed=5), np.array([2.0, 1.0, 0.5])),
    "shock_tube_64x8x8": lambda: (WL.shock_tube(64, 8, 8).pos, np.array([8.0, 1.0, 1.0])),
    "cubic_lattice_exact_ties": lambda: (lattice("sc", 8), np.ones(3)),
    "bcc_lattice": lambda: (lattice("bcc", 5), np.ones(3)),
    "fcc_degenerate_vertices": lambda: (lattice("fcc", 4), np.ones(3)),
    "n1": lambda: (np.array([[0.3, 0.6, 0.9]]), np.ones(3)),
    "n2": lambda: (np.array([[0.1, 0.5, 0.5], [0.6, 0.55, 0.45]]), np.ones(3)),
    "n5": lambda: (WL.random_points(5, seed=6), np.ones(3)),
    "n37": lambda: (WL.random_points(37, seed=7), np.ones(3)),
    # a dense core in a sparse background: cell volumes over five decades, crowded bins
    "clustered_6000": lambda: (WL.clustered_points(6000, seed=1), np.ones(3)),
}


@pytest.mark.parametrize("case", list(CASES))
def test_tessellation_matches_oracle(oracle, ctx, case):
    c, torch = ctx
    pos, box = CASES[case]()
    T = oracle.tessellate(pos, box, 0 if len(pos) <= 1100 else 1)
    mesh, P, G = H.gpu_tessellate(c, torch, pos, box)
    ncommon = H.compare_tessellations(oracle, T, G, pos, box, label=case)
    assert ncommon > 0
    H.check_incidence(G)
    assert abs(G["cell_volume"].sum() - np.prod(box)) <= 1e-11 * np.prod(box)


def lattice_at(kind, m, offset):
    """Exact lattice of m^3 cells in the unit box, basis shifted by `offset`
    cells (0.1 and 1/3-like offsets make coordinates inexact in binary)."""
    s = 1.0 / m
    basis = {"sc": [(0, 0, 0)], "bcc": [(0, 0, 0), (0.5, 0.5, 0.5)],
             "fcc": [(0, 0, 0), (0.5, 0.5, 0), (0.5, 0, 0.5), (0, 0.5, 0.5)]}[kind]
    pts = [((i + b[0] + offset) * s, (j + b[1] + offset) * s, (k + b[2] + offset) * s)
           for k in range(m) for j in range(m) for i in range(m) for b in basis]
    return np.array(pts) % 1.0


# (kind, cells per axis, basis offset, bin width, jitter in spacings): sizes
# and offsets whose coordinates are not exact in binary, where every Voronoi
# vertex is shared by more cells than three planes define (cube corners,
# rhombic-dodecahedron vertices) and rounding gives one point several slightly
# different values; and lattices perturbed by 1e-11 and 1e-15 of a spacing,
# within the tie margin of the plane tests and at the rounding level
LATTICES = [("sc", 6, 0.0, 1.0, 0.0), ("sc", 12, 0.25, 1.25, 0.0), ("sc", 24, 0.1, 1.0, 0.0),
            ("bcc", 12, 0.5, 1.25, 0.0), ("fcc", 4, 0.1, 1.0, 0.0), ("fcc", 6, 0.0, 1.25, 0.0),
            ("fcc", 12, 0.25, 1.0, 0.0), ("sc", 12, 0.25, 1.0, 1e-11), ("sc", 6, 0.1, 1.0, 1e-11),
            ("fcc", 6, 0.0, 1.0, 1e-11), ("sc", 12, 0.25, 1.0, 1e-15)]


@pytest.mark.parametrize("kind,m,offset,bin_scale,jitter", LATTICES)
def test_exact_lattices_at_inexact_sizes_and_offsets(oracle, ctx, kind, m, offset, bin_scale, jitter):
    """Perfect (and nearly perfect) lattices: every cell is the lattice's Voronoi
    cell (cube, truncated octahedron, rhombic dodecahedron): its volume 1/n,
    its face count 6, 14 or 12 (faces of the perturbed ones that a jitter of
    1e-11 spacings opens stay below the area threshold), and the mesh equals
    the oracle's (faces at or below the area threshold excepted, as
    everywhere)."""
    c, torch = ctx
    pos = lattice_at(kind, m, offset)
    n = len(pos)
    if jitter:
        rng = np.random.default_rng(11)
        pos = (pos + jitter / m * rng.standard_normal(pos.shape)) % 1.0
        pos = np.where(pos >= 1.0, 0.0, pos)
    box = np.ones(3)
    c.set_config(bin_scale=bin_scale)
    try:
        mesh, P, G = H.gpu_tessellate(c, torch, pos, box)
    finally:
        c.set_config(bin_scale=1.0)
    np.testing.assert_allclose(G["cell_volume"], 1.0 / n, rtol=1e-12 if not jitter else 1e-9, atol=0)
    faces = {"sc": 6, "bcc": 14, "fcc": 12}[kind]
    assert np.all(np.diff(G["inc_off"]) == faces)
    H.check_incidence(G)
    if n <= 4000:
        T = oracle.tessellate(pos, box, 0 if n <= 1100 else 1)
        H.compare_tessellations(oracle, T, G, pos, box, label=f"{kind}{m}+{offset}")


def _extreme(name):
    rng = np.random.default_rng(21)
    if name == "generators_on_a_plane":
        u = rng.uniform(0, 1, size=(600, 2))
        return np.column_stack([u, np.full(600, 0.5)]), np.ones(3)
    if name == "generators_on_a_line":
        return np.column_stack([rng.uniform(0, 1, 200), np.full(200, 0.3), np.full(200, 0.7)]), np.ones(3)
    if name == "hcp_lattice":
        m, a = 6, 1.0 / 6
        pts = [((i + 0.5 * (j % 2) + 0.5 * (k % 2)) * a, (j + (k % 2) / 3.0) * a * np.sqrt(3) / 2,
                k * a * np.sqrt(2.0 / 3.0)) for k in range(m) for j in range(m) for i in range(m)]
        box = np.array([1.0, m * a * np.sqrt(3) / 2, m * a * np.sqrt(2.0 / 3.0)])
        return np.array(pts) % box, box
    if name == "flat_box_100_to_1":
        box = np.array([1.0, 1.0, 0.01])
        return rng.uniform(0, 1, size=(1500, 3)) * box, box
    if name == "tight_cluster_in_a_large_box":
        return 0.5 + 1e-3 * rng.uniform(-1, 1, size=(800, 3)), np.ones(3)
    if name == "lattice_and_a_near_centred_point":
        return np.concatenate([lattice_at("sc", 6, 0.0), [[0.5 + 1e-12, 0.5, 0.5]]]) % 1.0, np.ones(3)
    raise KeyError(name)


@pytest.mark.parametrize("name", ["generators_on_a_plane", "generators_on_a_line", "hcp_lattice", "flat_box_100_to_1",
                                  "tight_cluster_in_a_large_box", "lattice_and_a_near_centred_point"])
def test_degenerate_and_extreme_generator_sets(oracle, ctx, name):
    """Generators on one plane or one line (cells are prisms and slabs through
    the whole box), the hcp lattice (co-spherical neighbours), a box 100 times
    thinner than wide, a cluster 1e-3 across in a unit box (cells over nine
    decades of volume), a cubic lattice with one more point 1e-12 off a cube
    corner: the tessellation closes (volumes sum to the box) and equals the
    oracle's.  The last case is checked for closure only: there the oracle's
    own volumes sum to the box only to 1.5e-8 (its clipping tolerance meets
    the point 1e-12 off the corner), while the device closes it to rounding."""
    c, torch = ctx
    pos, box = _extreme(name)
    mesh, P, G = H.gpu_tessellate(c, torch, pos, box)
    H.check_incidence(G)
    assert abs(G["cell_volume"].sum() - np.prod(box)) <= 1e-12 * np.prod(box)
    assert np.all(G["cell_volume"] > 0)
    if name == "lattice_and_a_near_centred_point":
        return
    T = oracle.tessellate(pos, box, 0 if len(pos) <= 1100 else 1)
    # the cluster's outer cells reach 500 times their generators' spacing: their
    # vertices come from nearly parallel planes (condition numbers near 1e5), and
    # two FP64 computations of a face agree to 1e-8 of it there, not 1e-9
    rtol = 1e-8 if name == "tight_cluster_in_a_large_box" else H.GEOM_RTOL
    H.compare_tessellations(oracle, T, G, pos, box, geom_rtol=rtol, label=name)


def test_tessellation_is_deterministic(ctx):
    c, torch = ctx
    pos = WL.random_points(3000, seed=8)
    _, _, A = H.gpu_tessellate(c, torch, pos, np.ones(3))
    _, _, B = H.gpu_tessellate(c, torch, pos, np.ones(3))
    for k in A:
        np.testing.assert_array_equal(A[k], B[k])


@pytest.mark.parametrize("case", ["random_1001", "smooth_wave_16^3", "fcc_degenerate_vertices",
                                  "cubic_lattice_exact_ties", "shock_tube_64x8x8", "n5"])
def test_filtered_clipping_gives_the_same_mesh_bit_for_bit(ctx, case):
    """clip_filter=1 classifies with FP32 plus an error bound and falls back to
    the FP64 test only near ties, and re-solves every final vertex in FP64:
    the mesh must equal the direct FP64 clipper's (clip_filter=0) exactly."""
    c, torch = ctx
    pos, box = CASES[case]()
    c.set_config(clip_filter=0)
    try:
        _, _, A = H.gpu_tessellate(c, torch, pos, box)
    finally:
        c.set_config(clip_filter=1)
    _, _, B = H.gpu_tessellate(c, torch, pos, box)
    for k in A:
        np.testing.assert_array_equal(A[k], B[k], err_msg=k)


def test_counters(ctx):
    c, torch = ctx
    pos = WL.random_points(4000, seed=11)
    c.set_config(collect_stats=1, clip_filter=0)
    try:
        H.gpu_tessellate(c, torch, pos, np.ones(3))
        s0 = c.mm_tess_stats()
        c.set_config(clip_filter=1)
        H.gpu_tessellate(c, torch, pos, np.ones(3))
        s1 = c.mm_tess_stats()
    finally:
        c.set_config(collect_stats=0, clip_filter=1)
    assert s0["cuts"] == s1["cuts"] > 10 * 4000
    assert s0["fp64_plane_tests"] > 100 * s1["fp64_plane_tests"]
    assert s0["max_planes"] <= 64 and s0["max_vertices"] <= 128


def test_rejects_bad_positions(ctx):
    from paper_1707_05333_gb300.binding import MMError
    c, torch = ctx
    pos = WL.random_points(100, seed=10)
    pos[17, 1] = 1.0  # == box: outside [0, L)
    with pytest.raises(MMError) as e:
        H.gpu_tessellate(c, torch, pos, np.ones(3))
    assert e.value.status == 1
    pos[17, 1] = np.nan
    with pytest.raises(MMError):
        H.gpu_tessellate(c, torch, pos, np.ones(3))
    # the context stays usable
    pos[17, 1] = 0.5
    H.gpu_tessellate(c, torch, pos, np.ones(3))


def test_full_size_shear_layer_sampled_cells(oracle, ctx):
    """The bench workload (256^3 generators): sampled cells against the
    oracle computed one by one, plus the tiling invariant over all cells."""
    c, torch = ctx
    w = WL.shear_layer(256)
    mesh, P, G = H.gpu_tessellate(c, torch, w.pos, w.box)
    n = w.n
    assert abs(G["cell_volume"].sum() - 1.0) <= 1e-10
    H.check_incidence(G)
    rng = np.random.default_rng(0)
    cells = np.sort(rng.choice(n, 64, replace=False))
    T = oracle.tessellate(w.pos, w.box, cells=cells)
    scale = (1.0 / n) ** (2.0 / 3.0)
    np.testing.assert_allclose(G["cell_volume"][cells], T["volume"][cells], rtol=1e-9)
    np.testing.assert_allclose(G["cell_centroid"][:, cells].T, T["centroid"][cells], atol=1e-9 * np.sqrt(scale))
    # per sampled cell: the directed oracle faces equal the GPU incident faces
    # (topology exact above the drop threshold, areas to 1e-9 of each face's
    # own area, face centroids to 1e-9 of its own size)
    thr = H.AREA_REL * scale
    excuse = thr * (1.0 + H.GEOM_RTOL)
    off, inc = G["inc_off"], G["inc_face"]
    nband = 0
    for ci in cells:
        ent = inc[off[ci]:off[ci + 1]]
        got = {}
        for e in ent:
            if e >= 0:
                got[(int(G["face_j"][e]), int(G["face_shift"][e]))] = (G["face_area"][e], G["face_centroid"][:, e])
            else:
                f = ~e
                # the face seen from cell j: its centroid moves to j's frame
                code = int(G["face_shift"][f])
                s3 = np.array([code % 3 - 1, (code // 3) % 3 - 1, code // 9 - 1], dtype=float)
                got[(int(G["face_i"][f]), 26 - code)] = (G["face_area"][f], G["face_centroid"][:, f] - s3 * w.box)
        sel = np.nonzero(T["cell"] == ci)[0]
        want = {(int(T["nb"][k]), int(oracle.shift_code(T["shift"][k]))): (T["area"][k], T["fcentroid"][k])
                for k in sel}
        nband += sum(1 for a, _ in want.values() if thr < a <= 1e-8 * scale)
        for k, (a, cen) in want.items():
            if k not in got:
                assert a <= excuse, (ci, k, a / scale)
                continue
            ga, gc = got[k]
            assert abs(ga - a) <= H.GEOM_RTOL * a, (ci, k, abs(ga - a) / a)
            assert np.abs(gc - cen).max() <= H.GEOM_RTOL * np.sqrt(a), (ci, k)
        for k, (ga, _) in got.items():
            if k not in want:
                assert ga <= excuse, (ci, k, ga / scale)
    print(f"[256^3 sampled cells] faces in the band (1e-10, 1e-8] of (V/n)^(2/3): {nband}")


@pytest.mark.parametrize("warps,cap,scale,sort", [(2, 32, 0.8, 0), (8, 64, 1.5, 1), (1, 48, 1.25, 0),
                                                  (4, 64, 2.5, 0), (2, 64, 1.25, 1)])
def test_tunable_settings_keep_the_mesh(oracle, ctx, warps, cap, scale, sort):
    c, torch = ctx
    pos = WL.random_points(1500, seed=12)
    T = oracle.tessellate(pos, np.ones(3), 1)
    c.set_config(clip_warps=warps, cand_cap=cap, bin_scale=scale, clip_sort=sort)
    try:
        _, _, G = H.gpu_tessellate(c, torch, pos, np.ones(3))
    finally:
        c.set_config(clip_warps=2, cand_cap=64, bin_scale=1.0, clip_sort=0)
    H.compare_tessellations(oracle, T, G, pos, np.ones(3))
    H.check_incidence(G)


def test_candidate_sorts_give_the_same_mesh_bit_for_bit(ctx):
    """clip_sort 0 (shared memory) and 1 (registers) order more than 32
    buffered candidates the same way: uniform random points, where such
    batches are common, give the same mesh bit for bit."""
    c, torch = ctx
    pos = WL.random_points(20000, seed=14)
    c.set_config(collect_stats=1)
    try:
        _, _, A = H.gpu_tessellate(c, torch, pos, np.ones(3))
        assert c.mm_tess_stats()["max_candidates"] > 32
        c.set_config(clip_sort=1)
        _, _, B = H.gpu_tessellate(c, torch, pos, np.ones(3))
    finally:
        c.set_config(collect_stats=0, clip_sort=0)
    for k in A:
        np.testing.assert_array_equal(A[k], B[k], err_msg=k)


def test_autotune_picks_a_valid_setting(ctx):
    c, torch = ctx
    w = WL.shear_layer(24)
    P = H.to_dev(torch, w.pos.T)
    best = c.mm_autotune(P, w.box, reps=1)
    try:
        assert best["clip_warps"] in (2, 4, 8) and best["cand_cap"] in (32, 64)
        assert best["bin_scale"] in (0.8, 1.0, 1.25, 1.5) and best["tessellate_ms"] > 0
        assert best["clip_sort"] in (0, 1)
        mesh = c.mm_tessellate(P, w.box)
        assert mesh.nfaces > 0
    finally:
        c.set_config(clip_warps=2, cand_cap=64, bin_scale=1.0, clip_sort=0)


def test_rejects_bad_sizes_and_boxes(ctx):
    """n outside [1, MM_MAX_CELLS], non-positive box sizes and empty boxes of a
    batch are refused with MM_EINVAL before any device memory is touched, and
    the context stays usable."""
    import ctypes
    from paper_1707_05333_gb300 import binding
    c, torch = ctx
    pos = H.to_dev(torch, WL.random_points(64, seed=12).T)
    p = ctypes.c_void_p(pos.data_ptr())
    box = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    for n in (0, -5, 100_000_001):
        assert c.L.mm_tessellate(c.h, p, n, box, ctypes.byref(binding.MeshStruct())) == 1
    bad = (ctypes.c_double * 3)(1.0, 0.0, 1.0)
    assert c.L.mm_tessellate(c.h, p, 64, bad, ctypes.byref(binding.MeshStruct())) == 1
    # box sizes outside [MM_MIN_BOX, MM_MAX_BOX] = [2^-40, 2^40] (the clipper's FP32 bounds)
    for L in (2.0 ** -41, 2.0 ** 41, float("inf"), float("nan")):
        big = (ctypes.c_double * 3)(1.0, L, 1.0)
        assert c.L.mm_tessellate(c.h, p, 64, big, ctypes.byref(binding.MeshStruct())) == 1
    # a batch whose second box is empty
    off = (ctypes.c_int64 * 3)(0, 64, 64)
    boxes = (ctypes.c_double * 6)(1.0, 1.0, 1.0, 1.0, 1.0, 1.0)
    U = torch.zeros((5, 64), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = binding.Context(stream=stream)
        st = b.L.mm_step_batched(b.h, p, ctypes.c_void_p(U.data_ptr()), 64, off, boxes, 2, None)
        assert st == 1
        b.close()
    _, _, G = H.gpu_tessellate(c, torch, WL.random_points(64, seed=12), np.ones(3))
    assert abs(G["cell_volume"].sum() - 1.0) < 1e-12


@pytest.mark.parametrize("k", [-36, -12, 12, 36])
def test_power_of_two_scaled_box_gives_the_scaled_mesh(ctx, k):
    """Positions and box scaled by 2^k (within [2^-40, 2^40]): every FP64 and
    FP32 operation of the tessellation scales exactly, so the mesh is the unit
    box's with areas times 4^k, volumes times 8^k and centroids times 2^k.
    Pins the scale handling of the FP32 bounds (bins, coverage radius,
    security limit)."""
    c, torch = ctx
    pos = WL.random_points(700, box=(1.0, 0.5, 2.0), seed=21)
    box = np.array([1.0, 0.5, 2.0])
    _, _, A = H.gpu_tessellate(c, torch, pos, box)
    s = 2.0 ** k
    _, _, B = H.gpu_tessellate(c, torch, pos * s, box * s)
    for key in ("face_i", "face_j", "face_shift", "inc_off", "inc_face"):
        np.testing.assert_array_equal(A[key], B[key], err_msg=key)
    np.testing.assert_allclose(B["cell_volume"], A["cell_volume"] * s ** 3, rtol=1e-14, atol=0)
    np.testing.assert_allclose(B["face_area"], A["face_area"] * s ** 2, rtol=1e-14, atol=0)
    np.testing.assert_allclose(B["cell_centroid"], A["cell_centroid"] * s, rtol=1e-14, atol=0)
    np.testing.assert_allclose(B["face_normal"], A["face_normal"], rtol=1e-14, atol=1e-15)
