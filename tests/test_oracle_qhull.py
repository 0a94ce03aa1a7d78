"""The oracle's periodic Voronoi cells (Sec. 3) against Qhull's.

Qhull builds the Voronoi diagram by another algorithm altogether: the
Delaunay triangulation as the lower convex hull of the points lifted onto a
paraboloid, the Voronoi vertices as the tetrahedra's circumcentres.  The
periodic box is unrolled into its 27 images; the cells of the central image
are then bounded, and each one is the oracle's cell of that generator.
Compared: the set of (cell, neighbour, image shift) faces, every face's area
and centroid, every cell's volume and centroid.  A dropped or extra face, a
wrong clipping plane, a wrong shift or a wrong polygon sum fails here
without any of the oracle's own formulas being used."""
import numpy as np
import pytest

from paper_1707_05333_gb300 import workloads as WL

spatial = pytest.importorskip("scipy.spatial")

SHIFTS = np.array([(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)])
CENTRE = 13  # index of the (0, 0, 0) image in SHIFTS


def _polygon(P, normal):
    """Area and centroid of a convex planar polygon given its vertices in any
    order: sorted by angle about their mean in the plane, then summed as a
    fan of triangles from the mean."""
    m = P.mean(axis=0)
    u = P[np.argmax(np.linalg.norm(P - m, axis=1))] - m
    u /= np.linalg.norm(u)
    v = np.cross(normal, u)
    ang = np.arctan2((P - m) @ v, (P - m) @ u)
    Q = P[np.argsort(ang)]
    R = np.roll(Q, -1, axis=0)
    a = 0.5 * np.linalg.norm(np.cross(Q - m, R - m), axis=1)
    area = a.sum()
    cen = (a[:, None] * (m + Q + R) / 3.0).sum(0) / area if area > 0 else m
    return area, cen


def _polyhedron(V):
    """Volume and centroid of the convex hull of V, as tetrahedra from the
    vertices' mean to Qhull's hull triangles."""
    hull = spatial.ConvexHull(V)
    o = V.mean(axis=0)
    A, B, C = (V[hull.simplices[:, k]] for k in range(3))
    w = np.abs(np.einsum("ij,ij->i", A - o, np.cross(B - o, C - o))) / 6.0
    vol = w.sum()
    return vol, (w[:, None] * (o + A + B + C) / 4.0).sum(0) / vol


def qhull_cells(pos, box):
    n = len(pos)
    pts = (pos[None, :, :] + SHIFTS[:, None, :] * box).reshape(-1, 3)
    vor = spatial.Voronoi(pts)
    vol = np.zeros(n)
    cen = np.zeros((n, 3))
    for i in range(n):
        reg = vor.regions[vor.point_region[CENTRE * n + i]]
        assert -1 not in reg, "a central cell reaches infinity: too few images"
        vol[i], cen[i] = _polyhedron(vor.vertices[reg])
    faces = {}
    for (p, q), rv in zip(vor.ridge_points, vor.ridge_vertices):
        for a, b in ((p, q), (q, p)):
            if a // n != CENTRE:
                continue
            assert -1 not in rv
            d = pts[b] - pts[a]
            area, fc = _polygon(vor.vertices[rv], d / np.linalg.norm(d))
            faces[(int(a % n), int(b % n), tuple(int(s) for s in SHIFTS[b // n]))] = (area, fc)
    return vol, cen, faces


def _min_image(d, box):
    return d - box * np.round(d / box)


def _lattice(kind, m, offset, jitter=0.0):
    """Cubic, BCC or FCC lattice of m^3 conventional cells in the unit box,
    shifted by `offset` spacings (inexact in binary), optionally perturbed
    by `jitter` spacings: every Voronoi vertex is shared by more cells than
    three planes define, the ties the clipper has to settle."""
    s = 1.0 / m
    basis = {"sc": [(0, 0, 0)], "bcc": [(0, 0, 0), (0.5, 0.5, 0.5)],
             "fcc": [(0, 0, 0), (0.5, 0.5, 0), (0.5, 0, 0.5), (0, 0.5, 0.5)]}[kind]
    p = np.array([((i + b[0] + offset) * s, (j + b[1] + offset) * s, (k + b[2] + offset) * s)
                  for k in range(m) for j in range(m) for i in range(m) for b in basis])
    if jitter:
        p = p + jitter * s * np.random.default_rng(3).standard_normal(p.shape)
    p = p % 1.0
    return np.where(p >= 1.0, 0.0, p), np.ones(3)


CASES = {
    "uniform_unit_box": lambda: (WL.random_points(200, seed=11), np.ones(3)),
    "uniform_flat_box": lambda: (WL.random_points(150, box=(2.0, 1.0, 0.5), seed=12),
                                 np.array([2.0, 1.0, 0.5])),
    "jittered_lattice": lambda: (WL.smooth_wave(5).pos, WL.smooth_wave(5).box),
    "clustered": lambda: (WL.clustered_points(400, seed=13), np.ones(3)),
    "cubic_5_offset_0.1": lambda: _lattice("sc", 5, 0.1),
    "bcc_4_offset_0.3": lambda: _lattice("bcc", 4, 0.3),
    "fcc_3_offset_0.1": lambda: _lattice("fcc", 3, 0.1),
    "cubic_6_jitter_1e-11": lambda: _lattice("sc", 6, 0.25, 1e-11),
    "fcc_3_jitter_1e-11": lambda: _lattice("fcc", 3, 0.0, 1e-11),
    # 80 of the 512 points of a grid of eighths: many cospherical ties, irregular cells
    "grid_eighths_subset": lambda: (np.random.default_rng(14).permutation(
        np.stack(np.meshgrid(*[np.arange(8) / 8.0] * 3, indexing="ij"), -1).reshape(-1, 3))[:80], np.ones(3)),
}


def mismatches(T, pos, box, qhull, area_rel):
    """Every way the oracle's tessellation T differs from Qhull's cells:
    volumes beyond 1e-9 relative, cell centroids beyond 1e-9 of the mean
    spacing h, faces above twice the drop threshold area_rel h^2 present on
    one side only (nearer the threshold rounding may keep a face on one side
    only), face areas beyond 1e-9 relative, face centroids beyond 1e-9 of the
    face's own size."""
    vq, cq, fq = qhull
    n = len(pos)
    h = (np.prod(box) / n) ** (1.0 / 3.0)
    out = []
    bad = np.flatnonzero(np.abs(T["volume"] - vq) > 1e-9 * vq)
    out += [f"volume of cell {i}" for i in bad[:5]]
    bad = np.flatnonzero(np.abs(_min_image(T["centroid"] - cq, box)).max(axis=1) > 1e-9 * h)
    out += [f"centroid of cell {i}" for i in bad[:5]]
    thr = 2.0 * area_rel * h * h
    fo = {(int(T["cell"][k]), int(T["nb"][k]), tuple(int(s) for s in T["shift"][k])): k
          for k in range(len(T["area"]))}
    big_q = {key for key, (a, _) in fq.items() if a > thr}
    big_o = {key for key, k in fo.items() if T["area"][k] > thr}
    out += [f"face {key} only in Qhull" for key in sorted(big_q - set(fo))[:5]]
    out += [f"face {key} only in the oracle" for key in sorted(big_o - set(fq))[:5]]
    for key in sorted(big_q & set(fo)):
        k = fo[key]
        a, fc = fq[key]
        if abs(T["area"][k] - a) > 1e-9 * a:
            out.append(f"area of face {key}")
        if np.linalg.norm(T["fcentroid"][k] - fc) > 1e-9 * np.sqrt(a):
            out.append(f"centroid of face {key}")
    return out, len(big_q), len(fq) - len(big_q), len(fo) - len(big_o)


@pytest.mark.parametrize("mode", [0, 1], ids=["brute", "grid"])
@pytest.mark.parametrize("case", list(CASES))
def test_cells_equal_qhull_voronoi_of_the_unrolled_box(oracle, case, mode):
    pos, box = CASES[case]()
    T = oracle.tessellate(pos, box, mode)
    bad, nf, sq, so = mismatches(T, pos, box, qhull_cells(pos, box), oracle.AREA_REL)
    print(f"[qhull {case} mode {mode}] {len(pos)} cells, {nf} faces above 2e-10 h^2, "
          f"{sq} Qhull slivers, {so} oracle slivers")
    assert not bad, bad[:10]


def _planted(T, what, box):
    """A copy of the oracle's output with one plausible mistake in it."""
    T = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in T.items()}
    k = int(np.argmax(T["area"]))
    if what == "dropped_face":
        keep = np.arange(len(T["area"])) != k
        for key in ("cell", "nb", "shift", "area", "normal", "fcentroid"):
            T[key] = T[key][keep]
    elif what == "wrong_shift":
        T["shift"][k] = -T["shift"][k] if np.any(T["shift"][k]) else np.array([1, 0, 0])
    elif what == "swapped_neighbour":
        T["nb"][k] = (T["nb"][k] + 1) % T["n"]
    elif what == "area_off_by_1e-8":
        T["area"][k] *= 1.0 + 1e-8
    elif what == "face_centroid_moved":
        T["fcentroid"][k] += 1e-8 * np.sqrt(T["area"][k])
    elif what == "volume_off_by_1e-8":
        T["volume"][3] *= 1.0 + 1e-8
    elif what == "centroid_in_the_wrong_image":
        T["centroid"][5] += 0.5 * box
    return T


@pytest.mark.parametrize("what", ["dropped_face", "wrong_shift", "swapped_neighbour", "area_off_by_1e-8",
                                  "face_centroid_moved", "volume_off_by_1e-8",
                                  "centroid_in_the_wrong_image"])
def test_the_comparison_sees_a_planted_mistake(oracle, what):
    pos, box = CASES["uniform_flat_box"]()
    T = oracle.tessellate(pos, box, 1)
    Q = qhull_cells(pos, box)
    assert not mismatches(T, pos, box, Q, oracle.AREA_REL)[0]
    assert mismatches(_planted(T, what, box), pos, box, Q, oracle.AREA_REL)[0]


def _fuzz_set(rng):
    """One random point set: uniform, with coordinates on the box walls,
    rounded to a grid of eighths (cospherical ties), or clustered, in a box
    of aspect ratio up to 10."""
    n = int(rng.integers(3, 120))
    box = np.exp(rng.uniform(np.log(0.3), np.log(3.0), 3))
    kind = int(rng.integers(0, 4))
    pos = rng.uniform(0.0, 1.0, (n, 3)) * box
    if kind == 1:
        pos[rng.random((n, 3)) < 0.2] = 0.0
    elif kind == 2:
        pos = np.unique(np.round(pos / box * 8.0) / 8.0 * box, axis=0)
    elif kind == 3:
        pos = (rng.uniform(0.0, 1.0, 3) * box + rng.normal(0.0, 0.05, (n, 3)) * box) % box
    pos = np.unique(np.where(pos >= box, 0.0, pos), axis=0)
    return pos, box


@pytest.mark.slow
def test_seeded_fuzz_against_qhull(oracle):
    rng = np.random.default_rng(2024)
    runs = 0
    while runs < 150:
        pos, box = _fuzz_set(rng)
        if len(pos) < 2:
            continue
        T = oracle.tessellate(pos, box, 1)
        bad = mismatches(T, pos, box, qhull_cells(pos, box), oracle.AREA_REL)[0]
        assert not bad, (pos.tolist(), box.tolist(), bad[:5])
        runs += 1
