"""Pins of the oracle's Voronoi tessellation (Sec. 3) against closed forms and
geometric invariants that do not depend on the oracle's own formulas."""
import math

import numpy as np
import pytest

from paper_1707_05333_gb300 import workloads as WL


def lattice(kind, m, a=1.0):
    """Points of a cubic, BCC or FCC lattice with m^3 conventional cells of side a/m."""
    s = a / m
    basis = {"sc": [(0, 0, 0)],
             "bcc": [(0, 0, 0), (0.5, 0.5, 0.5)],
             "fcc": [(0, 0, 0), (0.5, 0.5, 0), (0.5, 0, 0.5), (0, 0.5, 0.5)]}[kind]
    pts = []
    for k in range(m):
        for j in range(m):
            for i in range(m):
                for b in basis:
                    pts.append(((i + b[0] + 0.25) * s, (j + b[1] + 0.25) * s, (k + b[2] + 0.25) * s))
    return np.array(pts), s


def per_cell_faces(T):
    out = {}
    for k in range(len(T["area"])):
        out.setdefault(int(T["cell"][k]), []).append(k)
    return out


@pytest.mark.parametrize("mode", [0, 1])
def test_cubic_lattice_closed_form(oracle, mode):
    pos, h = lattice("sc", 4)
    T = oracle.tessellate(pos, np.ones(3), mode)
    np.testing.assert_allclose(T["volume"], h ** 3, rtol=1e-13)
    np.testing.assert_allclose(T["centroid"], pos, atol=1e-14)
    faces = per_cell_faces(T)
    for i in range(len(pos)):
        ks = faces[i]
        assert len(ks) == 6
        np.testing.assert_allclose(T["area"][ks], h * h, rtol=1e-13)
        # normals are the six axis directions
        nrm = np.round(T["normal"][ks]).astype(int)
        assert sorted(map(tuple, nrm)) == sorted([(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0),
                                                  (0, 0, 1), (0, 0, -1)])


def test_bcc_truncated_octahedra(oracle):
    pos, a = lattice("bcc", 3)
    T = oracle.tessellate(pos, np.ones(3), 1)
    np.testing.assert_allclose(T["volume"], a ** 3 / 2, rtol=1e-12)
    faces = per_cell_faces(T)
    hexa = 3 * math.sqrt(3) * a * a / 16
    square = a * a / 8
    for i in range(len(pos)):
        areas = np.sort(T["area"][faces[i]])
        assert len(areas) == 14
        np.testing.assert_allclose(areas[:6], square, rtol=1e-12)
        np.testing.assert_allclose(areas[6:], hexa, rtol=1e-12)


def test_fcc_rhombic_dodecahedra(oracle):
    pos, a = lattice("fcc", 2)
    T = oracle.tessellate(pos, np.ones(3), 0)
    np.testing.assert_allclose(T["volume"], a ** 3 / 4, rtol=1e-12)
    faces = per_cell_faces(T)
    for i in range(len(pos)):
        assert len(faces[i]) == 12
        np.testing.assert_allclose(T["area"][faces[i]], math.sqrt(2) * a * a / 8, rtol=1e-12)


def check_invariants(T, pos, box, tol=1e-9):
    # tol bounds the per-cell sums, which may lose faces below the 1e-10
    # relative area threshold; per-face properties are held to 1e-12.
    n = len(pos)
    vol = T["volume"]
    # the cells tile the periodic box
    assert abs(vol.sum() - np.prod(box)) <= tol * np.prod(box)
    faces = per_cell_faces(T)
    key = {}
    for k in range(len(T["area"])):
        key[(int(T["cell"][k]), int(T["nb"][k]), tuple(T["shift"][k]))] = k
    for i in range(n):
        ks = faces[i]
        A = T["area"][ks]
        nrm = T["normal"][ks]
        fc = T["fcentroid"][ks]
        scale = vol[i] ** (2.0 / 3.0)
        # closed surface: sum A n = 0
        assert np.all(np.abs((A[:, None] * nrm).sum(0)) <= tol * scale)
        # divergence theorem: V = 1/3 sum A n.(x_f - r_i), and
        # sum A n (x) (x_f - c_i) = V I (first moment about the centroid)
        rel = fc - pos[i]
        assert abs((A * np.sum(nrm * rel, axis=1)).sum() / 3.0 - vol[i]) <= tol * vol[i]
        mom = (A[:, None, None] * nrm[:, :, None] * (fc - T["centroid"][i])[:, None, :]).sum(0)
        np.testing.assert_allclose(mom, vol[i] * np.eye(3), atol=tol * 10 * vol[i])
        # the normal of a face is the direction to the neighbour's image
        for k in ks:
            j = int(T["nb"][k])
            q = pos[j] + T["shift"][k] * box - pos[i]
            np.testing.assert_allclose(T["normal"][k], q / np.linalg.norm(q), atol=1e-14)
            # the face lies on the bisector plane
            assert abs(np.dot(T["fcentroid"][k] - pos[i], q) - 0.5 * np.dot(q, q)) <= 1e-12 * np.dot(q, q)
            # and is seen from the other side with equal area, opposite normal
            m = key[(j, i, tuple(-T["shift"][k]))]
            assert abs(T["area"][m] - T["area"][k]) <= 1e-12 * scale
            np.testing.assert_allclose(T["normal"][m], -T["normal"][k], atol=1e-14)
            np.testing.assert_allclose(T["fcentroid"][m], T["fcentroid"][k] - T["shift"][k] * box,
                                       atol=1e-12)


def test_invariants_jittered_lattice(oracle):
    w = WL.smooth_wave(6)
    T = oracle.tessellate(w.pos, w.box, 1)
    check_invariants(T, w.pos, w.box)


def test_invariants_random_points(oracle):
    pos = WL.random_points(300, seed=1)
    T = oracle.tessellate(pos, np.ones(3), 1)
    check_invariants(T, pos, np.ones(3))


def test_invariants_elongated_box(oracle):
    w = WL.shock_tube(32, 4, 4)
    T = oracle.tessellate(w.pos, w.box, 1)
    check_invariants(T, w.pos, w.box)


@pytest.mark.parametrize("maker", ["lattice", "random", "tube"])
def test_bruteforce_equals_grid(oracle, maker):
    if maker == "lattice":
        w = WL.smooth_wave(6)
        pos, box = w.pos, w.box
    elif maker == "random":
        pos, box = WL.random_points(250, seed=2), np.ones(3)
    else:
        w = WL.shock_tube(16, 3, 3)
        pos, box = w.pos, w.box
    A = oracle.tessellate(pos, box, 0)
    B = oracle.tessellate(pos, box, 1)
    np.testing.assert_array_equal(A["cell"], B["cell"])
    np.testing.assert_array_equal(A["nb"], B["nb"])
    np.testing.assert_array_equal(A["shift"], B["shift"])
    np.testing.assert_allclose(A["area"], B["area"], rtol=1e-14)
    np.testing.assert_allclose(A["volume"], B["volume"], rtol=1e-14)


def test_single_generator_is_the_box(oracle):
    box = np.array([2.0, 1.0, 0.5])
    T = oracle.tessellate(np.array([[0.3, 0.7, 0.1]]), box, 0)
    assert T["volume"][0] == pytest.approx(1.0, rel=1e-14)
    F = oracle.unique_faces(T)
    # three shared faces, each the cell's contact with its own image
    assert len(F["area"]) == 3
    np.testing.assert_allclose(np.sort(F["area"]), [0.5, 1.0, 2.0], rtol=1e-14)
    assert np.all(F["i"] == 0) and np.all(F["j"] == 0)


def test_two_generators(oracle):
    # two points on the x axis of a unit box: two slabs of width 1/2 in x
    pos = np.array([[0.1, 0.5, 0.5], [0.6, 0.5, 0.5]])
    T = oracle.tessellate(pos, np.ones(3), 0)
    np.testing.assert_allclose(T["volume"], [0.5, 0.5], rtol=1e-14)
    F = oracle.unique_faces(T)
    pair = F["area"][(F["i"] == 0) & (F["j"] == 1)]
    np.testing.assert_allclose(np.sort(pair), [1.0, 1.0], rtol=1e-14)


def test_rejects_positions_outside_box(oracle):
    with pytest.raises(oracle.OracleError):
        oracle.tessellate(np.array([[1.0, 0.5, 0.5], [0.2, 0.2, 0.2]]), np.ones(3), 0)
    with pytest.raises(oracle.OracleError):
        oracle.tessellate(np.array([[np.nan, 0.5, 0.5]]), np.ones(3), 0)
