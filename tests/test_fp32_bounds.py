"""The FP32 bounds the kernels rely on, checked by emulating their FP32
arithmetic on the host (numpy float32, one rounding per operation, which is
never better than the kernels' fused multiply-adds) against FP64.

* The gradient limiter screens Delta = g . d in FP32 and trusts the FP32
  leader when it beats the runner-up by more than 2 B with
  B = 8e-7 |g|_1 max_j |d_j|_1 (+ 1e-36): every FP32 Delta must then lie
  within B of the FP64 one.
* The clipper's home-bin wall distances and ring coverage radius are FP32,
  lowered by a slack of 2e-6 max(L): the lowered values must never exceed the
  exact ones.
* The clipper's FP32 candidate filter keeps every neighbour image the exact
  security-radius test keeps.
* The clipper's FP32 vertices carry an error bound err, and its FP32 plane
  tests a bound B built on it: err must bound the distance to the exact
  vertex, B the error of the test value, and every sign B settles must be
  the exact test's (tie margin included)."""
import numpy as np

U32 = np.float32


def test_limiter_screening_error_bound():
    rng = np.random.default_rng(1707)
    worst = 0.0
    for scale_g, scale_d in ((1.0, 1.0), (1e-6, 1e3), (1e8, 1e-9), (3.0, 2.0 ** -20)):
        g = rng.normal(size=(20000, 3)) * scale_g * rng.uniform(0.01, 1.0, (20000, 1))
        d = rng.normal(size=(20000, 3)) * scale_d * rng.uniform(0.01, 1.0, (20000, 1))
        g32, d32 = g.astype(U32), d.astype(U32)
        # fmaf(g0, dx, fmaf(g1, dy, g2 * dz)) with separate roundings
        t = (g32[:, 2] * d32[:, 2]).astype(U32)
        t = (g32[:, 1] * d32[:, 1] + t).astype(U32)
        del32 = (g32[:, 0] * d32[:, 0] + t).astype(U32).astype(np.float64)
        del64 = g[:, 0] * d[:, 0] + g[:, 1] * d[:, 1] + g[:, 2] * d[:, 2]
        g1 = np.abs(g32.astype(np.float64)).sum(axis=1)
        d1 = np.abs(d32.astype(np.float64)).sum(axis=1)
        B = 8e-7 * g1 * d1 + 1e-36
        err = np.abs(del32 - del64)
        assert np.all(err <= B), np.max(err / B)
        worst = max(worst, float(np.max(err / B)))
    # the margin is real: the worst case uses well under half the bound
    assert worst < 0.5, worst


def test_clipper_wall_distances_stay_conservative():
    rng = np.random.default_rng(1708)
    for L in (1.0, 8.0, 2.0 ** -30, 2.0 ** 30, 0.37):
        for g in (1, 7, 64, 256, 4096):
            bs = L / g
            p = rng.uniform(0.0, L, 20000)
            p = p[p < L]
            pf = p.astype(U32)
            ibsf, bsf = U32(g / L), U32(bs)
            cb = np.clip(np.floor(pf * ibsf).astype(np.int64), 0, g - 1)
            slack = U32(2e-6) * U32(L)
            lo32 = (pf - (cb.astype(U32) * bsf).astype(U32)).astype(U32)
            hi32 = (((cb + 1).astype(U32) * bsf).astype(U32) - pf).astype(U32)
            edge32 = (np.minimum(lo32, hi32) - slack).astype(np.float64)
            # exact distances from p to the walls of bin cb (cb may differ from
            # p's true bin by one at a boundary: the distance is then negative)
            lo = p - cb * bs
            hi = (cb + 1) * bs - p
            assert np.all(edge32 <= np.minimum(lo, hi)), L
            # ring r covers radius edge + r bs; the FP32 form, lowered, never exceeds it
            for r in (1, 2, 5):
                R32 = (edge32.astype(U32) + U32(r) * bsf).astype(np.float64)
                assert np.all(R32 * (1 - 1e-6) <= np.minimum(lo, hi) + r * bs), (L, g, r)


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(U32)


def _fma(a, b, c):
    # a * b is exact in FP64 for FP32 a, b; one rounding to FP32 after the add
    return _f32(a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64))


def _mul(a, b):
    return _f32(a.astype(np.float64) * b.astype(np.float64))


def _vertex32(qa, oa, qb, ob, qc, oc):
    """The clipper's FP32 vertex of three planes q.v = o (Cramer's rule with
    fused multiply-adds and a correctly rounded reciprocal) and its error
    bound err = 3 u H (5.5 (|qa| + |qb| + |qc|) + 13 |v|_1), H = |qa||qb||qc| /
    |det|; +inf where the kernel solves in FP64 instead."""
    (ax, ay, az), (bx, by, bz), (cx, cy, cz) = (_f32(q).T for q in (qa, qb, qc))
    ao, bo, co = _f32(oa), _f32(ob), _f32(oc)
    bcx, bcy, bcz = _fma(by, cz, -_mul(bz, cy)), _fma(bz, cx, -_mul(bx, cz)), _fma(bx, cy, -_mul(by, cx))
    cax, cay, caz = _fma(cy, az, -_mul(cz, ay)), _fma(cz, ax, -_mul(cx, az)), _fma(cx, ay, -_mul(cy, ax))
    abx, aby, abz = _fma(ay, bz, -_mul(az, by)), _fma(az, bx, -_mul(ax, bz)), _fma(ax, by, -_mul(ay, bx))
    det = _fma(ax, bcx, _fma(ay, bcy, _mul(az, bcz)))
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        inv = _f32(1.0 / det.astype(np.float64))
        x = _mul(_fma(ao, bcx, _fma(bo, cax, _mul(co, abx))), inv)
        y = _mul(_fma(ao, bcy, _fma(bo, cay, _mul(co, aby))), inv)
        z = _mul(_fma(ao, bcz, _fma(bo, caz, _mul(co, abz))), inv)
        la, lb, lc = (np.sqrt(_mul(U32(2.0), o)) for o in (ao, bo, co))
        H = _mul(_mul(_mul(la, lb), lc), np.abs(inv))
        vn = np.abs(x) + np.abs(y) + np.abs(z)
        u = U32(5.9604645e-8)
        err = _mul(_mul(_mul(U32(3.0), u), H), U32(5.5) * (la + lb + lc) + U32(13.0) * vn)
        ok = (u * H < U32(1e-3)) & (err < U32(1e30)) & (np.minimum(np.minimum(la, lb), lc) >= U32(3.7252903e-9)) \
            & (np.maximum(np.maximum(la, lb), lc) <= U32(268435456.0))
    return np.stack([x, y, z], 1), np.where(ok, err, np.inf)


def test_clipper_vertex_and_plane_test_bounds():
    """The filtered clipper classifies a vertex against a plane in FP32 and
    trusts the sign of s = q.v - o only beyond its bound B = |q| err +
    16 u (|q_x v_x| + |q_y v_y| + |q_z v_z| + o).  Emulated here: the FP32
    vertex of three bisector planes and its err must bound the distance to
    the exact vertex, B the error of s, and every sign B settles must be
    the exact test's, the kernel's tie margin (2^13 units in the last place
    of o) included; the FP32 bound of |v|^2 the security radius uses must not
    fall below the exact one.  Planes are bisectors of neighbours at distances 0.3..3
    (o = |q|^2 / 2), some nearly parallel (ill-conditioned), at scales
    2^-20, 1 and 2^20."""
    rng = np.random.default_rng(1709)
    m = 40000
    worst_v, worst_s, settled = 0.0, 0.0, 0
    for scale in (2.0 ** -20, 1.0, 2.0 ** 20):
        def planes():
            d = rng.normal(size=(m, 3))
            d /= np.linalg.norm(d, axis=1, keepdims=True)
            return d * rng.uniform(0.3, 3.0, (m, 1)) * scale
        qa, qb, qc = planes(), planes(), planes()
        near = rng.random(m) < 0.3  # nearly parallel third plane
        qc[near] = qb[near] * (1.0 + 1e-3 * rng.normal(size=(near.sum(), 1))) + 1e-3 * scale * rng.normal(
            size=(near.sum(), 3))
        o = [0.5 * (q * q).sum(1) for q in (qa, qb, qc)]
        v32, err = _vertex32(qa, o[0], qb, o[1], qc, o[2])
        keep = np.isfinite(err)
        A = np.stack([qa, qb, qc], 1)[keep]
        v = np.linalg.solve(A, np.stack(o, 1)[keep][..., None])[..., 0]
        dv = np.linalg.norm(v32[keep].astype(np.float64) - v, axis=1)
        assert np.all(dv <= err[keep]), np.max(dv / err[keep])
        worst_v = max(worst_v, float(np.max(dv / err[keep])))
        # the security radius takes |v|^2 from the FP32 bound (|v| + err)^2 <=
        # |v|^2 + err (2 |v|_1 + err), widened by 1e-5: never below the exact one
        x, y, z = v32[keep].T
        e = err[keep]
        s2 = _fma(x, x, _fma(y, y, _mul(z, z)))
        l1 = np.abs(x) + np.abs(y) + np.abs(z)
        nr2 = _mul(_fma(e, _fma(U32(2.0) * np.ones_like(l1), l1, e), s2), U32(1.00001)).astype(np.float64)
        assert np.all(nr2 >= (v * v).sum(1)), np.min(nr2 / (v * v).sum(1))
        # test planes against the kept vertices
        qt = planes()[keep]
        ot = 0.5 * (qt * qt).sum(1)
        fq, fo = _f32(qt), _f32(ot)
        V = v32[keep]
        s32 = _fma(fq[:, 0], V[:, 0], _fma(fq[:, 1], V[:, 1], _fma(fq[:, 2], V[:, 2], -fo))).astype(np.float64)
        mag = (np.abs(_mul(fq[:, 0], V[:, 0])) + np.abs(_mul(fq[:, 1], V[:, 1])) + np.abs(_mul(fq[:, 2], V[:, 2]))
               + fo).astype(np.float64)
        fqn = (np.sqrt(_mul(U32(2.0), fo)) * U32(1.0000005)).astype(np.float64)
        B = fqn * err[keep].astype(np.float64) + 16.0 * 5.9604645e-8 * mag
        s = (qt * v).sum(1) - ot
        assert np.all(np.abs(s32 - s) <= B), np.max(np.abs(s32 - s) / B)
        worst_s = max(worst_s, float(np.max(np.abs(s32 - s) / B)))
        margin = np.spacing(ot) * 2.0 ** 13
        beyond, inside = s32 > B * 1.00001, s32 < -B
        assert np.all(s[beyond] > margin[beyond]) and np.all(s[inside] <= margin[inside])
        settled += int(beyond.sum() + inside.sum())
    print(f"[clipper bounds] worst |dv|/err {worst_v:.2f}, worst |ds|/B {worst_s:.2f}, {settled} tests settled in FP32")
    assert settled > 0.9 * 3 * m * 0.5


def test_clipper_candidate_filter_keeps_every_candidate_the_exact_test_keeps():
    """The clipper gathers candidates with an FP32 |q|^2 (the FP32 copy of the
    neighbour's position plus the FP32 image offset s L - p of the cell's
    generator) against limk = 4 m (1 + 1e-5) + 2e-6 max(L) sqrt(4 m), m the
    FP32 bound of the largest |v|^2; the exact test keeps |q|^2 <= 4 m.  At
    the tightest case, an exact |q|^2 just inside 4 m, the FP32 filter must
    keep it: separations from L/512 to L, image shifts of -1, 0, 1, boxes of
    several shapes and scales."""
    rng = np.random.default_rng(1710)
    n = 200000
    worst = 0.0
    for L in (np.array([1.0, 1.0, 1.0]), np.array([1.0, 0.5, 2.0]), 2.0 ** 20 * np.array([1.0, 1.0, 0.25]),
              2.0 ** -20 * np.array([3.0, 1.0, 1.0])):
        Lmax = L.max()
        p_i = rng.uniform(0.0, 1.0, (n, 3)) * L
        shift = rng.integers(-1, 2, (n, 3))
        # neighbour positions that put the exact separation at random lengths L/512..L
        d = rng.normal(size=(n, 3))
        d *= (Lmax * np.exp(rng.uniform(np.log(1.0 / 512), 0.0, (n, 1)))) / np.linalg.norm(d, axis=1, keepdims=True)
        p_j = p_i + d - shift * L
        ok = np.all((p_j >= 0.0) & (p_j < L), axis=1)
        assert ok.sum() > 5000, ok.sum()
        p_i, p_j, shift = p_i[ok], p_j[ok], shift[ok]
        q = p_j + shift * L - p_i  # the exact separation of the candidate image
        d2 = (q * q).sum(1)
        m = _f32(d2 / 4.0)
        m = np.where(4.0 * m.astype(np.float64) < d2, np.nextafter(m, U32(np.inf)), m)  # smallest FP32 with d2 <= 4 m
        off = _f32(shift * L - p_i)
        q32 = _f32(_f32(p_j).astype(np.float64) + off.astype(np.float64))
        d2f = _fma(q32[:, 0], q32[:, 0], _fma(q32[:, 1], q32[:, 1], _mul(q32[:, 2], q32[:, 2])))
        m4 = _mul(U32(4.0), m)
        slack = _f32(2e-6 * Lmax)
        limk = _fma(m4, U32(1.00001) * np.ones_like(m4), _mul(slack * np.ones_like(m4), np.sqrt(m4)))
        assert np.all(d2f <= limk), np.max(d2f.astype(np.float64) - limk)
        worst = max(worst, float(np.max((d2f.astype(np.float64) - 4.0 * m) / (limk.astype(np.float64) - 4.0 * m))))
    print(f"[candidate filter] worst use of the margin {worst:.2f}")
    assert worst < 1.0
