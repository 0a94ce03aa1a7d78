"""The FP32 bounds the kernels rely on, checked by emulating their FP32
arithmetic on the host (numpy float32, one rounding per operation, which is
never better than the kernels' fused multiply-adds) against FP64.

* The gradient limiter screens Delta = g . d in FP32 and trusts the FP32
  leader when it beats the runner-up by more than 2 B with
  B = 8e-7 |g|_1 max_j |d_j|_1 (+ 1e-36): every FP32 Delta must then lie
  within B of the FP64 one.
* The clipper's home-bin wall distances and ring coverage radius are FP32,
  lowered by a slack of 2e-6 max(L): the lowered values must never exceed the
  exact ones."""
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
