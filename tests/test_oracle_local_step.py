"""The oracle's local one-step sub-problem (rings 0..3 of a few cells, used
to check sampled cells of the full-size benchmark box) equals the oracle's
whole-box step on the same cells."""
import numpy as np
import pytest

from paper_1707_05333_gb300 import workloads as WL
from tests import helpers as H

CASES = {
    "S10": dict(limiter=1),
    "DM_roundness": dict(limiter=2, regularize=1),
    "face_centroid_limiter": dict(limiter=3),
    "HLL_entropy_switch": dict(limiter=1, riemann=1, entropy=1, mach_th=1.1),
}


@pytest.mark.parametrize("case", list(CASES))
def test_local_step_equals_the_whole_box_step(oracle, case):
    kw = CASES[case]
    ent = bool(kw.get("entropy", 0))
    w = WL.shear_layer(18)
    rho, vel, pres = WL.random_state(w.n, seed=len(case))
    U = oracle.charges_from_prims(np.full(w.n, 1.0 / w.n), rho, vel, pres, w.gamma, entropy=ent)
    cfg = oracle.make_cfg(gamma=w.gamma, cfl=w.cfl, **kw)
    S = oracle.step(w.pos, U, w.box, cfg, dt=1e-3)
    cells = np.array([0, 17, 2024, 3333, w.n - 1])
    Ul, pl, wl, m = H.oracle_local_step(oracle, w.pos, U, w.box, cfg, cells, 1e-3)
    assert m < w.n
    scale = np.abs(S["U"]).max(axis=0)
    np.testing.assert_allclose(Ul, S["U"][cells], rtol=0, atol=1e-14 * scale.max())
    np.testing.assert_array_equal(pl, S["pos"][cells])
    np.testing.assert_array_equal(wl, S["w"][cells])
