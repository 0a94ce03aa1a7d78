"""The Gresho-Chan vortex (Sec. 5.3): its initial state is a steady solution,
and the oracle's error against it converges with resolution.

The pins are independent of the formulas' transcription: radial balance
dP/dr = rho v_phi^2 / r is checked by finite differences of the printed
pressure, and the error norm is the paper's L1 of the tangential velocity
at the generators (Sec. 5.3)."""
import numpy as np
import pytest

from paper_1707_05333_gb300 import workloads as WL


def gresho_l1(pos, U):
    """L1 = mean_i |v_phi,i - v_phi(r_i)| over generators (Sec. 5.3)."""
    v = U[:, 1:4] / U[:, :1]
    dx, dy = pos[:, 0] - 0.5, pos[:, 1] - 0.5
    r = np.hypot(dx, dy)
    vphi = (-dy * v[:, 0] + dx * v[:, 1]) / r
    return float(np.mean(np.abs(vphi - WL.gresho_vphi(r))))


def test_gresho_profiles_are_in_radial_balance():
    """Centrifugal balance of a steady rotating column: dP/dr = rho v^2 / r
    with rho = 1, on every piece, and P and v continuous at r = 0.2, 0.4."""
    h = 1e-6
    for r in np.concatenate([np.linspace(0.01, 0.19, 7), np.linspace(0.21, 0.39, 7), [0.45, 0.7]]):
        dpdr = (WL.gresho_pressure(r + h) - WL.gresho_pressure(r - h)) / (2 * h)
        assert abs(dpdr - WL.gresho_vphi(r) ** 2 / r) < 1e-6, r
    for r in (0.2, 0.4):
        assert abs(WL.gresho_pressure(r - 1e-12) - WL.gresho_pressure(r)) < 1e-9
        assert abs(WL.gresho_vphi(r - 1e-12) - WL.gresho_vphi(r)) < 1e-9


def test_gresho_workload_shape():
    w = WL.gresho_vortex(32)
    assert w.n == 32 * 32 * 6
    assert np.allclose(w.box, [1.0, 1.0, 0.2])
    assert np.all(w.pos >= 0) and np.all(w.pos < w.box)
    assert np.all(w.vel[:, 2] == 0)
    dx, dy = w.pos[:, 0] - 0.5, w.pos[:, 1] - 0.5
    # velocity is purely azimuthal
    assert np.max(np.abs(dx * w.vel[:, 0] + dy * w.vel[:, 1])) < 1e-14


def run_oracle(oracle, n_side, t_end):
    w = WL.gresho_vortex(n_side)
    cfg = oracle.make_cfg(gamma=w.gamma, cfl=w.cfl, limiter=1, regularize=1)
    T = oracle.tessellate(w.pos, w.box)
    U = oracle.charges_from_prims(T["volume"], w.rho, w.vel, w.pres, w.gamma)
    pos, t = w.pos.copy(), 0.0
    assert gresho_l1(pos, U) < 1e-12  # sampled exactly at the generators
    while t < t_end:
        S = oracle.step(pos, U, w.box, cfg)
        if t + S["dt"] > t_end:
            S = oracle.step(pos, U, w.box, cfg, dt=t_end - t)
        pos, U, t = S["pos"], S["U"], t + S["dt"]
    return gresho_l1(pos, U)


@pytest.mark.slow
def test_oracle_gresho_error_converges(oracle):
    """The paper measures L1 ~ N^-0.88 at t = 2; at t = 0.1 the oracle's error
    must also fall with resolution (slope at least 0.5 between 16^2 and
    24^2) and stay a small fraction of the peak speed 1."""
    l16 = run_oracle(oracle, 16, 0.1)
    l24 = run_oracle(oracle, 24, 0.1)
    slope = np.log(l16 / l24) / np.log(24 / 16)
    assert l16 < 0.05 and l24 < l16
    assert slope > 0.5, (l16, l24, slope)
