"""One step of the oracle on a cubic lattice whose state varies along x only
is the one-dimensional MUSCL-Hancock scheme of Sec. 4 and Sec. 4.1.

On such a lattice every cell is a cube of side h; the Green-Gauss gradient
is the central difference along x; the transverse neighbours hold the cell's
own values, so the S10 limiter sees only the two x-neighbours and the
transverse faces carry equal and opposite fluxes; the face centroid is the
midpoint of the two generators, so a face moves with the mean velocity of
its generators.  The one-dimensional scheme below is written from those
passages directly:

  gradient g = (W_{i+1} - W_{i-1}) / 2h, limited by S10 (Sec. 4.1),
  half step W' = W - dt/2 dF/dx, dF/dx = (dF/dW) g, the derivative of the
        Euler flux taken by a complex step (no Jacobian formula involved),
  gradient of W', limited again (Sec. 4.1, two gradient estimates),
  face states W'_i + (h/2) g'_i and W'_{i+1} - (h/2) g'_{i+1},
  boost into the frame of the face, HLLC or HLL, back to the lab frame by the
        Galilean transformation of the Euler flux (Sec. 4 items 3-5),
  U_i <- U_i - dt h^2 (F_{i+1/2} - F_{i-1/2}) (Sec. 4, outward flux).

The Riemann solvers are the oracle's one-dimensional ones, pinned on their
own (Toro's exact star states, the jump conditions); everything the
three-dimensional step adds around them -- the tessellation's faces, the
Green-Gauss matrix, reconstruction offsets, boosts, the unique-face
bookkeeping and the sign of the update -- is checked here.  A mistake
planted in the one-dimensional scheme (a full instead of a half step, one
gradient pass instead of two, the reconstruction from the generator instead
of the centroid side, a face at rest, a back-boost without its energy term,
no limiter) moves the result by 1e-3 or more; the two agree to 1e-13 of the
largest charge (measured 5e-16)."""
import numpy as np
import pytest

from paper_1707_05333_gb300 import workloads as WL

GAMMA = 5.0 / 3.0


def conserved(rho, u, P):
    """Conserved state per volume (rho, rho u, 0, 0, rho e)."""
    W = np.zeros((len(rho), 5))
    W[:, 0] = rho
    W[:, 1] = rho * u
    W[:, 4] = P / (GAMMA - 1.0) + 0.5 * rho * u * u
    return W


def euler_flux_x(W):
    rho, mx, my, mz, E = W.T
    u = mx / rho
    P = (GAMMA - 1.0) * (E - 0.5 * (mx * mx + my * my + mz * mz) / rho)
    return np.stack([mx, mx * u + P, my * u, mz * u, (E + P) * u], axis=1)


def flux_derivative(W, g):
    """(dF_x/dW) g, exactly up to rounding, by a complex step."""
    eps = 1e-30
    return euler_flux_x(W + 1j * eps * g).imag / eps


def s10(W, g, h, to_face=False):
    """S10 limiter (Sec. 4.1) on the line: neighbourhood extremes including
    the cell, Delta = g (c_j - c_i) to both neighbours (g (x_f - c_i), half
    as far, for the face-centroid form), alpha = min(1, psi)."""
    Wm, Wp = np.roll(W, 1, axis=0), np.roll(W, -1, axis=0)
    hi = np.maximum(np.maximum(Wm, W), Wp)
    lo = np.minimum(np.minimum(Wm, W), Wp)
    a = np.ones_like(W)
    for d in ((0.5 * h, -0.5 * h) if to_face else (h, -h)):
        D = g * d
        with np.errstate(divide="ignore", invalid="ignore"):
            psi = np.where(D > 0, (hi - W) / D, np.where(D < 0, (lo - W) / D, 1.0))
        a = np.minimum(a, psi)
    return a


def dm(W, g, h, theta):
    """Duffell-MacFadyen factor (Sec. 4.1) on the line: min(1, min_j max(0,
    theta (W_j - W_i) / Delta_ij)) over the two neighbours with Delta != 0;
    the transverse neighbours have Delta = 0 and do not count."""
    a = np.ones_like(W)
    for Wj, d in ((np.roll(W, -1, axis=0), h), (np.roll(W, 1, axis=0), -h)):
        D = g * d
        with np.errstate(divide="ignore", invalid="ignore"):
            psi = np.where(D != 0, np.maximum(0.0, theta * (Wj - W) / D), 1.0)
        a = np.minimum(a, psi)
    return a


def prim_in_face_frame(W, wf):
    rho = W[0]
    u = W[1:4] / rho
    P = (GAMMA - 1.0) * (W[4] - 0.5 * rho * np.dot(u, u))
    return np.array([rho, u[0] - wf, u[1], u[2], P])


def step_1d(W, h, dt, eta, limiter, riemann, plant=None, theta=0.49):
    def grad(X):
        g = (np.roll(X, -1, axis=0) - np.roll(X, 1, axis=0)) / (2.0 * h)
        if not limiter or plant == "no_limiter":
            return g
        a = s10(X, g, h, to_face=limiter == 3)
        if limiter == 2:
            a = a * dm(X, g, h, theta)
        return a * g

    g0 = grad(W)
    Wh = W - (1.0 if plant == "full_step" else 0.5) * dt * flux_derivative(W, g0)
    g1 = g0 if plant == "one_gradient" else grad(Wh)
    off = -0.5 * h if plant == "wrong_side" else 0.5 * h
    WL = Wh + off * g1
    WR = np.roll(Wh - off * g1, -1, axis=0)
    v = W[:, 1] / W[:, 0]
    wf = np.zeros_like(v) if plant == "face_at_rest" else eta * 0.5 * (v + np.roll(v, -1))
    F = np.zeros_like(W)
    for k in range(len(W)):
        Fp = riemann(prim_in_face_frame(WL[k], wf[k]), prim_in_face_frame(WR[k], wf[k]), GAMMA)
        e_boost = 0.0 if plant == "no_energy_boost" else wf[k] * Fp[1] + 0.5 * wf[k] ** 2 * Fp[0]
        F[k] = [Fp[0], Fp[1] + wf[k] * Fp[0], Fp[2], Fp[3], Fp[4] + e_boost]
    return W - dt / h * (F - np.roll(F, 1, axis=0))


CASES = {
    "static_no_limiter_hllc": dict(eta=0.0, limiter=0, riemann=0),
    "static_s10_hllc": dict(eta=0.0, limiter=1, riemann=0),
    "moving_s10_hllc": dict(eta=1.0, limiter=1, riemann=0),
    "moving_s10_hll": dict(eta=1.0, limiter=1, riemann=1),
    "moving_s10_dm_hllc": dict(eta=1.0, limiter=2, riemann=0),
    "moving_face_centroid_s10_hllc": dict(eta=1.0, limiter=3, riemann=0),
}


def _run(oracle, nx, ny, nz, c):
    w = WL.planar_lattice(nx, ny, nz)  # h = 1/nx, not a power of two for nx = 30
    h = 1.0 / nx
    ix = np.rint(w.pos[:, 0] / h - 0.5).astype(int)
    W1d = conserved(*WL.planar_profile((np.arange(nx) + 0.5) * h))
    U = W1d[ix] * h ** 3
    rho, u = W1d[:, 0], W1d[:, 1] / W1d[:, 0]
    P = (GAMMA - 1.0) * (W1d[:, 4] - 0.5 * rho * u * u)
    dt = 0.3 * h / np.max(np.abs(u) + np.sqrt(GAMMA * P / rho))
    cfg = oracle.make_cfg(gamma=GAMMA, eta=c["eta"], limiter=c["limiter"], riemann=c["riemann"])
    out = oracle.step(w.pos, U, w.box, cfg, dt=dt)
    riemann = oracle.hll_1d if c["riemann"] else oracle.hllc_1d
    return out["U"], W1d, ix, h, dt, riemann


@pytest.mark.parametrize("shape", [(32, 1, 1), (32, 2, 2), (30, 3, 3)], ids=["32x1x1", "32x2x2", "30x3x3"])
@pytest.mark.parametrize("case", list(CASES))
def test_lattice_step_is_the_one_dimensional_scheme(oracle, case, shape):
    c = CASES[case]
    U3, W1d, ix, h, dt, riemann = _run(oracle, *shape, c)
    ref = step_1d(W1d, h, dt, c["eta"], c["limiter"], riemann)[ix] * h ** 3
    scale = np.abs(ref).max(axis=0)
    scale[2:4] = scale[1]  # transverse momentum stays zero: held to the x-momentum's scale
    err = np.abs(U3 - ref).max(axis=0) / scale
    print(f"[1d {case} {shape}] max error per component / max |U|: {err}")
    assert np.all(err <= 1e-13), err  # measured <= 4.6e-16
    # the charges really changed: the step is not the identity
    assert np.abs(U3 - W1d[ix] * h ** 3).max(axis=0)[[0, 1, 4]].min() > 1e-6 * scale[[0, 1, 4]].min()


@pytest.mark.parametrize("plant", ["full_step", "one_gradient", "wrong_side", "face_at_rest",
                                   "no_energy_boost", "no_limiter"])
def test_a_planted_mistake_in_the_scheme_is_seen(oracle, plant):
    c = CASES["moving_s10_hllc"]
    U3, W1d, ix, h, dt, riemann = _run(oracle, 32, 2, 2, c)
    bad = step_1d(W1d, h, dt, c["eta"], c["limiter"], riemann, plant=plant)[ix] * h ** 3
    err = (np.abs(U3 - bad).max(axis=0)[[0, 1, 4]] / np.abs(bad).max(axis=0)[[0, 1, 4]]).max()
    assert err > 1e-6, err
