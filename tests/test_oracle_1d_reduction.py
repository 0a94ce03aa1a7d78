"""One step of the oracle on a cubic lattice whose state varies along x only
is a one-dimensional finite-volume scheme written from Sec. 4 and Sec. 4.1.

On such a lattice every cell is a cube of side h; the Green-Gauss gradient
is the central difference along x; the transverse neighbours hold the cell's
own values, so the limiters see only the two x-neighbours and the transverse
faces carry equal and opposite fluxes; the face centroid is the midpoint of
the two generators, so a face moves with the mean velocity of its
generators.  The one-dimensional schemes below are written from those
passages directly:

  gradient g = (W_{i+1} - W_{i-1}) / 2h, limited by S10, S10 to the face
        centroid, or S10 and Duffell-MacFadyen (Sec. 4.1),
  half step W' = W - dt/2 dF/dx, dF/dx = (dF/dW) g, the derivative of the
        Euler flux taken by a complex step (no Jacobian formula involved),
  gradient of W', limited again (Sec. 4.1, two gradient estimates),
  face states W'_i + (h/2) g'_i and W'_{i+1} - (h/2) g'_{i+1},
  boost into the frame of the face (a vector: the flow has a transverse
        shear v_y(x)), HLLC or HLL, back to the lab frame by the Galilean
        transformation of the Euler flux (Sec. 4 items 3-5),
  U_i <- U_i - dt h^2 (F_{i+1/2} - F_{i-1/2}) (Sec. 4, outward flux);

Heun's flux averaging (Sec. 6) with every generator moving at one
velocity, so that the lattice translates and stays a lattice: two
forward-Euler stages reconstructing in space only, averaged with the start;
and the entropy column with the shock switch (Sec. 4.3): rho A predicted
through the complex-step derivative of its passive flux (rho A) u, its face
flux upwind of the contact, the faces' shock Mach numbers, and the switch
at the swept volume V'.

The Riemann solvers are the oracle's one-dimensional ones, pinned on their
own (Toro's exact star states, the jump conditions); everything the
three-dimensional step adds around them -- the tessellation's faces, the
Green-Gauss matrix, limiters, reconstruction offsets, boosts, the
unique-face bookkeeping and the sign of the update -- is checked here.  A
mistake planted in the one-dimensional scheme (a full instead of a half
step, one gradient pass instead of two, the reconstruction from the wrong
side, a face at rest, a back-boost without its energy term, no limiter)
moves the result by 1e-3 or more, and in the entropy scheme (the start
volume for V', the downwind side's A, the switch inverted) by 4e-5 or more;
the two agree to 1e-13 of the largest charge (measured 7.5e-15)."""
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
    """Euler flux along x; a sixth column rho A is carried passively, (rho A) u."""
    rho, mx, my, mz, E = W[:, :5].T
    u = mx / rho
    P = (GAMMA - 1.0) * (E - 0.5 * (mx * mx + my * my + mz * mz) / rho)
    cols = [mx, mx * u + P, my * u, mz * u, (E + P) * u]
    if W.shape[1] == 6:
        cols.append(W[:, 5] * u)
    return np.stack(cols, axis=1)


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
    """1-D primitives (rho, u_n, v_t1, v_t2, P) along +x in the frame of a
    face moving at the vector wf."""
    rho = W[0]
    u = W[1:4] / rho
    P = (GAMMA - 1.0) * (W[4] - 0.5 * rho * np.dot(u, u))
    v = u - wf
    return np.array([rho, v[0], v[1], v[2], P])


def limited_gradient(X, h, limiter, theta=0.49, plant=None):
    g = (np.roll(X, -1, axis=0) - np.roll(X, 1, axis=0)) / (2.0 * h)
    if not limiter or plant == "no_limiter":
        return g
    a = s10(X, g, h, to_face=limiter == 3)
    if limiter == 2:
        a = a * dm(X, g, h, theta)
    return a * g


def face_fluxes(WL, WR, wf, riemann, plant=None):
    """Lab-frame flux through the faces i+1/2 moving at wf[i]: the face-frame
    Riemann flux F' turned back by the Galilean transformation of the Euler
    flux, mass F'_m, momentum F'_p + w F'_m, energy F'_E + w.F'_p + w^2/2 F'_m."""
    F = np.zeros_like(WL)
    for k in range(len(WL)):
        w = wf[k]
        Fp = riemann(prim_in_face_frame(WL[k], w), prim_in_face_frame(WR[k], w), GAMMA)
        F[k, 0] = Fp[0]
        F[k, 1:4] = Fp[1:4] + w * Fp[0]
        F[k, 4] = Fp[4] + (0.0 if plant == "no_energy_boost" else np.dot(w, Fp[1:4]) + 0.5 * np.dot(w, w) * Fp[0])
    return F


def step_1d(W, h, dt, eta, limiter, riemann, plant=None):
    """The half-step scheme: two limited gradients, faces at the mean of the
    generators' velocities eta v."""
    g0 = limited_gradient(W, h, limiter, plant=plant)
    Wh = W - (1.0 if plant == "full_step" else 0.5) * dt * flux_derivative(W, g0)
    g1 = g0 if plant == "one_gradient" else limited_gradient(Wh, h, limiter, plant=plant)
    off = -0.5 * h if plant == "wrong_side" else 0.5 * h
    WL = Wh + off * g1
    WR = np.roll(Wh - off * g1, -1, axis=0)
    v = W[:, 1:4] / W[:, :1]
    wf = np.zeros_like(v) if plant == "face_at_rest" else eta * 0.5 * (v + np.roll(v, -1, axis=0))
    F = face_fluxes(WL, WR, wf, riemann, plant)
    return W - dt / h * (F - np.roll(F, 1, axis=0))


def heun_1d(W, h, dt, w, limiter, riemann):
    """Heun's flux averaging with every generator moving at the same w (the
    lattice translates and stays a lattice): two forward-Euler stages that
    reconstruct in space only, each with its own limited gradient, and the
    mean of the start and the second stage."""
    def stage(X):
        g = limited_gradient(X, h, limiter)
        F = face_fluxes(X + 0.5 * h * g, np.roll(X - 0.5 * h * g, -1, axis=0), np.tile(w, (len(X), 1)), riemann)
        return X - dt / h * (F - np.roll(F, 1, axis=0))

    return 0.5 * (W + stage(stage(W)))


def step_1d_entropy(W, h, dt, limiter, riemann, mach_th, oracle, plant=None):
    """The half-step scheme with the entropy column rho A (Sec. 4.3): rho A
    reconstructed and predicted like the other columns, its flux the mass
    flux times A of the contact's upwind side (HLLC) or the HLL average of
    rho A (HLL), unchanged by the boost; each face's shock Mach number from
    the Riemann problem; a cell whose faces all stay below mach_th takes its
    energy from its entropy, E = |m|^2/2M + A rho^gamma V'/(gamma - 1), at the
    volume V' = V + dt sum (+-) A (w_f . n) the faces sweep it to, and the
    other cells reset their entropy from their energy.  The transverse faces
    carry equal states: Mach number 0, or 1 up to rounding, below every
    threshold used here, and equal and opposite swept volumes."""
    g0 = limited_gradient(W, h, limiter)
    Wh = W - 0.5 * dt * flux_derivative(W, g0)
    g1 = limited_gradient(Wh, h, limiter)
    WL = Wh + 0.5 * h * g1
    WR = np.roll(Wh - 0.5 * h * g1, -1, axis=0)
    assert np.all(WL[:, 5] > 0) and np.all(WR[:, 5] > 0)
    v = W[:, 1:4] / W[:, :1]
    wf = 0.5 * (v + np.roll(v, -1, axis=0))
    F = face_fluxes(WL[:, :5], WR[:, :5], wf, oracle.hll_1d if riemann else oracle.hllc_1d)
    F = np.hstack([F, np.zeros((len(F), 1))])
    mach = np.zeros(len(F))
    for k in range(len(F)):
        pl, pr = prim_in_face_frame(WL[k], wf[k]), prim_in_face_frame(WR[k], wf[k])
        sl, ss, sr, _ = oracle.star_state(pl, pr, GAMMA)
        al, ar = WL[k, 5] / WL[k, 0], WR[k, 5] / WR[k, 0]
        if riemann:
            fl, fr = pl[0] * pl[1] * al, pr[0] * pr[1] * ar
            F[k, 5] = fl if sl >= 0 else fr if sr <= 0 else (sr * fl - sl * fr + sl * sr * (WR[k, 5] - WL[k, 5])) / (sr - sl)
        else:
            upwind_left = (ss >= 0) != (plant == "downwind_entropy")
            F[k, 5] = F[k, 0] * (al if upwind_left else ar)
        mach[k] = oracle.shock_mach(pl, pr, GAMMA)
    V = h ** 3
    U = W * V - dt * h * h * (F - np.roll(F, 1, axis=0))
    mc = np.maximum(mach, np.roll(mach, 1))
    Vn = V + (0.0 if plant == "start_volume" else 1.0) * dt * h * h * (wf[:, 0] - np.roll(wf[:, 0], 1))
    energy = (mc >= mach_th) != (plant == "switch_inverted")
    for i in range(len(U)):
        m2 = np.dot(U[i, 1:4], U[i, 1:4])
        if not energy[i]:
            P = (U[i, 5] / U[i, 0]) * (U[i, 0] / Vn[i]) ** GAMMA
            U[i, 4] = 0.5 * m2 / U[i, 0] + P * Vn[i] / (GAMMA - 1.0)
        else:
            P = (GAMMA - 1.0) * (U[i, 4] - 0.5 * m2 / U[i, 0]) / Vn[i]
            U[i, 5] = U[i, 0] * P / (U[i, 0] / Vn[i]) ** GAMMA
    return U, int(energy.sum())


CASES = {
    "static_no_limiter_hllc": dict(eta=0.0, limiter=0, riemann=0),
    "static_s10_hllc": dict(eta=0.0, limiter=1, riemann=0),
    "moving_s10_hllc": dict(eta=1.0, limiter=1, riemann=0),
    "moving_s10_hll": dict(eta=1.0, limiter=1, riemann=1),
    "moving_s10_dm_hllc": dict(eta=1.0, limiter=2, riemann=0),
    "moving_face_centroid_s10_hllc": dict(eta=1.0, limiter=3, riemann=0),
}


def _setup(nx, ny, nz):
    """The planar lattice with a transverse shear v_y(x) added to its flow
    (still one-dimensional: every field depends on x alone)."""
    w = WL.planar_lattice(nx, ny, nz)  # h = 1/nx, not a power of two for nx = 30
    h = 1.0 / nx
    ix = np.rint(w.pos[:, 0] / h - 0.5).astype(int)
    x = (np.arange(nx) + 0.5) * h
    rho, u, P = WL.planar_profile(x)
    vy = 0.05 + 0.15 * np.sin(2 * np.pi * x)
    W1d = conserved(rho, u, P)
    W1d[:, 2] = rho * vy
    W1d[:, 4] += 0.5 * rho * vy * vy
    dt = 0.3 * h / np.max(np.abs(u) + np.abs(vy) + np.sqrt(GAMMA * P / rho))
    return w, h, ix, W1d, dt


def _run(oracle, nx, ny, nz, c):
    w, h, ix, W1d, dt = _setup(nx, ny, nz)
    cfg = oracle.make_cfg(gamma=GAMMA, eta=c["eta"], limiter=c["limiter"], riemann=c["riemann"])
    out = oracle.step(w.pos, W1d[ix] * h ** 3, w.box, cfg, dt=dt)
    riemann = oracle.hll_1d if c["riemann"] else oracle.hllc_1d
    return out["U"], W1d, ix, h, dt, riemann


def _max_error(U3, ref):
    scale = np.abs(ref).max(axis=0)
    scale[1:4] = scale[1:4].max()  # momentum components to the momentum's scale (v_z stays zero)
    return np.abs(U3 - ref).max(axis=0) / scale


SHAPES = dict(argnames="shape", argvalues=[(32, 1, 1), (32, 2, 2), (30, 3, 3)], ids=["32x1x1", "32x2x2", "30x3x3"])


@pytest.mark.parametrize(**SHAPES)
@pytest.mark.parametrize("case", list(CASES))
def test_lattice_step_is_the_one_dimensional_scheme(oracle, case, shape):
    c = CASES[case]
    U3, W1d, ix, h, dt, riemann = _run(oracle, *shape, c)
    ref = step_1d(W1d, h, dt, c["eta"], c["limiter"], riemann)[ix] * h ** 3
    err = _max_error(U3, ref)
    print(f"[1d {case} {shape}] max error per component / max |U|: {err}")
    assert np.all(err <= 1e-13), err
    # the charges really changed: the step is not the identity
    assert np.all(_max_error(U3, W1d[ix] * h ** 3)[[0, 1, 2, 4]] > 1e-6)


@pytest.mark.parametrize(**SHAPES)
@pytest.mark.parametrize("limiter", [0, 1, 2], ids=["no_limiter", "s10", "s10_dm"])
def test_lattice_heun_step_is_the_one_dimensional_heun_scheme(oracle, limiter, shape):
    w, h, ix, W1d, dt = _setup(*shape)
    wmesh = np.array([0.07, -0.04, 0.03])
    cfg = oracle.make_cfg(gamma=GAMMA, limiter=limiter)
    out = oracle.step_heun(w.pos, W1d[ix] * h ** 3, w.box, cfg, dt=dt, w=np.tile(wmesh, (len(w.pos), 1)))
    ref = heun_1d(W1d, h, dt, wmesh, limiter, oracle.hllc_1d)[ix] * h ** 3
    err = _max_error(out["U"], ref)
    print(f"[1d heun limiter {limiter} {shape}] max error per component / max |U|: {err}")
    assert np.all(err <= 1e-13), err
    assert np.all(_max_error(out["U"], W1d[ix] * h ** 3)[[0, 1, 2, 4]] > 1e-6)


ENTROPY_CASES = {  # the faces' Mach numbers reach 1.07-1.10 at the block's edges: 1.05 splits the cells
    "switch_hllc": dict(riemann=0, mach_th=1.05),
    "switch_hll": dict(riemann=1, mach_th=1.05),
    "energy_everywhere": dict(riemann=0, mach_th=0.0),
    "entropy_everywhere": dict(riemann=0, mach_th=1e300),
}


@pytest.mark.parametrize(**SHAPES)
@pytest.mark.parametrize("case", list(ENTROPY_CASES))
def test_lattice_entropy_step_is_the_one_dimensional_scheme(oracle, case, shape):
    c = ENTROPY_CASES[case]
    w, h, ix, W1d, dt = _setup(*shape)
    rho = W1d[:, 0]
    P = (GAMMA - 1.0) * (W1d[:, 4] - 0.5 * (W1d[:, 1] ** 2 + W1d[:, 2] ** 2) / rho)
    W6 = np.hstack([W1d, (P / rho ** GAMMA * rho)[:, None]])
    cfg = oracle.make_cfg(gamma=GAMMA, limiter=1, riemann=c["riemann"], entropy=1, mach_th=c["mach_th"])
    out = oracle.step(w.pos, W6[ix] * h ** 3, w.box, cfg, dt=dt)
    ref, n_energy = step_1d_entropy(W6, h, dt, 1, c["riemann"], c["mach_th"], oracle)
    ref = ref[ix]
    err = _max_error(out["U"], ref)
    print(f"[1d entropy {case} {shape}] cells on the energy equation {n_energy} of {shape[0]}; error: {err}")
    assert np.all(err <= 1e-13), err
    if case.startswith("switch"):
        assert 0 < n_energy < shape[0]


@pytest.mark.parametrize("plant", ["start_volume", "downwind_entropy", "switch_inverted"])
def test_a_planted_mistake_in_the_entropy_scheme_is_seen(oracle, plant):
    w, h, ix, W1d, dt = _setup(32, 2, 2)
    rho = W1d[:, 0]
    P = (GAMMA - 1.0) * (W1d[:, 4] - 0.5 * (W1d[:, 1] ** 2 + W1d[:, 2] ** 2) / rho)
    W6 = np.hstack([W1d, (P / rho ** GAMMA * rho)[:, None]])
    cfg = oracle.make_cfg(gamma=GAMMA, limiter=1, entropy=1, mach_th=1.05)
    out = oracle.step(w.pos, W6[ix] * h ** 3, w.box, cfg, dt=dt)
    bad = step_1d_entropy(W6, h, dt, 1, 0, 1.05, oracle, plant=plant)[0][ix]
    err = _max_error(out["U"], bad)[[4, 5]].max()
    print(f"[entropy plant {plant}] {err:.2e}")
    assert err > 1e-8, err


@pytest.mark.parametrize("plant", ["full_step", "one_gradient", "wrong_side", "face_at_rest",
                                   "no_energy_boost", "no_limiter"])
def test_a_planted_mistake_in_the_scheme_is_seen(oracle, plant):
    c = CASES["moving_s10_hllc"]
    U3, W1d, ix, h, dt, riemann = _run(oracle, 32, 2, 2, c)
    bad = step_1d(W1d, h, dt, c["eta"], c["limiter"], riemann, plant=plant)[ix] * h ** 3
    err = _max_error(U3, bad)[[0, 1, 2, 4]].max()
    assert err > 1e-6, err
