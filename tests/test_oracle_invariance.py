"""Symmetries of the oracle's whole step (Sec. 2-4): relabelling the cells,
translating every generator through the periodic box, mirroring the box
(x -> L - x with the x velocity reversed) and changing the units of length
and velocity by powers of two each commute with one step, to the rounding of
sums taken in another order.  A mistake in an index (i for j),
an image shift, a normal's or a flux's sign, or a per-cell quantity read
for the wrong cell breaks one of them; none needs the method's own formulas
on this side."""
import numpy as np
import pytest

from paper_1707_05333_gb300 import workloads as WL

N = 240
BOX = np.array([1.0, 0.75, 1.25])

CONFIGS = {
    "s10_hllc": dict(limiter=1),
    "dm_regularized_entropy_switch": dict(limiter=2, regularize=1, entropy=1, mach_th=1.05),
    "face_centroid_hll": dict(limiter=3, riemann=1),
}


def _state(oracle, cfg, pos):
    rho, vel, pres = WL.random_state(N, seed=31, v_sigma=0.4)
    T = oracle.tessellate(pos, BOX, 1)
    return oracle.charges_from_prims(T["volume"], rho, vel, pres, cfg.gamma, entropy=bool(cfg.entropy))


def _wrap(p):
    p = np.mod(p, BOX)
    return np.where(p >= BOX, 0.0, p)


def _setup(oracle, name):
    cfg = oracle.make_cfg(**CONFIGS[name])
    pos = WL.random_points(N, box=BOX, seed=32)
    U = _state(oracle, cfg, pos)
    S = oracle.step(pos, U, BOX, cfg)
    return cfg, pos, U, S


def _close(a, b, rtol=1e-13):  # measured <= 9e-16
    scale = np.abs(b).max(axis=0)
    scale[1:4] = scale[1:4].max()
    return np.abs(a - b).max(axis=0) / scale <= rtol


@pytest.mark.parametrize("name", list(CONFIGS))
def test_relabelling_the_cells_relabels_the_step(oracle, name):
    cfg, pos, U, S = _setup(oracle, name)
    perm = np.random.default_rng(33).permutation(N)
    P = oracle.step(pos[perm], U[perm], BOX, cfg, dt=S["dt"])
    assert np.all(_close(P["U"], S["U"][perm]))
    np.testing.assert_allclose(P["pos"], S["pos"][perm], rtol=0, atol=1e-13)
    assert P["dt_cfl"] == pytest.approx(S["dt_cfl"], rel=1e-13)


@pytest.mark.parametrize("name", list(CONFIGS))
def test_a_periodic_translation_commutes_with_the_step(oracle, name):
    cfg, pos, U, S = _setup(oracle, name)
    t = np.array([0.3141, -0.2718, 0.5772]) * BOX
    P = oracle.step(_wrap(pos + t), U, BOX, cfg, dt=S["dt"])
    assert np.all(_close(P["U"], S["U"]))
    d = P["pos"] - _wrap(S["pos"] + t)
    d -= BOX * np.round(d / BOX)
    assert np.abs(d).max() <= 1e-12


@pytest.mark.parametrize("name", list(CONFIGS))
def test_the_mirror_image_steps_to_the_mirror_image(oracle, name):
    cfg, pos, U, S = _setup(oracle, name)
    m = pos.copy()
    m[:, 0] = BOX[0] - pos[:, 0]
    Um = U.copy()
    Um[:, 1] = -U[:, 1]
    P = oracle.step(_wrap(m), Um, BOX, cfg, dt=S["dt"])
    ref = S["U"].copy()
    ref[:, 1] = -ref[:, 1]
    assert np.all(_close(P["U"], ref))


def test_heun_step_commutes_with_relabelling_and_translation(oracle):
    cfg = oracle.make_cfg(limiter=2, regularize=1)
    pos = WL.random_points(N, box=BOX, seed=34)
    U = _state(oracle, cfg, pos)
    S = oracle.step_heun(pos, U, BOX, cfg)
    perm = np.random.default_rng(35).permutation(N)
    P = oracle.step_heun(pos[perm], U[perm], BOX, cfg, dt=S["dt"])
    assert np.all(_close(P["U"], S["U"][perm]))
    t = np.array([-0.123, 0.456, 0.789]) * BOX
    Q = oracle.step_heun(_wrap(pos + t), U, BOX, cfg, dt=S["dt"])
    assert np.all(_close(Q["U"], S["U"]))


def test_a_wrong_index_breaks_relabelling(oracle):
    """The relabelling check is not vacuous: charges paired with the wrong
    generators (a one-place shift of the labels) give another step."""
    cfg, pos, U, S = _setup(oracle, "s10_hllc")
    P = oracle.step(pos, np.roll(U, 1, axis=0), BOX, cfg, dt=S["dt"])
    assert not np.all(_close(P["U"], np.roll(S["U"], 1, axis=0), rtol=1e-6))


@pytest.mark.parametrize("name", list(CONFIGS))
@pytest.mark.parametrize("s,a", [(2.0 ** -20, 1.0), (2.0 ** 20, 1.0), (1.0, 2.0 ** 10), (2.0 ** -7, 2.0 ** 5)],
                         ids=["small", "large", "fast", "small_fast"])
def test_power_of_two_units_commute_with_the_step(oracle, name, s, a):
    """Lengths times s, velocities times a (pressures a^2, times s/a): the
    charges of one step scale as (s^3) (1, a, a, a, a^2 [, a^2]) and the CFL
    step as s/a.  Every tolerance inside the oracle is relative to a length
    or a value of the configuration; an absolute one would show here."""
    cfg, pos, U, S = _setup(oracle, name)
    k = np.array([1.0, a, a, a, a * a] + ([a * a] if cfg.entropy else [])) * s ** 3
    P = oracle.step(pos * s, U * k, BOX * s, cfg, dt=S["dt"] * s / a)
    assert np.all(_close(P["U"], S["U"] * k))
    assert P["dt_cfl"] == pytest.approx(S["dt_cfl"] * s / a, rel=1e-13)
    d = P["pos"] - S["pos"] * s
    d -= BOX * s * np.round(d / (BOX * s))
    assert np.abs(d).max() <= 1e-13 * s
