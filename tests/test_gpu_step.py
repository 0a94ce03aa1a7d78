"""GPU hydro stages and the whole step (mm_gradients, mm_mesh_velocity,
mm_timestep, mm_flux_step, mm_drift, mm_step) against the oracle."""
import numpy as np
import pytest

from paper_1707_05333_gb300 import workloads as WL
from tests import helpers as H

pytestmark = pytest.mark.gpu

RTOL_STEP = 1e-10  # one-step conserved states, FP64 path


@pytest.fixture(scope="module")
def gpu():
    c, torch = H.gpu_context()
    yield c, torch
    c.close()


@pytest.fixture(autouse=True)
def default_settings(gpu):
    """Every test starts from the default configuration (the parity cases
    switch limiters, solvers, the entropy column and the integrator)."""
    from paper_1707_05333_gb300 import binding
    c, _ = gpu
    d = binding.default_config()
    c.set_config(**{f: getattr(d, f) for f, _ in d._fields_})


def setup(oracle, w, rho=None, vel=None, pres=None, entropy=False):
    T = oracle.tessellate(w.pos, w.box, 1)
    U = oracle.charges_from_prims(T["volume"], w.rho if rho is None else rho, w.vel if vel is None else vel,
                                  w.pres if pres is None else pres, w.gamma, w.e_add, entropy=entropy)
    return T, U


def cfg_pair(oracle, gamma, **kw):
    from paper_1707_05333_gb300 import binding
    o = oracle.make_cfg(gamma=gamma, **kw)
    g = binding.default_config(gamma=gamma, **kw)
    return o, g


def assert_state_close(G, O, rtol=RTOL_STEP):
    # per component, relative to the component's scale; the momentum
    # components to the momentum's (a component can vanish, or stay zero up
    # to rounding, as the transverse momentum of a planar flow)
    assert G.shape[0] == O.shape[1]
    pscale = np.abs(O[:, 1:4]).max()
    for k in range(O.shape[1]):
        scale = pscale if 1 <= k <= 3 else np.abs(O[:, k]).max()
        np.testing.assert_allclose(G[k], O[:, k], rtol=rtol, atol=rtol * scale, err_msg=f"component {k}")


@pytest.mark.parametrize("limiter", [0, 1, 2, 3])
def test_gradients_match_oracle(oracle, gpu, limiter):
    c, torch = gpu
    w = WL.smooth_wave(12)
    rho, vel, pres = WL.random_state(w.n, seed=limiter)
    T, U = setup(oracle, w, rho, vel, pres)
    ocfg, gcfg = cfg_pair(oracle, w.gamma, limiter=limiter)
    c.set_config(**{f: getattr(gcfg, f) for f, _ in gcfg._fields_})
    mesh, P, G = H.gpu_tessellate(c, torch, w.pos, w.box)
    W = U / T["volume"][:, None]
    og = oracle.gradient(oracle.unique_faces(T), T["volume"], T["centroid"], w.box, W, ocfg)
    gg = c.mm_gradients(mesh, H.to_dev(torch, W.T)).cpu().numpy()
    og = og.reshape(w.n, 15).T
    for r in range(15):
        np.testing.assert_allclose(gg[r], og[r], rtol=1e-9, atol=1e-9 * np.abs(og[r]).max() + 1e-14)


CONFIGS = {
    "smooth_wave_16^3_S10": dict(maker=lambda: WL.smooth_wave(16), kw=dict(limiter=1)),
    "smooth_wave_random_state_DM_regularized": dict(maker=lambda: WL.smooth_wave(10), kw=dict(limiter=2, regularize=1),
                                                    random=True),
    "shock_tube_64x6x6": dict(maker=lambda: WL.shock_tube(64, 6, 6), kw=dict(limiter=1)),
    "point_blast_12^3": dict(maker=lambda: WL.point_blast(12), kw=dict(limiter=1)),
    "static_mesh_eta0": dict(maker=lambda: WL.smooth_wave(9), kw=dict(limiter=1, eta=0.0), random=True),
    "no_limiter_ragged_11^3": dict(maker=lambda: WL.smooth_wave(11), kw=dict(limiter=0), random=True),
    "hll_shock_tube_48x6x6": dict(maker=lambda: WL.shock_tube(48, 6, 6), kw=dict(limiter=1, riemann=1)),
    "face_centroid_limiter_random": dict(maker=lambda: WL.smooth_wave(10), kw=dict(limiter=3, regularize=1),
                                         random=True),
    "gresho_vortex_16x16x3_regularized": dict(maker=lambda: WL.gresho_vortex(16), kw=dict(limiter=1, regularize=1)),
    "clustered_6000_random_state_DM": dict(maker=lambda: WL.clustered_box(6000), kw=dict(limiter=2), random=True),
    # exact lattice of spacing 1/30 with a planar state: Delta toward the
    # equal-valued transverse neighbours is zero up to rounding, which the DM
    # limiter must not count
    "planar_lattice_30x3x3_DM": dict(maker=lambda: WL.planar_lattice(30, 3, 3), kw=dict(limiter=2)),
    # entropy column and switch (Sec. 4.3): cells at the shock keep the energy
    # equation, the rest take E from the entropy
    "entropy_switch_shock_tube_48x6x6": dict(maker=lambda: WL.shock_tube(48, 6, 6),
                                             kw=dict(limiter=1, entropy=1, mach_th=1.1)),
    "entropy_switch_hll_point_blast_12^3": dict(maker=lambda: WL.point_blast(12),
                                                kw=dict(limiter=2, riemann=1, entropy=1, mach_th=1.1)),
    "entropy_everywhere_random_regularized": dict(maker=lambda: WL.smooth_wave(10),
                                                  kw=dict(limiter=3, regularize=1, entropy=1, mach_th=1e300),
                                                  random=True),
}


@pytest.mark.parametrize("case", list(CONFIGS))
def test_one_step_matches_oracle(oracle, gpu, case):
    c, torch = gpu
    spec = CONFIGS[case]
    w = spec["maker"]()
    ent = bool(spec["kw"].get("entropy", 0))
    if spec.get("random"):
        rho, vel, pres = WL.random_state(w.n, seed=3)
        T, U = setup(oracle, w, rho, vel, pres, entropy=ent)
    else:
        T, U = setup(oracle, w, entropy=ent)
    ocfg, gcfg = cfg_pair(oracle, w.gamma, cfl=w.cfl, **spec["kw"])
    c.set_config(**{f: getattr(gcfg, f) for f, _ in gcfg._fields_})
    S = oracle.step(w.pos, U, w.box, ocfg, tess=T)
    # same dt on both sides: the oracle's CFL value
    pos = H.to_dev(torch, w.pos.T)
    Ud = H.to_dev(torch, U.T)
    dt_fixed = torch.tensor([S["dt"]], dtype=torch.float64, device="cuda")
    w_out = torch.empty((3, w.n), dtype=torch.float64, device="cuda")
    dt_out = torch.empty((1,), dtype=torch.float64, device="cuda")
    c.mm_step(pos, Ud, w.box, dt_fixed=dt_fixed, dt_out=dt_out, w_out=w_out)
    np.testing.assert_allclose(w_out.cpu().numpy().T, S["w"], rtol=1e-12, atol=1e-14)
    assert_state_close(Ud.cpu().numpy(), S["U"])
    dp = pos.cpu().numpy().T - S["pos"]
    dp -= np.round(dp / w.box) * w.box
    assert np.abs(dp).max() <= 1e-12
    # the CFL timestep itself, computed on the device
    c.mm_step(H.to_dev(torch, w.pos.T), H.to_dev(torch, U.T), w.box, dt_out=dt_out)
    assert float(dt_out.item()) == pytest.approx(S["dt_cfl"], rel=1e-13)


def test_stagewise_calls_equal_mm_step(oracle, gpu):
    c, torch = gpu
    w = WL.smooth_wave(10)
    rho, vel, pres = WL.random_state(w.n, seed=5)
    T, U = setup(oracle, w, rho, vel, pres)
    c.set_config(limiter=1, regularize=1, gamma=w.gamma, eta=1.0)
    pos = H.to_dev(torch, w.pos.T)
    Ud = H.to_dev(torch, U.T)
    mesh = c.mm_tessellate(pos, w.box)
    wv = c.mm_mesh_velocity(mesh, pos, Ud)
    dt = c.mm_timestep(mesh, Ud, wv)
    c.mm_flux_step(mesh, pos, wv, dt, Ud)
    c.mm_drift(pos, wv, dt, w.box)
    pos2 = H.to_dev(torch, w.pos.T)
    U2 = H.to_dev(torch, U.T)
    c.mm_step(pos2, U2, w.box)
    assert torch.equal(Ud, U2) and torch.equal(pos, pos2)


def test_conservation_and_determinism_on_device(oracle, gpu):
    c, torch = gpu
    w = WL.smooth_wave(20)
    rho, vel, pres = WL.random_state(w.n, seed=6)
    T, U = setup(oracle, w, rho, vel, pres)
    c.set_config(limiter=2, regularize=1, gamma=w.gamma)
    outs = []
    for _ in range(2):
        pos = H.to_dev(torch, w.pos.T)
        Ud = H.to_dev(torch, U.T)
        t0 = c.mm_totals(Ud).cpu().numpy()
        for _ in range(3):
            c.mm_step(pos, Ud, w.box)
        t1 = c.mm_totals(Ud).cpu().numpy()
        scale = np.abs(U).sum(0)
        scale[1:4] = scale[1:4].max()
        assert np.all(np.abs(t1 - t0) <= 1e-13 * scale)
        outs.append((pos.clone(), Ud.clone()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_uniform_flow_is_preserved(oracle, gpu):
    c, torch = gpu
    w = WL.smooth_wave(12)
    n = w.n
    T = oracle.tessellate(w.pos, w.box, 1)
    vel = np.tile([0.3, -0.2, 0.1], (n, 1))
    U = oracle.charges_from_prims(T["volume"], np.full(n, 1.2), vel, np.full(n, 0.8), w.gamma)
    c.set_config(limiter=1, regularize=0, gamma=w.gamma, eta=1.0)
    pos = H.to_dev(torch, w.pos.T)
    Ud = H.to_dev(torch, U.T)
    dt = torch.tensor([1e-3], dtype=torch.float64, device="cuda")
    c.mm_step(pos, Ud, w.box, dt_fixed=dt)
    np.testing.assert_allclose(Ud.cpu().numpy().T, U, rtol=1e-12, atol=1e-16)


def test_prims_to_charges(oracle, gpu):
    c, torch = gpu
    w = WL.smooth_wave(8)
    c.set_config(gamma=w.gamma)
    mesh, P, G = H.gpu_tessellate(c, torch, w.pos, w.box)
    U = c.mm_prims_to_charges(mesh, H.to_dev(torch, w.rho), H.to_dev(torch, w.vel.T), H.to_dev(torch, w.pres))
    O = oracle.charges_from_prims(G["cell_volume"], w.rho, w.vel, w.pres, w.gamma)
    np.testing.assert_allclose(U.cpu().numpy().T, O, rtol=1e-14, atol=1e-18)


def test_full_size_shear_layer_step_properties(gpu):
    """The bench workload: one full step conserves mass, momentum and energy
    and keeps every charge finite and positive."""
    c, torch = gpu
    w = WL.shear_layer(256)
    c.set_config(limiter=1, regularize=0, gamma=w.gamma, cfl=w.cfl, eta=1.0)
    pos = H.to_dev(torch, w.pos.T)
    mesh = c.mm_tessellate(pos, w.box)
    U = c.mm_prims_to_charges(mesh, H.to_dev(torch, w.rho), H.to_dev(torch, w.vel.T), H.to_dev(torch, w.pres))
    t0 = c.mm_totals(U).cpu().numpy()
    scale = U.abs().sum(1).cpu().numpy()
    dt = torch.empty((1,), dtype=torch.float64, device="cuda")
    c.mm_step(pos, U, w.box, dt_out=dt)
    t1 = c.mm_totals(U).cpu().numpy()
    # momentum components share one scale (one of them is identically zero here)
    scale[1:4] = scale[1:4].max()
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale)
    assert bool(torch.isfinite(U).all()) and bool((U[0] > 0).all())
    assert 0 < float(dt.item()) < 1e-2


FULL_SIZE_CASES = {
    "S10_HLLC": dict(limiter=1),
    "DM_roundness": dict(limiter=2, regularize=1),
    "HLL_entropy_switch": dict(limiter=1, riemann=1, entropy=1, mach_th=1.1),
}


@pytest.mark.parametrize("case", list(FULL_SIZE_CASES))
def test_full_size_shear_layer_sampled_cells_match_oracle(oracle, gpu, case):
    """The bench workload (256^3 generators, FP64 path): one whole step on the
    device against the oracle on sampled cells, each computed from the
    oracle's own tessellation of the cell's rings 0..3 (see
    helpers.oracle_local_step).  Inputs are identical on both sides: the
    shear-layer primitives turned into charges with the nominal volume 1/n
    (so W = U / V carries each cell's volume jitter), a fixed dt below the
    CFL value.  Charges to 1e-10 of each component's scale (momentum: the
    largest component's), positions to 1e-12."""
    c, torch = gpu
    kw = FULL_SIZE_CASES[case]
    ent = bool(kw.get("entropy", 0))
    w = WL.shear_layer(256)
    n = w.n
    U0 = oracle.charges_from_prims(np.full(n, 1.0 / n), w.rho, w.vel, w.pres, w.gamma, entropy=ent)
    dt = 2e-4
    ocfg, gcfg = cfg_pair(oracle, w.gamma, cfl=w.cfl, **kw)
    c.set_config(**{f: getattr(gcfg, f) for f, _ in gcfg._fields_})
    pos = H.to_dev(torch, w.pos.T)
    Ud = H.to_dev(torch, U0.T)
    del U0
    c.mm_step(pos, Ud, w.box, dt_fixed=torch.tensor([dt], dtype=torch.float64, device="cuda"))
    rng = np.random.default_rng(1)
    # random cells, plus cells on the two shear interfaces |y - 0.5| = 0.25
    y = w.pos[:, 1]
    near = np.nonzero(np.abs(np.abs(y - 0.5) - 0.25) < 0.5 / 256)[0]
    cells = np.concatenate([rng.choice(n, 12, replace=False), rng.choice(near, 4, replace=False)])
    G = Ud[:, torch.as_tensor(cells, device="cuda")].cpu().numpy().T
    GP = pos[:, torch.as_tensor(cells, device="cuda")].cpu().numpy().T
    del Ud, pos
    U0 = oracle.charges_from_prims(np.full(n, 1.0 / n), w.rho, w.vel, w.pres, w.gamma, entropy=ent)
    O, OP, _, m = H.oracle_local_step(oracle, w.pos, U0, w.box, ocfg, cells, dt)
    print(f"[256^3 one-step parity {case}] {len(cells)} sampled cells, {m} cells tessellated by the oracle")
    scale = np.abs(O).max(axis=0)
    scale[1:4] = scale[1:4].max()
    for k in range(O.shape[1]):
        np.testing.assert_allclose(G[:, k], O[:, k], rtol=0, atol=RTOL_STEP * scale[k], err_msg=f"component {k}")
    dp = GP - OP
    dp -= np.round(dp / w.box) * w.box
    assert np.abs(dp).max() <= 1e-12


def test_full_size_shear_layer_mixed_step_sampled_l1(oracle, gpu):
    """The mixed-precision path on the bench workload (256^3): one step
    against the FP64 oracle on 24 sampled cells (rings 0..3 of each
    tessellated by the oracle), identical inputs as above; relative L1 of
    density, momentum and energy over the sample <= 1e-5, and the device's
    totals conserved to 1e-12."""
    c, torch = gpu
    w = WL.shear_layer(256)
    n = w.n
    U0 = oracle.charges_from_prims(np.full(n, 1.0 / n), w.rho, w.vel, w.pres, w.gamma)
    dt = 2e-4
    ocfg, gcfg = cfg_pair(oracle, w.gamma, cfl=w.cfl, limiter=1)
    gcfg.precision = 1
    c.set_config(**{f: getattr(gcfg, f) for f, _ in gcfg._fields_})
    try:
        pos = H.to_dev(torch, w.pos.T)
        Ud = H.to_dev(torch, U0.T)
        del U0
        t0 = c.mm_totals(Ud).cpu().numpy()
        c.mm_step(pos, Ud, w.box, dt_fixed=torch.tensor([dt], dtype=torch.float64, device="cuda"))
        t1 = c.mm_totals(Ud).cpu().numpy()
        rng = np.random.default_rng(2)
        cells = rng.choice(n, 24, replace=False)
        G = Ud[:, torch.as_tensor(cells, device="cuda")].cpu().numpy().T
        del Ud, pos
    finally:
        c.set_config(precision=0)
    U0 = oracle.charges_from_prims(np.full(n, 1.0 / n), w.rho, w.vel, w.pres, w.gamma)
    scale = np.abs(U0).sum(0)
    scale[1:4] = max(scale[1:4].max(), np.sqrt(scale[0] * scale[4]))
    assert np.all(np.abs(t1 - t0) <= 1e-12 * scale), (t1 - t0) / scale
    O, _, _, m = H.oracle_local_step(oracle, w.pos, U0, w.box, ocfg, cells, dt)
    l1 = {}
    for name, cols in (("density", [0]), ("momentum", [1, 2, 3]), ("energy", [4])):
        l1[name] = np.abs(G[:, cols] - O[:, cols]).sum() / np.abs(O[:, cols]).sum()
    print("256^3 mixed step, sampled cells: relative L1 vs the FP64 oracle", {k: f"{v:.2e}" for k, v in l1.items()})
    assert max(l1.values()) <= 1e-5, l1


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_ensemble_largest_box_sampled_cells_match_oracle(oracle, gpu, precision):
    """The batched ensemble's largest box (uniform random generators,
    lognormal density from a k^-3 Gaussian field, Gaussian velocities, P = 1,
    gamma 5/3), one step on the device against the oracle's local step on 16
    sampled cells, identical inputs (primitives times the nominal volume 1/n,
    a fixed dt below the CFL step).  FP64: charges to 1e-10 of each
    component's scale, positions to 1e-12; mixed precision: relative L1 of
    density, momentum and energy over the sample <= 1e-5."""
    c, torch = gpu
    sizes = WL.ensemble_sizes(512)
    b = int(np.argmax(sizes))
    w = WL.ensemble_box(b, int(sizes[b]))
    n = w.n
    U0 = oracle.charges_from_prims(np.full(n, 1.0 / n), w.rho, w.vel, w.pres, w.gamma)
    dt = 3e-4  # below the CFL step of the box's smallest cells
    ocfg, gcfg = cfg_pair(oracle, w.gamma, cfl=w.cfl, limiter=1)
    gcfg.precision = precision
    c.set_config(**{f: getattr(gcfg, f) for f, _ in gcfg._fields_})
    try:
        pos = H.to_dev(torch, w.pos.T)
        Ud = H.to_dev(torch, U0.T)
        c.mm_step(pos, Ud, w.box, dt_fixed=torch.tensor([dt], dtype=torch.float64, device="cuda"))
        rng = np.random.default_rng(5)
        cells = rng.choice(n, 16, replace=False)
        G = Ud[:, torch.as_tensor(cells, device="cuda")].cpu().numpy().T
        GP = pos[:, torch.as_tensor(cells, device="cuda")].cpu().numpy().T
    finally:
        c.set_config(precision=0)
    O, OP, _, m = H.oracle_local_step(oracle, w.pos, U0, w.box, ocfg, cells, dt)
    print(f"[ensemble box {b}, {n} cells, precision {precision}] {len(cells)} sampled cells, "
          f"{m} tessellated by the oracle")
    if precision == 0:
        scale = np.abs(O).max(axis=0)
        scale[1:4] = scale[1:4].max()
        for k in range(O.shape[1]):
            np.testing.assert_allclose(G[:, k], O[:, k], rtol=0, atol=RTOL_STEP * scale[k], err_msg=f"component {k}")
        dp = GP - OP
        dp -= np.round(dp / w.box) * w.box
        assert np.abs(dp).max() <= 1e-12
    else:
        l1 = {}
        for name, cols in (("density", [0]), ("momentum", [1, 2, 3]), ("energy", [4])):
            l1[name] = np.abs(G[:, cols] - O[:, cols]).sum() / np.abs(O[:, cols]).sum()
        print("relative L1 vs the FP64 oracle", {k: f"{v:.2e}" for k, v in l1.items()})
        assert max(l1.values()) <= 1e-5, l1


MIXED_CASES = {  # (workload, limiter)
    "smooth_wave_16^3": (lambda: WL.smooth_wave(16), 1),
    "shear_layer_32^3": (lambda: WL.shear_layer(32), 1),
    "shock_tube_64x8x8": (lambda: WL.shock_tube(64, 8, 8), 1),
    "point_blast_16^3": (lambda: WL.point_blast(16), 1),
    "planar_lattice_30x3x3_DM": (lambda: WL.planar_lattice(30, 3, 3), 2),
}


@pytest.mark.parametrize("case", list(MIXED_CASES))
def test_mixed_step_l1_error_and_conservation(oracle, gpu, case):
    """precision=1: FP32 gradients, half step, reconstruction and fluxes, FP64
    update.  One step against the FP64 oracle: relative L1 error of density,
    momentum and energy <= 1e-5, and totals conserved to 1e-12."""
    c, torch = gpu
    maker, limiter = MIXED_CASES[case]
    w = maker()
    T, U = setup(oracle, w)
    ocfg, gcfg = cfg_pair(oracle, w.gamma, cfl=w.cfl, limiter=limiter)
    S = oracle.step(w.pos, U, w.box, ocfg, tess=T)
    gcfg.precision = 1
    c.set_config(**{f: getattr(gcfg, f) for f, _ in gcfg._fields_})
    try:
        pos = H.to_dev(torch, w.pos.T)
        Ud = H.to_dev(torch, U.T)
        t0 = c.mm_totals(Ud).cpu().numpy()
        dt = torch.tensor([S["dt"]], dtype=torch.float64, device="cuda")
        c.mm_step(pos, Ud, w.box, dt_fixed=dt)
        t1 = c.mm_totals(Ud).cpu().numpy()
    finally:
        c.set_config(precision=0)
    G = Ud.cpu().numpy().T
    O = S["U"]
    l1 = {}
    for name, cols in (("density", [0]), ("momentum", [1, 2, 3]), ("energy", [4])):
        l1[name] = np.abs(G[:, cols] - O[:, cols]).sum() / np.abs(O[:, cols]).sum()
    print(case, "relative L1 vs FP64 oracle:", {k: f"{v:.2e}" for k, v in l1.items()})
    assert l1["density"] <= 1e-5 and l1["energy"] <= 1e-5 and l1["momentum"] <= 1e-5, l1
    scale = np.abs(U).sum(0)
    # momentum scale sqrt(M E) (the momentum may start exactly at zero)
    scale[1:4] = max(scale[1:4].max(), np.sqrt(scale[0] * scale[4]))
    assert np.all(np.abs(t1 - t0) <= 1e-12 * scale), (t1 - t0) / scale


HEUN_CASES = {
    "smooth_random_regularized": dict(maker=lambda: WL.smooth_wave(10), kw=dict(limiter=1, regularize=1), random=True),
    "shock_tube_48x6x6_hll": dict(maker=lambda: WL.shock_tube(48, 6, 6), kw=dict(limiter=2, riemann=1)),
    "gresho_vortex_16x16x3": dict(maker=lambda: WL.gresho_vortex(16), kw=dict(limiter=3, regularize=1)),
}


@pytest.mark.parametrize("case", list(HEUN_CASES))
def test_heun_step_matches_oracle(oracle, gpu, case):
    """integrator = 1: stage on the start mesh, drift, second tessellation,
    stage on the end mesh, average (Sec. 6)."""
    c, torch = gpu
    spec = HEUN_CASES[case]
    w = spec["maker"]()
    if spec.get("random"):
        rho, vel, pres = WL.random_state(w.n, seed=13, v_sigma=0.2)
        T, U = setup(oracle, w, rho, vel, pres)
    else:
        T, U = setup(oracle, w)
    ocfg = oracle.make_cfg(gamma=w.gamma, cfl=w.cfl, **spec["kw"])
    from paper_1707_05333_gb300 import binding
    gcfg = binding.default_config(gamma=w.gamma, cfl=w.cfl, integrator=1, **spec["kw"])
    c.set_config(**{f: getattr(gcfg, f) for f, _ in gcfg._fields_})
    try:
        S = oracle.step_heun(w.pos, U, w.box, ocfg, tess=T)
        pos = H.to_dev(torch, w.pos.T)
        Ud = H.to_dev(torch, U.T)
        dt_fixed = torch.tensor([S["dt"]], dtype=torch.float64, device="cuda")
        dt_out = torch.empty((1,), dtype=torch.float64, device="cuda")
        c.mm_step(pos, Ud, w.box, dt_fixed=dt_fixed, dt_out=dt_out)
        assert_state_close(Ud.cpu().numpy(), S["U"])
        dp = pos.cpu().numpy().T - S["pos"]
        dp -= np.round(dp / w.box) * w.box
        assert np.abs(dp).max() <= 1e-12
        # the context's mesh is the end-of-step one
        G = {k: v.cpu().numpy() for k, v in c.mm_current_mesh().to_torch().items()}
        np.testing.assert_allclose(G["cell_volume"], S["tess1"]["volume"], rtol=1e-9)
        c.mm_step(H.to_dev(torch, w.pos.T), H.to_dev(torch, U.T), w.box, dt_out=dt_out)
        assert float(dt_out.item()) == pytest.approx(S["dt_cfl"], rel=1e-13)
    finally:
        c.set_config(integrator=0)
