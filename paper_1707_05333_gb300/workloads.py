"""Seeded synthetic inputs shaped like the paper's test problems.

This module is the only code shared by the CPU oracle and the CUDA path.  It
draws generator positions and samples initial primitive fields (density,
velocity, pressure) at those positions; it holds none of the method's
arithmetic (no tessellation, no charges, no fluxes).  Charges U = W V need the
cell volumes, so each side turns the primitives into charges itself.

Every workload uses numpy's PCG64 with seed 1707 + workload index (+ box index
for the ensemble), so both sides read identical bytes.

The paper's own initial conditions are built from a 4096-particle glass block
replicated 16^3 times (Sec. 5); that glass is not available, so a cubic lattice
with seeded uniform jitter of +-0.1 spacing stands in for it.
"""
from __future__ import annotations

import dataclasses

import numpy as np

SEED_BASE = 1707


@dataclasses.dataclass
class Workload:
    """One periodic box: generators plus initial primitives sampled at them.

    pos   (n, 3) float64, every coordinate in [0, box[d])
    rho   (n,)   float64 density
    vel   (n, 3) float64 velocity
    pres  (n,)   float64 pressure
    e_add (n,)   float64 energy *charge* added on top of the sampled state
                 (the point-blast deposit; zero elsewhere)
    """

    name: str
    pos: np.ndarray
    box: np.ndarray
    rho: np.ndarray
    vel: np.ndarray
    pres: np.ndarray
    e_add: np.ndarray
    gamma: float
    cfl: float
    steps: int

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def jittered_lattice(shape, box, rng, jitter=0.1):
    """Points (i+1/2, j+1/2, k+1/2) h + U(-jitter h, +jitter h)^3, x fastest."""
    nx, ny, nz = shape
    box = np.asarray(box, dtype=np.float64)
    h = box / np.array(shape, dtype=np.float64)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    base = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64) + 0.5
    pos = base * h
    if jitter > 0.0:
        pos = pos + rng.uniform(-jitter, jitter, size=pos.shape) * h
    return np.mod(pos, box)


def _finish(name, pos, box, rho, vel, pres, gamma, cfl, steps, e_add=None):
    n = pos.shape[0]
    return Workload(
        name=name,
        pos=np.ascontiguousarray(pos, dtype=np.float64),
        box=np.asarray(box, dtype=np.float64),
        rho=np.ascontiguousarray(rho, dtype=np.float64),
        vel=np.ascontiguousarray(vel, dtype=np.float64),
        pres=np.ascontiguousarray(pres, dtype=np.float64),
        e_add=np.zeros(n) if e_add is None else np.ascontiguousarray(e_add, dtype=np.float64),
        gamma=float(gamma),
        cfl=float(cfl),
        steps=int(steps),
    )


def smooth_wave(n_side=16, jitter=0.1, seed_offset=0):
    """Periodic unit box, rho=1, P=1, v = 0.01 sin(2 pi x) (1,1,1), gamma=5/3."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + seed_offset))
    box = np.ones(3)
    pos = jittered_lattice((n_side,) * 3, box, rng, jitter)
    n = pos.shape[0]
    s = 0.01 * np.sin(2.0 * np.pi * pos[:, 0])
    vel = np.stack([s, s, s], axis=1)
    return _finish(f"smooth_wave_{n_side}^3", pos, box, np.ones(n), vel, np.ones(n),
                   5.0 / 3.0, 0.3, 1)


def shock_tube(nx=128, ny=16, nz=16, length=8.0, jitter=0.1):
    """Sod tube in a periodic length x 1 x 1 box, gamma=1.4 (Sec. 5.1 analogue).

    x < length/2: rho=1, P=1; else rho=0.125, P=0.1; v=0.  Run to t=0.2.
    """
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 1))
    box = np.array([length, 1.0, 1.0])
    pos = jittered_lattice((nx, ny, nz), box, rng, jitter)
    left = pos[:, 0] < 0.5 * length
    rho = np.where(left, 1.0, 0.125)
    pres = np.where(left, 1.0, 0.1)
    vel = np.zeros_like(pos)
    return _finish(f"shock_tube_{nx}x{ny}x{nz}", pos, box, rho, vel, pres, 1.4, 0.3, 0)


def point_blast(n_side=64, jitter=0.1):
    """Sedov-Taylor analogue (Sec. 5.2): rho=1, P=1e-5, gamma=5/3, and a
    thermal energy of 1 split equally over the 8 generators nearest the
    box centre (ties broken by index)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 2))
    box = np.ones(3)
    pos = jittered_lattice((n_side,) * 3, box, rng, jitter)
    n = pos.shape[0]
    d2 = np.sum((pos - 0.5) ** 2, axis=1)
    order = np.lexsort((np.arange(n), d2))
    e_add = np.zeros(n)
    e_add[order[:8]] = 1.0 / 8.0
    return _finish(f"point_blast_{n_side}^3", pos, box, np.ones(n), np.zeros((n, 3)),
                   np.full(n, 1e-5), 5.0 / 3.0, 0.3, 200, e_add)


def shear_layer(n_side=256, jitter=0.1):
    """3-D shear layer in the periodic unit box, gamma=5/3, P=2.5:
    rho=2, vx=+0.5 for |y-0.5|<0.25, else rho=1, vx=-0.5; vy=0.01 sin(4 pi x)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 3))
    box = np.ones(3)
    pos = jittered_lattice((n_side,) * 3, box, rng, jitter)
    n = pos.shape[0]
    inner = np.abs(pos[:, 1] - 0.5) < 0.25
    rho = np.where(inner, 2.0, 1.0)
    vel = np.zeros((n, 3))
    vel[:, 0] = np.where(inner, 0.5, -0.5)
    vel[:, 1] = 0.01 * np.sin(4.0 * np.pi * pos[:, 0])
    return _finish(f"shear_layer_{n_side}^3", pos, box, rho, vel, np.full(n, 2.5),
                   5.0 / 3.0, 0.3, 20)


def gresho_vphi(r):
    """Tangential velocity of the Gresho-Chan vortex (Sec. 5.3): 5r inside
    r < 0.2, 2 - 5r on 0.2 <= r < 0.4, zero beyond."""
    r = np.asarray(r, dtype=np.float64)
    return np.where(r < 0.2, 5.0 * r, np.where(r < 0.4, 2.0 - 5.0 * r, 0.0))


def gresho_pressure(r):
    """Pressure of the Gresho-Chan vortex (Sec. 5.3): 5 + 12.5 r^2 inside
    r < 0.2, 9 + 12.5 r^2 - 20 r + 4 ln(5r) on 0.2 <= r < 0.4, 3 + 4 ln 2
    beyond."""
    r = np.asarray(r, dtype=np.float64)
    mid = 9.0 + 12.5 * r * r - 20.0 * r + 4.0 * np.log(np.maximum(5.0 * r, 1e-300))
    return np.where(r < 0.2, 5.0 + 12.5 * r * r, np.where(r < 0.4, mid, 3.0 + 4.0 * np.log(2.0)))


def gresho_vortex(n_side=64, jitter=0.1, gamma=5.0 / 3.0):
    """Gresho-Chan vortex (Sec. 5.3) in the periodic 1 x 1 x 0.2 box, centred
    at (0.5, 0.5): rho = 1, v = v_phi(r) e_phi, P(r), run to t = 2.  The
    lattice is n x n x round(0.2 n), so the equivalent 2-D resolution is n^2
    (the paper's run: n = 64, about 50K generators).  gamma is not stated
    for this test; 5/3 as in the other tests."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 1000 + n_side))
    nz = max(1, int(round(0.2 * n_side)))
    box = np.array([1.0, 1.0, 0.2])
    pos = jittered_lattice((n_side, n_side, nz), box, rng, jitter)
    n = pos.shape[0]
    dx, dy = pos[:, 0] - 0.5, pos[:, 1] - 0.5
    r = np.hypot(dx, dy)
    vphi = gresho_vphi(r)
    inv = np.where(r > 0, 1.0 / np.maximum(r, 1e-300), 0.0)
    vel = np.zeros((n, 3))
    vel[:, 0] = -vphi * dy * inv
    vel[:, 1] = vphi * dx * inv
    return _finish(f"gresho_vortex_{n_side}x{n_side}x{nz}", pos, box, np.ones(n), vel, gresho_pressure(r),
                   gamma, 0.3, 0)


def gaussian_random_field(rng, n_grid=64, slope=-3.0):
    """Unit-variance periodic Gaussian random field with power spectrum k^slope."""
    k = np.fft.fftfreq(n_grid) * n_grid
    kx, ky, kz = np.meshgrid(k, k, k, indexing="ij")
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(kk)
    nz = kk > 0
    amp[nz] = kk[nz] ** (0.5 * slope)
    noise = rng.standard_normal((n_grid,) * 3)
    field = np.real(np.fft.ifftn(np.fft.fftn(noise) * amp))
    field -= field.mean()
    field /= field.std()
    return field


def trilinear_periodic(field, pos):
    """Sample a periodic grid field (cell-centred on the unit box) at pos."""
    n = field.shape[0]
    x = pos * n - 0.5
    i0 = np.floor(x).astype(np.int64)
    f = x - i0
    out = np.zeros(pos.shape[0])
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = ((f[:, 0] if dx else 1 - f[:, 0]) *
                     (f[:, 1] if dy else 1 - f[:, 1]) *
                     (f[:, 2] if dz else 1 - f[:, 2]))
                out += w * field[(i0[:, 0] + dx) % n, (i0[:, 1] + dy) % n, (i0[:, 2] + dz) % n]
    return out


def ensemble_box(b, n_cells):
    """One box of the batched ensemble: uniform random generators in the unit
    box, lognormal density exp(0.5 g - 0.125) from a k^-3 Gaussian random
    field g, Gaussian velocities (sigma 0.1), P=1, gamma=5/3."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 4 + 1 + b))
    box = np.ones(3)
    pos = rng.uniform(0.0, 1.0, size=(n_cells, 3))
    g = trilinear_periodic(gaussian_random_field(rng), pos)
    rho = np.exp(0.5 * g - 0.125)
    vel = rng.normal(0.0, 0.1, size=(n_cells, 3))
    return _finish(f"ensemble_box_{b}", pos, box, rho, vel, np.ones(n_cells), 5.0 / 3.0, 0.3, 1)


def ensemble_sizes(n_boxes=512, lo_log2=10.0, hi_log2=16.0):
    """Cell counts round(2^U(lo, hi)) for the batched ensemble (seeded)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 4))
    return np.rint(2.0 ** rng.uniform(lo_log2, hi_log2, size=n_boxes)).astype(np.int64)


def random_points(n, box=(1.0, 1.0, 1.0), seed=0):
    """Uniform random generators, for tests (seed relative to the base)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 100 + seed))
    box = np.asarray(box, dtype=np.float64)
    return rng.uniform(0.0, 1.0, size=(n, 3)) * box


def random_state(n, seed=0, rho_range=(0.5, 2.0), v_sigma=0.3, p_range=(0.5, 2.0)):
    """Random smooth-free primitives for unit tests (seeded)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 200 + seed))
    rho = rng.uniform(*rho_range, size=n)
    vel = rng.normal(0.0, v_sigma, size=(n, 3))
    pres = rng.uniform(*p_range, size=n)
    return rho, vel, pres


WORKLOADS = {
    "smooth_wave": smooth_wave,
    "shock_tube": shock_tube,
    "point_blast": point_blast,
    "shear_layer": shear_layer,
    "gresho_vortex": gresho_vortex,
}


def planar_profile(x):
    """Primitives (rho, u, P) of a planar state along x in [0, 1): a smooth
    wave with a raised block in density and pressure on [0.3, 0.6) (a
    contact and two jumps), flowing at u = 0.1 + 0.2 cos 2 pi x."""
    blk = ((x >= 0.3) & (x < 0.6)).astype(np.float64)
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * x) + 0.5 * blk
    u = 0.1 + 0.2 * np.cos(2 * np.pi * x)
    P = 1.0 + 0.2 * np.sin(4 * np.pi * x) + 0.6 * blk
    return rho, u, P


def planar_lattice(nx, ny, nz):
    """An exact cubic lattice of spacing h = 1/nx (no jitter) in the box
    (1, ny h, nz h), cells in x-major order, carrying planar_profile along x
    (gamma = 5/3): the mesh is the Cartesian grid and the flow one-dimensional."""
    h = 1.0 / nx
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
    pos = np.stack([(ix + 0.5) * h, (iy + 0.5) * h, (iz + 0.5) * h], axis=1)
    rho, u, P = planar_profile(pos[:, 0])
    vel = np.zeros((len(pos), 3))
    vel[:, 0] = u
    return _finish(f"planar_lattice_{nx}x{ny}x{nz}", pos, np.array([1.0, ny * h, nz * h]), rho, vel, P,
                   5.0 / 3.0, 0.3, 1)


def clustered_points(n, core_fraction=0.5, core_scale=0.02, seed=0):
    """Strongly clustered generators for robustness tests (seeded): a
    fraction of the points in a Plummer-like core (radius drawn so that the
    enclosed fraction is r^3 / (r^2 + a^2)^(3/2), a = core_scale) about the
    box centre, the rest uniform; positions wrapped into the unit box."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 300 + seed))
    nc = int(round(core_fraction * n))
    u = rng.uniform(1e-6, 0.999, size=nc)
    r = core_scale / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
    d = rng.normal(size=(nc, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    core = 0.5 + np.minimum(r, 0.45)[:, None] * d
    rest = rng.uniform(0.0, 1.0, size=(n - nc, 3))
    return np.concatenate([core, rest]) % 1.0


def clustered_box(n=6000, seed=1):
    """A clustered point set (clustered_points) in the periodic unit box with
    a uniform gas at rest (rho = 1, P = 1, gamma = 5/3): the mesh, not the
    flow, is the test."""
    pos = clustered_points(n, seed=seed)
    return _finish(f"clustered_{n}", pos, np.ones(3), np.ones(n), np.zeros((n, 3)), np.ones(n), 5.0 / 3.0, 0.3, 1)
