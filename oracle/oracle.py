"""ctypes wrapper of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this module.  It builds ``mm_oracle.c`` with gcc into ``oracle/_build`` and
composes one hydro step in the order of the paper's outline (Sec. 2):
tessellate -> charges to states -> mesh velocity and CFL timestep ->
limited gradient and half step -> limited half-step gradient -> face fluxes
in the face frame -> charge update -> drift.

Arrays are array-of-structs float64: pos (n,3), W and U (n,ng), grad (n,ng,3),
with ng = 5, or 6 when the entropy column rho A (A = P / rho^gamma) is on.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "mm_oracle.c")
_HDR = os.path.join(_HERE, "mm_oracle.h")
_LIB = os.path.join(_BUILD, "libmm_oracle.so")
_lock = threading.Lock()
_lib = None

AREA_REL = 1e-10  # faces below this fraction of V^(2/3) are dropped (tie rule)


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, no fast-math) if it is out of date."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Cfg(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("cfl", ctypes.c_double), ("eta", ctypes.c_double),
                ("chi", ctypes.c_double), ("zeta", ctypes.c_double), ("theta", ctypes.c_double),
                ("rho_floor", ctypes.c_double), ("eps_floor", ctypes.c_double),
                ("limiter", ctypes.c_int), ("regularize", ctypes.c_int), ("riemann", ctypes.c_int),
                ("entropy", ctypes.c_int), ("mach_th", ctypes.c_double)]


def make_cfg(gamma=5.0 / 3.0, cfl=0.3, eta=1.0, chi=1.0, zeta=0.25, theta=0.49,
             rho_floor=1e-10, eps_floor=1e-10, limiter=1, regularize=0, riemann=0, entropy=0,
             mach_th=1.1) -> Cfg:
    return Cfg(gamma, cfl, eta, chi, zeta, theta, rho_floor, eps_floor, limiter, regularize, riemann, entropy,
               mach_th)


def width(cfg) -> int:
    """State components per cell: 5, or 6 with the entropy column."""
    return 6 if cfg.entropy else 5


_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_tessellate.argtypes = [_I64, _P, _P, ctypes.c_int, ctypes.c_double, _P, _P, _I64, _P,
                                         _P, _P, _P, _P, _P, _P]
            L.orc_tessellate.restype = ctypes.c_int
            L.orc_tessellate_subset.argtypes = [_I64, _P, _P, ctypes.c_double, _I64, _P, _P, _P, _I64,
                                                _P, _P, _P, _P, _P, _P, _P]
            L.orc_tessellate_subset.restype = ctypes.c_int
            L.orc_gradient.argtypes = [_I64, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]
            L.orc_half_step.argtypes = [_I64, _P, _P, _P, ctypes.c_double, _P]
            L.orc_face_flux.argtypes = [_I64, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                        _P, _P, _P, _P]
            L.orc_update.argtypes = [_I64, _I64, _P, _P, _P, _P, _P, ctypes.c_double, _P, _P, _P]
            L.orc_mesh_velocity.argtypes = [_I64, _P, _P, _P, _P, _P, _P]
            L.orc_timestep.argtypes = [_I64, _P, _P, _P, _P]
            L.orc_timestep.restype = ctypes.c_double
            L.orc_drift.argtypes = [_I64, _P, _P, ctypes.c_double, _P]
            L.orc_floor_state.argtypes = [_P, _P, _P, _P]
            L.orc_euler_flux.argtypes = [_P, _P, ctypes.c_double, _P]
            L.orc_flux_jacobian.argtypes = [_P, ctypes.c_int, ctypes.c_double, _P]
            L.orc_riemann_lab.argtypes = [_P, _P, _P, _P, _P, _P, _P]
            L.orc_heun_average.argtypes = [_I64, _P, _P, _P, _P]
            L.orc_star_state.argtypes = [_P, _P, ctypes.c_double, _P, _P, _P, _P]
            L.orc_shock_mach.argtypes = [_P, _P, ctypes.c_double]
            L.orc_shock_mach.restype = ctypes.c_double
            L.orc_hllc_1d.argtypes = [_P, _P, ctypes.c_double, _P]
            L.orc_hll_1d.argtypes = [_P, _P, ctypes.c_double, _P]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


class OracleError(RuntimeError):
    pass


def tessellate(pos, box, mode=1, area_rel=AREA_REL, cells=None):
    """Voronoi cells of the periodic box (Sec. 3).  Returns a dict with
    volume (n,), centroid (n,3) and the directed faces cell, nb, shift (k,3),
    area, normal (k,3), centroid (k,3).  ``cells`` restricts the work to a
    subset (grid mode); volume/centroid are then only valid on that subset."""
    pos = _c(pos)
    box = _c(box)
    n = pos.shape[0]
    m = n if cells is None else len(cells)
    cap = max(64, 48 * m)
    vol = np.zeros(n)
    cen = np.zeros((n, 3))
    f_cell = np.zeros(cap, np.int32)
    f_nb = np.zeros(cap, np.int32)
    f_sh = np.zeros((cap, 3), np.int32)
    f_a = np.zeros(cap)
    f_n = np.zeros((cap, 3))
    f_c = np.zeros((cap, 3))
    nf = ctypes.c_int64(0)
    L = lib()
    if cells is None:
        rc = L.orc_tessellate(n, _p(pos), _p(box), mode, area_rel, _p(vol), _p(cen), cap,
                              ctypes.byref(nf), _p(f_cell), _p(f_nb), _p(f_sh), _p(f_a), _p(f_n),
                              _p(f_c))
    else:
        cl = _c(cells, np.int64)
        rc = L.orc_tessellate_subset(n, _p(pos), _p(box), area_rel, m, _p(cl), _p(vol), _p(cen),
                                     cap, ctypes.byref(nf), _p(f_cell), _p(f_nb), _p(f_sh), _p(f_a),
                                     _p(f_n), _p(f_c))
    if rc != 0:
        raise OracleError(f"orc_tessellate failed with code {rc}")
    k = nf.value
    return dict(volume=vol, centroid=cen, cell=f_cell[:k].copy(), nb=f_nb[:k].copy(),
                shift=f_sh[:k].copy(), area=f_a[:k].copy(), normal=f_n[:k].copy(),
                fcentroid=f_c[:k].copy(), box=box.copy(), n=n)


def shift_code(shift):
    s = np.asarray(shift)
    return (s[..., 0] + 1) + 3 * (s[..., 1] + 1) + 9 * (s[..., 2] + 1)


def unique_faces(T):
    """One record per shared face: i < j, or i == j with the image shift
    whose code is above the zero-shift code (the other copy is its mirror)."""
    code = shift_code(T["shift"])
    keep = (T["cell"] < T["nb"]) | ((T["cell"] == T["nb"]) & (code > 13))
    return dict(i=T["cell"][keep].copy(), j=T["nb"][keep].copy(), shift=T["shift"][keep].copy(),
                area=T["area"][keep].copy(), normal=T["normal"][keep].copy(),
                centroid=T["fcentroid"][keep].copy())


def charges_from_prims(volume, rho, vel, pres, gamma, e_add=None, entropy=False):
    """U = W V with W = (rho, rho v, P/(gamma-1) + rho v^2/2) (Sec. 4), plus
    rho A with A = P / rho^gamma when the entropy column is on (Sec. 4.3; an
    energy deposit e_add raises P accordingly)."""
    vol = np.asarray(volume)
    W = np.zeros((vol.shape[0], 6 if entropy else 5))
    W[:, 0] = rho
    W[:, 1:4] = rho[:, None] * vel
    W[:, 4] = pres / (gamma - 1.0) + 0.5 * rho * np.sum(vel * vel, axis=1)
    U = W * vol[:, None]
    if e_add is not None:
        U[:, 4] += e_add
    if entropy:
        P = pres + (0.0 if e_add is None else (gamma - 1.0) * np.asarray(e_add) / vol)
        U[:, 5] = U[:, 0] * P / np.power(np.asarray(rho, dtype=np.float64), gamma)
    return U


def gradient(F, volume, centroid, box, W, cfg):
    n = W.shape[0]
    assert W.shape[1] == width(cfg)
    grad = np.zeros((n, width(cfg), 3))
    fi, fj, sh = _c(F["i"], np.int32), _c(F["j"], np.int32), _c(F["shift"], np.int32)
    area, nrm, fc = _c(F["area"]), _c(F["normal"]), _c(F["centroid"])
    cen, box, W = _c(centroid), _c(box), _c(W)
    lib().orc_gradient(n, fi.shape[0], _p(fi), _p(fj), _p(sh), _p(area), _p(nrm), _p(fc), _p(cen), _p(box),
                       _p(W), ctypes.byref(cfg), _p(grad))
    return grad


def half_step(W, grad, cfg, dt):
    W, grad = _c(W), _c(grad)
    Wh = np.zeros_like(W)
    lib().orc_half_step(W.shape[0], _p(W), _p(grad), ctypes.byref(cfg), float(dt), _p(Wh))
    return Wh


def face_flux(F, pos, centroid, box, Wh, grad, w, cfg, return_aux=False):
    """Face fluxes A F (nf, ng); with return_aux also (shock Mach number,
    swept-volume rate A w_f . n) per face."""
    nf = F["i"].shape[0]
    flux = np.zeros((nf, width(cfg)))
    mach = np.zeros(nf)
    vrate = np.zeros(nf)
    fi, fj, sh = _c(F["i"], np.int32), _c(F["j"], np.int32), _c(F["shift"], np.int32)
    area, nrm, fc = _c(F["area"]), _c(F["normal"]), _c(F["centroid"])
    pos, cen, box, Wh, grad, w = _c(pos), _c(centroid), _c(box), _c(Wh), _c(grad), _c(w)
    lib().orc_face_flux(Wh.shape[0], nf, _p(fi), _p(fj), _p(sh), _p(area), _p(nrm), _p(fc), _p(pos),
                        _p(cen), _p(box), _p(Wh), _p(grad), _p(w), ctypes.byref(cfg), _p(flux), _p(mach),
                        _p(vrate))
    return (flux, dict(mach=mach, vrate=vrate)) if return_aux else flux


def update(F, flux, dt, volume, cfg, U, aux=None):
    U = _c(U).copy()
    fi, fj = _c(F["i"], np.int32), _c(F["j"], np.int32)
    flux, vol = _c(flux), _c(volume)
    z = np.zeros(fi.shape[0])
    mach = _c(z if aux is None else aux["mach"])
    vrate = _c(z if aux is None else aux["vrate"])
    lib().orc_update(U.shape[0], fi.shape[0], _p(fi), _p(fj), _p(flux), _p(mach), _p(vrate), float(dt), _p(vol),
                     ctypes.byref(cfg), _p(U))
    return U


def mesh_velocity(pos, U, volume, centroid, cfg):
    pos, U, vol, cen = _c(pos), _c(U), _c(volume), _c(centroid)
    w = np.zeros((U.shape[0], 3))
    lib().orc_mesh_velocity(U.shape[0], _p(pos), _p(U), _p(vol), _p(cen), ctypes.byref(cfg), _p(w))
    return w


def timestep(U, volume, w, cfg):
    U, vol, w = _c(U), _c(volume), _c(w)
    return lib().orc_timestep(U.shape[0], _p(U), _p(vol), _p(w), ctypes.byref(cfg))


def drift(pos, w, dt, box):
    pos = _c(pos).copy()
    w, box = _c(w), _c(box)
    lib().orc_drift(pos.shape[0], _p(pos), _p(w), float(dt), _p(box))
    return pos


def floor_state(W, cfg):
    W = _c(W)
    out = np.zeros(5)
    ch = ctypes.c_int(0)
    lib().orc_floor_state(_p(W), ctypes.byref(cfg), _p(out), ctypes.byref(ch))
    return out, bool(ch.value)


def euler_flux(W, nrm, gamma):
    W, nrm = _c(W), _c(nrm)
    F = np.zeros(5)
    lib().orc_euler_flux(_p(W), _p(nrm), float(gamma), _p(F))
    return F


def flux_jacobian(W, d, gamma):
    W = _c(W)
    A = np.zeros((5, 5))
    lib().orc_flux_jacobian(_p(W), int(d), float(gamma), _p(A))
    return A


def riemann_lab(WL, WR, nrm, wface, cfg, return_mach=False):
    WL, WR, nrm, wface = _c(WL), _c(WR), _c(nrm), _c(wface)
    F = np.zeros(width(cfg))
    m = ctypes.c_double(0.0)
    lib().orc_riemann_lab(_p(WL), _p(WR), _p(nrm), _p(wface), ctypes.byref(cfg), _p(F), ctypes.byref(m))
    return (F, m.value) if return_mach else F


def star_state(primL, primR, gamma):
    """(S_L, S*, S_R, P*) of the HLLC model for 1-D states (rho, u, v1, v2, P)."""
    L, R = _c(primL), _c(primR)
    out = [ctypes.c_double() for _ in range(4)]
    lib().orc_star_state(_p(L), _p(R), float(gamma), *[ctypes.byref(o) for o in out])
    return tuple(o.value for o in out)


def shock_mach(primL, primR, gamma):
    L, R = _c(primL), _c(primR)
    return lib().orc_shock_mach(_p(L), _p(R), float(gamma))


def hll_1d(primL, primR, gamma):
    L, R = _c(primL), _c(primR)
    F = np.zeros(5)
    lib().orc_hll_1d(_p(L), _p(R), float(gamma), _p(F))
    return F


def hllc_1d(primL, primR, gamma):
    L, R = _c(primL), _c(primR)
    F = np.zeros(5)
    lib().orc_hllc_1d(_p(L), _p(R), float(gamma), _p(F))
    return F


def step(pos, U, box, cfg, mode=1, dt=None, tess=None, w=None):
    """One step of the moving-mesh method (Sec. 2), returning every stage.
    w, if given, prescribes the generator velocities instead of Sec. 4.2's."""
    pos = _c(pos)
    T = tess if tess is not None else tessellate(pos, box, mode)
    F = unique_faces(T)
    vol, cen = T["volume"], T["centroid"]
    W = U / vol[:, None]
    w = mesh_velocity(pos, U, vol, cen, cfg) if w is None else _c(w)
    dt_cfl = timestep(U, vol, w, cfg)
    if dt is None:
        dt = dt_cfl
    g0 = gradient(F, vol, cen, box, W, cfg)
    Wh = half_step(W, g0, cfg, dt)
    g1 = gradient(F, vol, cen, box, Wh, cfg)
    flux, aux = face_flux(F, pos, cen, box, Wh, g1, w, cfg, return_aux=True)
    U1 = update(F, flux, dt, vol, cfg, U, aux)
    pos1 = drift(pos, w, dt, box)
    return dict(tess=T, faces=F, W=W, w=w, dt=dt, dt_cfl=dt_cfl, grad0=g0, Wh=Wh, grad1=g1,
                flux=flux, mach=aux["mach"], vrate=aux["vrate"], U=U1, pos=pos1)


def heun_average(U0, U, volume, cfg):
    U0, vol = _c(U0), _c(volume)
    U = _c(U).copy()
    lib().orc_heun_average(U.shape[0], _p(U0), _p(vol), ctypes.byref(cfg), _p(U))
    return U


def stage(F, pos, vol, cen, box, U, w, dt, cfg):
    """One forward-Euler stage of Heun's method on a fixed mesh: limited
    gradient of W = U / V, reconstruction in space only (no half step),
    face fluxes with the generators moving at w, and the charge update."""
    W = U / vol[:, None]
    g = gradient(F, vol, cen, box, W, cfg)
    flux = face_flux(F, pos, cen, box, W, g, w, cfg)
    return update(F, flux, dt, vol, cfg, U)


def step_heun(pos, U, box, cfg, mode=1, dt=None, tess=None, w=None):
    """Second-order time integration by Heun's method (Sec. 6, future item
    "true second order time integration"): fluxes at the start of the step
    on the start mesh and at its end on the mesh of the drifted generators
    are averaged.  The generators move at their start velocity w throughout
    (Sec. 4.2's, or the one given)."""
    assert not cfg.entropy, "the entropy switch is defined for the half-step scheme only"
    pos = _c(pos)
    T0 = tess if tess is not None else tessellate(pos, box, mode)
    F0 = unique_faces(T0)
    vol0, cen0 = T0["volume"], T0["centroid"]
    w = mesh_velocity(pos, U, vol0, cen0, cfg) if w is None else _c(w)
    dt_cfl = timestep(U, vol0, w, cfg)
    if dt is None:
        dt = dt_cfl
    U1 = stage(F0, pos, vol0, cen0, box, U, w, dt, cfg)
    pos1 = drift(pos, w, dt, box)
    T1 = tessellate(pos1, box, mode)
    F1 = unique_faces(T1)
    U2 = stage(F1, pos1, T1["volume"], T1["centroid"], box, U1, w, dt, cfg)
    U3 = heun_average(U, U2, T1["volume"], cfg)
    return dict(tess=T0, tess1=T1, w=w, dt=dt, dt_cfl=dt_cfl, U1=U1, U2=U2, U=U3, pos=pos1)
