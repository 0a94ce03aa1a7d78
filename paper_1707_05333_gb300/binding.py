"""Python binding of libmm (the C ABI in include/mm.h), argument marshalling only.

Every stage of the step runs in the CUDA library; this module only passes
torch tensors' device pointers and sizes through ctypes and turns status codes
into exceptions.  There is no fallback: without the built library (see
``build.py``) and a CUDA device, every call raises.

Layouts follow the C ABI: positions (3, n), charges and per-volume states
(5, n) or (6, n) with the entropy column, velocities (3, n), gradients (15, n)
or (18, n); all float64, contiguous, on the
context's device.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

_lib = None

_c_i64 = ctypes.c_int64
_c_p = ctypes.c_void_p


class MMError(RuntimeError):
    """A libmm call returned a nonzero mm_status."""

    def __init__(self, name, status, msg):
        super().__init__(f"{name} failed with status {status} ({STATUS.get(status, '?')}): {msg}")
        self.status = status


STATUS = {0: "MM_OK", 1: "MM_EINVAL", 2: "MM_ENOMEM", 3: "MM_ECAPACITY", 4: "MM_EDEGENERATE",
          5: "MM_ECUDA", 6: "MM_ETIMEOUT"}


class Config(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("cfl", ctypes.c_double), ("eta", ctypes.c_double),
                ("chi", ctypes.c_double), ("zeta", ctypes.c_double), ("theta", ctypes.c_double),
                ("rho_floor", ctypes.c_double), ("eps_floor", ctypes.c_double),
                ("area_rel", ctypes.c_double), ("limiter", ctypes.c_int), ("regularize", ctypes.c_int),
                ("precision", ctypes.c_int), ("collect_stats", ctypes.c_int),
                ("riemann", ctypes.c_int), ("clip_warps", ctypes.c_int), ("cand_cap", ctypes.c_int),
                ("clip_filter", ctypes.c_int), ("bin_scale", ctypes.c_double),
                ("mach_th", ctypes.c_double), ("entropy", ctypes.c_int), ("integrator", ctypes.c_int),
                ("clip_sort", ctypes.c_int)]


class MeshStruct(ctypes.Structure):
    _fields_ = [("n", _c_i64), ("nfaces", _c_i64), ("nincident", _c_i64), ("face_stride", _c_i64),
                ("box", ctypes.c_double * 3), ("nboxes", _c_i64), ("cell_box", _c_p), ("box_size", _c_p),
                ("face_i", _c_p), ("face_j", _c_p), ("face_shift", _c_p), ("face_area", _c_p),
                ("face_normal", _c_p), ("face_centroid", _c_p), ("cell_volume", _c_p),
                ("cell_centroid", _c_p), ("inc_off", _c_p), ("inc_face", _c_p)]


EXPORTS = ["mm_default_config", "mm_create", "mm_destroy", "mm_last_error", "mm_set_config",
           "mm_tessellate", "mm_gradients", "mm_mesh_velocity", "mm_timestep", "mm_flux_step",
           "mm_drift", "mm_step", "mm_prims_to_charges", "mm_totals", "mm_copy", "mm_tess_stats",
           "mm_set_timing", "mm_stage_times", "mm_kernel_launches", "mm_totals_noalloc", "mm_step_batched",
           "mm_sync_status", "mm_current_mesh", "mm_get_config", "mm_autotune", "mm_step_host"]

STATS = ["max_candidates", "max_planes", "max_vertices", "multi_ring_cells", "cuts", "fp64_plane_tests",
         "fp64_vertex_solves", "fp64_fan_terms", "candidates_tested", "retried_cells"]

STAGES = ["bin", "clip", "faces", "mesh_velocity", "gradient_half_step", "gradient", "face_flux", "update",
          "drift"]


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libmm.so (built in-tree).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libmm.so is not built ({path}); run paper_1707_05333_gb300.build.build()")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    L.mm_default_config.argtypes = [P(Config)]
    L.mm_default_config.restype = None
    L.mm_create.argtypes = [P(_c_p), P(Config), _c_p]
    L.mm_destroy.argtypes = [_c_p]
    L.mm_destroy.restype = None
    L.mm_last_error.argtypes = [_c_p]
    L.mm_last_error.restype = ctypes.c_char_p
    L.mm_set_config.argtypes = [_c_p, P(Config)]
    L.mm_tessellate.argtypes = [_c_p, _c_p, _c_i64, P(ctypes.c_double), P(MeshStruct)]
    L.mm_gradients.argtypes = [_c_p, P(MeshStruct), _c_p, _c_p]
    L.mm_mesh_velocity.argtypes = [_c_p, P(MeshStruct), _c_p, _c_p, _c_p]
    L.mm_timestep.argtypes = [_c_p, P(MeshStruct), _c_p, _c_p, _c_p]
    L.mm_flux_step.argtypes = [_c_p, P(MeshStruct), _c_p, _c_p, _c_p, _c_p]
    L.mm_drift.argtypes = [_c_p, _c_p, _c_i64, _c_p, _c_p, P(ctypes.c_double)]
    L.mm_step.argtypes = [_c_p, _c_p, _c_p, _c_i64, P(ctypes.c_double), _c_p, _c_p, _c_p]
    L.mm_prims_to_charges.argtypes = [_c_p, P(MeshStruct), _c_p, _c_p, _c_p, _c_p]
    L.mm_totals.argtypes = [_c_p, _c_p, _c_i64, _c_p]
    L.mm_copy.argtypes = [_c_p, _c_p, _c_p, _c_i64]
    L.mm_tess_stats.argtypes = [_c_p, P(_c_i64)]
    L.mm_set_timing.argtypes = [_c_p, ctypes.c_int]
    L.mm_stage_times.argtypes = [_c_p, P(ctypes.c_double), P(_c_i64)]
    L.mm_step_batched.argtypes = [_c_p, _c_p, _c_p, _c_i64, P(_c_i64), P(ctypes.c_double), ctypes.c_int, _c_p]
    L.mm_step_host.argtypes = [_c_p, _c_p, _c_p, _c_i64, P(ctypes.c_double), _c_p]
    L.mm_sync_status.argtypes = [_c_p]
    L.mm_get_config.argtypes = [_c_p, P(Config)]
    L.mm_autotune.argtypes = [_c_p, _c_p, _c_i64, P(ctypes.c_double), ctypes.c_int, P(ctypes.c_double)]
    L.mm_current_mesh.argtypes = [_c_p, P(MeshStruct)]
    L.mm_totals_noalloc.argtypes = [_c_p, _c_i64, _c_p, _c_p, ctypes.c_char_p, _c_i64]
    L.mm_kernel_launches.argtypes = [_c_p]
    L.mm_kernel_launches.restype = _c_i64
    for name in EXPORTS:
        if name not in ("mm_default_config", "mm_destroy", "mm_last_error", "mm_kernel_launches"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def mm_totals_noalloc(U: torch.Tensor, totals: torch.Tensor, stream: torch.cuda.Stream | None = None) -> None:
    """Totals of U (5, n) into totals (5,) through the allocation-free entry point."""
    L = load()
    n = U.shape[1]
    buf = ctypes.create_string_buffer(256)
    s = stream or torch.cuda.current_stream()
    st = L.mm_totals_noalloc(_ptr(U, (5, n)), n, _ptr(totals, (5,)), _c_p(s.cuda_stream), buf, len(buf))
    if st != 0:
        raise MMError("mm_totals_noalloc", st, buf.value.decode())


def default_config(**kw) -> Config:
    cfg = Config()
    load().mm_default_config(ctypes.byref(cfg))
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise KeyError(f"unknown mm_config field {k}")
        setattr(cfg, k, v)
    return cfg


def _ptr(t: torch.Tensor | None, shape=None, dtype=torch.float64):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libmm takes device tensors")
    if t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(t: torch.Tensor | None, shape=None, dtype=torch.float64):
    """Pointer to a contiguous host tensor (the host-buffer step)."""
    if t is None:
        return None
    if t.device.type != "cpu":
        raise ValueError("expected a host tensor")
    if t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Mesh:
    """The context-owned mesh of the last tessellation (valid until the next)."""

    def __init__(self, ctx: "Context", s: MeshStruct):
        self.ctx = ctx
        self.s = s

    @property
    def n(self):
        return int(self.s.n)

    @property
    def nfaces(self):
        return int(self.s.nfaces)

    def _copy(self, ptr, shape, dtype, stride=None):
        out = torch.empty(shape, dtype=dtype, device=self.ctx.device)
        nbytes = out.numel() * out.element_size()
        if out.numel() == 0:
            return out
        if stride is None:
            self.ctx._call("mm_copy", self.ctx.h, _ptr(out, dtype=dtype), ctypes.c_void_p(ptr), nbytes)
        else:
            row = shape[1] * out.element_size()
            for r in range(shape[0]):
                self.ctx._call("mm_copy", self.ctx.h, ctypes.c_void_p(out[r].data_ptr()),
                               ctypes.c_void_p(ptr + r * stride * out.element_size()), row)
        return out

    def to_torch(self) -> dict:
        """Copies of the mesh arrays as torch tensors (same layouts as the ABI)."""
        s = self.s
        n, nf, ni = int(s.n), int(s.nfaces), int(s.nincident)
        return dict(
            face_i=self._copy(s.face_i, (nf,), torch.int32),
            face_j=self._copy(s.face_j, (nf,), torch.int32),
            face_shift=self._copy(s.face_shift, (nf,), torch.int32),
            face_area=self._copy(s.face_area, (nf,), torch.float64),
            face_normal=self._copy(s.face_normal, (3, nf), torch.float64, stride=int(s.face_stride)),
            face_centroid=self._copy(s.face_centroid, (3, nf), torch.float64, stride=int(s.face_stride)),
            cell_volume=self._copy(s.cell_volume, (n,), torch.float64),
            cell_centroid=self._copy(s.cell_centroid, (3, n), torch.float64),
            inc_off=self._copy(s.inc_off, (n + 1,), torch.int32),
            inc_face=self._copy(s.inc_face, (ni,), torch.int32),
        )


class Context:
    """An mm_ctx bound to one CUDA stream of the current device."""

    def __init__(self, config: Config | None = None, stream: torch.cuda.Stream | None = None, **kw):
        if not torch.cuda.is_available():
            raise RuntimeError("libmm needs a CUDA device")
        self.L = load()
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream or torch.cuda.current_stream()
        self.config = config or default_config(**kw)
        h = _c_p()
        st = self.L.mm_create(ctypes.byref(h), ctypes.byref(self.config), _c_p(self.stream.cuda_stream))
        if st != 0:
            raise MMError("mm_create", st, "context creation failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.mm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, *args):
        st = getattr(self.L, name)(*args)
        if st != 0:
            raise MMError(name, st, self.L.mm_last_error(self.h).decode())

    def set_config(self, **kw):
        for k, v in kw.items():
            setattr(self.config, k, v)
        self._call("mm_set_config", self.h, ctypes.byref(self.config))

    def mm_tessellate(self, pos: torch.Tensor, box) -> Mesh:
        n = pos.shape[1]
        b = (ctypes.c_double * 3)(*[float(x) for x in box])
        s = MeshStruct()
        self._call("mm_tessellate", self.h, _ptr(pos, (3, n)), n, b, ctypes.byref(s))
        return Mesh(self, s)

    @property
    def ng(self) -> int:
        """Rows of the charges: 5, or 6 with the entropy column."""
        return 6 if self.config.entropy else 5

    def mm_gradients(self, mesh: Mesh, W: torch.Tensor) -> torch.Tensor:
        grad = torch.empty((3 * self.ng, mesh.n), dtype=torch.float64, device=self.device)
        self._call("mm_gradients", self.h, ctypes.byref(mesh.s), _ptr(W, (self.ng, mesh.n)), _ptr(grad))
        return grad

    def mm_mesh_velocity(self, mesh: Mesh, pos, U) -> torch.Tensor:
        w = torch.empty((3, mesh.n), dtype=torch.float64, device=self.device)
        self._call("mm_mesh_velocity", self.h, ctypes.byref(mesh.s), _ptr(pos, (3, mesh.n)),
                   _ptr(U, (self.ng, mesh.n)), _ptr(w))
        return w

    def mm_timestep(self, mesh: Mesh, U, w) -> torch.Tensor:
        dt = torch.empty((1,), dtype=torch.float64, device=self.device)
        self._call("mm_timestep", self.h, ctypes.byref(mesh.s), _ptr(U, (self.ng, mesh.n)), _ptr(w, (3, mesh.n)),
                   _ptr(dt))
        return dt

    def mm_flux_step(self, mesh: Mesh, pos, w, dt: torch.Tensor, U: torch.Tensor) -> None:
        self._call("mm_flux_step", self.h, ctypes.byref(mesh.s), _ptr(pos, (3, mesh.n)), _ptr(w, (3, mesh.n)),
                   _ptr(dt, (1,)), _ptr(U, (self.ng, mesh.n)))

    def mm_drift(self, pos, w, dt: torch.Tensor, box) -> None:
        n = pos.shape[1]
        b = (ctypes.c_double * 3)(*[float(x) for x in box])
        self._call("mm_drift", self.h, _ptr(pos, (3, n)), n, _ptr(w, (3, n)), _ptr(dt, (1,)), b)

    def mm_step(self, pos, U, box, dt_fixed: torch.Tensor | None = None, dt_out=None, w_out=None):
        n = pos.shape[1]
        b = (ctypes.c_double * 3)(*[float(x) for x in box])
        self._call("mm_step", self.h, _ptr(pos, (3, n)), _ptr(U, (self.ng, n)), n, b,
                   _ptr(dt_fixed, (1,)), _ptr(dt_out, (1,)), _ptr(w_out, (3, n)))

    def mm_step_host(self, pos, U, box, dt_out=None):
        """One step on host tensors (pos [3][n], U [5 or 6][n], float64, in place;
        page-locked memory lets the library overlap the copies with the step).
        dt_out: optional host float64 tensor of one element."""
        n = pos.shape[1]
        b = (ctypes.c_double * 3)(*[float(x) for x in box])
        self._call("mm_step_host", self.h, _hptr(pos, (3, n)), _hptr(U, (self.ng, n)), n, b, _hptr(dt_out, (1,)))

    def mm_step_batched(self, pos, U, box_off, boxes, dt_out=None):
        """One step of independent periodic boxes stored back to back (replays a
        captured CUDA graph after the first call with the same arguments)."""
        import numpy as _np
        n = pos.shape[1]
        off = _np.ascontiguousarray(box_off, dtype=_np.int64)
        bx = _np.ascontiguousarray(boxes, dtype=_np.float64).reshape(-1)
        nbox = len(off) - 1
        self._keep = (off, bx)
        self._call("mm_step_batched", self.h, _ptr(pos, (3, n)), _ptr(U, (self.ng, n)), n,
                   off.ctypes.data_as(ctypes.POINTER(_c_i64)), bx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                   nbox, _ptr(dt_out, (nbox,)))

    def mm_get_config(self) -> Config:
        cfg = Config()
        self._call("mm_get_config", self.h, ctypes.byref(cfg))
        return cfg

    def mm_autotune(self, pos, box, reps: int = 1) -> dict:
        """Time the clipper over its tunable settings and keep the fastest."""
        n = pos.shape[1]
        b = (ctypes.c_double * 3)(*[float(x) for x in box])
        best = ctypes.c_double(0.0)
        self._call("mm_autotune", self.h, _ptr(pos, (3, n)), n, b, int(reps), ctypes.byref(best))
        cfg = self.mm_get_config()
        self.config = cfg
        return {"clip_warps": cfg.clip_warps, "cand_cap": cfg.cand_cap, "bin_scale": cfg.bin_scale,
                "clip_sort": cfg.clip_sort, "tessellate_ms": best.value}

    def mm_sync_status(self) -> None:
        self._call("mm_sync_status", self.h)

    def mm_current_mesh(self) -> Mesh:
        s = MeshStruct()
        self._call("mm_current_mesh", self.h, ctypes.byref(s))
        return Mesh(self, s)

    def mm_prims_to_charges(self, mesh: Mesh, rho, vel, P) -> torch.Tensor:
        U = torch.empty((self.ng, mesh.n), dtype=torch.float64, device=self.device)
        self._call("mm_prims_to_charges", self.h, ctypes.byref(mesh.s), _ptr(rho, (mesh.n,)),
                   _ptr(vel, (3, mesh.n)), _ptr(P, (mesh.n,)), _ptr(U))
        return U

    def mm_totals(self, U) -> torch.Tensor:
        n = U.shape[1]
        out = torch.empty((5,), dtype=torch.float64, device=self.device)
        self._call("mm_totals", self.h, _ptr(U, (U.shape[0], n)), n, _ptr(out))
        return out

    def mm_set_timing(self, on: bool) -> None:
        self._call("mm_set_timing", self.h, 1 if on else 0)

    def mm_stage_times(self) -> dict:
        """{stage: (total ms, runs)} since mm_set_timing(True)."""
        ms = (ctypes.c_double * len(STAGES))()
        runs = (_c_i64 * len(STAGES))()
        self._call("mm_stage_times", self.h, ms, runs)
        return {name: (ms[k], runs[k]) for k, name in enumerate(STAGES)}

    def mm_kernel_launches(self) -> int:
        return int(self.L.mm_kernel_launches(self.h))

    def mm_tess_stats(self) -> dict:
        """Counters of the last tessellation made with collect_stats=1."""
        arr = (_c_i64 * len(STATS))()
        self._call("mm_tess_stats", self.h, arr)
        return dict(zip(STATS, list(arr)))
