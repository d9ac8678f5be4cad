"""ctypes binding of liblapfoam.so (include/lapfoam.h), same names as the C ABI.

Argument marshalling only: every step of the time step runs in the CUDA library. Loading
fails loudly when the library cannot be built or loaded; there is no fallback path.
Functions raise :class:`LfmError` on a non-OK status (except where a status is the result,
e.g. ``lfm_query``).
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int32, c_size_t, c_uint64, c_void_p
from typing import Optional, Sequence

import numpy as np

from . import _build

LFM_OK, LFM_EINVAL, LFM_ENOMEM, LFM_ECUDA = 0, -1, -2, -3
LFM_ESINGULAR, LFM_ENONFINITE, LFM_ETIMEOUT, LFM_ESTATE = -4, -5, -6, -7
LFM_FIXED_VALUE, LFM_ZERO_GRADIENT = 0, 1
LFM_FP64, LFM_MIXED, LFM_DF64 = 0, 1, 2
LFM_BOTH = -1

_NAMES = {0: "LFM_OK", -1: "LFM_EINVAL", -2: "LFM_ENOMEM", -3: "LFM_ECUDA", -4: "LFM_ESINGULAR",
          -5: "LFM_ENONFINITE", -6: "LFM_ETIMEOUT", -7: "LFM_ESTATE"}


class LfmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class lfm_mesh(ctypes.Structure):
    _fields_ = [("n_cells", c_int32), ("n_faces", c_int32),
                ("owner", POINTER(c_int32)), ("neighbour", POINTER(c_int32)),
                ("V", POINTER(c_double)), ("magSf", POINTER(c_double)), ("deltaCoeffs", POINTER(c_double)),
                ("n_patches", c_int32),
                ("patch_start", POINTER(c_int32)), ("patch_size", POINTER(c_int32)),
                ("n_bfaces", c_int32),
                ("bface_cell", POINTER(c_int32)),
                ("bmagSf", POINTER(c_double)), ("bdeltaCoeffs", POINTER(c_double))]


class lfm_geometry(ctypes.Structure):
    _fields_ = [("Sf", POINTER(c_double)), ("weights", POINTER(c_double)), ("corr_vec", POINTER(c_double)),
                ("bSf", POINTER(c_double))]


class lfm_solver_opts(ctypes.Structure):
    _fields_ = [("tol", c_double), ("rel_tol", c_double), ("max_iter", c_int32),
                ("min_iter", c_int32), ("precision", c_int32)]


class lfm_step_stats(ctypes.Structure):
    _fields_ = [("iters", c_int32), ("converged", c_int32), ("sweeps", c_int32), ("status", c_int32),
                ("init_res", c_double), ("final_res", c_double), ("norm_factor", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lfm_dd_counts(ctypes.Structure):
    _fields_ = [("first_label", c_int32), ("n_owned", c_int32), ("n_ghost", c_int32), ("n_send", c_int32)]


_ctx_p = c_void_p
_SIGS = {
    "lfm_version": ([], c_char_p),
    "lfm_mesh_check": ([POINTER(lfm_mesh), c_char_p, c_size_t], c_int),
    "lfm_face_addressing": ([c_int32, c_int32, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32),
                             POINTER(c_int32), POINTER(c_int32)], c_int),
    "lfm_workspace_bytes": ([POINTER(lfm_mesh), c_int32], c_size_t),
    "lfm_workspace_bytes_geometry": ([POINTER(lfm_mesh), c_int32], c_size_t),
    "lfm_upload_mesh_geometry": ([_ctx_p, POINTER(lfm_mesh), POINTER(lfm_geometry)], c_int),
    "lfm_set_nonorth_correctors": ([_ctx_p, c_int32], c_int),
    "lfm_set_diffusivity_cells": ([_ctx_p, POINTER(c_double), POINTER(c_double)], c_int),
    "lfm_set_source": ([_ctx_p, POINTER(c_double), POINTER(c_double)], c_int),
    "lfm_get_addressing": ([_ctx_p, POINTER(c_int32), POINTER(c_int32), POINTER(ctypes.c_uint32),
                            POINTER(c_int32), POINTER(c_int32)], c_int),
    "lfm_grad": ([_ctx_p, POINTER(c_double), POINTER(c_double)], c_int),
    "lfm_create": ([POINTER(_ctx_p), c_int, c_void_p], c_int),
    "lfm_bind_workspace": ([_ctx_p, c_void_p, c_size_t, c_int32], c_int),
    "lfm_upload_mesh": ([_ctx_p, POINTER(lfm_mesh)], c_int),
    "lfm_box_counts": ([c_int32, c_int32, c_int32, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32),
                        POINTER(c_int32)], c_int),
    "lfm_box_layout": ([c_int32, c_int32, c_int32, POINTER(c_double), POINTER(c_double), POINTER(c_double),
                        POINTER(c_int32), POINTER(c_int32), POINTER(ctypes.c_uint32), POINTER(c_double),
                        POINTER(c_double), POINTER(c_double),
                        POINTER(c_int32), POINTER(c_int32), POINTER(c_int32), POINTER(c_double),
                        POINTER(c_double)], c_int),
    "lfm_upload_box": ([_ctx_p, c_int32, c_int32, c_int32, POINTER(c_double), POINTER(c_double),
                        POINTER(c_double)], c_int),
    "lfm_workspace_bytes_box": ([c_int32, c_int32, c_int32, c_int32], c_size_t),
    "lfm_upload_mesh_shared": ([_ctx_p, _ctx_p], c_int),
    "lfm_workspace_bytes_shared": ([_ctx_p, c_int32], c_size_t),
    "lfm_fill_field": ([_ctx_p, c_double], c_int),
    "lfm_set_diffusivity": ([_ctx_p, c_double, POINTER(c_double), POINTER(c_double)], c_int),
    "lfm_set_patch": ([_ctx_p, c_int32, c_int32, POINTER(c_double), c_double], c_int),
    "lfm_set_time_step": ([_ctx_p, c_double], c_int),
    "lfm_set_solver": ([_ctx_p, POINTER(lfm_solver_opts)], c_int),
    "lfm_set_field": ([_ctx_p, POINTER(c_double)], c_int),
    "lfm_set_field_device": ([_ctx_p, c_void_p], c_int),
    "lfm_advance": ([_ctx_p, c_int32, POINTER(lfm_step_stats)], c_int),
    "lfm_advance_async": ([_ctx_p, c_int32], c_int),
    "lfm_query": ([_ctx_p], c_int),
    "lfm_finish": ([_ctx_p, POINTER(lfm_step_stats), c_int32], c_int),
    "lfm_get_field": ([_ctx_p, POINTER(c_double), POINTER(c_double)], c_int),
    "lfm_field_device_ptr": ([_ctx_p, POINTER(c_void_p)], c_int),
    "lfm_get_matrix": ([_ctx_p, POINTER(c_double), POINTER(c_double), POINTER(c_double)], c_int),
    "lfm_get_launch": ([_ctx_p, POINTER(c_int32), POINTER(c_int32)], c_int),
    "lfm_get_phase_times": ([_ctx_p, POINTER(c_double)], c_int),
    "lfm_set_launch": ([_ctx_p, c_int32, c_int32], c_int),
    "lfm_set_barrier_timeout": ([_ctx_p, c_uint64], c_int),
    "lfm_debug_skip_arrival": ([_ctx_p, c_int32], c_int),
    "lfm_debug_stage_rows": ([_ctx_p, c_int32], c_int),
    "lfm_debug_skip_stage_copy": ([_ctx_p, c_int32], c_int),
    "lfm_debug_staged_passes": ([_ctx_p, POINTER(ctypes.c_int64)], c_int),
    "lfm_pcg_solve_static": ([c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                              POINTER(lfm_solver_opts), POINTER(lfm_step_stats), c_void_p], c_int),
    "lfm_destroy": ([_ctx_p], c_int),
    "lfm_measure_fp64_fma_rate": ([c_int, POINTER(c_double)], c_int),
    "lfm_face_coeffs_device": ([c_int32, c_int32, c_int32] + [c_void_p] * 15, c_int),
    "lfm_dd_plan": ([c_int32, c_int32, c_void_p, c_void_p, c_int32, c_int32, POINTER(lfm_dd_counts), c_void_p,
                     c_void_p, c_void_p, c_void_p], c_int),
    "lfm_dd_create": ([POINTER(c_void_p), _ctx_p, c_int32], c_int),
    "lfm_dd_part_counts": ([c_void_p, c_int32, POINTER(lfm_dd_counts)], c_int),
    "lfm_dd_set_field": ([c_void_p, c_void_p], c_int),
    "lfm_dd_get_field": ([c_void_p, c_void_p], c_int),
    "lfm_dd_advance": ([c_void_p, c_int32, POINTER(lfm_step_stats)], c_int),
    "lfm_dd_destroy": ([c_void_p], c_int),
    "lfm_dd_last_error": ([c_void_p], c_char_p),
    "lfm_batch_create": ([POINTER(c_void_p), c_int, c_void_p], c_int),
    "lfm_batch_add": ([c_void_p, _ctx_p, POINTER(c_int32)], c_int),
    "lfm_batch_remove": ([c_void_p, c_int32], c_int),
    "lfm_batch_size": ([c_void_p], c_int),
    "lfm_batch_set_launch": ([c_void_p, c_int32, POINTER(c_int32)], c_int),
    "lfm_batch_debug_stage_rows": ([c_void_p, c_int32], c_int),
    "lfm_batch_get_launch": ([c_void_p, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32)], c_int),
    "lfm_batch_set_barrier_timeout": ([c_void_p, c_uint64], c_int),
    "lfm_batch_advance_async": ([c_void_p, c_int32, c_int32], c_int),
    "lfm_batch_advance_capped_async": ([c_void_p, c_int32, c_int32, POINTER(c_int32), c_int32], c_int),
    "lfm_batch_results": ([c_void_p, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32), c_int32], c_int),
    "lfm_batch_query": ([c_void_p], c_int),
    "lfm_batch_finish": ([c_void_p], c_int),
    "lfm_batch_case_status": ([c_void_p, c_int32], c_int),
    "lfm_batch_case_iters": ([c_void_p, c_int32], c_int),
    "lfm_batch_case_stats": ([c_void_p, c_int32, POINTER(lfm_step_stats), c_int32], c_int),
    "lfm_batch_destroy": ([c_void_p], c_int),
    "lfm_batch_last_error": ([c_void_p], c_char_p),
    "lfm_last_error": ([_ctx_p], c_char_p),
    "lfm_checked_build": ([], c_int),
    "lfm_debug_check_inject": ([_ctx_p, c_int32], c_int),
}

_lib = None


def checked_requested() -> bool:
    """LFM_CHECKED=1 in the environment selects the checked build (liblapfoam_checked.so:
    every index a kernel reads from the mesh addressing is tested before use)."""
    return os.environ.get("LFM_CHECKED", "") == "1"


def library_path() -> str:
    return _build.lib_path(checked_requested())


def load(build: bool = True) -> ctypes.CDLL:
    """Loads liblapfoam.so, or the checked build when LFM_CHECKED=1 (building it first when
    stale). Raises when that fails."""
    global _lib
    if _lib is None:
        checked = checked_requested()
        path = _build.build(checked=checked) if build else _build.lib_path(checked)
        lib = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def declared_symbols() -> Sequence[str]:
    return list(_SIGS)


def _err(ctx) -> str:
    msg = load().lfm_last_error(ctx)
    return msg.decode() if msg else ""


def _check(rc: int, ctx=None) -> int:
    if rc != LFM_OK:
        raise LfmError(rc, _err(ctx))
    return rc


def _f64(a: Optional[np.ndarray]):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a: Optional[np.ndarray], t):
    if a is None:
        return ctypes.cast(None, POINTER(t))
    return a.ctypes.data_as(POINTER(t))


class MeshArgs:
    """Keeps the arrays of an ``lfm_mesh`` alive while the struct is in use."""

    def __init__(self, m):
        self.arrays = dict(owner=_i32(m.owner), neighbour=_i32(m.neighbour), V=_f64(m.V),
                           magSf=_f64(m.magSf), deltaCoeffs=_f64(m.deltaCoeffs),
                           patch_start=_i32(m.patch_start), patch_size=_i32(m.patch_size),
                           bface_cell=_i32(m.bface_cell), bmagSf=_f64(m.bmagSf),
                           bdeltaCoeffs=_f64(m.bdeltaCoeffs))
        a = self.arrays
        self.struct = lfm_mesh(int(m.n_cells), int(m.n_faces), _ptr(a["owner"], c_int32),
                               _ptr(a["neighbour"], c_int32), _ptr(a["V"], c_double),
                               _ptr(a["magSf"], c_double), _ptr(a["deltaCoeffs"], c_double),
                               len(a["patch_start"]), _ptr(a["patch_start"], c_int32),
                               _ptr(a["patch_size"], c_int32), int(m.n_bfaces),
                               _ptr(a["bface_cell"], c_int32), _ptr(a["bmagSf"], c_double),
                               _ptr(a["bdeltaCoeffs"], c_double))


# ---- functions with the C names --------------------------------------------------------

def lfm_version() -> str:
    return load().lfm_version().decode()


def lfm_mesh_check(mesh) -> str:
    """'' when the mesh is valid, else the reason."""
    args = MeshArgs(mesh)
    buf = ctypes.create_string_buffer(512)
    rc = load().lfm_mesh_check(ctypes.byref(args.struct), buf, 512)
    return "" if rc == LFM_OK else buf.value.decode()


def lfm_face_addressing(n_cells: int, owner, neighbour):
    owner, neighbour = _i32(owner), _i32(neighbour)
    F = len(owner)
    own_start = np.empty(n_cells + 1, np.int32)
    lo_start = np.empty(n_cells + 1, np.int32)
    losort = np.empty(max(F, 1), np.int32)
    _check(load().lfm_face_addressing(n_cells, F, _ptr(owner, c_int32), _ptr(neighbour, c_int32),
                                      _ptr(own_start, c_int32), _ptr(losort, c_int32),
                                      _ptr(lo_start, c_int32)))
    return own_start, losort[:F], lo_start


def lfm_workspace_bytes(mesh, precision: int = LFM_BOTH) -> int:
    args = MeshArgs(mesh)
    return int(load().lfm_workspace_bytes(ctypes.byref(args.struct), precision))


def lfm_create(device: int = 0, stream: Optional[int] = None) -> c_void_p:
    ctx = c_void_p()
    _check(load().lfm_create(ctypes.byref(ctx), device, c_void_p(stream) if stream else None))
    return ctx


def lfm_bind_workspace(ctx, dev_ptr: int, nbytes: int, precision: int = LFM_BOTH):
    _check(load().lfm_bind_workspace(ctx, c_void_p(dev_ptr), nbytes, precision), ctx)


def lfm_upload_mesh(ctx, mesh):
    args = MeshArgs(mesh)
    _check(load().lfm_upload_mesh(ctx, ctypes.byref(args.struct)), ctx)


class GeometryArgs:
    """Keeps the arrays of an ``lfm_geometry`` alive while the struct is in use."""

    def __init__(self, g):
        self.arrays = dict(Sf=_f64(g.Sf), weights=_f64(g.weights), corr_vec=_f64(g.corr_vec), bSf=_f64(g.bSf))
        a = self.arrays
        self.struct = lfm_geometry(_ptr(a["Sf"], c_double), _ptr(a["weights"], c_double),
                                   _ptr(a["corr_vec"], c_double), _ptr(a["bSf"], c_double))


def lfm_workspace_bytes_geometry(mesh, precision: int = LFM_BOTH) -> int:
    args = MeshArgs(mesh)
    return int(load().lfm_workspace_bytes_geometry(ctypes.byref(args.struct), precision))


def lfm_upload_mesh_geometry(ctx, mesh, geometry):
    """``geometry``: an object with Sf [F, 3], weights [F], corr_vec [F, 3], bSf [NB, 3]."""
    args = MeshArgs(mesh)
    gargs = GeometryArgs(geometry)
    _check(load().lfm_upload_mesh_geometry(ctx, ctypes.byref(args.struct), ctypes.byref(gargs.struct)), ctx)


def lfm_set_diffusivity_cells(ctx, DT_cells, weights=None):
    DT_cells = _f64(DT_cells)
    weights = _f64(weights)
    _check(load().lfm_set_diffusivity_cells(ctx, _ptr(DT_cells, c_double), _ptr(weights, c_double)), ctx)


def lfm_get_addressing(ctx, n_cells: int, n_faces: int, n_bfaces: int, W: int) -> dict:
    out = dict(slot_other=np.empty(max(W * n_cells, 1), np.int32), slot_face=np.empty(max(W * n_cells, 1), np.int32),
               face_slots=np.empty(max(2 * n_faces, 2), np.uint32), b_start=np.empty(n_cells + 1, np.int32),
               b_face=np.empty(max(n_bfaces, 1), np.int32))
    _check(load().lfm_get_addressing(ctx, _ptr(out["slot_other"], c_int32), _ptr(out["slot_face"], c_int32),
                                     _ptr(out["face_slots"], ctypes.c_uint32), _ptr(out["b_start"], c_int32),
                                     _ptr(out["b_face"], c_int32)), ctx)
    out["slot_other"], out["slot_face"] = out["slot_other"][:W * n_cells], out["slot_face"][:W * n_cells]
    out["face_slots"], out["b_face"] = out["face_slots"][:2 * n_faces], out["b_face"][:n_bfaces]
    return out


def lfm_set_source(ctx, Su=None, Sp=None):
    Su, Sp = _f64(Su), _f64(Sp)
    _check(load().lfm_set_source(ctx, _ptr(Su, c_double), _ptr(Sp, c_double)), ctx)


def lfm_set_nonorth_correctors(ctx, n_corr: int):
    _check(load().lfm_set_nonorth_correctors(ctx, int(n_corr)), ctx)


def lfm_grad(ctx, n_cells: int, n_bfaces: int, boundary: bool = True):
    """Gauss gradient of the current T: (cells [N, 3], boundary faces [NB, 3] or None)."""
    G = np.empty((n_cells, 3))
    Gb = np.empty((max(n_bfaces, 1), 3)) if boundary else None
    _check(load().lfm_grad(ctx, _ptr(G, c_double), _ptr(Gb, c_double) if boundary else None), ctx)
    return G, (Gb[:n_bfaces] if boundary else None)


def lfm_box_counts(nx: int, ny: int, nz: int):
    n, f, nb, w = c_int32(), c_int32(), c_int32(), c_int32()
    _check(load().lfm_box_counts(nx, ny, nz, ctypes.byref(n), ctypes.byref(f), ctypes.byref(nb), ctypes.byref(w)))
    return n.value, f.value, nb.value, w.value


def lfm_box_layout(xs, ys, zs):
    """Host replica of the device box builder; returns a dict of arrays."""
    xs, ys, zs = _f64(xs), _f64(ys), _f64(zs)
    nx, ny, nz = len(xs) - 1, len(ys) - 1, len(zs) - 1
    N, F, NB, W = lfm_box_counts(nx, ny, nz)
    out = dict(slot_other=np.empty(max(W * N, 1), np.int32), slot_face=np.empty(max(W * N, 1), np.int32),
               face_slots=np.empty(max(2 * F, 2), np.uint32),
               V=np.empty(N), magSf=np.empty(max(F, 1)), deltaCoeffs=np.empty(max(F, 1)),
               b_start=np.empty(N + 1, np.int32), b_face=np.empty(NB, np.int32), bface_cell=np.empty(NB, np.int32),
               bmagSf=np.empty(NB), bdeltaCoeffs=np.empty(NB))
    _check(load().lfm_box_layout(nx, ny, nz, _ptr(xs, c_double), _ptr(ys, c_double), _ptr(zs, c_double),
                                 *[_ptr(out[k], {np.dtype(np.int32): c_int32, np.dtype(np.uint32): ctypes.c_uint32,
                                                 np.dtype(np.float64): c_double}[out[k].dtype])
                                   for k in ("slot_other", "slot_face", "face_slots", "V", "magSf", "deltaCoeffs",
                                             "b_start",
                                             "b_face", "bface_cell", "bmagSf", "bdeltaCoeffs")]))
    out["slot_other"], out["slot_face"] = out["slot_other"][:W * N], out["slot_face"][:W * N]
    out["face_slots"] = out["face_slots"][:2 * F]
    out["magSf"], out["deltaCoeffs"] = out["magSf"][:F], out["deltaCoeffs"][:F]
    out.update(n_cells=N, n_faces=F, n_bfaces=NB, W=W)
    return out


def lfm_upload_box(ctx, xs, ys, zs):
    xs, ys, zs = _f64(xs), _f64(ys), _f64(zs)
    _check(load().lfm_upload_box(ctx, len(xs) - 1, len(ys) - 1, len(zs) - 1, _ptr(xs, c_double),
                                 _ptr(ys, c_double), _ptr(zs, c_double)), ctx)


def lfm_workspace_bytes_box(nx: int, ny: int, nz: int, precision: int = LFM_BOTH) -> int:
    return int(load().lfm_workspace_bytes_box(nx, ny, nz, precision))


def lfm_upload_mesh_shared(ctx, src_ctx):
    _check(load().lfm_upload_mesh_shared(ctx, src_ctx), ctx)


def lfm_workspace_bytes_shared(src_ctx, precision: int = LFM_BOTH) -> int:
    return int(load().lfm_workspace_bytes_shared(src_ctx, precision))


def lfm_fill_field(ctx, value: float):
    _check(load().lfm_fill_field(ctx, float(value)), ctx)


def lfm_set_diffusivity(ctx, uniform: float, DT_faces=None, DT_bfaces=None):
    a, b = _f64(DT_faces), _f64(DT_bfaces)
    _check(load().lfm_set_diffusivity(ctx, float(uniform), _ptr(a, c_double), _ptr(b, c_double)), ctx)


def lfm_set_patch(ctx, patch: int, ptype: int, values=None, uniform: float = 0.0):
    v = _f64(values)
    _check(load().lfm_set_patch(ctx, patch, ptype, _ptr(v, c_double), float(uniform)), ctx)


def lfm_set_time_step(ctx, dt: float):
    _check(load().lfm_set_time_step(ctx, float(dt)), ctx)


def lfm_set_solver(ctx, tol: float, rel_tol: float = 0.0, max_iter: int = 1000, min_iter: int = 0,
                   precision: int = LFM_FP64):
    o = lfm_solver_opts(float(tol), float(rel_tol), int(max_iter), int(min_iter), int(precision))
    _check(load().lfm_set_solver(ctx, ctypes.byref(o)), ctx)


def lfm_set_field(ctx, T: np.ndarray):
    T = _f64(T)
    _check(load().lfm_set_field(ctx, _ptr(T, c_double)), ctx)


def lfm_set_field_device(ctx, dev_ptr: int):
    _check(load().lfm_set_field_device(ctx, c_void_p(dev_ptr)), ctx)


def lfm_advance(ctx, n_steps: int):
    out = (lfm_step_stats * max(n_steps, 1))()
    _check(load().lfm_advance(ctx, n_steps, out), ctx)
    return [out[i] for i in range(n_steps)]


def lfm_advance_async(ctx, n_steps: int):
    _check(load().lfm_advance_async(ctx, n_steps), ctx)


def lfm_query(ctx) -> int:
    rc = load().lfm_query(ctx)
    if rc < 0:
        raise LfmError(rc, _err(ctx))
    return rc


def lfm_finish(ctx, n: int):
    out = (lfm_step_stats * max(n, 1))()
    rc = load().lfm_finish(ctx, out, n)
    stats = [out[i] for i in range(n)]
    if rc != LFM_OK:
        raise LfmError(rc, _err(ctx))
    return stats


def lfm_finish_status(ctx, n: int):
    """Like lfm_finish but returns (status, stats) instead of raising."""
    out = (lfm_step_stats * max(n, 1))()
    rc = load().lfm_finish(ctx, out, n)
    return rc, [out[i] for i in range(n)]


def lfm_get_field(ctx, n_cells: int, n_bfaces: int = 0, out: Optional[np.ndarray] = None,
                  boundary: bool = False):
    T = out if out is not None else np.empty(n_cells)
    Tb = np.empty(n_bfaces) if boundary else None
    _check(load().lfm_get_field(ctx, _ptr(T, c_double), _ptr(Tb, c_double)), ctx)
    return (T, Tb) if boundary else T


def lfm_field_device_ptr(ctx) -> int:
    p = c_void_p()
    _check(load().lfm_field_device_ptr(ctx, ctypes.byref(p)), ctx)
    return int(p.value)


def lfm_get_matrix(ctx, n_cells: int, n_faces: int):
    d, u, s = np.empty(n_cells), np.empty(max(n_faces, 1)), np.empty(n_cells)
    _check(load().lfm_get_matrix(ctx, _ptr(d, c_double), _ptr(u, c_double), _ptr(s, c_double)), ctx)
    return d, u[:n_faces], s


PHASES = ("assembly_faces", "rows_initial_residual", "p_update", "amul_dot", "update_dots", "fp64_correction")


def lfm_get_phase_times(ctx) -> dict:
    ms = (c_double * 8)()
    _check(load().lfm_get_phase_times(ctx, ms), ctx)
    return {name: ms[i] for i, name in enumerate(PHASES)}


def lfm_get_launch(ctx):
    a, b = c_int32(), c_int32()
    _check(load().lfm_get_launch(ctx, ctypes.byref(a), ctypes.byref(b)), ctx)
    return a.value, b.value


def lfm_set_launch(ctx, ctas: int, threads: int):
    _check(load().lfm_set_launch(ctx, int(ctas), int(threads)), ctx)


def lfm_set_barrier_timeout(ctx, ns: int):
    _check(load().lfm_set_barrier_timeout(ctx, int(ns)), ctx)


def lfm_debug_skip_arrival(ctx, cta: int):
    _check(load().lfm_debug_skip_arrival(ctx, int(cta)), ctx)


def lfm_debug_stage_rows(ctx, on: bool):
    _check(load().lfm_debug_stage_rows(ctx, 1 if on else 0), ctx)


def lfm_debug_skip_stage_copy(ctx, cta: int):
    _check(load().lfm_debug_skip_stage_copy(ctx, int(cta)), ctx)


def lfm_debug_staged_passes(ctx) -> int:
    n = ctypes.c_int64(0)
    _check(load().lfm_debug_staged_passes(ctx, ctypes.byref(n)), ctx)
    return n.value


def lfm_checked_build() -> bool:
    return bool(load().lfm_checked_build())


def lfm_debug_check_inject(ctx, site: int):
    _check(load().lfm_debug_check_inject(ctx, int(site)), ctx)


def lfm_pcg_solve_static(n_cells: int, n_faces: int, owner_ptr: int, neighbour_ptr: int, diag_ptr: int,
                         upper_ptr: int, source_ptr: int, x_ptr: int, tol: float, rel_tol: float = 0.0,
                         max_iter: int = 1000, min_iter: int = 0, stream: Optional[int] = None):
    """Allocation-free FP64 solve of a device-resident LDU system (pointers are device
    addresses). Returns (status, stats); does not raise on a solver status."""
    o = lfm_solver_opts(float(tol), float(rel_tol), int(max_iter), int(min_iter), LFM_FP64)
    st = lfm_step_stats()
    rc = load().lfm_pcg_solve_static(int(n_cells), int(n_faces), c_void_p(owner_ptr), c_void_p(neighbour_ptr),
                                     c_void_p(diag_ptr), c_void_p(upper_ptr), c_void_p(source_ptr),
                                     c_void_p(x_ptr), ctypes.byref(o), ctypes.byref(st),
                                     c_void_p(stream) if stream else None)
    return rc, st


def lfm_destroy(ctx):
    load().lfm_destroy(ctx)


def lfm_face_coeffs_device(n_cells: int, n_faces: int, n_bfaces: int, owner, neighbour, Sf, Cf, C, bface_cell,
                           bSf, bCf, weights, magSf, deltaCoeffs, corr_vec, bmagSf, bdeltaCoeffs, stream=0):
    """Face weights and corrected-laplacian coefficients on the device; every array argument
    is a device address (int), stream a cudaStream_t handle (0: the legacy default)."""
    ptrs = [owner, neighbour, Sf, Cf, C, bface_cell, bSf, bCf, weights, magSf, deltaCoeffs, corr_vec, bmagSf,
            bdeltaCoeffs, stream]
    rc = load().lfm_face_coeffs_device(int(n_cells), int(n_faces), int(n_bfaces),
                                       *[c_void_p(int(p)) if p else None for p in ptrs])
    if rc != LFM_OK:
        raise LfmError(rc, _err(None))


def lfm_measure_fp64_fma_rate(device: int = 0) -> float:
    """FP64 fused multiply-adds per second measured on the device."""
    v = c_double(0.0)
    rc = load().lfm_measure_fp64_fma_rate(int(device), ctypes.byref(v))
    if rc != LFM_OK:
        raise LfmError(rc, _err(None))
    return v.value


def lfm_last_error(ctx=None) -> str:
    return _err(ctx)


# ---- batched form ------------------------------------------------------------------------

def _berr(b) -> str:
    msg = load().lfm_batch_last_error(b)
    return msg.decode() if msg else ""


def _bcheck(rc: int, b=None) -> int:
    if rc != LFM_OK:
        raise LfmError(rc, _berr(b))
    return rc


def lfm_batch_create(device: int = 0, stream: Optional[int] = None) -> c_void_p:
    b = c_void_p()
    _bcheck(load().lfm_batch_create(ctypes.byref(b), device, c_void_p(stream) if stream else None))
    return b


def lfm_batch_add(b, ctx) -> int:
    cid = c_int32()
    _bcheck(load().lfm_batch_add(b, ctx, ctypes.byref(cid)), b)
    return cid.value


def lfm_batch_remove(b, case_id: int):
    _bcheck(load().lfm_batch_remove(b, int(case_id)), b)


def lfm_batch_size(b) -> int:
    return int(load().lfm_batch_size(b))


def lfm_batch_set_launch(b, threads: int, cells_per_thread=None):
    arr = None if cells_per_thread is None else (c_int32 * 3)(*[int(v) for v in cells_per_thread])
    _bcheck(load().lfm_batch_set_launch(b, int(threads), arr), b)


def lfm_batch_get_launch(b):
    ctas, thr, cpt = c_int32(), c_int32(), (c_int32 * 3)()
    _bcheck(load().lfm_batch_get_launch(b, ctypes.byref(ctas), ctypes.byref(thr), cpt), b)
    return ctas.value, thr.value, list(cpt)


def lfm_batch_set_barrier_timeout(b, ns: int):
    _bcheck(load().lfm_batch_set_barrier_timeout(b, int(ns)), b)


def lfm_batch_debug_stage_rows(b, on: bool):
    _bcheck(load().lfm_batch_debug_stage_rows(b, 1 if on else 0), b)


def lfm_batch_advance_async(b, n_steps: int, use_graph: bool = True):
    _bcheck(load().lfm_batch_advance_async(b, int(n_steps), 1 if use_graph else 0), b)


def lfm_batch_advance_capped_async(b, n_steps: int, caps, use_graph: bool = True):
    """caps: per case id, at most this many of the n_steps (a sequence of ints)."""
    n = len(caps)
    arr = (c_int32 * max(n, 1))(*[int(x) for x in caps])
    _bcheck(load().lfm_batch_advance_capped_async(b, int(n_steps), 1 if use_graph else 0, arr, n), b)


def lfm_batch_results(b, n: int):
    """(status, steps, iterations) lists for case ids 0 .. n-1 after the last advance."""
    st, sp, it = (c_int32 * max(n, 1))(), (c_int32 * max(n, 1))(), (c_int32 * max(n, 1))()
    _bcheck(load().lfm_batch_results(b, st, sp, it, int(n)), b)
    return list(st[:n]), list(sp[:n]), list(it[:n])


def lfm_batch_query(b) -> int:
    rc = load().lfm_batch_query(b)
    if rc < 0:
        raise LfmError(rc, _berr(b))
    return rc


def lfm_batch_finish(b) -> int:
    """Waits; returns LFM_OK or the first failing case's status (does not raise on those)."""
    rc = load().lfm_batch_finish(b)
    if rc == LFM_ECUDA:
        raise LfmError(rc, _berr(b))
    return rc


def lfm_batch_case_status(b, case_id: int) -> int:
    return int(load().lfm_batch_case_status(b, int(case_id)))


def lfm_batch_case_iters(b, case_id: int) -> int:
    return int(load().lfm_batch_case_iters(b, int(case_id)))


def lfm_batch_case_stats(b, case_id: int, n: int):
    out = (lfm_step_stats * max(n, 1))()
    _bcheck(load().lfm_batch_case_stats(b, int(case_id), out, int(n)), b)
    return [out[i] for i in range(n)]


def lfm_batch_destroy(b):
    load().lfm_batch_destroy(b)


def lfm_batch_last_error(b=None) -> str:
    return _berr(b)


# ---- one case decomposed into parts -----------------------------------------------------

def _dderr(d=None) -> str:
    msg = load().lfm_dd_last_error(d)
    return msg.decode() if msg else ""


def _ddcheck(rc: int, d=None) -> int:
    if rc != LFM_OK:
        raise LfmError(rc, _dderr(d))
    return rc


def lfm_dd_plan(owner, neighbour, n_cells: int, n_parts: int, part: int):
    """(counts, ghost labels, send sources, send parts, send slots) of one part (host only)."""
    import numpy as np
    owner = np.ascontiguousarray(owner, dtype=np.int32)
    neighbour = np.ascontiguousarray(neighbour, dtype=np.int32)
    cnt = lfm_dd_counts()
    args = (int(n_cells), len(owner), owner.ctypes.data, neighbour.ctypes.data, int(n_parts), int(part))
    _ddcheck(load().lfm_dd_plan(*args, ctypes.byref(cnt), None, None, None, None))
    g = np.zeros(max(cnt.n_ghost, 1), np.int32)
    src, prt, slt = (np.zeros(max(cnt.n_send, 1), np.int32) for _ in range(3))
    _ddcheck(load().lfm_dd_plan(*args, ctypes.byref(cnt), g.ctypes.data, src.ctypes.data, prt.ctypes.data,
                                slt.ctypes.data))
    return cnt, g[:cnt.n_ghost], src[:cnt.n_send], prt[:cnt.n_send], slt[:cnt.n_send]


def lfm_dd_create(ctx, n_parts: int):
    d = c_void_p()
    _ddcheck(load().lfm_dd_create(ctypes.byref(d), ctx, int(n_parts)))
    return d


def lfm_dd_part_counts(d, part: int):
    cnt = lfm_dd_counts()
    _ddcheck(load().lfm_dd_part_counts(d, int(part), ctypes.byref(cnt)), d)
    return cnt


def lfm_dd_set_field(d, T):
    import numpy as np
    T = np.ascontiguousarray(T, dtype=np.float64)
    _ddcheck(load().lfm_dd_set_field(d, T.ctypes.data), d)


def lfm_dd_get_field(d, n_cells: int):
    import numpy as np
    T = np.empty(n_cells)
    _ddcheck(load().lfm_dd_get_field(d, T.ctypes.data), d)
    return T


def lfm_dd_advance(d, n_steps: int):
    out = (lfm_step_stats * max(n_steps, 1))()
    _ddcheck(load().lfm_dd_advance(d, int(n_steps), out), d)
    return [out[i] for i in range(n_steps)]


def lfm_dd_destroy(d):
    load().lfm_dd_destroy(d)
