"""CPU oracle for one laplacianFoam time step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline arm of ``bench.py`` may
import this package. It is a thin ctypes driver around ``oracle.c`` (plain serial FP64 C);
it shares nothing with the CUDA path except the seeded raw-case description from
:mod:`lapcase`, from which it derives geometry, addressing, matrix and solve on its own.

Paper passages followed (arXiv 2507.18268): Eq. (1) and the laplacianFoam listing (one
``fvm::ddt(T) - fvm::laplacian(DT, T)`` solve per step), the face addressing of section
"OpenFOAM", the face-loop pattern of the listing "First cycle in the gradf routine", and the
PCG + diagonal preconditioner named in section "Evaluation"; for general hexahedral meshes
the gradient passes of section "Code Porting" (listings "weights", "dotInterpolate", the
two gradf cycles, the field division and correctBoundaryConditions) and the corrected
laplacian. The formulae the paper does not print are listed in ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import tempfile
from typing import List, Optional

import numpy as np

import lapcase

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)


class _Box(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("xs", _f64p), ("ys", _f64p), ("zs", _f64p), ("perm", _i64p),
                ("DT_uniform", ctypes.c_double), ("DTx", _f64p), ("DTy", _f64p), ("DTz", _f64p)]


class _Hex(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("pts", _f64p)]


class _Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("singular", ctypes.c_int32), ("nonfinite", ctypes.c_int32),
                ("init_res", ctypes.c_double), ("final_res", ctypes.c_double),
                ("norm_factor", ctypes.c_double)]


@dataclasses.dataclass
class Stats:
    iters: int
    converged: bool
    singular: bool
    nonfinite: bool
    init_res: float
    final_res: float
    norm_factor: float


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain C, no FMA contraction so that x86 and Arm
    hosts round identically)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.ora_box_counts.argtypes = [ctypes.POINTER(_Box), _i64p, _i64p, _i64p]
        lib.ora_box_mesh.argtypes = [ctypes.POINTER(_Box), _i32p, _i32p, _f64p, _f64p, _f64p, _f64p,
                                     _i32p, _i32p, _f64p, _f64p, _f64p]
        lib.ora_box_mesh.restype = ctypes.c_int
        lib.ora_assemble.argtypes = [ctypes.c_int64, ctypes.c_int64, _i32p, _i32p, _f64p, _f64p, _f64p,
                                     _f64p, ctypes.c_int64, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p,
                                     ctypes.c_double, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
        lib.ora_cell_dt_to_faces.argtypes = [ctypes.c_int64, ctypes.c_int64, _i32p, _i32p, _f64p, _i32p, _f64p,
                                             _f64p, _f64p]
        lib.ora_amul.argtypes = [ctypes.c_int64, ctypes.c_int64, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p]
        lib.ora_pcg.argtypes = [ctypes.c_int64, ctypes.c_int64, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p,
                                ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                ctypes.POINTER(_Stats), _f64p, ctypes.c_int32]
        lib.ora_pcg.restype = ctypes.c_int
        lib.ora_advance.argtypes = [ctypes.c_int64, ctypes.c_int64, _i32p, _i32p, _f64p, _f64p, _f64p,
                                    _f64p, ctypes.c_int64, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p,
                                    ctypes.c_double, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int32, ctypes.c_int32, _f64p, _f64p, _f64p, ctypes.POINTER(_Stats)]
        lib.ora_advance.restype = ctypes.c_int
        lib.ora_boundary_values.argtypes = [ctypes.c_int64, _i32p, _i32p, _f64p, _f64p, _f64p]
        lib.ora_hex_counts.argtypes = [ctypes.POINTER(_Hex), _i64p, _i64p, _i64p]
        lib.ora_hex_mesh.argtypes = [ctypes.POINTER(_Hex), _i32p, _i32p, _f64p, _f64p, _i32p, _i32p, _f64p,
                                     _f64p, _f64p, _f64p]
        lib.ora_hex_mesh.restype = ctypes.c_int
        lib.ora_hex_coeffs.argtypes = [ctypes.c_int64, ctypes.c_int64, _i32p, _i32p, _f64p, _f64p, _f64p, _i32p,
                                       _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
        lib.ora_gauss_grad.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _i32p, _i32p, _f64p,
                                       _f64p, _f64p, _i32p, _f64p, _f64p, _f64p, _f64p]
        lib.ora_gauss_grad.restype = ctypes.c_int
        lib.ora_grad_boundary.argtypes = [ctypes.c_int64, _i32p, _f64p, _f64p, _i32p, _f64p, _f64p, _f64p,
                                          _f64p]
        lib.ora_advance_corrected.argtypes = [ctypes.c_int64, ctypes.c_int64, _i32p, _i32p, _f64p, _f64p,
                                              _f64p, _f64p, _f64p, _f64p, _f64p, ctypes.c_int64, _i32p, _i32p,
                                              _f64p, _f64p, _f64p, _f64p, _f64p, ctypes.c_double,
                                              ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_int32, ctypes.c_int32, _f64p, _f64p,
                                              _f64p, ctypes.POINTER(_Stats)]
        lib.ora_advance_corrected.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a: Optional[np.ndarray], t):
    if a is None:
        return ctypes.cast(None, t)
    return a.ctypes.data_as(t)


@dataclasses.dataclass
class Mesh:
    """LDU mesh as the oracle builds it (labels after the case's relabelling)."""
    n_cells: int
    n_faces: int
    n_bfaces: int
    owner: np.ndarray
    neighbour: np.ndarray
    V: np.ndarray
    magSf: np.ndarray
    delta: np.ndarray
    DTf: np.ndarray
    bcell: np.ndarray
    bpatch: np.ndarray
    bmagSf: np.ndarray
    bdelta: np.ndarray
    DTb: np.ndarray
    # general hexahedral geometry (None for the rectilinear box); ``delta`` then holds the
    # nonOrthDeltaCoeffs used by the implicit laplacian
    Sf: Optional[np.ndarray] = None      # [F, 3] owner -> neighbour
    Cf: Optional[np.ndarray] = None      # [F, 3]
    C: Optional[np.ndarray] = None       # [N, 3]
    w: Optional[np.ndarray] = None       # [F] interpolation weight of the owner value
    corr: Optional[np.ndarray] = None    # [F, 3] non-orthogonal correction vectors
    bSf: Optional[np.ndarray] = None     # [NB, 3] outward
    bCf: Optional[np.ndarray] = None     # [NB, 3]


def box_mesh(case: lapcase.RawCase) -> Mesh:
    lib = _load()
    keep = []

    def f64(a):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=np.float64)
        keep.append(a)
        return a

    xs, ys, zs = f64(case.xs), f64(case.ys), f64(case.zs)
    perm = None if case.perm is None else np.ascontiguousarray(case.perm, dtype=np.int64)
    DTx, DTy, DTz = f64(case.DTx), f64(case.DTy), f64(case.DTz)
    box = _Box(case.nx, case.ny, case.nz, _p(xs, _f64p), _p(ys, _f64p), _p(zs, _f64p),
               _p(perm, _i64p), float(case.DT_uniform), _p(DTx, _f64p), _p(DTy, _f64p),
               _p(DTz, _f64p))
    N, F, NB = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    lib.ora_box_counts(ctypes.byref(box), ctypes.byref(N), ctypes.byref(F), ctypes.byref(NB))
    N, F, NB = N.value, F.value, NB.value
    m = Mesh(N, F, NB, np.empty(F, np.int32), np.empty(F, np.int32), np.empty(N), np.empty(F),
             np.empty(F), np.empty(F), np.empty(NB, np.int32), np.empty(NB, np.int32),
             np.empty(NB), np.empty(NB), np.empty(NB))
    rc = lib.ora_box_mesh(ctypes.byref(box), _p(m.owner, _i32p), _p(m.neighbour, _i32p), _p(m.V, _f64p),
                          _p(m.magSf, _f64p), _p(m.delta, _f64p), _p(m.DTf, _f64p), _p(m.bcell, _i32p),
                          _p(m.bpatch, _i32p), _p(m.bmagSf, _f64p), _p(m.bdelta, _f64p), _p(m.DTb, _f64p))
    if rc != 0:
        raise MemoryError("oracle mesh build ran out of memory")
    return m


def hex_mesh(case: lapcase.RawCase) -> Mesh:
    """General hexahedral mesh of a case with ``points``: topology and per-face DT from the
    box description (natural numbering), geometry and discretisation coefficients from the
    vertex positions."""
    if case.points is None:
        raise ValueError("case has no vertex array")
    if case.perm is not None:
        raise ValueError("general hexahedral cases use natural numbering")
    lib = _load()
    base = box_mesh(case)  # topology, patches and per-face DT (its rectilinear geometry is unused)
    pts = np.ascontiguousarray(case.points, dtype=np.float64)
    if pts.shape != (case.nz + 1, case.ny + 1, case.nx + 1, 3):
        raise ValueError("points must have shape (nz+1, ny+1, nx+1, 3)")
    h = _Hex(case.nx, case.ny, case.nz, _p(pts, _f64p))
    N, F, NB = base.n_cells, base.n_faces, base.n_bfaces
    owner, neighbour = np.empty(F, np.int32), np.empty(F, np.int32)
    Sf, Cf, bSf, bCf = np.empty((F, 3)), np.empty((F, 3)), np.empty((NB, 3)), np.empty((NB, 3))
    bcell, bpatch = np.empty(NB, np.int32), np.empty(NB, np.int32)
    V, C = np.empty(N), np.empty((N, 3))
    rc = lib.ora_hex_mesh(ctypes.byref(h), _p(owner, _i32p), _p(neighbour, _i32p), _p(Sf, _f64p), _p(Cf, _f64p),
                          _p(bcell, _i32p), _p(bpatch, _i32p), _p(bSf, _f64p), _p(bCf, _f64p), _p(V, _f64p),
                          _p(C, _f64p))
    if rc != 0:
        raise MemoryError("oracle hex mesh ran out of memory")
    assert np.array_equal(owner, base.owner) and np.array_equal(neighbour, base.neighbour)
    assert np.array_equal(bcell, base.bcell) and np.array_equal(bpatch, base.bpatch)
    w, magSf, nod, corr = np.empty(F), np.empty(F), np.empty(F), np.empty((F, 3))
    bmagSf, bdelta = np.empty(NB), np.empty(NB)
    lib.ora_hex_coeffs(F, NB, _p(owner, _i32p), _p(neighbour, _i32p), _p(Sf, _f64p), _p(Cf, _f64p), _p(C, _f64p),
                       _p(bcell, _i32p), _p(bSf, _f64p), _p(bCf, _f64p), _p(w, _f64p), _p(magSf, _f64p),
                       _p(nod, _f64p), _p(corr, _f64p), _p(bmagSf, _f64p), _p(bdelta, _f64p))
    return Mesh(N, F, NB, owner, neighbour, V, magSf, nod, base.DTf, bcell, bpatch, bmagSf, bdelta, base.DTb,
                Sf=Sf, Cf=Cf, C=C, w=w, corr=corr, bSf=bSf, bCf=bCf)


def interpolation_weights(case: lapcase.RawCase, mesh: Mesh) -> np.ndarray:
    """Owner interpolation weights of the mesh's internal faces (from the general geometry;
    for a rectilinear box, from the geometry of its vertex lattice)."""
    if mesh.w is not None:
        return mesh.w
    if case.perm is not None:
        raise ValueError("cell-field DT needs natural numbering")
    return hex_mesh(case.with_(points=lapcase.box_points(case.xs, case.ys, case.zs), n_nonorth_corr=0)).w


def cell_dt_to_faces(case: lapcase.RawCase, mesh: Mesh):
    """(DTf, DTb) of the case's cell-field DT."""
    lib = _load()
    DTc = np.ascontiguousarray(case.cell_array(case.DT_cells))
    w = np.ascontiguousarray(interpolation_weights(case, mesh))
    DTf, DTb = np.empty(mesh.n_faces), np.empty(mesh.n_bfaces)
    lib.ora_cell_dt_to_faces(mesh.n_faces, mesh.n_bfaces, _p(mesh.owner, _i32p), _p(mesh.neighbour, _i32p),
                             _p(w, _f64p), _p(mesh.bcell, _i32p), _p(DTc, _f64p), _p(DTf, _f64p), _p(DTb, _f64p))
    return DTf, DTb


def mesh_of(case: lapcase.RawCase) -> Mesh:
    """The case's mesh, with the face diffusivities of a cell-field DT when the case has one."""
    m = hex_mesh(case) if case.points is not None else box_mesh(case)
    if case.DT_cells is not None:
        m.DTf, m.DTb = cell_dt_to_faces(case, m)
    return m


def source_arrays(case: lapcase.RawCase):
    """(Su, Sp) per cell label, or None."""
    if case.perm is not None and (case.Su is not None or case.Sp is not None):
        raise ValueError("sources need natural numbering")
    return case.cell_array(case.Su), case.cell_array(case.Sp)


def gauss_grad(mesh: Mesh, T: np.ndarray, Tb: np.ndarray) -> np.ndarray:
    """Gauss linear gradient [N, 3] of the cell field T with boundary-face values Tb."""
    lib = _load()
    T = np.ascontiguousarray(T, dtype=np.float64)
    Tb = np.ascontiguousarray(Tb, dtype=np.float64)
    G = np.empty((mesh.n_cells, 3))
    rc = lib.ora_gauss_grad(mesh.n_cells, mesh.n_faces, mesh.n_bfaces, _p(mesh.owner, _i32p),
                            _p(mesh.neighbour, _i32p), _p(mesh.Sf, _f64p), _p(mesh.w, _f64p), _p(mesh.V, _f64p),
                            _p(mesh.bcell, _i32p), _p(mesh.bSf, _f64p), _p(Tb, _f64p), _p(T, _f64p), _p(G, _f64p))
    if rc != 0:
        raise MemoryError("oracle gradient ran out of memory")
    return G


def grad_boundary(mesh: Mesh, btype: np.ndarray, bvalue: np.ndarray, T: np.ndarray, G: np.ndarray) -> np.ndarray:
    """Boundary-face values [NB, 3] of the gradient after correctBoundaryConditions."""
    lib = _load()
    T = np.ascontiguousarray(T, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    Gb = np.empty((mesh.n_bfaces, 3))
    lib.ora_grad_boundary(mesh.n_bfaces, _p(mesh.bcell, _i32p), _p(mesh.bSf, _f64p), _p(mesh.bdelta, _f64p),
                          _p(btype, _i32p), _p(bvalue, _f64p), _p(T, _f64p), _p(G, _f64p), _p(Gb, _f64p))
    return Gb


def grad(case: lapcase.RawCase, mesh: Mesh, T: np.ndarray):
    """Gauss linear gradient of T with the case's boundary conditions: (cells [N, 3],
    boundary faces [NB, 3])."""
    btype, bvalue = boundary_types_values(case, mesh)
    G = gauss_grad(mesh, T, boundary_values(case, mesh, T))
    return G, grad_boundary(mesh, btype, bvalue, T, G)


def boundary_types_values(case: lapcase.RawCase, mesh: Mesh):
    """Per-boundary-face patch type and value from the case's six patches."""
    types = np.array([int(t) for t, _ in case.patches], dtype=np.int32)
    vals = np.array([float(v) for _, v in case.patches], dtype=np.float64)
    return np.ascontiguousarray(types[mesh.bpatch]), np.ascontiguousarray(vals[mesh.bpatch])


def initial_field(case: lapcase.RawCase) -> np.ndarray:
    """Initial T indexed by cell label."""
    T0 = case.T0_natural()
    if case.perm is None:
        return T0.copy()
    T = np.empty_like(T0)
    T[np.asarray(case.perm)] = T0
    return T


def assemble(mesh: Mesh, btype: np.ndarray, bvalue: np.ndarray, dt: float, T_old: np.ndarray,
             Su: Optional[np.ndarray] = None, Sp: Optional[np.ndarray] = None):
    """Returns (diag, upper, source) of fvm::ddt(T) - fvm::laplacian(DT, T) (- the source
    S_T = Su + Sp T when given, per cell label)."""
    lib = _load()
    T_old = np.ascontiguousarray(T_old, dtype=np.float64)
    Su = None if Su is None else np.ascontiguousarray(Su, dtype=np.float64)
    Sp = None if Sp is None else np.ascontiguousarray(Sp, dtype=np.float64)
    diag, upper, source = np.empty(mesh.n_cells), np.empty(mesh.n_faces), np.empty(mesh.n_cells)
    lib.ora_assemble(mesh.n_cells, mesh.n_faces, _p(mesh.owner, _i32p), _p(mesh.neighbour, _i32p),
                     _p(mesh.V, _f64p), _p(mesh.magSf, _f64p), _p(mesh.delta, _f64p), _p(mesh.DTf, _f64p),
                     mesh.n_bfaces, _p(mesh.bcell, _i32p), _p(btype, _i32p), _p(bvalue, _f64p),
                     _p(mesh.bmagSf, _f64p), _p(mesh.bdelta, _f64p), _p(mesh.DTb, _f64p), float(dt),
                     _p(T_old, _f64p), _p(Su, _f64p), _p(Sp, _f64p), _p(diag, _f64p), _p(upper, _f64p),
                     _p(source, _f64p))
    return diag, upper, source


def amul(mesh: Mesh, diag: np.ndarray, upper: np.ndarray, x: np.ndarray) -> np.ndarray:
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(mesh.n_cells)
    lib.ora_amul(mesh.n_cells, mesh.n_faces, _p(mesh.owner, _i32p), _p(mesh.neighbour, _i32p),
                 _p(diag, _f64p), _p(upper, _f64p), _p(x, _f64p), _p(y, _f64p))
    return y


def _stats(s: _Stats) -> Stats:
    return Stats(int(s.iters), bool(s.converged), bool(s.singular), bool(s.nonfinite),
                 float(s.init_res), float(s.final_res), float(s.norm_factor))


def pcg(owner, neighbour, diag, upper, source, psi, tol, rel_tol=0.0, max_iter=1000, min_iter=0,
        trace: int = 0):
    """Solves A psi = source from the initial guess psi (not modified). Returns
    (solution, Stats, trace_of_search_directions or None)."""
    lib = _load()
    owner = np.ascontiguousarray(owner, dtype=np.int32)
    neighbour = np.ascontiguousarray(neighbour, dtype=np.int32)
    diag = np.ascontiguousarray(diag, dtype=np.float64)
    upper = np.ascontiguousarray(upper, dtype=np.float64)
    source = np.ascontiguousarray(source, dtype=np.float64)
    x = np.array(psi, dtype=np.float64, copy=True)
    N, F = len(diag), len(upper)
    tr = np.zeros((trace, N)) if trace else None
    st = _Stats()
    rc = lib.ora_pcg(N, F, _p(owner, _i32p), _p(neighbour, _i32p), _p(diag, _f64p), _p(upper, _f64p),
                     _p(source, _f64p), _p(x, _f64p), float(tol), float(rel_tol), int(max_iter),
                     int(min_iter), ctypes.byref(st), _p(tr, _f64p), int(trace))
    if rc != 0:
        raise MemoryError("oracle PCG ran out of memory")
    return x, _stats(st), tr


def advance(case: lapcase.RawCase, n_steps: Optional[int] = None, mesh: Optional[Mesh] = None,
            T: Optional[np.ndarray] = None):
    """Runs ``n_steps`` (default: the case's) implicit steps. Returns (T by label, [Stats])."""
    lib = _load()
    mesh = mesh or mesh_of(case)
    n_steps = case.n_steps if n_steps is None else n_steps
    btype, bvalue = boundary_types_values(case, mesh)
    T = initial_field(case) if T is None else np.array(T, dtype=np.float64, copy=True)
    stats = (_Stats * max(n_steps, 1))()
    Su, Sp = source_arrays(case)
    if mesh.Sf is not None:
        rc = lib.ora_advance_corrected(
            mesh.n_cells, mesh.n_faces, _p(mesh.owner, _i32p), _p(mesh.neighbour, _i32p), _p(mesh.V, _f64p),
            _p(mesh.magSf, _f64p), _p(mesh.delta, _f64p), _p(mesh.DTf, _f64p), _p(mesh.Sf, _f64p),
            _p(mesh.w, _f64p), _p(mesh.corr, _f64p), mesh.n_bfaces, _p(mesh.bcell, _i32p), _p(btype, _i32p),
            _p(bvalue, _f64p), _p(mesh.bmagSf, _f64p), _p(mesh.bdelta, _f64p), _p(mesh.DTb, _f64p),
            _p(mesh.bSf, _f64p), float(case.dt), int(n_steps), int(case.n_nonorth_corr), float(case.tol),
            float(case.rel_tol), int(case.max_iter), int(case.min_iter), _p(Su, _f64p), _p(Sp, _f64p),
            _p(T, _f64p), stats)
        if rc != 0:
            raise MemoryError("oracle advance ran out of memory")
        return T, [_stats(stats[i]) for i in range(n_steps)]
    rc = lib.ora_advance(mesh.n_cells, mesh.n_faces, _p(mesh.owner, _i32p), _p(mesh.neighbour, _i32p),
                         _p(mesh.V, _f64p), _p(mesh.magSf, _f64p), _p(mesh.delta, _f64p),
                         _p(mesh.DTf, _f64p), mesh.n_bfaces, _p(mesh.bcell, _i32p), _p(btype, _i32p),
                         _p(bvalue, _f64p), _p(mesh.bmagSf, _f64p), _p(mesh.bdelta, _f64p),
                         _p(mesh.DTb, _f64p), float(case.dt), int(n_steps), float(case.tol),
                         float(case.rel_tol), int(case.max_iter), int(case.min_iter), _p(Su, _f64p),
                         _p(Sp, _f64p), _p(T, _f64p), stats)
    if rc != 0:
        raise MemoryError("oracle advance ran out of memory")
    return T, [_stats(stats[i]) for i in range(n_steps)]


def boundary_values(case: lapcase.RawCase, mesh: Mesh, T: np.ndarray) -> np.ndarray:
    lib = _load()
    btype, bvalue = boundary_types_values(case, mesh)
    T = np.ascontiguousarray(T, dtype=np.float64)
    Tb = np.empty(mesh.n_bfaces)
    lib.ora_boundary_values(mesh.n_bfaces, _p(mesh.bcell, _i32p), _p(btype, _i32p), _p(bvalue, _f64p),
                            _p(T, _f64p), _p(Tb, _f64p))
    return Tb


def dense_matrix(mesh: Mesh, diag: np.ndarray, upper: np.ndarray) -> np.ndarray:
    """The LDU matrix written out densely (small meshes only)."""
    A = np.diag(np.asarray(diag, dtype=np.float64)).copy()
    A[mesh.owner, mesh.neighbour] += upper
    A[mesh.neighbour, mesh.owner] += upper
    return A
