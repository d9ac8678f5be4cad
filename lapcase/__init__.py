"""Seeded synthetic inputs for the laplacianFoam time step (shared by the CUDA path and the oracle).

This module draws random numbers and writes down mesh *specifications*; it holds none of
the finite-volume arithmetic (no volumes, face areas, distances, matrix coefficients or
solver steps). Both consumers derive those independently from a :class:`RawCase`.

A raw case is a rectilinear hexahedral box (the blockMesh-style meshes of the paper's
evaluation, section "Evaluation", Table "Mesh dimensions") described by:

* ``xs, ys, zs`` -- vertex coordinates along each axis (lengths nx+1, ny+1, nz+1);
* ``perm`` -- optional relabelling of cells: natural cell id ``i + nx*(j + ny*k)`` gets label
  ``perm[id]`` (None = identity);
* diffusivity ``DT`` per geometric face: either the scalar ``DT_uniform`` or three arrays
  ``DTx[k, j, i]`` (shape nz, ny, nx+1; i indexes x-normal face planes 0..nx, boundary planes
  included), ``DTy[k, j, i]`` (nz, ny+1, nx) and ``DTz[k, j, i]`` (nz+1, ny, nx);
* six patches in the fixed order x0, x1, y0, y1, z0, z1, each ``(type, value)`` with type
  ``FIXED_VALUE`` or ``ZERO_GRADIENT``;
* the initial field ``T0`` (scalar, or an array over natural cell ids), the time step ``dt``,
  the number of steps and the PCG controls (tolerance, relTol, maxIter, minIter).

Face conventions every consumer must follow (they define the order of the LDU arrays):

* internal faces: one per pair of face-adjacent cells; owner = smaller label, neighbour =
  larger label; faces sorted by (owner, neighbour) -- OpenFOAM's upper-triangular order
  (section "OpenFOAM": every face has an owner, only internal faces a neighbour; the face
  normal points from owner to neighbour);
* boundary faces: grouped by patch in the order above; inside an x-patch faces run over
  (k, j) with j fastest, inside a y-patch over (k, i) with i fastest, inside a z-patch over
  (j, i) with i fastest.

Optional physics (section "The laplacianFoam application", Eq. (1)): ``DT_cells`` gives the
diffusivity as a cell field (over natural cell ids; it replaces the per-face DT and is
interpolated to faces by the consumer), ``Su`` and ``Sp`` a volumetric source
S_T = Su + Sp T per unit volume (scalars or arrays over natural cell ids). Cases with
``DT_cells`` use natural numbering.

General (non-orthogonal) hexahedral boxes add ``points`` -- vertex coordinates of shape
(nz+1, ny+1, nx+1, 3), vertex (i, j, k) at ``points[k, j, i]`` -- which replace the
rectilinear geometry (xs, ys, zs then only give the cell counts), and ``n_nonorth_corr``,
the number of extra non-orthogonal corrector passes per time step (OpenFOAM's
nNonOrthogonalCorrectors). Such cases use natural numbering (no ``perm``). Face point order
(it fixes each face's orientation): the +x face of cell (i, j, k) -- shared with (i+1, j, k)
-- has the points at i+1 in the order (j, k), (j+1, k), (j+1, k+1), (j, k+1); the +y face
the points at j+1 in the order (i, k), (i, k+1), (i+1, k+1), (i+1, k); the +z face the
points at k+1 in the order (i, j), (i+1, j), (i+1, j+1), (i, j+1). A boundary face on a
"1" patch (x1, y1, z1) uses the same order as the internal face in its direction; on a "0"
patch the reverse cycle starting from the same first point (x0: (j, k), (j, k+1),
(j+1, k+1), (j+1, k); y0: (i, k), (i+1, k), (i+1, k+1), (i, k+1); z0: (i, j), (i, j+1),
(i+1, j+1), (i+1, j)), so that boundary normals point out of the domain.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

FIXED_VALUE = 0
ZERO_GRADIENT = 1
PATCH_NAMES = ("x0", "x1", "y0", "y1", "z0", "z1")

FP64 = 0
MIXED = 1
DF64 = 2


@dataclasses.dataclass
class RawCase:
    xs: np.ndarray
    ys: np.ndarray
    zs: np.ndarray
    perm: Optional[np.ndarray] = None
    DT_uniform: float = 0.0
    DTx: Optional[np.ndarray] = None
    DTy: Optional[np.ndarray] = None
    DTz: Optional[np.ndarray] = None
    patches: Sequence[Tuple[int, float]] = ((FIXED_VALUE, 373.0), (FIXED_VALUE, 273.0),
                                           (ZERO_GRADIENT, 0.0), (ZERO_GRADIENT, 0.0),
                                           (ZERO_GRADIENT, 0.0), (ZERO_GRADIENT, 0.0))
    T0: object = 273.0
    dt: float = 0.005
    n_steps: int = 20
    tol: float = 1e-6
    rel_tol: float = 0.0
    max_iter: int = 1000
    min_iter: int = 0
    precision: int = FP64
    name: str = "case"
    points: Optional[np.ndarray] = None
    n_nonorth_corr: int = 0
    DT_cells: Optional[np.ndarray] = None
    Su: object = None
    Sp: object = None

    def cell_array(self, v) -> Optional[np.ndarray]:
        """A scalar or per-natural-cell quantity as an array over natural cell ids."""
        if v is None:
            return None
        if np.isscalar(v):
            return np.full(self.n_cells, float(v))
        return np.ascontiguousarray(v, dtype=np.float64).reshape(self.n_cells)

    @property
    def nx(self) -> int:
        return len(self.xs) - 1

    @property
    def ny(self) -> int:
        return len(self.ys) - 1

    @property
    def nz(self) -> int:
        return len(self.zs) - 1

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_internal_faces(self) -> int:
        nx, ny, nz = self.nx, self.ny, self.nz
        return (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)

    @property
    def n_boundary_faces(self) -> int:
        nx, ny, nz = self.nx, self.ny, self.nz
        return 2 * (ny * nz + nx * nz + nx * ny)

    def T0_natural(self) -> np.ndarray:
        """Initial field over natural cell ids (float64)."""
        if np.isscalar(self.T0):
            return np.full(self.n_cells, float(self.T0))
        return np.ascontiguousarray(self.T0, dtype=np.float64).reshape(self.n_cells)

    def with_(self, **kw) -> "RawCase":
        return dataclasses.replace(self, **kw)


def uniform_axis(n: int, length: float = 1.0) -> np.ndarray:
    return np.linspace(0.0, length, n + 1)


def graded_axis(n: int, ratio: float, length: float = 1.0) -> np.ndarray:
    """Vertex coordinates with each cell ``ratio`` times wider than the previous one."""
    widths = ratio ** np.arange(n, dtype=np.float64)
    widths *= length / widths.sum()
    xs = np.concatenate(([0.0], np.cumsum(widths)))
    xs[-1] = length
    return xs


def _log_uniform(rng: np.random.Generator, lo: float, hi: float, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def face_dt_arrays(nx: int, ny: int, nz: int, rng: np.random.Generator, lo: float, hi: float):
    """Per-geometric-face diffusivity drawn log-uniform in [lo, hi] (boundary faces included)."""
    DTx = _log_uniform(rng, lo, hi, (nz, ny, nx + 1))
    DTy = _log_uniform(rng, lo, hi, (nz, ny + 1, nx))
    DTz = _log_uniform(rng, lo, hi, (nz + 1, ny, nx))
    return DTx, DTy, DTz


# ---------------------------------------------------------------------------------------
# The five workloads (20^3 plain, 100^3 permuted, 200^3 graded, a batch of 512, a serving
# stream) and small variants of them for tests.
# ---------------------------------------------------------------------------------------

def plain_box(n: int = 20) -> RawCase:
    """n^3 unit cube, natural numbering, DT=4e-5, dt=0.005, 20 steps, x0=373 K, x1=273 K
    fixedValue, other faces zeroGradient, T0=273 K, tol 1e-6, relTol 0."""
    ax = uniform_axis(n)
    return RawCase(xs=ax, ys=ax.copy(), zs=ax.copy(), DT_uniform=4e-5, dt=0.005, n_steps=20,
                   tol=1e-6, rel_tol=0.0, T0=273.0, name=f"plain{n}")


def permuted_box(n: int = 100, seed_perm: int = 1, seed_dt: int = 2, n_steps: int = 50) -> RawCase:
    """n^3 unit cube with a seeded random cell relabelling and per-face DT log-uniform in
    [1e-6, 1e-4]; dt=0.01, tol 1e-8, boundary conditions and T0 as the plain box."""
    ax = uniform_axis(n)
    perm = np.random.default_rng(seed_perm).permutation(n ** 3).astype(np.int64)
    DTx, DTy, DTz = face_dt_arrays(n, n, n, np.random.default_rng(seed_dt), 1e-6, 1e-4)
    return RawCase(xs=ax, ys=ax.copy(), zs=ax.copy(), perm=perm, DTx=DTx, DTy=DTy, DTz=DTz,
                   dt=0.01, n_steps=n_steps, tol=1e-8, rel_tol=0.0, T0=273.0,
                   name=f"permuted{n}")


def graded_box(n: int = 200, ratio: float = 1.02, n_steps: int = 100,
               precision: int = FP64) -> RawCase:
    """n^3 unit cube graded in x (each cell ``ratio`` times the previous), uniform in y and z,
    boundary conditions and T0 as the plain box, DT=4e-5, dt=0.005, tol 1e-6."""
    return RawCase(xs=graded_axis(n, ratio), ys=uniform_axis(n), zs=uniform_axis(n),
                   DT_uniform=4e-5, dt=0.005, n_steps=n_steps, tol=1e-6, rel_tol=0.0,
                   T0=273.0, precision=precision, name=f"graded{n}")


def batch_cases(n_cases: int = 512, seed: int = 3, n_min: int = 16, n_max: int = 96,
                n_steps: int = 10, precision: int = FP64) -> List[RawCase]:
    """Independent cases: edge n log-uniform in [n_min, n_max], DT log-uniform in
    [1e-6, 1e-4], dt log-uniform in [1e-3, 1e-1], fixedValue temperatures U(250, 400) on
    x0 and x1 (drawn independently), zeroGradient elsewhere, T0 uniform = the x1 value."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_cases):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        DT = float(_log_uniform(rng, 1e-6, 1e-4))
        dt = float(_log_uniform(rng, 1e-3, 1e-1))
        Ta, Tb = (float(v) for v in rng.uniform(250.0, 400.0, 2))
        ax = uniform_axis(n)
        patches = ((FIXED_VALUE, Ta), (FIXED_VALUE, Tb)) + ((ZERO_GRADIENT, 0.0),) * 4
        out.append(RawCase(xs=ax, ys=ax.copy(), zs=ax.copy(), DT_uniform=DT, dt=dt,
                           n_steps=n_steps, tol=1e-6, rel_tol=0.0, T0=Tb, patches=patches,
                           precision=precision, name=f"batch{c}_n{n}"))
    return out


@dataclasses.dataclass
class Request:
    arrival_s: float
    case: RawCase


def serving_stream(n_requests: int = 2000, seed: int = 4, rate_per_s: float = 200.0,
                   n_min: int = 32, n_max: int = 160, max_steps: int = 50) -> List[Request]:
    """Poisson arrivals (exponential gaps, mean 1/rate) of solve requests: edge n
    log-uniform in [n_min, n_max], steps uniform in 1..max_steps, precision FP64 or mixed
    with probability 1/2, DT, dt and boundary values drawn as for :func:`batch_cases`."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(n_requests):
        t += float(rng.exponential(1.0 / rate_per_s))
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        steps = int(rng.integers(1, max_steps + 1))
        precision = MIXED if rng.random() < 0.5 else FP64
        DT = float(_log_uniform(rng, 1e-6, 1e-4))
        dt = float(_log_uniform(rng, 1e-3, 1e-1))
        Ta, Tb = (float(v) for v in rng.uniform(250.0, 400.0, 2))
        ax = uniform_axis(n)
        patches = ((FIXED_VALUE, Ta), (FIXED_VALUE, Tb)) + ((ZERO_GRADIENT, 0.0),) * 4
        out.append(Request(t, RawCase(xs=ax, ys=ax.copy(), zs=ax.copy(), DT_uniform=DT, dt=dt,
                                      n_steps=steps, tol=1e-6, rel_tol=0.0, T0=Tb,
                                      patches=patches, precision=precision,
                                      name=f"req{r}_n{n}")))
    return out


def random_small_case(seed: int, nx: int = 4, ny: int = 4, nz: int = 4, permute: bool = True,
                      face_dt: bool = True, graded: bool = True,
                      patch_types: Optional[Sequence[int]] = None) -> RawCase:
    """A small randomised case for validation: optional permutation, per-face DT, grading
    in all three axes, random patch values and a random initial field."""
    rng = np.random.default_rng(seed)

    def axis(n):
        if not graded:
            return uniform_axis(n)
        w = rng.uniform(0.5, 1.5, n)
        return np.concatenate(([0.0], np.cumsum(w / w.sum())))

    xs, ys, zs = axis(nx), axis(ny), axis(nz)
    N = nx * ny * nz
    perm = rng.permutation(N).astype(np.int64) if permute else None
    if face_dt:
        DTx, DTy, DTz = face_dt_arrays(nx, ny, nz, rng, 1e-3, 1e-1)
        DTu = 0.0
    else:
        DTx = DTy = DTz = None
        DTu = float(_log_uniform(rng, 1e-3, 1e-1))
    if patch_types is None:
        patch_types = [FIXED_VALUE if rng.random() < 0.5 else ZERO_GRADIENT for _ in range(6)]
    patches = tuple((int(t), float(rng.uniform(250, 400))) for t in patch_types)
    T0 = rng.uniform(250, 400, N)
    return RawCase(xs=xs, ys=ys, zs=zs, perm=perm, DT_uniform=DTu, DTx=DTx, DTy=DTy, DTz=DTz,
                   patches=patches, T0=T0, dt=float(_log_uniform(rng, 1e-3, 1.0)), n_steps=3,
                   tol=1e-12, rel_tol=0.0, name=f"small{seed}")


# ---------------------------------------------------------------------------------------
# General (non-orthogonal) hexahedral boxes
# ---------------------------------------------------------------------------------------

def box_points(xs: np.ndarray, ys: np.ndarray, zs: np.ndarray) -> np.ndarray:
    """Vertex array (nz+1, ny+1, nx+1, 3) of the rectilinear box on the given axes."""
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return np.ascontiguousarray(np.stack([X, Y, Z], axis=-1), dtype=np.float64)


def mapped_box(case: RawCase, M, shift=(0.0, 0.0, 0.0), n_nonorth_corr: int = 1) -> RawCase:
    """The case's box mapped by the affine map p -> M p + shift (faces stay planar; cells
    are parallelepipeds when M is not diagonal)."""
    P = box_points(case.xs, case.ys, case.zs)
    P = P @ np.asarray(M, dtype=np.float64).T + np.asarray(shift, dtype=np.float64)
    return case.with_(points=np.ascontiguousarray(P), n_nonorth_corr=n_nonorth_corr, perm=None,
                      name=case.name + "_mapped")


def perturbed_box(case: RawCase, amp: float = 0.2, seed: int = 5, n_nonorth_corr: int = 1) -> RawCase:
    """The case's box with every interior vertex moved along each axis by up to ``amp``
    times the smaller adjacent cell width (seeded, uniform); boundary vertices stay, so the
    faces inside the domain become warped quadrilaterals. amp < 0.5 keeps cells valid."""
    rng = np.random.default_rng(seed)
    P = box_points(case.xs, case.ys, case.zs)
    shape = P.shape[:3]
    interior = np.zeros(shape, dtype=bool)
    interior[1:-1, 1:-1, 1:-1] = True
    for a, v in enumerate((case.xs, case.ys, case.zs)):
        w = np.zeros(len(v))
        if len(v) > 2:
            w[1:-1] = np.minimum(np.diff(v)[:-1], np.diff(v)[1:])
        bshape = [1, 1, 1]
        bshape[2 - a] = len(v)
        P[..., a] += np.where(interior, amp * rng.uniform(-1.0, 1.0, shape) * w.reshape(bshape), 0.0)
    return case.with_(points=np.ascontiguousarray(P), n_nonorth_corr=n_nonorth_corr, perm=None,
                      name=case.name + "_perturbed")


def skewed_box(n: int = 200, n_steps: int = 100, precision: int = FP64) -> RawCase:
    """The graded n^3 box (graded200 for n=200) sheared by x' = x + 0.25 y + 0.15 z, with one
    non-orthogonal corrector per step; DT, dt, boundary conditions and tolerances as the
    graded box."""
    base = graded_box(n, n_steps=n_steps, precision=precision)
    M = [[1.0, 0.25, 0.15], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]]
    return mapped_box(base, M, n_nonorth_corr=1).with_(name=f"skewed{n}")


def two_material_box(n: int = 24, ratio: float = 20.0, n_steps: int = 5) -> RawCase:
    """A graded box split at x = 0.5 into two materials (DT 1e-2 and 1e-2 / ratio as a cell
    field), x0 = 373 K / x1 = 273 K fixedValue, insulated elsewhere."""
    xs = graded_axis(n, 1.05)
    cx = 0.5 * (xs[1:] + xs[:-1])
    DTc = np.where(cx < 0.5, 1e-2, 1e-2 / ratio)
    nat = np.broadcast_to(DTc[None, None, :], (n, n, n)).ravel().copy()
    return RawCase(xs=xs, ys=uniform_axis(n), zs=uniform_axis(n), DT_cells=nat, dt=0.5, n_steps=n_steps,
                   tol=1e-10, T0=300.0, name=f"two_material{n}")


def heated_box(n: int = 20, Su: float = 50.0, Sp: float = -0.5, n_steps: int = 5, seed: int = 6) -> RawCase:
    """A uniform box with a seeded random heat source Su in [0, 2 Su] per cell and a uniform
    implicit sink Sp, x0 = 373 K / x1 = 273 K fixedValue, insulated elsewhere."""
    rng = np.random.default_rng(seed)
    ax = uniform_axis(n)
    return RawCase(xs=ax, ys=ax.copy(), zs=ax.copy(), DT_uniform=4e-3, dt=0.05, n_steps=n_steps, tol=1e-10,
                   T0=300.0, Su=rng.uniform(0.0, 2.0 * Su, n ** 3), Sp=Sp, name=f"heated{n}")
