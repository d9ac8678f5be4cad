"""Hexahedral box meshes in OpenFOAM's LDU face addressing (the blockMesh role).

Turns a box specification (:class:`lapcase.RawCase`: vertex coordinates per axis, optional
cell relabelling, per-face diffusivity, six patches) into the arrays ``lfm_upload_mesh``
takes (section "OpenFOAM" of arXiv 2507.18268: owner < neighbour per internal face, faces in
upper-triangular order, boundary faces grouped by patch; Table "Mesh dimensions" for the
box meshes of the evaluation).

Geometry of an orthogonal hexahedral mesh: cell volume dx*dy*dz; an internal face's area is
the product of the two widths parallel to it and its deltaCoeff is the inverse distance
between the two cell centres; a boundary face's deltaCoeff is the inverse distance from the
cell centre to the face centre.
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

import lapcase


@dataclasses.dataclass
class LduMesh:
    n_cells: int
    n_faces: int
    n_bfaces: int
    owner: np.ndarray          # int32 [F]
    neighbour: np.ndarray      # int32 [F]
    V: np.ndarray              # float64 [N]
    magSf: np.ndarray          # float64 [F]
    deltaCoeffs: np.ndarray    # float64 [F]
    patch_start: np.ndarray    # int32 [P]
    patch_size: np.ndarray     # int32 [P]
    bface_cell: np.ndarray     # int32 [NB]
    bmagSf: np.ndarray         # float64 [NB]
    bdeltaCoeffs: np.ndarray   # float64 [NB]
    DT_faces: np.ndarray       # float64 [F]   diffusivity per internal face
    DT_bfaces: np.ndarray      # float64 [NB]  diffusivity per boundary face
    cell_of_label: np.ndarray  # int64 [N]     natural cell id of each label

    @property
    def n_patches(self) -> int:
        return len(self.patch_start)


def _dt_array(arr, uniform, shape):
    if arr is None:
        return np.full(shape, float(uniform))
    return np.asarray(arr, dtype=np.float64).reshape(shape)


def box_mesh(case: lapcase.RawCase) -> LduMesh:
    nx, ny, nz = case.nx, case.ny, case.nz
    N = nx * ny * nz
    xs, ys, zs = (np.asarray(a, dtype=np.float64) for a in (case.xs, case.ys, case.zs))
    hx, hy, hz = np.diff(xs), np.diff(ys), np.diff(zs)
    cx, cy, cz = 0.5 * (xs[:-1] + xs[1:]), 0.5 * (ys[:-1] + ys[1:]), 0.5 * (zs[:-1] + zs[1:])
    label = np.arange(N, dtype=np.int64) if case.perm is None else np.asarray(case.perm, dtype=np.int64)
    lab3 = label.reshape(nz, ny, nx)  # [k, j, i]
    DTx = _dt_array(case.DTx, case.DT_uniform, (nz, ny, nx + 1))
    DTy = _dt_array(case.DTy, case.DT_uniform, (nz, ny + 1, nx))
    DTz = _dt_array(case.DTz, case.DT_uniform, (nz + 1, ny, nx))

    V = np.empty(N)
    V[lab3] = (hx[None, None, :] * hy[None, :, None]) * hz[:, None, None]

    a_list, b_list, area, dcoef, dtf = [], [], [], [], []
    # x-normal internal faces: (i, j, k) - (i+1, j, k)
    a_list.append(lab3[:, :, :-1].ravel())
    b_list.append(lab3[:, :, 1:].ravel())
    area.append(np.broadcast_to((hy[None, :, None] * hz[:, None, None]), (nz, ny, nx - 1)).ravel())
    dcoef.append(np.broadcast_to(1.0 / (cx[1:] - cx[:-1]), (nz, ny, nx - 1)).ravel())
    dtf.append(DTx[:, :, 1:nx].ravel())
    # y-normal
    a_list.append(lab3[:, :-1, :].ravel())
    b_list.append(lab3[:, 1:, :].ravel())
    area.append(np.broadcast_to((hx[None, None, :] * hz[:, None, None]), (nz, ny - 1, nx)).ravel())
    dcoef.append(np.broadcast_to((1.0 / (cy[1:] - cy[:-1]))[None, :, None], (nz, ny - 1, nx)).ravel())
    dtf.append(DTy[:, 1:ny, :].ravel())
    # z-normal
    a_list.append(lab3[:-1, :, :].ravel())
    b_list.append(lab3[1:, :, :].ravel())
    area.append(np.broadcast_to((hx[None, None, :] * hy[None, :, None]), (nz - 1, ny, nx)).ravel())
    dcoef.append(np.broadcast_to((1.0 / (cz[1:] - cz[:-1]))[:, None, None], (nz - 1, ny, nx)).ravel())
    dtf.append(DTz[1:nz, :, :].ravel())

    a = np.concatenate(a_list)
    b = np.concatenate(b_list)
    own = np.minimum(a, b)
    nei = np.maximum(a, b)
    order = np.lexsort((nei, own))
    owner = own[order].astype(np.int32)
    neighbour = nei[order].astype(np.int32)
    magSf = np.concatenate(area)[order]
    deltaCoeffs = np.concatenate(dcoef)[order]
    DT_faces = np.concatenate(dtf)[order]

    # boundary patches x0, x1, y0, y1, z0, z1
    cells, barea, bdel, bdt, sizes = [], [], [], [], []
    for side in (0, 1):
        i = nx - 1 if side else 0
        fx = xs[nx] if side else xs[0]
        cells.append(lab3[:, :, i].ravel())
        barea.append((hy[None, :] * hz[:, None]).ravel())
        bdel.append(np.full(ny * nz, 1.0 / abs(fx - cx[i])))
        bdt.append(DTx[:, :, nx if side else 0].ravel())
        sizes.append(ny * nz)
    for side in (0, 1):
        j = ny - 1 if side else 0
        fy = ys[ny] if side else ys[0]
        cells.append(lab3[:, j, :].ravel())
        barea.append((hx[None, :] * hz[:, None]).ravel())
        bdel.append(np.full(nx * nz, 1.0 / abs(fy - cy[j])))
        bdt.append(DTy[:, ny if side else 0, :].ravel())
        sizes.append(nx * nz)
    for side in (0, 1):
        k = nz - 1 if side else 0
        fz = zs[nz] if side else zs[0]
        cells.append(lab3[k, :, :].ravel())
        barea.append((hx[None, :] * hy[:, None]).ravel())
        bdel.append(np.full(nx * ny, 1.0 / abs(fz - cz[k])))
        bdt.append(DTz[nz if side else 0, :, :].ravel())
        sizes.append(nx * ny)
    sizes = np.array(sizes, dtype=np.int32)
    starts = np.concatenate(([0], np.cumsum(sizes)[:-1])).astype(np.int32)
    cell_of_label = np.empty(N, dtype=np.int64)
    cell_of_label[label] = np.arange(N, dtype=np.int64)
    return LduMesh(
        n_cells=N, n_faces=len(owner), n_bfaces=int(sizes.sum()), owner=owner, neighbour=neighbour,
        V=V, magSf=np.ascontiguousarray(magSf), deltaCoeffs=np.ascontiguousarray(deltaCoeffs),
        patch_start=starts, patch_size=sizes,
        bface_cell=np.concatenate(cells).astype(np.int32),
        bmagSf=np.ascontiguousarray(np.concatenate(barea)),
        bdeltaCoeffs=np.ascontiguousarray(np.concatenate(bdel)),
        DT_faces=np.ascontiguousarray(DT_faces), DT_bfaces=np.ascontiguousarray(np.concatenate(bdt)),
        cell_of_label=cell_of_label)


def field_by_label(case: lapcase.RawCase, mesh: LduMesh) -> np.ndarray:
    """The case's initial field T0 indexed by cell label."""
    return np.ascontiguousarray(case.T0_natural()[mesh.cell_of_label])


def uniform_dt(case: lapcase.RawCase) -> bool:
    return case.DTx is None and case.DTy is None and case.DTz is None
