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
from typing import List, Optional

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
    weights: Optional[np.ndarray] = None  # float64 [F] owner interpolation weight (rectilinear: h_N / (h_P + h_N))

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

    a_list, b_list, area, dcoef, dtf, wts = [], [], [], [], [], []
    # x-normal internal faces: (i, j, k) - (i+1, j, k)
    a_list.append(lab3[:, :, :-1].ravel())
    b_list.append(lab3[:, :, 1:].ravel())
    area.append(np.broadcast_to((hy[None, :, None] * hz[:, None, None]), (nz, ny, nx - 1)).ravel())
    dcoef.append(np.broadcast_to(1.0 / (cx[1:] - cx[:-1]), (nz, ny, nx - 1)).ravel())
    dtf.append(DTx[:, :, 1:nx].ravel())
    wts.append(np.broadcast_to(hx[1:] / (hx[:-1] + hx[1:]), (nz, ny, nx - 1)).ravel())
    # y-normal
    a_list.append(lab3[:, :-1, :].ravel())
    b_list.append(lab3[:, 1:, :].ravel())
    area.append(np.broadcast_to((hx[None, None, :] * hz[:, None, None]), (nz, ny - 1, nx)).ravel())
    dcoef.append(np.broadcast_to((1.0 / (cy[1:] - cy[:-1]))[None, :, None], (nz, ny - 1, nx)).ravel())
    dtf.append(DTy[:, 1:ny, :].ravel())
    wts.append(np.broadcast_to((hy[1:] / (hy[:-1] + hy[1:]))[None, :, None], (nz, ny - 1, nx)).ravel())
    # z-normal
    a_list.append(lab3[:-1, :, :].ravel())
    b_list.append(lab3[1:, :, :].ravel())
    area.append(np.broadcast_to((hx[None, None, :] * hy[None, :, None]), (nz - 1, ny, nx)).ravel())
    dcoef.append(np.broadcast_to((1.0 / (cz[1:] - cz[:-1]))[:, None, None], (nz - 1, ny, nx)).ravel())
    dtf.append(DTz[1:nz, :, :].ravel())
    wts.append(np.broadcast_to((hz[1:] / (hz[:-1] + hz[1:]))[:, None, None], (nz - 1, ny, nx)).ravel())

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
    # owner weight: the neighbour cell's share of the centre distance, with owner/neighbour
    # possibly swapped by the relabelling
    w_nat = np.concatenate(wts)
    weights = np.where(a <= b, w_nat, 1.0 - w_nat)[order]

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
        cell_of_label=cell_of_label, weights=np.ascontiguousarray(weights))


def field_by_label(case: lapcase.RawCase, mesh: LduMesh) -> np.ndarray:
    """The case's initial field T0 indexed by cell label."""
    return np.ascontiguousarray(case.T0_natural()[mesh.cell_of_label])


def uniform_dt(case: lapcase.RawCase) -> bool:
    return case.DTx is None and case.DTy is None and case.DTz is None


# ---------------------------------------------------------------------------------------
# General (non-orthogonal) hexahedral boxes from vertex positions
# ---------------------------------------------------------------------------------------

@dataclasses.dataclass
class HexGeometry:
    """The arrays ``lfm_upload_mesh_geometry`` takes, plus the centres they derive from."""
    Sf: np.ndarray        # [F, 3] internal face area vectors, owner -> neighbour
    weights: np.ndarray   # [F]    linear-interpolation weight of the owner value
    corr_vec: np.ndarray  # [F, 3] non-orthogonal correction vectors
    bSf: np.ndarray       # [NB, 3] boundary face area vectors, outward
    Cf: np.ndarray        # [F, 3] face centres
    bCf: np.ndarray       # [NB, 3]
    C: np.ndarray         # [N, 3] cell centres


def _dot3(a, b):
    return (a[:, 0] * b[:, 0] + a[:, 1] * b[:, 1]) + a[:, 2] * b[:, 2]


def _quad_geometry(q: np.ndarray):
    """Centres and area vectors of quadrilaterals q [M, 4, 3]: triangles (p_i, p_i+1, c) about
    the average point c of the four points; the area vector is half the sum of the triangle
    normals (p_i+1 - p_i) x (c - p_i), the centre the triangle centroids weighted by the
    normals' lengths."""
    fc = (((q[:, 0] + q[:, 1]) + q[:, 2]) + q[:, 3]) / 4.0
    sumN = np.zeros_like(fc)
    sumA = np.zeros(len(q))
    sumAc = np.zeros_like(fc)
    for p in range(4):
        a, b = q[:, p], q[:, (p + 1) % 4]
        e, t = b - a, fc - a
        n = np.stack([e[:, 1] * t[:, 2] - e[:, 2] * t[:, 1], e[:, 2] * t[:, 0] - e[:, 0] * t[:, 2],
                      e[:, 0] * t[:, 1] - e[:, 1] * t[:, 0]], axis=1)
        mag = np.sqrt(_dot3(n, n))
        sumN += n
        sumA += mag
        sumAc += mag[:, None] * ((a + b) + fc)
    ok = sumA > 1e-300
    Cf = np.where(ok[:, None], (1.0 / 3.0) * sumAc / np.where(ok, sumA, 1.0)[:, None], fc)
    return Cf, 0.5 * sumN


def _face_coeffs_on_device(device: int, N: int, owner, neighbour, Sf, Cf, C, bcell, bSf, bCf):
    """The per-face coefficients of hex_mesh computed on GPU ``device`` by the library's
    kernel (lfm_face_coeffs_device): weights, |Sf|, deltaCoeffs, correction vectors, boundary
    |Sf| and deltaCoeffs, returned as host arrays."""
    import torch

    from . import binding as B

    dev = torch.device("cuda", device)

    def up(a, dtype):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).to(dev)

    F, NB = len(owner), len(bcell)
    own, nei, bc = up(owner, np.int32), up(neighbour, np.int32), up(bcell, np.int32)
    sf, cf, c, bsf, bcf = (up(a, np.float64) for a in (Sf, Cf, C, bSf, bCf))
    f64 = dict(dtype=torch.float64, device=dev)
    w, mag, delta, corr = torch.empty(F, **f64), torch.empty(F, **f64), torch.empty(F, **f64), torch.empty((F, 3), **f64)
    bmag, bdelta = torch.empty(NB, **f64), torch.empty(NB, **f64)
    stream = torch.cuda.current_stream(dev)
    with torch.cuda.device(dev):
        B.lfm_face_coeffs_device(N, F, NB, own.data_ptr(), nei.data_ptr(), sf.data_ptr(), cf.data_ptr(), c.data_ptr(),
                                 bc.data_ptr(), bsf.data_ptr(), bcf.data_ptr(), w.data_ptr(), mag.data_ptr(),
                                 delta.data_ptr(), corr.data_ptr(), bmag.data_ptr(), bdelta.data_ptr(),
                                 stream.cuda_stream)
    return tuple(t.cpu().numpy() for t in (w, mag, delta, corr, bmag, bdelta))


def hex_mesh(case: lapcase.RawCase, device: Optional[int] = None):
    """LDU mesh and geometry of a general hexahedral box (``case.points``; natural
    numbering). Face point order as documented in :mod:`lapcase`. Returns
    (LduMesh, HexGeometry); the mesh's deltaCoeffs are the non-orthogonal implicit
    coefficients 1 / max(n.d, 0.05 |d|) and bdeltaCoeffs the inverse patch-normal
    distances 1 / |n.(Cf - C_P)|. With ``device`` the per-face coefficients (the
    interpolation weights, the implicit coefficients, the correction vectors) are computed
    on that GPU by the library's kernel; without it, here on the host, by the same formulas
    in the same order."""
    if case.points is None:
        raise ValueError("case has no vertex array")
    if case.perm is not None:
        raise ValueError("general hexahedral boxes use natural numbering")
    nx, ny, nz = case.nx, case.ny, case.nz
    P = np.asarray(case.points, dtype=np.float64)
    if P.shape != (nz + 1, ny + 1, nx + 1, 3):
        raise ValueError("points must have shape (nz+1, ny+1, nx+1, 3)")
    base = box_mesh(case)  # topology, patches and per-face DT (natural numbering)
    N, F, NB = base.n_cells, base.n_faces, base.n_bfaces
    nat = np.arange(N, dtype=np.int64).reshape(nz, ny, nx)

    def quads(*corners):
        return np.stack([c.reshape(-1, 3) for c in corners], axis=1)

    # internal faces by direction, then merged into (owner, neighbour) order
    qx = quads(P[:-1, :-1, 1:-1], P[:-1, 1:, 1:-1], P[1:, 1:, 1:-1], P[1:, :-1, 1:-1])
    qy = quads(P[:-1, 1:-1, :-1], P[1:, 1:-1, :-1], P[1:, 1:-1, 1:], P[:-1, 1:-1, 1:])
    qz = quads(P[1:-1, :-1, :-1], P[1:-1, :-1, 1:], P[1:-1, 1:, 1:], P[1:-1, 1:, :-1])
    own = np.concatenate([nat[:, :, :-1].ravel(), nat[:, :-1, :].ravel(), nat[:-1, :, :].ravel()])
    nei = np.concatenate([nat[:, :, 1:].ravel(), nat[:, 1:, :].ravel(), nat[1:, :, :].ravel()])
    order = np.lexsort((nei, own))
    q = np.concatenate([qx, qy, qz])[order]
    assert np.array_equal(own[order], base.owner) and np.array_equal(nei[order], base.neighbour)
    Cf, Sf = _quad_geometry(q)

    # boundary faces: x0, x1 over (k, j); y0, y1 over (k, i); z0, z1 over (j, i)
    bq = np.concatenate([
        quads(P[:-1, :-1, 0], P[1:, :-1, 0], P[1:, 1:, 0], P[:-1, 1:, 0]),
        quads(P[:-1, :-1, nx], P[:-1, 1:, nx], P[1:, 1:, nx], P[1:, :-1, nx]),
        quads(P[:-1, 0, :-1], P[:-1, 0, 1:], P[1:, 0, 1:], P[1:, 0, :-1]),
        quads(P[:-1, ny, :-1], P[1:, ny, :-1], P[1:, ny, 1:], P[:-1, ny, 1:]),
        quads(P[0, :-1, :-1], P[0, 1:, :-1], P[0, 1:, 1:], P[0, :-1, 1:]),
        quads(P[nz, :-1, :-1], P[nz, :-1, 1:], P[nz, 1:, 1:], P[nz, 1:, :-1]),
    ])
    bCf, bSf = _quad_geometry(bq)
    bcell = base.bface_cell.astype(np.int64)
    owner, neighbour = base.owner.astype(np.int64), base.neighbour.astype(np.int64)

    # cell centres and volumes: pyramids from each face to the average of the face centres,
    # contributions taken face by face (owner, then neighbour), boundary faces last
    targets = np.concatenate([np.stack([owner, neighbour], 1).ravel(), bcell])
    cEst = np.zeros((N, 3))
    np.add.at(cEst, targets, np.concatenate([np.repeat(Cf, 2, axis=0), bCf]))
    cEst /= np.bincount(targets, minlength=N)[:, None].astype(np.float64)
    fcs = np.concatenate([np.repeat(Cf, 2, axis=0), bCf])
    sfs = np.concatenate([np.repeat(Sf, 2, axis=0), bSf])
    sign_out = np.concatenate([np.tile([1.0, -1.0], F), np.ones(NB)])  # outward from the target cell
    pv = np.maximum(sign_out * _dot3(sfs, fcs - cEst[targets]), 1e-300)
    Csum = np.zeros((N, 3))
    vol = np.zeros(N)
    np.add.at(Csum, targets, pv[:, None] * (0.75 * fcs + 0.25 * cEst[targets]))
    np.add.at(vol, targets, pv)
    C = Csum / vol[:, None]
    V = vol / 3.0

    if device is not None:
        weights, magSf, delta, corr, bmagSf, bdelta = _face_coeffs_on_device(device, N, owner, neighbour, Sf, Cf, C,
                                                                           bcell, bSf, bCf)
        return _hex_result(base, V, magSf, delta, bmagSf, bdelta, Sf, weights, corr, bSf, Cf, bCf, C)

    # interpolation weights, implicit coefficients, correction vectors
    SfdOwn = np.abs(_dot3(Sf, Cf - C[owner]))
    SfdNei = np.abs(_dot3(Sf, C[neighbour] - Cf))
    tot = SfdOwn + SfdNei
    weights = np.where(np.abs(tot) > 1e-150, SfdNei / np.where(tot != 0, tot, 1.0), 0.5)
    magSf = np.sqrt(_dot3(Sf, Sf))
    n = Sf / magSf[:, None]
    d = C[neighbour] - C[owner]
    nd = np.maximum(_dot3(n, d), 0.05 * np.sqrt(_dot3(d, d)))
    delta = 1.0 / nd
    corr = n - d * delta[:, None]
    bmagSf = np.sqrt(_dot3(bSf, bSf))
    bn = bSf / bmagSf[:, None]
    bdelta = 1.0 / np.abs(_dot3(bn, bCf - C[bcell]))

    return _hex_result(base, V, magSf, delta, bmagSf, bdelta, Sf, weights, corr, bSf, Cf, bCf, C)


def _hex_result(base, V, magSf, delta, bmagSf, bdelta, Sf, weights, corr, bSf, Cf, bCf, C):
    mesh = dataclasses.replace(base, V=V, magSf=np.ascontiguousarray(magSf), deltaCoeffs=np.ascontiguousarray(delta),
                               bmagSf=np.ascontiguousarray(bmagSf), bdeltaCoeffs=np.ascontiguousarray(bdelta))
    geo = HexGeometry(Sf=np.ascontiguousarray(Sf), weights=np.ascontiguousarray(weights),
                      corr_vec=np.ascontiguousarray(corr), bSf=np.ascontiguousarray(bSf), Cf=Cf, bCf=bCf, C=C)
    return mesh, geo
