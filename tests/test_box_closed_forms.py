"""The device box builder's closed forms, checked on the host (no GPU needed).

``lfm_box_layout`` runs the same per-cell routine as the device kernel behind
``lfm_upload_box``; its arrays must equal, bit for bit, what the general path produces for
the same box: the numpy mesh builder, the counting-sort face addressing, the slot layout
(neighbour-side faces ascending, owned faces ascending, padding), each face's slot in its
owner's and its neighbour's row, and the cell-side boundary lists. This also proves every
index the kernel writes is in range.
"""
import numpy as np
import pytest

import lapcase
from paper_2507_18268_gb300 import binding as B
from paper_2507_18268_gb300.mesh import box_mesh


def general_path(case):
    m = box_mesh(case)
    N, F = m.n_cells, m.n_faces
    own_start, losort, lo_start = B.lfm_face_addressing(N, m.owner, m.neighbour)
    deg = (np.diff(own_start) + np.diff(lo_start))
    W = int(deg.max()) if N else 0
    so = np.empty(W * N, np.int32)
    sf = np.empty(W * N, np.int32)
    fs = np.full(2 * F, 0xffffffff, np.uint32)
    for c in range(N):
        slots = [(int(m.owner[f]), int(f), 1) for f in losort[lo_start[c]:lo_start[c + 1]]]
        slots += [(int(m.neighbour[f]), int(f), 0) for f in range(own_start[c], own_start[c + 1])]
        slots += [(c, -1, -1)] * (W - len(slots))
        for k, (o, f, side) in enumerate(slots):
            so[k * N + c], sf[k * N + c] = o, f
            if side >= 0:
                fs[2 * f + side] = k * N + c
    counts = np.bincount(m.bface_cell, minlength=N)
    b_start = np.concatenate(([0], np.cumsum(counts))).astype(np.int32)
    b_face = np.argsort(m.bface_cell, kind="stable").astype(np.int32)
    return dict(slot_other=so, slot_face=sf, face_slots=fs, V=m.V, magSf=m.magSf, deltaCoeffs=m.deltaCoeffs, b_start=b_start,
                b_face=b_face, bface_cell=m.bface_cell, bmagSf=m.bmagSf, bdeltaCoeffs=m.bdeltaCoeffs, W=W)


SHAPES = [(1, 1, 1), (1, 1, 5), (2, 1, 1), (2, 2, 2), (3, 1, 2), (1, 4, 3), (4, 3, 2), (5, 5, 5), (7, 3, 4),
          (2, 3, 1), (6, 1, 6), (3, 3, 3)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("graded", [False, True])
def test_box_layout_matches_general_path(shape, graded):
    nx, ny, nz = shape
    rng = np.random.default_rng(nx * 100 + ny * 10 + nz)

    def axis(n):
        if not graded:
            return lapcase.uniform_axis(n)
        w = rng.uniform(0.5, 1.5, n)
        return np.concatenate(([0.0], np.cumsum(w / w.sum())))

    case = lapcase.RawCase(xs=axis(nx), ys=axis(ny), zs=axis(nz), DT_uniform=1.0)
    ref = general_path(case)
    got = B.lfm_box_layout(case.xs, case.ys, case.zs)
    assert got["W"] == ref["W"]
    for key in ("slot_other", "slot_face", "face_slots", "V", "magSf", "deltaCoeffs", "b_start", "b_face", "bface_cell",
                "bmagSf", "bdeltaCoeffs"):
        assert np.array_equal(got[key], ref[key]), key


def test_box_counts_and_rejections():
    assert B.lfm_box_counts(4, 3, 2) == (24, 3 * 3 * 2 + 4 * 2 * 2 + 4 * 3 * 1, 2 * (6 + 8 + 12), 5)
    with pytest.raises(B.LfmError):
        B.lfm_box_counts(0, 3, 2)
    with pytest.raises(B.LfmError):
        B.lfm_box_layout(np.array([0.0, 1.0, 0.5]), np.array([0.0, 1.0]), np.array([0.0, 1.0]))
