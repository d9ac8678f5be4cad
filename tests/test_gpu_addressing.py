"""Face-to-cell addressing built on the device at upload equals, entry for entry, the
host reference built here from the counting-sort lists of ``lfm_face_addressing`` (GPU
required): slot rows, face slot positions, boundary lists."""
import numpy as np
import pytest

import lapcase
from paper_2507_18268_gb300 import Solver
from paper_2507_18268_gb300 import binding as B
from paper_2507_18268_gb300.mesh import box_mesh, hex_mesh

pytestmark = pytest.mark.gpu


def host_reference(m):
    N, F = m.n_cells, m.n_faces
    own_start, losort, lo_start = B.lfm_face_addressing(N, m.owner, m.neighbour)
    deg = np.diff(own_start) + np.diff(lo_start)
    W = int(deg.max()) if N else 0
    so = np.empty(W * N, np.int32)
    sf = np.empty(W * N, np.int32)
    fs = np.zeros(2 * F, np.uint32)
    for c in range(N):
        row = [(int(m.owner[f]), int(f), 1) for f in losort[lo_start[c]:lo_start[c + 1]]]
        row += [(int(m.neighbour[f]), int(f), 0) for f in range(own_start[c], own_start[c + 1])]
        row += [(c, -1, -1)] * (W - len(row))
        for k, (o, f, side) in enumerate(row):
            so[k * N + c], sf[k * N + c] = o, f
            if side >= 0:
                fs[2 * f + side] = k * N + c
    counts = np.bincount(m.bface_cell, minlength=N)
    b_start = np.concatenate(([0], np.cumsum(counts))).astype(np.int32)
    b_face = np.argsort(m.bface_cell, kind="stable").astype(np.int32)
    return dict(slot_other=so, slot_face=sf, face_slots=fs, b_start=b_start, b_face=b_face), W


MESHES = {
    "permuted_small": lambda: box_mesh(lapcase.random_small_case(1, nx=6, ny=5, nz=4)),
    "permuted_ragged": lambda: box_mesh(lapcase.random_small_case(2, nx=9, ny=2, nz=3)),
    "permuted30": lambda: box_mesh(lapcase.permuted_box(30)),
    "line": lambda: box_mesh(lapcase.RawCase(xs=lapcase.uniform_axis(40), ys=lapcase.uniform_axis(1),
                                             zs=lapcase.uniform_axis(1))),
    "one_cell": lambda: box_mesh(lapcase.RawCase(xs=np.array([0.0, 1.0]), ys=np.array([0.0, 1.0]),
                                                 zs=np.array([0.0, 1.0]))),
    "general": lambda: hex_mesh(lapcase.perturbed_box(lapcase.random_small_case(3, permute=False)))[0],
}


@pytest.mark.parametrize("name", list(MESHES))
def test_device_addressing_equals_host_reference(name):
    m = MESHES[name]()
    ref, W = host_reference(m)
    with Solver(m) as s:
        got = B.lfm_get_addressing(s.ctx, m.n_cells, m.n_faces, m.n_bfaces, W)
    for k in ("slot_other", "slot_face", "face_slots", "b_start", "b_face"):
        assert np.array_equal(got[k], ref[k]), k


def test_device_addressing_is_deterministic_on_a_large_mesh():
    m = box_mesh(lapcase.permuted_box(100))
    with Solver(m) as s1, Solver(m) as s2:
        a = B.lfm_get_addressing(s1.ctx, m.n_cells, m.n_faces, m.n_bfaces, 6)
        b = B.lfm_get_addressing(s2.ctx, m.n_cells, m.n_faces, m.n_bfaces, 6)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    # every face sits in exactly one slot of its owner's row and one of its neighbour's
    N = m.n_cells
    fs = a["face_slots"].astype(np.int64)
    assert np.array_equal(fs[0::2] % N, m.owner) and np.array_equal(fs[1::2] % N, m.neighbour)
    assert np.array_equal(a["slot_face"][fs[0::2]], np.arange(m.n_faces))
    assert np.array_equal(a["slot_face"][fs[1::2]], np.arange(m.n_faces))
