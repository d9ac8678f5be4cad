"""C-ABI library: loads and exports every declared symbol; host-side validation and
face-to-cell addressing (no GPU needed, no compute call)."""
import os
import re

import numpy as np
import pytest

import lapcase
from paper_2507_18268_gb300 import binding as B
from paper_2507_18268_gb300 import mesh as pm

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lapfoam.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lfm_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound():
    lib = B.load()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(B.declared_symbols())
    assert "sm_103a" in B.lfm_version()


def test_library_is_built_for_sm_103a_only():
    from paper_2507_18268_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _mesh(seed=0):
    return pm.box_mesh(lapcase.random_small_case(seed, nx=5, ny=4, nz=3))


def test_mesh_check_accepts_generated_meshes():
    for seed in range(3):
        assert B.lfm_mesh_check(_mesh(seed)) == ""


@pytest.mark.parametrize("mutation,needle", [
    ("owner_ge_neighbour", "owner"),
    ("out_of_range", "out of range"),
    ("unsorted", "upper-triangular"),
    ("nonpositive_volume", "V["),
    ("nan_area", "magSf"),
    ("bad_bcell", "boundary face"),
    ("patch_gap", "patch"),
])
def test_mesh_check_rejects(mutation, needle):
    m = _mesh(1)
    if mutation == "owner_ge_neighbour":
        m.owner = m.owner.copy(); m.owner[3] = m.neighbour[3]
    elif mutation == "out_of_range":
        m.neighbour = m.neighbour.copy(); m.neighbour[-1] = m.n_cells
    elif mutation == "unsorted":
        o, n = m.owner.copy(), m.neighbour.copy()
        o[[2, 7]] = o[[7, 2]]; n[[2, 7]] = n[[7, 2]]
        m.owner, m.neighbour = o, n
    elif mutation == "nonpositive_volume":
        m.V = m.V.copy(); m.V[4] = 0.0
    elif mutation == "nan_area":
        m.magSf = m.magSf.copy(); m.magSf[5] = np.nan
    elif mutation == "bad_bcell":
        m.bface_cell = m.bface_cell.copy(); m.bface_cell[0] = -1
    elif mutation == "patch_gap":
        m.patch_size = m.patch_size.copy(); m.patch_size[2] -= 1
    why = B.lfm_mesh_check(m)
    assert needle in why, why


@pytest.mark.parametrize("seed,permute", [(0, False), (1, True), (2, True)])
def test_face_addressing_matches_brute_force(seed, permute):
    case = lapcase.random_small_case(seed, nx=6, ny=5, nz=4, permute=permute)
    m = pm.box_mesh(case)
    own_start, losort, lo_start = B.lfm_face_addressing(m.n_cells, m.owner, m.neighbour)
    for c in range(m.n_cells):
        own = list(range(own_start[c], own_start[c + 1]))
        assert own == [f for f in range(m.n_faces) if m.owner[f] == c]
        lo = list(losort[lo_start[c]:lo_start[c + 1]])
        assert lo == [f for f in range(m.n_faces) if m.neighbour[f] == c]
    # every (cell, face) pair appears exactly once across both lists
    assert own_start[-1] == m.n_faces and lo_start[-1] == m.n_faces
    assert sorted(losort.tolist()) == list(range(m.n_faces))


def test_face_addressing_rejects_bad_input():
    with pytest.raises(B.LfmError) as e:
        B.lfm_face_addressing(3, [0, 1], [1, 1])
    assert e.value.code == B.LFM_EINVAL


def test_workspace_bytes_grow_with_mesh_and_precision():
    small = pm.box_mesh(lapcase.plain_box(8))
    big = pm.box_mesh(lapcase.plain_box(16))
    assert B.lfm_workspace_bytes(small) < B.lfm_workspace_bytes(big)
    w64 = B.lfm_workspace_bytes(big, B.LFM_FP64)
    w32 = B.lfm_workspace_bytes(big, B.LFM_MIXED)
    wb = B.lfm_workspace_bytes(big, B.LFM_BOTH)
    assert max(w32, w64) < wb < w32 + w64
    N, F = big.n_cells, big.n_faces
    # FP64 solve: at least the matrix (diag, upper, source, rD), the field and 4 vectors
    assert w64 >= 8 * (4 * N + F) + 8 * N + 8 * 4 * N


def test_product_mesh_builder_agrees_with_oracle_geometry():
    # two independent derivations of the same LDU mesh from one box specification
    import oracle
    for case in (lapcase.plain_box(6), lapcase.permuted_box(7, n_steps=1), lapcase.graded_box(5),
                 lapcase.random_small_case(3, nx=5, ny=4, nz=3)):
        m, o = pm.box_mesh(case), oracle.box_mesh(case)
        for a, b in ((m.owner, o.owner), (m.neighbour, o.neighbour), (m.V, o.V), (m.magSf, o.magSf),
                     (m.deltaCoeffs, o.delta), (m.DT_faces, o.DTf), (m.bface_cell, o.bcell),
                     (m.bmagSf, o.bmagSf), (m.bdeltaCoeffs, o.bdelta), (m.DT_bfaces, o.DTb)):
            assert np.array_equal(a, b)


def test_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(B.LfmError) as e:
        B.lfm_create(0, None)
    assert e.value.code == B.LFM_ECUDA


def test_workspace_sizes_by_precision():
    # host arithmetic only: the layout of each precision's solver buffers (8-byte FP64 /
    # double-float arrays, 4-byte FP32 arrays, the df64 block with its 4-byte triple-float part)
    m = _mesh(2)
    N, F, W = m.n_cells, m.n_faces, 6
    b64 = B.lfm_workspace_bytes(m, B.LFM_FP64)
    bmx = B.lfm_workspace_bytes(m, B.LFM_MIXED)
    bdf = B.lfm_workspace_bytes(m, B.LFM_DF64)
    ball = B.lfm_workspace_bytes(m, B.LFM_BOTH)
    assert 0 < b64 < bdf < ball and bmx < ball
    assert B.lfm_workspace_bytes(m, 7) == ball  # an unknown value lays out every form
    # the df64 block: x2, e2, diag2, rD2, vdt2 [8N], xlo, xolo [4N], g2 [8WN], each 256-aligned
    df_block = bdf - b64
    assert 5 * 8 * N + 2 * 4 * N + 8 * W * N <= df_block <= 5 * 8 * N + 2 * 4 * N + 8 * W * N + 8 * 256
    # every form's box workspace agrees with the general one for the same box
    case = lapcase.plain_box(7)
    bm = pm.box_mesh(case)
    for prec in (B.LFM_FP64, B.LFM_MIXED, B.LFM_DF64, B.LFM_BOTH):
        assert B.lfm_workspace_bytes_box(7, 7, 7, prec) == B.lfm_workspace_bytes(bm, prec)


def test_solver_log_layout():
    from paper_2507_18268_gb300 import solver_log
    st = [{"iters": 12, "converged": 1, "sweeps": 1, "status": 0, "init_res": 1.0, "final_res": 9.51e-07,
           "norm_factor": 3.2},
          {"iters": 0, "converged": 1, "sweeps": 0, "status": 0, "init_res": 4.0e-07, "final_res": 4.0e-07,
           "norm_factor": 3.1},
          {"iters": 3, "converged": 0, "sweeps": 1, "status": B.LFM_ENONFINITE, "init_res": 0.5,
           "final_res": float("nan"), "norm_factor": 3.0}]
    lines = solver_log(st, dt=0.005).split("\n")
    assert lines[0] == "Time = 0.005" and lines[1] == ""
    assert lines[2] == ("diagonalPCG:  Solving for T, Initial residual = 1, Final residual = 9.51e-07, "
                        "No Iterations 12")
    assert lines[3] == "Time = 0.01"
    assert lines[5].endswith("No Iterations 0")
    assert lines[8].endswith("No Iterations 3, status LFM_ENONFINITE")
    assert solver_log(st[:1], mixed=True).endswith("No Iterations 12, sweeps 1")
