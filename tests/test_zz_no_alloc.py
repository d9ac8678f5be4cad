"""Allocation-free solve (lfm_pcg_solve_static) against the context path (GPU required).

The allocation-free entry point is for callers that cannot allocate device memory; it keeps
its working memory in a fixed array inside the library. Here it must reproduce what
lfm_advance computes for the same systems: two consecutive implicit steps of a relabelled
case with per-face DT, solved one after the other through the C ABI, within the FP64
parity tolerance (1e-10 relative) and with the same iteration counts -- on a small case and
at the documented limit of 65,536 cells. Systems the kernel must reject (faces not sorted
by owner, a cell with more internal faces than the limit) return LFM_EINVAL with x left
as it was, and every rejection names its reason in lfm_last_error(NULL).
"""
import numpy as np
import pytest

import lapcase
from paper_2507_18268_gb300 import Solver
from paper_2507_18268_gb300 import binding as B

pytestmark = pytest.mark.gpu

RTOL64 = 1e-10


def _dev(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _limit_case():
    # 64 x 32 x 32 = 65,536 cells (the limit), 191,488 faces, relabelled, per-face DT
    nx, ny, nz = 64, 32, 32
    rng = np.random.default_rng(11)
    perm = rng.permutation(nx * ny * nz).astype(np.int64)
    DTx, DTy, DTz = lapcase.face_dt_arrays(nx, ny, nz, rng, 1e-6, 1e-4)
    return lapcase.RawCase(xs=lapcase.uniform_axis(nx), ys=lapcase.uniform_axis(ny), zs=lapcase.uniform_axis(nz),
                           perm=perm, DTx=DTx, DTy=DTy, DTz=DTz, dt=0.01, n_steps=2, tol=1e-8)


@pytest.mark.parametrize("which", ["permuted20", "limit65536"])
def test_static_solve_matches_context_path_two_calls(which):
    import torch
    case = lapcase.permuted_box(20, n_steps=2) if which == "permuted20" else _limit_case()
    with Solver.from_case(case) as s:
        m = s.mesh
        owner = _dev(m.owner, torch.int32)
        neighbour = _dev(m.neighbour, torch.int32)
        T = s.field().copy()
        assert which != "limit65536" or m.n_cells == 65536
        x = _dev(T, torch.float64)
        for step in range(2):
            diag, upper, source = s.matrix()          # the system lfm_advance solves next
            ref = s.advance(1)[0]                     # existing entry point
            T_ref = s.field()
            d, u, b = _dev(diag, torch.float64), _dev(upper, torch.float64), _dev(source, torch.float64)
            torch.cuda.synchronize()
            rc, st = B.lfm_pcg_solve_static(m.n_cells, m.n_faces, owner.data_ptr(), neighbour.data_ptr(),
                                            d.data_ptr(), u.data_ptr(), b.data_ptr(), x.data_ptr(),
                                            case.tol, case.rel_tol, case.max_iter, case.min_iter)
            assert rc == B.LFM_OK, B.lfm_last_error()
            assert st.iters == ref["iters"] and st.converged == ref["converged"]
            got = x.cpu().numpy()
            assert np.max(np.abs(got - T_ref) / np.abs(T_ref)) <= RTOL64, step
            # continue the next step from the context path's state, as lfm_advance does
            x.copy_(_dev(T_ref, torch.float64))


def test_static_solve_rejects_oversized_systems():
    import torch
    one = torch.zeros(4, dtype=torch.float64, device="cuda")
    idx = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc, _ = B.lfm_pcg_solve_static(65537, 0, idx.data_ptr(), idx.data_ptr(), one.data_ptr(), one.data_ptr(),
                                   one.data_ptr(), one.data_ptr(), 1e-6)
    assert rc == B.LFM_EINVAL and "exceed the fixed limits" in B.lfm_last_error()
    rc, _ = B.lfm_pcg_solve_static(4, 262145, idx.data_ptr(), idx.data_ptr(), one.data_ptr(), one.data_ptr(),
                                   one.data_ptr(), one.data_ptr(), 1e-6)
    assert rc == B.LFM_EINVAL


def _static(m_cells, owner, neighbour, d, u, b, x, tol=1e-8):
    return B.lfm_pcg_solve_static(m_cells, len(owner), owner.data_ptr(), neighbour.data_ptr(), d.data_ptr(),
                                  u.data_ptr(), b.data_ptr(), x.data_ptr(), tol)


def test_static_solve_rejects_unsorted_owners_and_leaves_x():
    import torch
    case = lapcase.permuted_box(8, n_steps=1)
    with Solver.from_case(case) as s:
        m = s.mesh
        diag, upper, source = s.matrix()
        T = s.field().copy()
    own = np.array(m.owner, dtype=np.int32)
    nbr = np.array(m.neighbour, dtype=np.int32)
    f = int(np.argmax(own[1:] > own[:-1])) + 1       # first face of the second owner
    own[[f - 1, f]] = own[[f, f - 1]]                 # two faces out of owner order
    nbr[[f - 1, f]] = nbr[[f, f - 1]]
    assert np.all(nbr > own) and np.any(own[1:] < own[:-1])
    x = _dev(T, torch.float64)
    rc, _ = _static(m.n_cells, _dev(own, torch.int32), _dev(nbr, torch.int32), _dev(diag, torch.float64),
                    _dev(upper, torch.float64), _dev(source, torch.float64), x)
    assert rc == B.LFM_EINVAL
    assert "not sorted by owner" in B.lfm_last_error()
    assert np.array_equal(x.cpu().numpy(), T)
    # the same call with the faces in order still solves (the shared array recovers)
    rc, st = _static(m.n_cells, _dev(m.owner, torch.int32), _dev(m.neighbour, torch.int32), _dev(diag, torch.float64),
                     _dev(upper, torch.float64), _dev(source, torch.float64), x)
    assert rc == B.LFM_OK and st.converged


def test_static_solve_rejects_a_cell_above_the_face_limit():
    import torch
    # a star: cell 0 owns a face to each of 39 other cells (more than 32 internal faces)
    N = 40
    own = np.zeros(N - 1, dtype=np.int32)
    nbr = np.arange(1, N, dtype=np.int32)
    d = np.full(N, 50.0)
    u = np.full(N - 1, -1.0)
    b = np.ones(N)
    x0 = np.full(N, 2.0)
    x = _dev(x0, torch.float64)
    rc, _ = _static(N, _dev(own, torch.int32), _dev(nbr, torch.int32), _dev(d, torch.float64),
                    _dev(u, torch.float64), _dev(b, torch.float64), x)
    assert rc == B.LFM_EINVAL
    assert "more than 32 internal faces" in B.lfm_last_error()
    assert np.array_equal(x.cpu().numpy(), x0)


def test_static_solve_rejects_x_overlapping_an_input():
    import torch
    N = 8
    own = _dev(np.arange(N - 1, dtype=np.int32), torch.int32)
    nbr = _dev(np.arange(1, N, dtype=np.int32), torch.int32)
    d = _dev(np.full(N, 4.0), torch.float64)
    u = _dev(np.full(N - 1, -1.0), torch.float64)
    b = _dev(np.ones(N), torch.float64)
    rc, _ = _static(N, own, nbr, d, u, b, b)          # in place on the source
    assert rc == B.LFM_EINVAL and "overlaps" in B.lfm_last_error()
    rc, _ = _static(N, own, nbr, d, u, b, d)
    assert rc == B.LFM_EINVAL


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")  # nothing is captured: that is the point
def test_static_solve_refuses_a_capturing_stream():
    # the call synchronises its stream, so on a stream under capture it must refuse before
    # any device work and leave the capture intact; the same call afterwards solves
    import torch
    N = 8
    own = _dev(np.arange(N - 1, dtype=np.int32), torch.int32)
    nbr = _dev(np.arange(1, N, dtype=np.int32), torch.int32)
    d = _dev(np.full(N, 4.0), torch.float64)
    u = _dev(np.full(N - 1, -1.0), torch.float64)
    b = _dev(np.ones(N), torch.float64)
    x = _dev(np.zeros(N), torch.float64)
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        graph.capture_begin(capture_error_mode="thread_local")
        try:
            rc, _ = B.lfm_pcg_solve_static(N, N - 1, own.data_ptr(), nbr.data_ptr(), d.data_ptr(), u.data_ptr(),
                                           b.data_ptr(), x.data_ptr(), 1e-10, stream=side.cuda_stream)
        finally:
            graph.capture_end()
    assert rc == B.LFM_ESTATE and "captured" in B.lfm_last_error()
    rc, st = B.lfm_pcg_solve_static(N, N - 1, own.data_ptr(), nbr.data_ptr(), d.data_ptr(), u.data_ptr(),
                                    b.data_ptr(), x.data_ptr(), 1e-10, stream=side.cuda_stream)
    assert rc == B.LFM_OK and st.converged
    A = np.diag(np.full(N, 4.0)) - np.diag(np.ones(N - 1), 1) - np.diag(np.ones(N - 1), -1)
    assert np.allclose(x.cpu().numpy(), np.linalg.solve(A, np.ones(N)), rtol=1e-8)
