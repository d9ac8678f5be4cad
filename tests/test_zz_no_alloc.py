"""Allocation-free solve (lfm_pcg_solve_static) against the context path (GPU required).

The allocation-free entry point is for callers that cannot allocate device memory; it keeps
its working memory in a fixed array inside the library. Here it must reproduce what
lfm_advance computes for the same systems: two consecutive implicit steps of a relabelled
case with per-face DT, solved one after the other through the C ABI, within the FP64
parity tolerance (1e-10 relative) and with the same iteration counts.
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


def test_static_solve_matches_context_path_two_calls():
    import torch
    case = lapcase.permuted_box(20, n_steps=2)
    with Solver.from_case(case) as s:
        m = s.mesh
        owner = _dev(m.owner, torch.int32)
        neighbour = _dev(m.neighbour, torch.int32)
        T = s.field().copy()
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
    assert rc == B.LFM_EINVAL
    rc, _ = B.lfm_pcg_solve_static(4, 262145, idx.data_ptr(), idx.data_ptr(), one.data_ptr(), one.data_ptr(),
                                   one.data_ptr(), one.data_ptr(), 1e-6)
    assert rc == B.LFM_EINVAL
