"""One case decomposed into parts on the GPU against the CPU oracle (GPU required).

Each part keeps its own vectors and receives its neighbours' interface values only through
the exchange (T once per step, p once per PCG iteration), with the global sums over all
parts -- the paper's multi-GPU data flow (section "Evaluation"), emulated in one launch on one
GPU. Bar: as the FP64 form, 1e-10 relative and the oracle's iteration count on every step,
for 1 to 7 parts on natural, relabelled, graded and ragged meshes; bitwise repeatable.
"""
import numpy as np
import pytest

import lapcase
import oracle
from paper_2507_18268_gb300 import Solver
from paper_2507_18268_gb300 import binding as B
from paper_2507_18268_gb300.decomp import Decomposed

pytestmark = pytest.mark.gpu

CASES = {
    "plain20": lambda: lapcase.plain_box(20),
    "permuted20": lambda: lapcase.permuted_box(20, n_steps=10),
    "graded40": lambda: lapcase.graded_box(40, n_steps=10),
    "ragged": lambda: lapcase.random_small_case(21, nx=7, ny=5, nz=3).with_(tol=1e-9, n_steps=4),
    "line": lambda: lapcase.RawCase(xs=lapcase.graded_axis(50, 1.05), ys=lapcase.uniform_axis(1),
                                    zs=lapcase.uniform_axis(1), DT_uniform=1e-2, dt=0.5, n_steps=5, tol=1e-12),
}


def relerr(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def dd_run(case, P):
    with Solver.from_case(case) as s:
        with Decomposed(s, P) as d:
            st = d.advance(case.n_steps)
            T = d.field()
            counts = d.counts()
    return T, st, counts


@pytest.mark.parametrize("P", [1, 2, 3, 4, 7])
@pytest.mark.parametrize("name", list(CASES))
def test_decomposed_matches_oracle(name, P):
    case = CASES[name]()
    To, so = oracle.advance(case)
    T, st, counts = dd_run(case, P)
    assert sum(c.n_owned for c in counts) == case.n_cells
    if P > 1 and name != "line":
        assert all(c.n_ghost > 0 for c in counts)
    assert [x["iters"] for x in st] == [x.iters for x in so], name
    assert all(x["converged"] and x["status"] == 0 for x in st)
    assert relerr(T, To) <= 1e-10


def test_decomposed_full_size_relabelled_100cubed():
    # 1M cells, relabelled with per-face DT: every part talks to every other
    case = lapcase.permuted_box(100, n_steps=5)
    To, so = oracle.advance(case)
    T, st, counts = dd_run(case, 4)
    assert [x["iters"] for x in st] == [x.iters for x in so]
    assert relerr(T, To) <= 1e-10
    assert all(c.n_send > 0 for c in counts)


def test_decomposed_is_bitwise_repeatable_and_resumable():
    case = CASES["permuted20"]()
    T1, s1, _ = dd_run(case, 3)
    T2, s2, _ = dd_run(case, 3)
    assert np.array_equal(T1, T2) and s1 == s2
    with Solver.from_case(case) as s:
        with Decomposed(s, 3) as d:
            d.advance(5)
            mid = d.field()
            d.set_field(mid)  # round trip through the host
            d.advance(5)
            T3 = d.field()
    assert np.array_equal(T3, T1)


def test_decomposed_rejects_what_it_does_not_cover():
    case = CASES["plain20"]()
    with Solver.from_case(case) as s:
        s.set_solver(case.tol, 0.0, 1000, 0, B.LFM_MIXED)
        with pytest.raises(B.LfmError) as e:
            Decomposed(s, 2)
        assert e.value.code == B.LFM_EINVAL
        s.set_solver(case.tol, 0.0, 1000, 0, B.LFM_FP64)
        with pytest.raises(B.LfmError) as e:
            Decomposed(s, 100000)
        assert e.value.code == B.LFM_EINVAL
