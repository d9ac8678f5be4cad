"""The mixed form's FP32 A p with its matrix rows streamed into shared memory by bulk copies
(cp.async.bulk, completed on mbarriers) against the same pass loading the rows into
registers (GPU required).

Both forms give every thread the same cells and form every value by the same operations in
the same order, so field and statistics must agree bit for bit: on meshes with one or many
tiles per CTA, CTA ranges that end inside a tile, launch shapes from one CTA to many, and on
meshes whose cell count is not a multiple of 4, where both runs take the register form.
"""
import numpy as np
import pytest

from paper_2507_18268_gb300 import Solver
from paper_2507_18268_gb300 import binding as B

from test_gpu_parity import CASES

pytestmark = pytest.mark.gpu

STAT_KEYS = ("iters", "sweeps", "converged", "status", "init_res", "final_res", "norm_factor")


def run(case, prec, stage: bool, ctas=0, threads=0, n_steps=None, staged=None):
    """Field and statistics of a run; `staged` (a list) receives the number of passes that
    ran with staged rows, as the device counted them."""
    with Solver.from_case(case) as s:
        s.set_solver(case.tol, case.rel_tol, case.max_iter, case.min_iter, prec)
        if ctas or threads:
            s.set_launch(ctas, threads)
        B.lfm_debug_stage_rows(s.ctx, stage)
        st = s.advance(case.n_steps if n_steps is None else n_steps)
        if staged is not None:
            staged.append(B.lfm_debug_staged_passes(s.ctx))
        return s.field().copy(), st


def assert_same(a, b):
    Ta, sa = a
    Tb, sb = b
    assert np.array_equal(Ta, Tb), float(np.max(np.abs(Ta - Tb)))
    assert len(sa) == len(sb)
    for x, y in zip(sa, sb):
        for k in STAT_KEYS:
            assert x[k] == y[k], (k, x, y)


PRECS = [B.LFM_MIXED]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["plain20", "permuted20", "graded40", "small_perm_graded", "insulated",
                                  "plain7", "ragged", "line"])
def test_staged_rows_bitwise_equal_to_register_rows(name, prec):
    case = CASES[name]()
    n_on, n_off = [], []
    assert_same(run(case, prec, True, staged=n_on), run(case, prec, False, staged=n_off))
    # the staged form really ran where it applies (six slots, N a multiple of 4), and only there
    assert n_off == [0]
    if case.n_cells % 4 == 0 and min(case.nx, case.ny, case.nz) > 1:
        assert n_on[0] > 0
    else:
        assert n_on == [0]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("ctas,threads", [(1, 256), (1, 1024), (3, 256), (7, 512), (64, 256), (10000, 512)])
def test_staged_rows_across_launch_shapes(ctas, threads, prec):
    # graded40: 64,000 cells; one CTA takes 32+ tiles, 10,000 CTAs (clamped to what fits)
    # leave ranges shorter than a tile
    case = CASES["graded40"]()
    assert_same(run(case, prec, True, ctas, threads), run(case, prec, False, ctas, threads))


@pytest.mark.parametrize("prec", PRECS)
def test_staged_rows_on_a_full_size_mesh(prec):
    # the 1 M-cell relabelled box: gathers without locality, many tiles per CTA
    case = CASES["permuted100"]()
    assert_same(run(case, prec, True, n_steps=2), run(case, prec, False, n_steps=2))


def batch_run(cases, n_steps, stage: bool, use_graph: bool):
    from paper_2507_18268_gb300.batch import Batch
    with Batch() as bt:
        ids = [bt.add_case(c) for c in cases]
        B.lfm_batch_debug_stage_rows(bt.handle, stage)
        assert bt.advance(n_steps, use_graph=use_graph) == B.LFM_OK
        return [(bt.field(cid).copy(), bt.stats(cid, n_steps)) for cid in ids]


@pytest.mark.parametrize("use_graph", [True, False])
def test_staged_rows_in_the_batched_kernel(use_graph):
    # mixed cases with even and odd edges (N a multiple of 4 or not), teams of one to many
    # CTAs, beside FP64 and df64 cases that keep the register form
    import lapcase
    n_steps = 3
    cases = []
    for i, c in enumerate(lapcase.batch_cases(n_cases=12, seed=21, n_min=6, n_max=60, n_steps=n_steps)):
        prec = [lapcase.MIXED, lapcase.MIXED, lapcase.FP64, lapcase.DF64][i % 4]
        cases.append(c.with_(precision=prec))
    on = batch_run(cases, n_steps, True, use_graph)
    off = batch_run(cases, n_steps, False, use_graph)
    for a, b in zip(on, off):
        assert_same(a, b)


def test_a_staged_copy_that_never_lands_times_out_and_the_context_recovers():
    # CTA 1 issues no copy for its first tile: its bounded wait runs out (LFM_ETIMEOUT, the
    # other CTAs leave at their next barrier), and the same context then solves exactly as a
    # fresh one does (no GPU fault: every wait is bounded and the kernel returns)
    import oracle
    case = CASES["graded40"]()
    fresh = run(case, B.LFM_MIXED, True)
    with Solver.from_case(case) as s:
        s.set_solver(case.tol, case.rel_tol, case.max_iter, case.min_iter, B.LFM_MIXED)
        B.lfm_set_barrier_timeout(s.ctx, 200_000_000)  # 0.2 s
        B.lfm_debug_skip_stage_copy(s.ctx, 1)
        B.lfm_advance_async(s.ctx, 1)
        rc, _ = B.lfm_finish_status(s.ctx, 1)
        assert rc == B.LFM_ETIMEOUT
        s.set_field(oracle.initial_field(case))
        st = s.advance(case.n_steps)
        again = (s.field().copy(), st)
    assert_same(again, fresh)
