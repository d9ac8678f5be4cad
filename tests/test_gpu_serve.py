"""Serving form: each request's result is the same alone and in the mix (GPU required).

Requests arrive faster than they finish, under an HBM budget that holds only a few cases,
so later requests wait for admission and join running batches. Every finished field is
compared with the same request solved alone: FP64 to 1e-10, mixed precision to 1e-5 (and to
the FP64 oracle to 1e-5).
"""
import numpy as np
import pytest

import lapcase
import oracle
from paper_2507_18268_gb300 import Solver
from paper_2507_18268_gb300 import binding as B
from paper_2507_18268_gb300.serve import Server, serve_serial_fp64

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def test_served_results_match_alone_under_a_tight_budget():
    reqs = lapcase.serving_stream(n_requests=40, seed=9, rate_per_s=4000.0, n_min=6, n_max=16, max_steps=6)
    biggest = max(B.lfm_workspace_bytes_box(r.case.nx, r.case.ny, r.case.nz, B.LFM_BOTH) for r in reqs)
    budget = 4 * biggest
    server = Server(budget_bytes=budget)
    try:
        rep = server.run(reqs, keep_fields=True)
    finally:
        server.close()
    assert rep["requests"] == len(reqs) and rep["failed"] == 0
    assert rep["peak_hbm_bytes"] <= budget
    waited = [d for d in rep["done"] if d.admitted_s > d.arrival_s + 1e-3]
    assert waited, "the budget should have made some requests wait"
    for d in rep["done"]:
        case = reqs[d.index].case
        with Solver.from_box_case(case) as s:
            st = s.advance(case.n_steps)
            alone = s.field()
        if case.precision == B.LFM_FP64:
            assert relerr(d.field, alone) <= 1e-10, d.index
        else:
            assert relerr(d.field, alone) <= 1e-5, d.index
            To, _ = oracle.advance(case)
            assert relerr(d.field, To) <= 1e-5, d.index


def test_serial_baseline_runs_every_request():
    reqs = lapcase.serving_stream(n_requests=6, seed=2, rate_per_s=1000.0, n_min=6, n_max=10, max_steps=3)
    rep = serve_serial_fp64(reqs, keep_fields=True)
    assert rep["requests"] == 6 and len(rep["fields"]) == 6
    for r, T in zip(reqs, rep["fields"]):
        To, _ = oracle.advance(r.case.with_(precision=B.LFM_FP64))
        assert relerr(T, To) <= 1e-10
