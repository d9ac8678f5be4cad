"""The df64 form (double-float arithmetic on the FP32 pipe) against the FP64 CPU oracle
(GPU required).

Bar, as for FP64: max |T_gpu - T_oracle| / |T_oracle| <= 1e-10 after every run and PCG
iteration counts equal to the oracle's on every step. The df64 form keeps 48 significand
bits instead of 53, so it is rounding-level close to FP64 (~1e-13 relative on these cases),
not bitwise; its reported normFactor and initial residual are checked against the oracle's
within the derived rounding bound (test_gpu_parity.py::test_stats_within_rounding_bound).
"""
import functools

import numpy as np
import pytest

import lapcase
import oracle
from paper_2507_18268_gb300 import Solver
from paper_2507_18268_gb300 import binding as B
from paper_2507_18268_gb300.batch import Batch

from test_gpu_parity import CASES, oracle_run, relerr

pytestmark = pytest.mark.gpu

RTOL = 1e-10


def df_run(case, n_steps=None, ctas=0, threads=0, layout=B.LFM_BOTH):
    s = Solver.from_case(case, layout=layout)
    try:
        s.set_solver(case.tol, case.rel_tol, case.max_iter, case.min_iter, B.LFM_DF64)
        if ctas or threads:
            s.set_launch(ctas, threads)
        st = s.advance(case.n_steps if n_steps is None else n_steps)
        T = s.field()
        launch = s.launch()
    finally:
        s.close()
    return T, st, launch


def assert_df_parity(T, st, To, so):
    assert len(st) == len(so)
    for k, (g, o) in enumerate(zip(st, so)):
        assert g["iters"] == o.iters, (k, g, o)
        assert bool(g["converged"]) == o.converged
        assert g["status"] == 0
    # normFactor and the initial residual of every step are checked against the derived
    # rounding bound in test_gpu_parity.py::test_stats_within_rounding_bound (df64 form)
    assert relerr(T, To) <= RTOL


@pytest.mark.parametrize("name", ["plain20", "plain7", "permuted20", "graded40", "ragged",
                                  "small_perm_graded", "line", "one_cell", "insulated"])
def test_df64_parity(name):
    T, st, _ = df_run(CASES[name]())
    To, so = oracle_run(name)
    assert_df_parity(T, st, To, so)


def test_df64_parity_permuted_100cubed_full():
    T, st, launch = df_run(CASES["permuted100"]())
    assert launch[0] > 1
    To, so = oracle_run("permuted100")
    assert_df_parity(T, st, To, so)


def test_graded200_full_size_all_forms():
    # the bench's workload at full size (200^3 graded box, 8 M cells), two steps, default
    # launch shape, every cell against the oracle: FP64 and df64 to 1e-10 with the oracle's
    # iteration counts, mixed to 1e-5
    case = lapcase.graded_box(200, n_steps=2)
    To, so = oracle.advance(case)
    for prec in (B.LFM_FP64, B.LFM_DF64, B.LFM_MIXED):
        with Solver.from_case(case.with_(precision=prec)) as s:
            st = s.advance(case.n_steps)
            T = s.field()
            assert s.launch()[0] >= 152
        if prec == B.LFM_MIXED:
            assert relerr(T, To) <= 1e-5
        else:
            assert_df_parity(T, st, To, so)


@functools.lru_cache(maxsize=None)
def _graded_oracle(n):
    return oracle.advance(lapcase.graded_box(n, n_steps=100))


@pytest.mark.parametrize("prec", [B.LFM_FP64, B.LFM_DF64])
@pytest.mark.parametrize("n", [40, 100])
def test_long_run_parity(prec, n):
    # 100 steps of the graded box's recipe: each step changes T by a small fraction, so the
    # initial residual is a small difference (see the flux form of the df64 row pass)
    case = lapcase.graded_box(n, n_steps=100)
    To, so = _graded_oracle(n)
    with Solver.from_case(case.with_(precision=prec)) as s:
        st = s.advance(case.n_steps)
        T = s.field()
    assert_df_parity(T, st, To, so)


@pytest.mark.parametrize("ctas,threads", [(1, 256), (1, 1024), (3, 256), (7, 512), (64, 256), (10000, 512)])
def test_df64_launch_shapes(ctas, threads):
    T, st, launch = df_run(CASES["permuted20"](), ctas=ctas, threads=threads)
    assert launch[1] == threads
    To, so = oracle_run("permuted20")
    assert_df_parity(T, st, To, so)


def test_df64_bitwise_deterministic():
    case = CASES["permuted20"]()
    T1, s1, _ = df_run(case, ctas=37, threads=256)
    T2, s2, _ = df_run(case, ctas=37, threads=256)
    assert np.array_equal(T1, T2)
    assert s1 == s2


def test_df64_only_workspace():
    case = CASES["ragged"]()
    T1, s1, _ = df_run(case, layout=B.LFM_DF64)
    T2, s2, _ = df_run(case, layout=B.LFM_BOTH)
    assert np.array_equal(T1, T2)
    with Solver.from_case(case, layout=B.LFM_DF64) as s:
        with pytest.raises(B.LfmError) as e:
            s.set_solver(case.tol, 0.0, 1000, 0, B.LFM_MIXED)
        assert e.value.code == B.LFM_ENOMEM
    with Solver.from_case(case.with_(precision=lapcase.MIXED), layout=B.LFM_MIXED) as s:
        with pytest.raises(B.LfmError) as e:
            s.set_solver(case.tol, 0.0, 1000, 0, B.LFM_DF64)
        assert e.value.code == B.LFM_ENOMEM


def test_df64_zero_diffusivity_and_iteration_limits():
    case = lapcase.plain_box(6).with_(DT_uniform=0.0, T0=np.linspace(250, 300, 216))
    T, st, _ = df_run(case, n_steps=2)
    To, so = oracle.advance(case, n_steps=2)
    assert all(s["iters"] == 0 and s["converged"] for s in st)
    assert relerr(T, To) <= 1e-14  # T passes through the 48-bit format once per launch
    case = CASES["permuted20"]().with_(min_iter=5, n_steps=2)
    T, st, _ = df_run(case)
    To, so = oracle.advance(case)
    assert [s["iters"] for s in st] == [s.iters for s in so]
    assert relerr(T, To) <= RTOL
    case = CASES["permuted20"]().with_(tol=1e-14, max_iter=3, n_steps=2)
    T, st, _ = df_run(case)
    To, so = oracle.advance(case)
    assert [s["iters"] for s in st] == [3, 3] and not st[0]["converged"]
    assert relerr(T, To) <= RTOL


def test_df64_dt_change_and_precision_switch():
    # the df64 conductances and V/dt are rebuilt after DT and dt change; switching to FP64 and
    # back continues from the same field
    case = CASES["permuted20"]().with_(n_steps=3)
    c2 = case.with_(DT_uniform=2.5e-3, DTx=None, DTy=None, DTz=None, dt=0.02)
    To, _ = oracle.advance(case)
    To2, _ = oracle.advance(c2, n_steps=3, T=To)
    with Solver.from_case(case) as s:
        s.set_solver(case.tol, 0.0, 1000, 0, B.LFM_DF64)
        s.advance(3)
        assert relerr(s.field(), To) <= RTOL
        B.lfm_set_diffusivity(s.ctx, 2.5e-3, None, None)
        B.lfm_set_time_step(s.ctx, 0.02)
        s.set_solver(case.tol, 0.0, 1000, 0, B.LFM_FP64)
        s.advance(1)
        s.set_solver(case.tol, 0.0, 1000, 0, B.LFM_DF64)
        s.advance(2)
        T = s.field()
    assert relerr(T, To2) <= RTOL


def test_df64_matrix_readback_is_the_fp64_assembly():
    case = CASES["graded40"]()
    with Solver.from_case(case) as s:
        d0, u0, s0 = s.matrix()
    with Solver.from_case(case) as s:
        s.set_solver(case.tol, 0.0, 1000, 0, B.LFM_DF64)
        s.advance(1)
        s.set_field(oracle.initial_field(case))
        d, u, src = s.matrix()
    assert np.array_equal(d, d0) and np.array_equal(u, u0) and np.array_equal(src, s0)


def test_df64_sources_and_correctors_on_orthogonal_mesh():
    case = lapcase.random_small_case(33, nx=7, ny=6, nz=5, permute=False).with_(
        Su=150.0, Sp=-0.3, tol=1e-10, n_steps=3)
    To, so = oracle.advance(case)
    T, st, _ = df_run(case)
    assert relerr(T, To) <= RTOL
    assert [s["iters"] for s in st] == [s.iters for s in so]
    # extra passes on a box uploaded without geometry: zero correction, re-solves only
    base = lapcase.random_small_case(10, nx=6, ny=6, nz=5, permute=False).with_(tol=1e-11, n_steps=3)
    To, so = oracle.advance(base.with_(points=lapcase.box_points(base.xs, base.ys, base.zs), n_nonorth_corr=2))
    with Solver.from_case(base) as s:
        s.set_solver(base.tol, 0.0, 1000, 0, B.LFM_DF64)
        B.lfm_set_nonorth_correctors(s.ctx, 2)
        st = s.advance(base.n_steps)
        T = s.field()
    assert relerr(T, To) <= RTOL
    assert [x["iters"] for x in st] == [x.iters for x in so]


def test_df64_general_geometry_in_a_df64_only_workspace():
    # general geometry with the df64 form in a workspace laid out for it alone, and in a batch
    base = lapcase.random_small_case(3, nx=6, ny=5, nz=4, permute=False)
    case = lapcase.perturbed_box(base, amp=0.2, seed=3).with_(tol=1e-10, n_steps=3, precision=lapcase.DF64)
    To, so = oracle.advance(case)
    with Solver.from_case(case, layout=B.LFM_DF64) as s:
        st = s.advance(case.n_steps)
        T = s.field()
    assert relerr(T, To) <= RTOL
    with Solver.from_case(case.with_(precision=lapcase.MIXED), layout=B.LFM_MIXED) as s:
        with pytest.raises(B.LfmError) as e:
            s.set_solver(case.tol, 0.0, 1000, 0, B.LFM_DF64)
        assert e.value.code == B.LFM_ENOMEM
    with Batch() as bt:
        ids = [bt.add_case(case), bt.add_case(case.with_(precision=lapcase.FP64))]
        bt.set_launch(256, (1, 1, 1))
        assert bt.advance(case.n_steps) == B.LFM_OK
        for cid in ids:
            assert relerr(bt.field(cid), To) <= RTOL


def test_df64_batched_matches_alone_and_oracle():
    n_steps = 4
    cases = lapcase.batch_cases(n_cases=12, seed=21, n_min=5, n_max=30, n_steps=n_steps)
    cases = [c.with_(precision=[lapcase.DF64, lapcase.FP64, lapcase.MIXED][i % 3]) for i, c in enumerate(cases)]
    with Batch() as bt:
        ids = [bt.add_case(c) for c in cases]
        bt.set_launch(256, (1, 1, 1))  # several CTAs per case
        assert bt.advance(n_steps) == B.LFM_OK
        for cid, c in zip(ids, cases):
            T = bt.field(cid)
            st = bt.stats(cid, n_steps)
            To, so = oracle.advance(c, n_steps=n_steps)
            if c.precision == lapcase.MIXED:
                assert relerr(T, To) <= 1e-5
                continue
            assert [x["iters"] for x in st] == [x.iters for x in so]
            assert relerr(T, To) <= RTOL
            if c.precision == lapcase.DF64:
                Ta, sa, _ = df_run(c, n_steps=n_steps)
                assert relerr(T, Ta) <= 1e-13


@pytest.mark.parametrize("prec", [B.LFM_DF64, B.LFM_MIXED])
def test_field_carried_between_launches(prec):
    # the triple-float field persists across launches: 3 + 3 steps equal 6 steps bitwise
    case = CASES["permuted20"]().with_(precision=prec)
    with Solver.from_case(case) as s:
        s.advance(3)
        s.advance(3)
        Ta = s.field()
    with Solver.from_case(case) as s:
        s.advance(6)
        Tb = s.field()
    assert np.array_equal(Ta, Tb)
    # a field written from the host replaces it: the same as a fresh case started there
    with Solver.from_case(case) as s:
        s.advance(3)
        T3 = s.field().copy()
        s.set_field(T3)
        s.advance(3)
        Tc = s.field()
    with Solver.from_case(case) as s:
        s.set_field(T3)
        s.advance(3)
        Td = s.field()
    assert np.array_equal(Tc, Td)
    # an FP64 launch in between writes the FP64 field: the next df launch starts from it
    with Solver.from_case(case) as s:
        s.advance(2)
        s.set_solver(case.tol, 0.0, 1000, 0, B.LFM_FP64)
        s.advance(1)
        T3 = s.field().copy()
        s.set_solver(case.tol, 0.0, 1000, 0, prec)
        s.advance(2)
        Te = s.field()
    with Solver.from_case(case) as s:
        s.set_field(T3)
        s.advance(2)
        Tf = s.field()
    assert np.array_equal(Te, Tf)


@pytest.mark.parametrize("name,tol,max_iter,min_iter,sweeps", [
    ("plain20", None, 1000, 0, "conv"),      # every step converges
    ("permuted20", None, 1000, 0, "more"),   # verifications that ask for another sweep
    ("graded40", 1e-11, 1000, 0, "more"),
    ("graded40", None, 1, 0, "cap"),         # steps that end at the iteration limit, not converged
    ("graded40", None, 3, 0, "any"),         # some steps end at the iteration limit
])
def test_mixed_fused_verification_bitwise(name, tol, max_iter, min_iter, sweeps):
    # Every mixed step after the first starts from the previous step's verification pass
    # (its rows and first residual formed there) -- within a launch, and across launches when
    # nothing changed in between (the seed carried in device memory); a step after a change
    # starts with its own sum and row passes. Same field, same statistics, bit for bit, for
    # one launch, one-step launches, and one-step launches with the seed invalidated between
    # them (a no-op change: the same time step set again).
    case = CASES[name]().with_(precision=B.LFM_MIXED)
    if tol is not None:
        case = case.with_(tol=tol)
    n = 5

    def run(chunks, touch=False):
        with Solver.from_case(case) as s:
            s.set_solver(case.tol, case.rel_tol, max_iter, min_iter, B.LFM_MIXED)
            st = []
            for k in chunks:
                if touch:
                    B.lfm_set_time_step(s.ctx, case.dt)
                st += s.advance(k)
            return s.field(), st

    Ta, sa = run([n])
    Tb, sb = run([1] * n)
    Tc, sc = run([1] * n, touch=True)
    assert np.array_equal(Ta, Tb) and np.array_equal(Ta, Tc)
    assert sa == sb == sc
    most = max(s["sweeps"] for s in sa)
    if sweeps == "conv":
        assert all(s["converged"] for s in sa)
    elif sweeps == "more":
        assert most > 1 and all(s["converged"] for s in sa)
    elif sweeps == "cap":
        assert not all(s["converged"] for s in sa)
    else:
        assert all(s["iters"] <= max_iter for s in sa)


def _scaled_case(kind):
    base = lapcase.random_small_case(41, nx=9, ny=7, nz=6).with_(tol=1e-10, n_steps=4)
    if kind == "celsius":
        # a field that crosses zero: leading parts of neighbouring values differ in sign
        return base.with_(patches=((lapcase.FIXED_VALUE, 50.0), (lapcase.FIXED_VALUE, -50.0),
                                   (lapcase.ZERO_GRADIENT, 0.0), (lapcase.ZERO_GRADIENT, 0.0),
                                   (lapcase.FIXED_VALUE, 0.0), (lapcase.ZERO_GRADIENT, 0.0)), T0=0.0)
    if kind == "micro":
        # a 1 mm box, small time step: V/dt and the conductances far from one
        return base.with_(xs=base.xs * 1e-3, ys=base.ys * 1e-3, zs=base.zs * 1e-3, dt=1e-4, DT_uniform=1e-7,
                          DTx=None, DTy=None, DTz=None)
    if kind == "large":
        # a 1 km box with a large diffusivity and time step
        return base.with_(xs=base.xs * 1e3, ys=base.ys * 1e3, zs=base.zs * 1e3, dt=1e5, DT_uniform=30.0,
                          DTx=None, DTy=None, DTz=None)
    raise KeyError(kind)


@pytest.mark.parametrize("kind", ["celsius", "micro", "large"])
def test_df64_and_mixed_at_extreme_scales(kind):
    case = _scaled_case(kind)
    To, so = oracle.advance(case)
    T, st, _ = df_run(case)
    scale = float(np.max(np.abs(To)))  # relative to the field's magnitude (T crosses zero)
    assert float(np.max(np.abs(T - To))) <= 1e-10 * scale
    assert [s["iters"] for s in st] == [s.iters for s in so]
    with Solver.from_case(case.with_(precision=lapcase.MIXED)) as s:
        s.advance(case.n_steps)
        Tm = s.field()
    assert float(np.max(np.abs(Tm - To))) <= 1e-5 * scale


@pytest.mark.parametrize("prec", [B.LFM_DF64, B.LFM_MIXED])
def test_timeout_and_nonfinite_in_the_df64_forms(prec):
    # a CTA that never arrives makes the others' bounded waits run out: LFM_ETIMEOUT, and the
    # same context then solves correctly (no GPU fault: the kernel returns)
    case = CASES["permuted20"]().with_(precision=prec)
    To, _ = oracle.advance(case)
    with Solver.from_case(case) as s:
        s.set_launch(4, 256)
        B.lfm_set_barrier_timeout(s.ctx, 200_000_000)  # 0.2 s
        B.lfm_debug_skip_arrival(s.ctx, 1)
        B.lfm_advance_async(s.ctx, 1)
        rc, _ = B.lfm_finish_status(s.ctx, 1)
        assert rc == B.LFM_ETIMEOUT
        s.set_field(oracle.initial_field(case))
        s.advance(case.n_steps)
        T = s.field()
    tol = RTOL if prec == B.LFM_DF64 else 1e-5
    assert relerr(T, To) <= tol
    # a non-finite field is reported, not propagated silently
    with Solver.from_case(case) as s:
        T0 = oracle.initial_field(case)
        T0[7] = np.nan
        s.set_field(T0)
        with pytest.raises(B.LfmError) as e:
            s.advance(1)
        assert e.value.code == B.LFM_ENONFINITE


def test_mixed_seed_is_not_carried_across_a_change():
    # a launch after a change of the time step must not start from the rows the last launch
    # left for the old one: equal to a new context started from the same field (up to the
    # triple-float field's rounding to FP64, which the new context starts from; rows of the
    # old time step would be off by far more)
    case = CASES["graded40"]().with_(precision=B.LFM_MIXED)
    with Solver.from_case(case) as s:
        s.set_solver(case.tol, 0.0, 1000, 0, B.LFM_MIXED)
        s.advance(3)
        T3 = s.field().copy()
        B.lfm_set_time_step(s.ctx, 2.5 * case.dt)
        st_a = s.advance(3)
        Ta = s.field()
    with Solver.from_case(case.with_(dt=2.5 * case.dt)) as t:
        t.set_solver(case.tol, 0.0, 1000, 0, B.LFM_MIXED)
        t.set_field(T3)
        st_b = t.advance(3)
        Tb = t.field()
    assert [x["iters"] for x in st_a] == [x["iters"] for x in st_b]
    assert [x["sweeps"] for x in st_a] == [x["sweeps"] for x in st_b]
    assert relerr(Ta, Tb) <= 1e-12
