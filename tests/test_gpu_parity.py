"""CUDA path against the CPU oracle (GPU required).

FP64 bar: max |T_gpu - T_oracle| / |T_oracle| <= 1e-10 after every run and PCG iteration
counts equal to the oracle's on every step (the same recurrence; only summation order
differs). Assembly: bitwise equal (same products, same summation order, no FMA).
normFactor and the initial residual of every step, in every form (FP64, df64, mixed):
within the rounding bound derived in stat_bounds.py, the GPU step and the oracle's step
started from the same field.
Mixed precision bar: within 1e-5 of the FP64 oracle.
"""
import functools

import numpy as np
import pytest

import lapcase
import oracle
import stat_bounds
from paper_2507_18268_gb300 import Solver, box_mesh
from paper_2507_18268_gb300 import binding as B

pytestmark = pytest.mark.gpu

RTOL64 = 1e-10
RTOL_MIXED = 1e-5


def _cases():
    return {
        "plain20": lambda: lapcase.plain_box(20),
        "plain7": lambda: lapcase.plain_box(7).with_(DT_uniform=3e-3),
        "permuted20": lambda: lapcase.permuted_box(20, n_steps=10),
        "permuted100": lambda: lapcase.permuted_box(100),
        "graded40": lambda: lapcase.graded_box(40, n_steps=10),
        "ragged": lambda: lapcase.random_small_case(21, nx=7, ny=5, nz=3).with_(tol=1e-9, n_steps=4),
        "small_perm_graded": lambda: lapcase.random_small_case(5, nx=9, ny=6, nz=4).with_(tol=1e-8, n_steps=3),
        "line": lambda: lapcase.RawCase(xs=lapcase.graded_axis(50, 1.05), ys=lapcase.uniform_axis(1),
                                        zs=lapcase.uniform_axis(1), DT_uniform=1e-2, dt=0.5, n_steps=5,
                                        tol=1e-12),
        "one_cell": lambda: lapcase.RawCase(xs=np.array([0.0, 1.0]), ys=np.array([0.0, 1.0]),
                                            zs=np.array([0.0, 1.0]), DT_uniform=0.3, dt=0.1, n_steps=3,
                                            tol=1e-12),
        "insulated": lambda: lapcase.random_small_case(8, nx=8, ny=8, nz=8,
                                                       patch_types=[1] * 6).with_(tol=1e-9, n_steps=3),
    }


CASES = _cases()


@functools.lru_cache(maxsize=None)
def oracle_run(name, n_steps=None):
    case = CASES[name]()
    T, st = oracle.advance(case, n_steps=n_steps)
    return T, st


def gpu_run(case, n_steps=None, ctas=0, threads=0, precision=None, workspace="torch"):
    s = Solver.from_case(case, workspace=workspace)
    try:
        if precision is not None:
            s.set_solver(case.tol, case.rel_tol, case.max_iter, case.min_iter, precision)
        if ctas or threads:
            s.set_launch(ctas, threads)
        st = s.advance(case.n_steps if n_steps is None else n_steps)
        T = s.field()
        launch = s.launch()
    finally:
        s.close()
    return T, st, launch


def relerr(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def assert_parity(name, T, st, n_steps=None):
    To, so = oracle_run(name, n_steps)
    assert len(st) == len(so)
    for k, (g, o) in enumerate(zip(st, so)):
        assert g["iters"] == o.iters, (k, g, o)
        assert bool(g["converged"]) == o.converged
        assert g["status"] == 0
    # normFactor and the initial residual: per step from the same field, within the rounding
    # bound of stat_bounds (test_stats_within_rounding_bound)
    assert relerr(T, To) <= RTOL64


# ---- normFactor and the initial residual: within the derived rounding bound --------------

FORMS = {"fp64": B.LFM_FP64, "df64": B.LFM_DF64, "mixed": B.LFM_MIXED}


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("name", ["plain20", "plain7", "permuted20", "graded40", "ragged",
                                  "small_perm_graded", "line", "one_cell", "insulated", "permuted100"])
def test_stats_within_rounding_bound(name, form):
    # every step of the GPU run against the oracle's step from the GPU's own starting field;
    # the mixed form's normFactor and first residual are FP64-class as well (df64 outer
    # passes on these orthogonal meshes), so the same derivation bounds them
    case = CASES[name]()
    _, recs = stat_bounds.gpu_walk(case, FORMS[form], form, n_steps=10 if name == "permuted100" else None)
    stat_bounds.assert_walk(recs, iters_equal=form != "mixed")


# ---- assembly: bitwise ----------------------------------------------------------------

@pytest.mark.parametrize("name", ["plain7", "permuted20", "graded40", "ragged", "small_perm_graded",
                                  "one_cell", "insulated"])
def test_assembly_bitwise(name):
    case = CASES[name]()
    om = oracle.box_mesh(case)
    bt, bv = oracle.boundary_types_values(case, om)
    d0, u0, s0 = oracle.assemble(om, bt, bv, case.dt, oracle.initial_field(case))
    with Solver.from_case(case) as s:
        d, u, src = s.matrix()
    assert np.array_equal(d, d0)
    assert np.array_equal(u, u0)
    assert np.array_equal(src, s0)


# ---- FP64 solves ------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["plain20", "plain7", "permuted20", "graded40", "ragged",
                                  "small_perm_graded", "line", "one_cell", "insulated"])
def test_fp64_parity(name):
    T, st, _ = gpu_run(CASES[name]())
    assert_parity(name, T, st)


def test_fp64_parity_permuted_100cubed_full():
    # the 1M-cell relabelled case with per-face DT, all 50 steps, default launch
    T, st, launch = gpu_run(CASES["permuted100"]())
    assert launch[0] > 1
    assert_parity("permuted100", T, st)


@pytest.mark.parametrize("ctas,threads", [(1, 256), (1, 1024), (2, 512), (3, 256), (7, 512), (64, 256),
                                          (10000, 512)])
def test_fp64_launch_shapes(ctas, threads):
    # more CTAs than cells per CTA, ragged last CTA, clamped oversubscription
    T, st, launch = gpu_run(CASES["permuted20"](), ctas=ctas, threads=threads)
    assert launch[1] == threads
    assert_parity("permuted20", T, st)


def test_fp64_bitwise_deterministic():
    case = CASES["permuted20"]()
    T1, s1, _ = gpu_run(case, ctas=37, threads=256)
    T2, s2, _ = gpu_run(case, ctas=37, threads=256)
    assert np.array_equal(T1, T2)
    assert s1 == s2


def test_library_owned_workspace_matches_torch_workspace():
    case = CASES["ragged"]()
    T1, s1, _ = gpu_run(case, workspace="torch")
    T2, s2, _ = gpu_run(case, workspace="library")
    assert np.array_equal(T1, T2)


def test_checkpoint_resume_bitwise():
    case = CASES["permuted20"]()
    with Solver.from_case(case) as a:
        a.advance(10)
        a.advance(10)
        T_full_ref = a.field()
    with Solver.from_case(case) as b:
        b.advance(10)
        saved = b.field().copy()
    with Solver.from_case(case) as c:
        c.set_field(saved)
        c.advance(10)
        T_resumed = c.field()
    assert np.array_equal(T_full_ref, T_resumed)


def test_boundary_values():
    case = CASES["small_perm_graded"]()
    om = oracle.box_mesh(case)
    with Solver.from_case(case) as s:
        s.advance(2)
        T, Tb = s.fields()
    Tb0 = oracle.boundary_values(case, om, T)
    assert np.array_equal(Tb, Tb0)


def test_zero_diffusivity_takes_no_iteration():
    case = lapcase.plain_box(6).with_(DT_uniform=0.0, T0=np.linspace(250, 300, 216))
    T, st, _ = gpu_run(case, n_steps=2)
    assert all(s["iters"] == 0 and s["converged"] for s in st)
    assert np.array_equal(T, np.linspace(250, 300, 216)[box_mesh(case).cell_of_label])


def test_min_and_max_iter():
    case = CASES["permuted20"]().with_(min_iter=5, n_steps=2)
    T, st, _ = gpu_run(case)
    To, so = oracle.advance(case)
    assert [s["iters"] for s in st] == [s.iters for s in so] and all(s["iters"] >= 5 for s in st)
    assert relerr(T, To) <= RTOL64
    case = CASES["permuted20"]().with_(tol=1e-14, max_iter=3, n_steps=2)
    T, st, _ = gpu_run(case)
    To, so = oracle.advance(case)
    assert [s["iters"] for s in st] == [3, 3] == [s.iters for s in so] and not st[0]["converged"]
    assert relerr(T, To) <= RTOL64


def _two_cell_unequal():
    # the hand-worked case of tests/golden/two_cell_unequal.json (unequal volumes)
    return lapcase.RawCase(xs=np.array([0.0, 0.5, 2.0]), ys=np.array([0.0, 1.0]), zs=np.array([0.0, 1.0]),
                           DT_uniform=0.75, dt=0.5,
                           patches=((lapcase.FIXED_VALUE, 10.0),) + ((lapcase.ZERO_GRADIENT, 0.0),) * 5,
                           T0=np.array([1.0, 2.0]), n_steps=1, tol=1e-13)


@pytest.mark.parametrize("precision", [B.LFM_FP64, B.LFM_DF64])
def test_convergence_test_is_strict_at_a_tie(precision):
    # res == tol must not stop the solve: a run repeats its own residuals bit for bit, so a
    # tolerance set to the residual after one iteration (or to the initial residual) is an
    # exact tie, which a strict '<' resolves by iterating on
    case = _two_cell_unequal()

    def run(tol, max_iter=1000):
        with Solver.from_case(case) as s:
            s.set_solver(tol, 0.0, max_iter, 0, precision)
            return s.advance(1)[0]

    one = run(1e-13, max_iter=1)
    assert one["iters"] == 1 and not one["converged"]
    assert run(one["final_res"])["iters"] == 2
    assert run(float(np.nextafter(one["final_res"], 1.0)))["iters"] == 1
    assert run(one["init_res"])["iters"] >= 1
    assert run(float(np.nextafter(one["init_res"], 1.0)))["iters"] == 0
    # and the hand-worked values themselves
    g = run(1e-13)
    assert g["iters"] == 2
    assert abs(g["norm_factor"] - 31.5) <= 1e-13 * 31.5 and abs(g["init_res"] - 19 / 21) <= 1e-13


# ---- failure paths (no fault: host-made or bounded waits) -------------------------------

def test_barrier_timeout_returns_status_and_context_stays_usable():
    case = CASES["permuted20"]()
    with Solver.from_case(case) as s:
        s.set_launch(4, 256)
        B.lfm_set_barrier_timeout(s.ctx, 200_000_000)  # 0.2 s
        B.lfm_debug_skip_arrival(s.ctx, 1)
        B.lfm_advance_async(s.ctx, 1)
        rc, _ = B.lfm_finish_status(s.ctx, 1)
        assert rc == B.LFM_ETIMEOUT
        # the same context keeps working
        s.set_field(oracle.initial_field(case))
        st = s.advance(case.n_steps)
        T = s.field()
    assert_parity("permuted20", T, st)


def test_nonfinite_field_is_reported():
    case = CASES["plain7"]()
    with Solver.from_case(case) as s:
        T0 = oracle.initial_field(case)
        T0[5] = np.nan
        s.set_field(T0)
        with pytest.raises(B.LfmError) as e:
            s.advance(1)
        assert e.value.code == B.LFM_ENONFINITE


def test_out_of_order_and_bad_arguments():
    ctx = B.lfm_create(0, None)
    try:
        with pytest.raises(B.LfmError) as e:
            B.lfm_advance(ctx, 1)
        assert e.value.code == B.LFM_ESTATE
        m = box_mesh(lapcase.plain_box(4))
        B.lfm_upload_mesh(ctx, m)
        for bad in (lambda: B.lfm_set_time_step(ctx, 0.0), lambda: B.lfm_set_time_step(ctx, float("nan")),
                    lambda: B.lfm_set_patch(ctx, 6, 0), lambda: B.lfm_set_patch(ctx, 0, 7),
                    lambda: B.lfm_set_diffusivity(ctx, -1.0),
                    lambda: B.lfm_set_solver(ctx, 1e-6, 0, 0, 0, 0)):
            with pytest.raises(B.LfmError) as e:
                bad()
            assert e.value.code == B.LFM_EINVAL
    finally:
        B.lfm_destroy(ctx)


def test_bound_workspace_too_small():
    import torch
    m = box_mesh(lapcase.plain_box(6))
    need = B.lfm_workspace_bytes(m, B.LFM_MIXED)
    ws = torch.empty(need - 4096, dtype=torch.uint8, device="cuda")
    ctx = B.lfm_create(0, None)
    try:
        B.lfm_bind_workspace(ctx, ws.data_ptr(), need - 4096, B.LFM_MIXED)
        with pytest.raises(B.LfmError) as e:
            B.lfm_upload_mesh(ctx, m)
        assert e.value.code == B.LFM_ENOMEM
    finally:
        B.lfm_destroy(ctx)


# ---- mixed precision ------------------------------------------------------------------

@pytest.mark.parametrize("name", ["plain20", "graded40", "permuted20", "ragged", "insulated", "line", "permuted100"])
def test_mixed_within_1e5_of_fp64_oracle(name):
    case = CASES[name]()
    T, st, _ = gpu_run(case, precision=B.LFM_MIXED)
    To, so = oracle_run(name)
    assert relerr(T, To) <= RTOL_MIXED
    for g, o in zip(st, so):
        assert g["converged"] and g["final_res"] < case.tol
        assert g["sweeps"] <= 5


def test_mixed_workspace_only_layout():
    import torch
    case = CASES["graded40"]()
    m = box_mesh(case)
    need = B.lfm_workspace_bytes(m, B.LFM_MIXED)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    ctx = B.lfm_create(0, None)
    try:
        B.lfm_bind_workspace(ctx, ws.data_ptr(), need, B.LFM_MIXED)
        B.lfm_upload_mesh(ctx, m)
        with pytest.raises(B.LfmError) as e:
            B.lfm_set_solver(ctx, 1e-6, 0, 1000, 0, B.LFM_FP64)
        assert e.value.code == B.LFM_ENOMEM
        B.lfm_set_solver(ctx, case.tol, 0, 1000, 0, B.LFM_MIXED)
    finally:
        B.lfm_destroy(ctx)
