"""General (non-orthogonal) hexahedral meshes on the GPU against the CPU oracle: the Gauss
gradient (lfm_grad), the corrected assembly and the non-orthogonal corrector passes, in
FP64, mixed precision, several launch shapes and the batched form (GPU required).

Bars: FP64 and df64 fields within 1e-10 of the oracle and iteration counts within one per step
(the gradient divides by V through a rounded reciprocal, so the correction term -- and
with it the source -- agrees to rounding, not bitwise); normFactor and the initial residual
within the rounding bound of stat_bounds.py; the implicit matrix bitwise; the gradient
within 1e-12; mixed precision within 1e-5 of the FP64 oracle.
"""
import numpy as np
import pytest

import lapcase
import oracle
import stat_bounds
from paper_2507_18268_gb300 import Solver
from paper_2507_18268_gb300 import binding as B
from paper_2507_18268_gb300.batch import Batch
from paper_2507_18268_gb300.mesh import hex_mesh

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def perturbed(seed, nx=6, ny=5, nz=4, amp=0.3, n_corr=1, **kw):
    base = lapcase.random_small_case(seed, nx=nx, ny=ny, nz=nz, permute=False, **kw)
    return lapcase.perturbed_box(base, amp=amp, seed=seed + 100, n_nonorth_corr=n_corr).with_(tol=1e-10, n_steps=4)


CASES = {
    "perturbed_corr0": lambda: perturbed(1, n_corr=0),
    "perturbed_corr1": lambda: perturbed(2, n_corr=1),
    "perturbed_corr2_facedt": lambda: perturbed(3, n_corr=2, face_dt=True),
    "perturbed_insulated": lambda: perturbed(4, patch_types=[lapcase.ZERO_GRADIENT] * 6),
    "ragged_line": lambda: perturbed(5, nx=9, ny=2, nz=1, amp=0.2),
    "mapped24": lambda: lapcase.mapped_box(lapcase.graded_box(24, n_steps=5),
                                           [[1.0, 0.25, 0.15], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]], n_nonorth_corr=1),
    "perturbed40": lambda: lapcase.perturbed_box(lapcase.graded_box(40, n_steps=5), amp=0.25, n_nonorth_corr=1),
}


def gpu_advance(case, precision=None, launch=None):
    with Solver.from_case(case) as s:
        if precision is not None:
            s.set_solver(case.tol, case.rel_tol, case.max_iter, case.min_iter, precision)
        if launch:
            s.set_launch(*launch)
        st = s.advance(case.n_steps)
        return s.field(), st


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_parity(name):
    case = CASES[name]()
    To, so = oracle.advance(case)
    T, st = gpu_advance(case)
    assert rel(T, To) <= 1e-10, name
    for a, b in zip(st, so):
        assert abs(a["iters"] - b.iters) <= 1, (a, b)
        assert a["converged"] == 1


@pytest.mark.parametrize("form", ["fp64", "df64"])
@pytest.mark.parametrize("name", list(CASES))
def test_stats_within_rounding_bound(name, form):
    # normFactor and the first pass's initial residual of every step against the oracle's
    # step from the GPU's own field, within the derived rounding bound (stat_bounds.py; on
    # general meshes it includes the explicit correction's rounding); iterations within one
    case = CASES[name]()
    prec = B.LFM_FP64 if form == "fp64" else B.LFM_DF64
    _, recs = stat_bounds.gpu_walk(case, prec, form)
    stat_bounds.assert_walk(recs, iters_equal=False)
    for rec in recs:
        assert abs(rec["g"]["iters"] - rec["o"].iters) <= 1, rec


@pytest.mark.parametrize("name", list(CASES))
def test_df64_parity(name):
    # the df64 form on general meshes: gradient in difference form, correction in df64
    case = CASES[name]()
    To, so = oracle.advance(case)
    T, st = gpu_advance(case, precision=B.LFM_DF64)
    assert rel(T, To) <= 1e-10, name
    for a, b in zip(st, so):
        assert abs(a["iters"] - b.iters) <= 1, (a, b)
        assert a["converged"] == 1


@pytest.mark.parametrize("launch", [(1, 256), (7, 512), (0, 1024)])
def test_df64_parity_launch_shapes(launch):
    case = CASES["perturbed40"]()
    To, _ = oracle.advance(case)
    T, _ = gpu_advance(case, precision=B.LFM_DF64, launch=launch)
    assert rel(T, To) <= 1e-10


@pytest.mark.parametrize("launch", [(1, 256), (3, 512), (0, 1024)])
def test_fp64_parity_launch_shapes(launch):
    case = CASES["perturbed40"]()
    To, _ = oracle.advance(case)
    T, _ = gpu_advance(case, launch=launch)
    assert rel(T, To) <= 1e-10


@pytest.mark.parametrize("name", ["perturbed_corr1", "perturbed40", "mapped24"])
def test_mixed_precision(name):
    case = CASES[name]()
    To, _ = oracle.advance(case)
    T, st = gpu_advance(case, precision=B.LFM_MIXED)
    assert rel(T, To) <= 1e-5
    assert all(x["converged"] for x in st)


@pytest.mark.parametrize("name", ["perturbed_corr2_facedt", "mapped24", "perturbed_insulated"])
def test_gradient_matches_oracle(name):
    case = CASES[name]()
    om = oracle.hex_mesh(case)
    T0 = oracle.initial_field(case)
    G0, Gb0 = oracle.grad(case, om, T0)
    with Solver.from_case(case) as s:
        G, Gb = s.grad()
        s.advance(2)
        T2 = s.field()
        G2, Gb2 = s.grad()
    assert rel(G, G0) <= 1e-12 and rel(Gb, Gb0) <= 1e-12
    H2, Hb2 = oracle.grad(case, om, T2)
    assert rel(G2, H2) <= 1e-12 and rel(Gb2, Hb2) <= 1e-12


def test_corrected_assembly():
    case = CASES["perturbed_corr2_facedt"]()
    om = oracle.hex_mesh(case)
    bt, bv = oracle.boundary_types_values(case, om)
    T0 = oracle.initial_field(case)
    d0, u0, s0 = oracle.assemble(om, bt, bv, case.dt, T0)
    # the explicit correction of the first pass, from the oracle's gradient
    G = oracle.gauss_grad(om, T0, oracle.boundary_values(case, om, T0))
    Gf = om.w[:, None] * (G[om.owner] - G[om.neighbour]) + G[om.neighbour]
    flux = om.DTf * om.magSf * np.einsum("fi,fi->f", om.corr, Gf)
    divc = np.zeros(om.n_cells)
    np.add.at(divc, om.owner, flux)
    np.add.at(divc, om.neighbour, -flux)
    with Solver.from_case(case) as s:
        d, u, src = s.matrix()
    assert np.array_equal(d, d0) and np.array_equal(u, u0)
    assert rel(src, s0 + divc) <= 1e-13
    assert rel(src, s0) > 1e-6  # the correction is not negligible on this mesh


def test_rectilinear_box_through_the_general_path():
    base = lapcase.random_small_case(9, nx=7, ny=5, nz=6, permute=False, face_dt=True).with_(tol=1e-11, n_steps=3)
    hexcase = base.with_(points=lapcase.box_points(base.xs, base.ys, base.zs), n_nonorth_corr=1)
    To, _ = oracle.advance(base)
    T, _ = gpu_advance(hexcase)
    assert rel(T, To) <= 1e-10


def test_correctors_on_an_orthogonal_mesh():
    # extra passes on a box uploaded without geometry: zero correction, re-solves only
    base = lapcase.random_small_case(10, nx=6, ny=6, nz=5, permute=False).with_(tol=1e-11, n_steps=3)
    To, so = oracle.advance(base.with_(points=lapcase.box_points(base.xs, base.ys, base.zs), n_nonorth_corr=2))
    with Solver.from_case(base) as s:
        B.lfm_set_nonorth_correctors(s.ctx, 2)
        st = s.advance(base.n_steps)
        T = s.field()
    assert rel(T, To) <= 1e-10
    assert [x["iters"] for x in st] == [x.iters for x in so]


def test_batched_general_meshes_match_alone():
    cases = [perturbed(20 + i, nx=5 + i, ny=4, nz=3 + (i % 2), n_corr=i % 3) for i in range(5)]
    cases.append(CASES["mapped24"]())
    solvers = [Solver.from_case(c) for c in cases]
    try:
        bt = Batch()
        for s in solvers:
            bt.add(s)
        bt.advance(3)
        got = [s.field() for s in solvers]
        bt.close()
    finally:
        for s in solvers:
            s.close()
    for c, T in zip(cases, got):
        To, _ = oracle.advance(c, n_steps=3)
        assert rel(T, To) <= 1e-10, c.name


def test_geometry_validation_and_state():
    case = CASES["perturbed_corr1"]()
    mesh, geo = hex_mesh(case)
    ctx = B.lfm_create(0, None)
    try:
        bad = type(geo)(**{**geo.__dict__, "weights": np.where(np.arange(len(geo.weights)) == 3, 1.5, geo.weights)})
        with pytest.raises(B.LfmError) as e:
            B.lfm_upload_mesh_geometry(ctx, mesh, bad)
        assert e.value.code == B.LFM_EINVAL
        bad = type(geo)(**{**geo.__dict__, "Sf": geo.Sf * 1.001})
        with pytest.raises(B.LfmError) as e:
            B.lfm_upload_mesh_geometry(ctx, mesh, bad)
        assert e.value.code == B.LFM_EINVAL
        B.lfm_upload_mesh(ctx, mesh)  # without geometry: no gradient
        with pytest.raises(B.LfmError) as e:
            B.lfm_grad(ctx, mesh.n_cells, mesh.n_bfaces)
        assert e.value.code == B.LFM_ESTATE
        with pytest.raises(B.LfmError):
            B.lfm_set_nonorth_correctors(ctx, -1)
    finally:
        B.lfm_destroy(ctx)


def test_batched_general_meshes_with_ragged_slot_widths():
    # a 2-cell-thick and a 1-cell-thick mesh force the generic-width batch kernel
    cases = [perturbed(50, nx=8, ny=2, nz=3, n_corr=1), perturbed(51, nx=7, ny=1, nz=5, amp=0.2, n_corr=2),
             perturbed(52, n_corr=0)]
    solvers = [Solver.from_case(c) for c in cases]
    try:
        bt = Batch()
        for s in solvers:
            bt.add(s)
        bt.advance(3)
        got = [s.field() for s in solvers]
        bt.close()
    finally:
        for s in solvers:
            s.close()
    for c, T in zip(cases, got):
        To, _ = oracle.advance(c, n_steps=3)
        assert rel(T, To) <= 1e-10, c.name


def test_shared_general_mesh_matches_alone():
    case = CASES["perturbed_corr2_facedt"]()
    To, _ = oracle.advance(case)
    mesh, geo = hex_mesh(case)
    with Solver(mesh, geometry=geo) as owner:
        with Solver.sharing(owner, case) as s:
            s.advance(case.n_steps)
            T = s.field()
            G, _ = s.grad()
    assert rel(T, To) <= 1e-10
    G0, _ = oracle.grad(case, oracle.hex_mesh(case), To)
    assert rel(G, G0) <= 1e-12


def test_corrector_count_limits():
    with Solver.from_case(CASES["perturbed_corr1"]()) as s:
        with pytest.raises(B.LfmError) as e:
            B.lfm_set_nonorth_correctors(s.ctx, 65)
        assert e.value.code == B.LFM_EINVAL
        B.lfm_set_nonorth_correctors(s.ctx, 64)
