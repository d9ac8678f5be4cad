"""Cell-field diffusivity and volumetric sources on the GPU against the CPU oracle (GPU
required). FP64 within 1e-10 of the oracle; mixed precision within 1e-5; the assembled
matrix with a source bitwise (orthogonal mesh, face DT), with a cell-field DT to rounding
(the interpolation weights come from the product's and the oracle's own geometry)."""
import numpy as np
import pytest

import lapcase
import oracle
from paper_2507_18268_gb300 import Solver
from paper_2507_18268_gb300 import binding as B
from paper_2507_18268_gb300.batch import Batch

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def cell_dt_general(seed=31):
    base = lapcase.random_small_case(seed, nx=6, ny=5, nz=4, permute=False)
    rng = np.random.default_rng(seed)
    case = lapcase.perturbed_box(base, amp=0.25, seed=seed, n_nonorth_corr=1)
    return case.with_(DT_cells=rng.uniform(1e-3, 1e-1, base.n_cells), Su=rng.uniform(-20, 20, base.n_cells),
                      Sp=-rng.uniform(0, 2, base.n_cells), tol=1e-10, n_steps=4)


CASES = {
    "two_material": lambda: lapcase.two_material_box(24),
    "heated": lambda: lapcase.heated_box(20),
    "heated_graded_facedt": lambda: lapcase.random_small_case(33, nx=7, ny=6, nz=5, permute=False).with_(
        Su=150.0, Sp=-0.3, tol=1e-10, n_steps=3),
    "general_cell_dt_source": cell_dt_general,
}


def run(case, precision=None):
    with Solver.from_case(case) as s:
        if precision is not None:
            s.set_solver(case.tol, case.rel_tol, case.max_iter, case.min_iter, precision)
        st = s.advance(case.n_steps)
        return s.field(), st


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_parity(name):
    case = CASES[name]()
    To, so = oracle.advance(case)
    T, st = run(case)
    assert rel(T, To) <= 1e-10
    for a, b in zip(st, so):
        assert abs(a["iters"] - b.iters) <= 1


@pytest.mark.parametrize("name", ["two_material", "heated", "general_cell_dt_source"])
def test_mixed_precision(name):
    case = CASES[name]()
    To, _ = oracle.advance(case)
    T, st = run(case, precision=B.LFM_MIXED)
    assert rel(T, To) <= 1e-5 and all(x["converged"] for x in st)


def test_assembly_with_source_is_bitwise():
    case = CASES["heated_graded_facedt"]()
    om = oracle.mesh_of(case)
    bt, bv = oracle.boundary_types_values(case, om)
    Su, Sp = oracle.source_arrays(case)
    d0, u0, s0 = oracle.assemble(om, bt, bv, case.dt, oracle.initial_field(case), Su, Sp)
    with Solver.from_case(case) as s:
        d, u, src = s.matrix()
    assert np.array_equal(d, d0) and np.array_equal(u, u0) and np.array_equal(src, s0)


def test_assembly_with_cell_dt():
    case = CASES["two_material"]()
    om = oracle.mesh_of(case)
    bt, bv = oracle.boundary_types_values(case, om)
    d0, u0, s0 = oracle.assemble(om, bt, bv, case.dt, oracle.initial_field(case))
    with Solver.from_case(case) as s:
        d, u, src = s.matrix()
    assert rel(u, u0) <= 1e-14 and rel(d, d0) <= 1e-14 and rel(src, s0) <= 1e-14


def test_batched_sources_match_alone():
    cases = [CASES["heated"]().with_(n_steps=3), CASES["two_material"]().with_(n_steps=3),
             cell_dt_general(40).with_(n_steps=3)]
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


def test_source_can_be_removed_and_arguments_checked():
    case = CASES["heated"]()
    plain = case.with_(Su=None, Sp=None)
    To, _ = oracle.advance(plain)
    with Solver.from_case(case) as s:
        B.lfm_set_source(s.ctx, None, None)
        s.set_field(oracle.initial_field(case))
        s.advance(case.n_steps)
        assert rel(s.field(), To) <= 1e-10
        with pytest.raises(B.LfmError) as e:
            B.lfm_set_diffusivity_cells(s.ctx, np.full(case.n_cells, 1e-3))  # no geometry, no weights
        assert e.value.code == B.LFM_EINVAL
        with pytest.raises(B.LfmError):
            B.lfm_set_diffusivity_cells(s.ctx, np.full(case.n_cells, -1.0), np.full(s.mesh.n_faces, 0.5))
        with pytest.raises(B.LfmError):
            B.lfm_set_source(s.ctx, np.full(case.n_cells, np.nan), None)
