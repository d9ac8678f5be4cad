"""The rounding bound of stat_bounds.py on the CPU (no GPU needed).

An independent numpy evaluation of normFactor and the initial residual -- row sums formed
as V/dt + the fixedValue conductances (as the GPU forms them), pairwise sums, products and
sums in numpy's order -- must lie within the bound of the oracle's values; the bound must be
far tighter than the quantities themselves; and a formula mistake (a volume-weighted mean
in normFactor) must fall outside it, so the bound can tell rounding from a wrong formula.
"""
import numpy as np
import pytest

import lapcase
import oracle
import stat_bounds


def _numpy_stats(case, om, T, weighted_mean=False):
    bt, bv = oracle.boundary_types_values(case, om)
    d, up, b = oracle.assemble(om, bt, bv, case.dt, T)
    Ax = d * T
    np.add.at(Ax, om.owner, up * T[om.neighbour])
    np.add.at(Ax, om.neighbour, up * T[om.owner])
    fv = bt == lapcase.FIXED_VALUE
    gb = np.zeros(om.n_cells)
    np.add.at(gb, om.bcell[fv], ((om.DTb * om.bmagSf) * om.bdelta)[fv])
    s = gb + om.V / case.dt
    xb = np.sum(om.V * T) / np.sum(om.V) if weighted_mean else np.sum(T) / om.n_cells
    nf = np.sum(np.abs(Ax - s * xb) + np.abs(b - s * xb)) + 1e-20
    return nf, np.sum(np.abs(b - Ax)) / nf


CASES = {
    "plain20": lambda: lapcase.plain_box(20),
    "graded24": lambda: lapcase.graded_box(24, n_steps=3),
    "permuted12": lambda: lapcase.permuted_box(12, n_steps=3),
    "small": lambda: lapcase.random_small_case(3, nx=7, ny=5, nz=4),
    "insulated": lambda: lapcase.random_small_case(8, nx=6, ny=6, nz=6, patch_types=[1] * 6),
}


@pytest.mark.parametrize("name", list(CASES))
def test_independent_evaluation_within_bound(name):
    case = CASES[name]()
    om = oracle.mesh_of(case)
    T = oracle.initial_field(case)
    for step in range(3):
        _, so = oracle.advance(case, n_steps=1, mesh=om, T=T)
        o = so[0]
        nf, ir = _numpy_stats(case, om, T)
        # launch (1, 1): a serial sum of all N values on the other side, the longest depth
        B_nf, B_ir = stat_bounds.step_bounds(case, om, T, "fp64", (1, 1), o.norm_factor, o.init_res)
        assert abs(nf - o.norm_factor) <= B_nf, (step, nf, o.norm_factor, B_nf)
        assert abs(ir - o.init_res) <= B_ir, (step, ir, o.init_res, B_ir)
        # non-vacuous: far below the values themselves
        assert B_nf < 1e-6 * o.norm_factor and B_ir < 1e-6 * o.init_res
        T, _ = oracle.advance(case, n_steps=1, mesh=om, T=T)


def test_a_wrong_mean_falls_outside_the_bound():
    case = lapcase.graded_box(20, n_steps=2)
    om = oracle.mesh_of(case)
    T, _ = oracle.advance(case, n_steps=1, mesh=om)
    _, so = oracle.advance(case, n_steps=1, mesh=om, T=T)
    nf, _ = _numpy_stats(case, om, T, weighted_mean=True)
    B_nf, _ = stat_bounds.step_bounds(case, om, T, "df64", (1, 1), so[0].norm_factor, so[0].init_res)
    assert abs(nf - so[0].norm_factor) > 10 * B_nf
