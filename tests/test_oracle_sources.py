"""Pins of the oracle's cell-field diffusivity and volumetric sources (CPU only).

  * a cell-field DT reaches the faces by linear interpolation: a uniform field stays uniform,
    a field linear in x gives its value at the face plane;
  * the steady state of a two-material slab equals the series-conductance solution computed
    here from the geometry alone;
  * the source S_T = Su + Sp T: uniform fields follow the closed form of one implicit Euler
    step, insulated boxes balance energy exactly, a heated slab rises above the linear profile.
"""
import numpy as np
import pytest

import lapcase
import oracle


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_uniform_cell_dt_equals_uniform_dt():
    base = lapcase.random_small_case(3, nx=5, ny=4, nz=3, permute=False, face_dt=False)
    D = 0.037
    m = oracle.mesh_of(base.with_(DT_cells=np.full(base.n_cells, D)))
    assert rel(m.DTf, np.full(m.n_faces, D)) < 3e-16 and np.all(m.DTb == D)
    T1, _ = oracle.advance(base.with_(DT_uniform=D))
    T2, _ = oracle.advance(base.with_(DT_uniform=0.0, DT_cells=np.full(base.n_cells, D)))
    assert rel(T2, T1) < 1e-12


def test_linear_cell_dt_interpolates_exactly():
    nx, ny, nz = 6, 3, 2
    xs = lapcase.graded_axis(nx, 1.4)
    case = lapcase.RawCase(xs=xs, ys=lapcase.uniform_axis(ny), zs=lapcase.uniform_axis(nz))
    cx = 0.5 * (xs[1:] + xs[:-1])
    DTc = np.broadcast_to((0.5 + 2.0 * cx)[None, None, :], (nz, ny, nx)).ravel().copy()
    m = oracle.mesh_of(case.with_(DT_cells=DTc))
    # x-normal faces: DT at the face plane; y/z-normal faces join cells with equal DT
    i_own = m.owner % nx
    xface = m.neighbour == m.owner + 1
    expect = np.where(xface, 0.5 + 2.0 * xs[i_own + 1], 0.5 + 2.0 * cx[i_own])
    assert rel(m.DTf, expect) < 1e-14


def test_two_material_steady_state_is_the_series_conductance_solution():
    n = 12
    case = lapcase.two_material_box(n).with_(ys=lapcase.uniform_axis(2), zs=lapcase.uniform_axis(2), dt=1e9,
                                             n_steps=3, tol=1e-14)
    nx = n
    DTc = np.where(0.5 * (case.xs[1:] + case.xs[:-1]) < 0.5, 1e-2, 1e-2 / 20.0)
    case = case.with_(DT_cells=np.broadcast_to(DTc[None, None, :], (2, 2, nx)).ravel().copy())
    T, _ = oracle.advance(case)
    # conductances per unit area of the x-chain: boundary half cells and interpolated faces
    h = np.diff(case.xs)
    gb0, gb1 = DTc[0] / (h[0] / 2), DTc[-1] / (h[-1] / 2)
    w = h[1:] / (h[:-1] + h[1:])
    DTf = w * DTc[:-1] + (1 - w) * DTc[1:]
    g = DTf / ((h[:-1] + h[1:]) / 2)
    R = 1 / gb0 + np.sum(1 / g) + 1 / gb1
    q = (373.0 - 273.0) / R
    Tc = np.empty(nx)
    Tc[0] = 373.0 - q / gb0
    for i in range(nx - 1):
        Tc[i + 1] = Tc[i] - q / g[i]
    got = T.reshape(2, 2, nx)
    assert rel(got, np.broadcast_to(Tc, (2, 2, nx))) < 1e-9


def test_uniform_source_step_has_the_closed_form():
    ax = lapcase.uniform_axis(4)
    ins = ((lapcase.ZERO_GRADIENT, 0.0),) * 6
    for Su, Sp in ((3.0, 0.0), (3.0, -0.8), (0.0, -2.5)):
        case = lapcase.RawCase(xs=ax, ys=ax.copy(), zs=ax.copy(), DT_uniform=0.1, dt=0.2, n_steps=1, tol=1e-14,
                               T0=300.0, patches=ins, Su=Su, Sp=Sp)
        T, _ = oracle.advance(case)
        expect = (300.0 + 0.2 * Su) / (1.0 - 0.2 * Sp)
        assert rel(T, np.full(case.n_cells, expect)) < 1e-13


def test_insulated_box_energy_balance_with_sources():
    base = lapcase.random_small_case(12, nx=5, ny=4, nz=3, permute=False, patch_types=[lapcase.ZERO_GRADIENT] * 6)
    rng = np.random.default_rng(1)
    Su = rng.uniform(-5, 5, base.n_cells)
    Sp = -rng.uniform(0, 1, base.n_cells)
    case = base.with_(Su=Su, Sp=Sp, n_steps=1, tol=1e-14)
    m = oracle.mesh_of(case)
    T0 = oracle.initial_field(case)
    T1, _ = oracle.advance(case, mesh=m)
    lhs = np.dot(m.V, T1 - T0) / case.dt
    rhs = np.dot(m.V, Su + Sp * T1)
    assert abs(lhs - rhs) < 1e-10 * np.dot(m.V, np.abs(Su) + np.abs(Sp * T1))


def test_heat_source_raises_the_steady_profile():
    ax = lapcase.uniform_axis(10)
    case = lapcase.RawCase(xs=ax, ys=lapcase.uniform_axis(1), zs=lapcase.uniform_axis(1), DT_uniform=1.0,
                           dt=1e9, n_steps=2, tol=1e-14, T0=300.0, Su=400.0)
    T, _ = oracle.advance(case)
    cx = 0.5 * (ax[1:] + ax[:-1])
    linear = 373.0 - 100.0 * cx
    assert np.all(T > linear)
    # 1D: T'' = -Su / DT, T(0) = 373, T(1) = 273 -> T = linear + Su/2 x (1 - x) at the centres,
    # which the two-point flux reproduces at interior cells up to the half-cell boundary terms
    exact = linear + 200.0 * cx * (1 - cx)
    assert rel(T, exact) < 2e-2
