"""Pins of the oracle's general-hexahedron path (CPU only): geometry, Gauss gradient,
correctBoundaryConditions and the corrected laplacian with non-orthogonal correctors.

What fixes each function (independently of the oracle's own code):
  * geometry: closed forms on rectilinear boxes; the transformation rules of volume,
    centroid and area vector under an affine map; closed cells (zero net area vector);
  * Gauss linear gradient: exact for linear fields when faces are planar and face centres
    lie on the segment between cell centres (rectilinear and affine-mapped uniform boxes);
    zero for a constant field;
  * correctBoundaryConditions: normal component = patch snGrad, tangential part = the cell's;
  * corrected laplacian: per-face flux of a linear field equals DT Sf.grad T exactly; the
    rectilinear limit equals the orthogonal path; the corrector fixed point satisfies the
    cell-by-cell balance recomputed here in numpy; energy is conserved with insulated
    boundaries; the correction brings a perturbed-mesh steady state closer to the exact one.
"""
import numpy as np
import pytest

import lapcase
import oracle


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def graded_case(nx=4, ny=3, nz=5, seed=0):
    return lapcase.random_small_case(seed, nx=nx, ny=ny, nz=nz, permute=False, face_dt=False)


def as_hex(case):
    return case.with_(points=lapcase.box_points(case.xs, case.ys, case.zs), n_nonorth_corr=0)


def test_rectilinear_box_geometry_matches_closed_forms():
    case = graded_case()
    m = oracle.hex_mesh(as_hex(case))
    b = oracle.box_mesh(case)
    assert rel(m.V, b.V) < 1e-13
    assert rel(m.magSf, b.magSf) < 1e-13
    assert rel(m.delta, b.delta) < 1e-13          # nonOrthDeltaCoeffs = 1/|d| when n || d
    assert rel(m.bmagSf, b.bmagSf) < 1e-13
    assert rel(m.bdelta, b.bdelta) < 1e-13
    assert np.max(np.abs(m.corr)) < 1e-13         # no non-orthogonality
    # cell centres at the midpoints of the vertex planes
    nx, ny, nz = case.nx, case.ny, case.nz
    cx = 0.5 * (case.xs[1:] + case.xs[:-1])
    cy = 0.5 * (case.ys[1:] + case.ys[:-1])
    cz = 0.5 * (case.zs[1:] + case.zs[:-1])
    Z, Y, X = np.meshgrid(cz, cy, cx, indexing="ij")
    assert rel(m.C, np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)) < 1e-13
    # weights: the owner weight is the neighbour's share of the centre distance
    d_own = np.abs(np.einsum("fi,fi->f", m.Sf, m.Cf - m.C[m.owner])) / m.magSf
    d_nei = np.abs(np.einsum("fi,fi->f", m.Sf, m.C[m.neighbour] - m.Cf)) / m.magSf
    assert rel(m.w, d_nei / (d_own + d_nei)) < 1e-13


def test_affine_map_transforms_geometry():
    case = graded_case(3, 4, 2, seed=3)
    M = np.array([[1.2, 0.3, -0.1], [0.05, 0.9, 0.2], [0.1, -0.2, 1.1]])
    t = np.array([0.3, -1.0, 2.0])
    base = oracle.hex_mesh(as_hex(case))
    m = oracle.hex_mesh(lapcase.mapped_box(case, M, t, n_nonorth_corr=0))
    det = np.linalg.det(M)
    cof = det * np.linalg.inv(M).T
    assert rel(m.V, abs(det) * base.V) < 1e-12
    assert rel(m.C, base.C @ M.T + t) < 1e-12
    assert rel(m.Cf, base.Cf @ M.T + t) < 1e-12
    assert rel(m.Sf, base.Sf @ cof.T) < 1e-12
    assert rel(m.bSf, base.bSf @ cof.T) < 1e-12
    assert abs(m.V.sum() - abs(det)) < 1e-12
    assert np.max(np.abs(m.corr)) > 1e-3          # genuinely non-orthogonal


@pytest.mark.parametrize("amp", [0.0, 0.2, 0.35])
def test_cells_are_closed(amp):
    case = lapcase.perturbed_box(graded_case(4, 4, 4, seed=5), amp=amp)
    m = oracle.hex_mesh(case)
    net = np.zeros((m.n_cells, 3))
    np.add.at(net, m.owner, m.Sf)
    np.add.at(net, m.neighbour, -m.Sf)
    np.add.at(net, m.bcell, m.bSf)
    scale = np.max(np.abs(m.Sf))
    assert np.max(np.abs(net)) < 1e-13 * scale
    assert np.all(m.V > 0) and abs(m.V.sum() - 1.0) < 1e-12  # boundary vertices stay on the unit cube


def linear_field(m, g, a=3.0):
    T = a + m.C @ g
    Tb = a + m.bCf @ g
    return T, Tb


@pytest.mark.parametrize("mapped", [False, True])
def test_gauss_gradient_is_exact_for_linear_fields(mapped):
    ax = lapcase.uniform_axis(5)
    case = lapcase.RawCase(xs=ax, ys=lapcase.uniform_axis(4), zs=lapcase.uniform_axis(3), DT_uniform=1.0)
    if mapped:
        case = lapcase.mapped_box(case, [[1.0, 0.4, 0.2], [0.1, 1.0, -0.3], [0.0, 0.2, 0.8]], n_nonorth_corr=0)
    else:
        case = as_hex(case.with_(xs=lapcase.graded_axis(5, 1.3)))
    m = oracle.hex_mesh(case)
    g = np.array([2.0, -1.5, 0.75])
    T, Tb = linear_field(m, g)
    G = oracle.gauss_grad(m, T, Tb)
    assert rel(G, np.tile(g, (m.n_cells, 1))) < 1e-12


def test_gauss_gradient_of_a_constant_vanishes():
    case = lapcase.perturbed_box(graded_case(5, 4, 3, seed=7), amp=0.3)
    m = oracle.hex_mesh(case)
    G = oracle.gauss_grad(m, np.full(m.n_cells, 300.0), np.full(m.n_bfaces, 300.0))
    h = np.min(m.V) ** (1 / 3)
    assert np.max(np.abs(G)) < 1e-10 * 300.0 / h


def test_boundary_gradient_normal_component_is_the_patch_sngrad():
    case = lapcase.perturbed_box(lapcase.random_small_case(2, permute=False, face_dt=False), amp=0.25)
    m = oracle.hex_mesh(case)
    T = oracle.initial_field(case)
    G, Gb = oracle.grad(case, m, T)
    btype, bvalue = oracle.boundary_types_values(case, m)
    n = m.bSf / np.linalg.norm(m.bSf, axis=1)[:, None]
    sn = np.where(btype == lapcase.FIXED_VALUE, (bvalue - T[m.bcell]) * m.bdelta, 0.0)
    assert rel(np.einsum("bi,bi->b", n, Gb), sn) < 1e-12
    Gc = G[m.bcell]
    tang_b = Gb - np.einsum("bi,bi->b", n, Gb)[:, None] * n
    tang_c = Gc - np.einsum("bi,bi->b", n, Gc)[:, None] * n
    assert rel(tang_b, tang_c) < 1e-12


def test_corrected_face_flux_of_a_linear_field_is_exact():
    ax = lapcase.uniform_axis(4)
    case = lapcase.mapped_box(lapcase.RawCase(xs=ax, ys=ax.copy(), zs=ax.copy(), DT_uniform=1.0),
                              [[1.0, 0.5, 0.3], [0.0, 1.0, 0.4], [0.2, 0.0, 1.0]], n_nonorth_corr=0)
    m = oracle.hex_mesh(case)
    g = np.array([1.0, -2.0, 0.5])
    T, Tb = linear_field(m, g)
    G = oracle.gauss_grad(m, T, Tb)
    Gf = m.w[:, None] * (G[m.owner] - G[m.neighbour]) + G[m.neighbour]
    flux = m.magSf * (m.delta * (T[m.neighbour] - T[m.owner]) + np.einsum("fi,fi->f", m.corr, Gf))
    assert rel(flux, m.Sf @ g) < 1e-12
    # and the uncorrected (orthogonal-only) flux is not exact on this mesh
    assert rel(m.magSf * m.delta * (T[m.neighbour] - T[m.owner]), m.Sf @ g) > 1e-3


def test_rectilinear_limit_equals_the_orthogonal_path():
    case = lapcase.random_small_case(4, nx=4, ny=3, nz=5, permute=False, face_dt=True)
    T_box, st_box = oracle.advance(case)
    T_hex, st_hex = oracle.advance(as_hex(case).with_(n_nonorth_corr=1))
    assert rel(T_hex, T_box) < 1e-10
    # one corrector pass doubles the solves; with zero correction the second solve starts
    # converged or close to it
    assert all(h.iters >= b.iters for h, b in zip(st_hex, st_box))


def balance_residual(case, m, T, T_old):
    """V/dt (T - T_old) minus the sum of corrected face fluxes into each cell (numpy)."""
    btype, bvalue = oracle.boundary_types_values(case, m)
    G = oracle.gauss_grad(m, T, oracle.boundary_values(case, m, T))
    Gf = m.w[:, None] * (G[m.owner] - G[m.neighbour]) + G[m.neighbour]
    flux = m.DTf * m.magSf * (m.delta * (T[m.neighbour] - T[m.owner]) + np.einsum("fi,fi->f", m.corr, Gf))
    inflow = np.zeros(m.n_cells)
    np.add.at(inflow, m.owner, flux)
    np.add.at(inflow, m.neighbour, -flux)
    fv = btype == lapcase.FIXED_VALUE
    bflux = np.where(fv, m.DTb * m.bmagSf * m.bdelta * (bvalue - T[m.bcell]), 0.0)
    np.add.at(inflow, m.bcell, bflux)
    return m.V / case.dt * (T - T_old) - inflow, m.V / case.dt * np.abs(T - T_old) + np.abs(inflow)


def test_corrector_fixed_point_satisfies_the_cell_balance():
    base = lapcase.random_small_case(6, nx=4, ny=4, nz=3, permute=False, face_dt=True)
    case = lapcase.perturbed_box(base, amp=0.3).with_(n_nonorth_corr=25, tol=1e-14, n_steps=1)
    m = oracle.hex_mesh(case)
    T0 = oracle.initial_field(case)
    T1, st = oracle.advance(case, mesh=m)
    res, scale = balance_residual(case, m, T1, T0)
    assert np.max(np.abs(res)) < 1e-9 * np.max(scale)
    # a single pass leaves the correction lagged: its balance residual is much larger
    T1a, _ = oracle.advance(case.with_(n_nonorth_corr=0), mesh=m)
    res_a, _ = balance_residual(case, m, T1a, T0)
    assert np.max(np.abs(res_a)) > 1e3 * np.max(np.abs(res))


def test_insulated_box_conserves_energy_with_correction():
    base = lapcase.random_small_case(8, nx=4, ny=3, nz=4, permute=False, face_dt=True,
                                     patch_types=[lapcase.ZERO_GRADIENT] * 6)
    case = lapcase.perturbed_box(base, amp=0.3).with_(n_nonorth_corr=2, tol=1e-13, n_steps=4)
    m = oracle.hex_mesh(case)
    T0 = oracle.initial_field(case)
    T1, _ = oracle.advance(case, mesh=m)
    assert abs(np.dot(m.V, T1) - np.dot(m.V, T0)) < 1e-12 * np.dot(m.V, np.abs(T0))


def test_correction_reduces_the_steady_state_error_on_a_perturbed_mesh():
    n = 8
    ax = lapcase.uniform_axis(n)
    base = lapcase.RawCase(xs=ax, ys=ax.copy(), zs=ax.copy(), DT_uniform=1.0, dt=1e6, n_steps=3,
                           tol=1e-13, T0=300.0)   # x0 = 373 K, x1 = 273 K fixedValue, others insulated
    case = lapcase.perturbed_box(base, amp=0.3, seed=11)
    m = oracle.hex_mesh(case)
    exact = 373.0 - 100.0 * m.C[:, 0]
    T_corr, _ = oracle.advance(case.with_(n_nonorth_corr=4), mesh=m)
    m0 = oracle.hex_mesh(case)
    m0.corr = np.zeros_like(m0.corr)   # the same mesh without the explicit correction
    T_plain, _ = oracle.advance(case.with_(n_nonorth_corr=0), mesh=m0)
    err_corr = np.max(np.abs(T_corr - exact))
    err_plain = np.max(np.abs(T_plain - exact))
    assert err_corr < 0.5 * err_plain


def test_correction_vectors_are_tangential_to_the_faces():
    # the over-relaxed split Sf = |Sf| (d / (n.d) + k): the implicit part runs along d and
    # the explicit correction vector k lies in the face plane
    case = lapcase.perturbed_box(graded_case(4, 5, 3, seed=9), amp=0.3)
    m = oracle.hex_mesh(case)
    n = m.Sf / m.magSf[:, None]
    assert np.max(np.abs(np.einsum("fi,fi->f", m.corr, n))) < 1e-12
    assert np.max(np.linalg.norm(m.corr, axis=1)) > 1e-2
