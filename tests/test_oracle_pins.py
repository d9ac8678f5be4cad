"""Pins of the CPU oracle to facts outside itself (no GPU needed).

Each test ties the oracle to mathematics the paper fixes (Eq. (1), the implicit TEqn of the
laplacianFoam listing, the LDU face addressing of section "OpenFOAM", PCG + diagonal
preconditioner of section "Evaluation"): a dense direct solve, closed-form steady and
transient solutions, exact matrix invariants, discrete conservation, relabelling
invariance, CG's finite termination and a hand-worked two-cell example.
"""
import json
import math
import os

import numpy as np
import pytest

import lapcase
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _assembled(case, T_old=None):
    mesh = oracle.box_mesh(case)
    btype, bvalue = oracle.boundary_types_values(case, mesh)
    T_old = oracle.initial_field(case) if T_old is None else T_old
    diag, upper, source = oracle.assemble(mesh, btype, bvalue, case.dt, T_old)
    return mesh, btype, bvalue, T_old, diag, upper, source


def _centres(v):
    v = np.asarray(v)
    return 0.5 * (v[:-1] + v[1:])


# ---------------------------------------------------------------------------------------
# Mesh addressing (section "OpenFOAM": owner/neighbour; upper-triangular face order)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1])
def test_mesh_addressing_brute_force(seed):
    case = lapcase.random_small_case(seed, nx=5, ny=3, nz=4)
    m = oracle.box_mesh(case)
    assert m.n_faces == case.n_internal_faces and m.n_bfaces == case.n_boundary_faces
    assert np.all(m.owner < m.neighbour)
    keys = m.owner.astype(np.int64) * m.n_cells + m.neighbour
    assert np.all(np.diff(keys) > 0), "faces not in strict (owner, neighbour) order"
    # brute force: the set of face-adjacent label pairs from the (i,j,k) lattice
    nx, ny, nz = case.nx, case.ny, case.nz
    perm = case.perm
    lab = lambda i, j, k: int(perm[i + nx * (j + ny * k)])
    pairs = set()
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for di, dj, dk in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
                    if i + di < nx and j + dj < ny and k + dk < nz:
                        a, b = lab(i, j, k), lab(i + di, j + dj, k + dk)
                        pairs.add((min(a, b), max(a, b)))
    assert pairs == set(zip(m.owner.tolist(), m.neighbour.tolist()))
    # every cell of a box has 6 faces (internal + boundary)
    deg = np.bincount(m.owner, minlength=m.n_cells) + np.bincount(m.neighbour, minlength=m.n_cells) \
        + np.bincount(m.bcell, minlength=m.n_cells)
    assert np.all(deg == 6)
    # the volumes tile the unit cube
    assert abs(m.V.sum() - 1.0) < 1e-14
    assert np.all(m.V > 0)


# ---------------------------------------------------------------------------------------
# Matrix invariants: symmetry, exact row sums, sign pattern, dominance
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_matrix_symmetry_and_row_sums(seed):
    case = lapcase.random_small_case(seed)
    mesh, btype, bvalue, T_old, diag, upper, source = _assembled(case)
    A = oracle.dense_matrix(mesh, diag, upper)
    assert np.array_equal(A, A.T)
    vdt = mesh.V / case.dt
    rows = A.sum(axis=1)
    fixed_cells = np.unique(mesh.bcell[btype == lapcase.FIXED_VALUE])
    interior = np.setdiff1d(np.arange(mesh.n_cells), fixed_cells)
    eps = np.finfo(float).eps
    # row sum = V/dt exactly (to rounding of the summation) away from fixedValue patches
    assert np.all(np.abs(rows[interior] - vdt[interior]) <= 8 * eps * diag[interior])
    # next to fixedValue patches the row sum exceeds V/dt (boundary conductance > 0)
    assert np.all(rows[fixed_cells] > vdt[fixed_cells])
    off = A - np.diag(np.diag(A))
    assert np.all(off <= 0.0)
    assert np.all(diag > 0)
    assert np.all(diag - np.abs(off).sum(axis=1) >= vdt * (1 - 1e-12))


def test_single_cell_reduces_to_boundary_conductances():
    # one unit cell, all six faces fixedValue at T_b: each face conducts DT*|S|/d = 0.3*1/0.5,
    # so one step from T0 gives (V/dt*T0 + 6*0.6*T_b) / (V/dt + 6*0.6) exactly.
    ax = np.array([0.0, 1.0])
    case = lapcase.RawCase(xs=ax, ys=ax, zs=ax, DT_uniform=0.3, dt=1e9,
                           patches=((lapcase.FIXED_VALUE, 300.0),) * 6, T0=0.0, tol=1e-14)
    T, st = oracle.advance(case, n_steps=1)
    assert math.isclose(T[0], 3.6 * 300.0 / (3.6 + 1e-9), rel_tol=1e-14)
    mesh, btype, bvalue, _, diag, upper, source = _assembled(case)
    assert mesh.n_faces == 0 and mesh.n_cells == 1
    # six faces with DT*|S|/d = 0.3*1/0.5
    assert math.isclose(diag[0] - 1.0 / 1e9, 6 * 0.3 * 2.0, rel_tol=1e-14)


# ---------------------------------------------------------------------------------------
# PCG against a dense direct solve (4^3 meshes)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("variant", ["uniform", "face_dt", "permuted", "graded", "all"])
def test_pcg_matches_dense_lu(variant):
    kw = dict(permute=False, face_dt=False, graded=False)
    if variant == "face_dt":
        kw["face_dt"] = True
    elif variant == "permuted":
        kw["permute"] = True
    elif variant == "graded":
        kw["graded"] = True
    elif variant == "all":
        kw = dict(permute=True, face_dt=True, graded=True)
    case = lapcase.random_small_case(11, **kw)
    mesh, btype, bvalue, T_old, diag, upper, source = _assembled(case)
    A = oracle.dense_matrix(mesh, diag, upper)
    x_lu = np.linalg.solve(A, source)
    x, st, _ = oracle.pcg(mesh.owner, mesh.neighbour, diag, upper, source, T_old, tol=1e-14,
                          max_iter=1000)
    assert st.converged
    assert np.max(np.abs(x - x_lu) / np.abs(x_lu)) <= 1e-12


def test_pcg_search_directions_are_A_conjugate():
    case = lapcase.random_small_case(5)
    mesh, btype, bvalue, T_old, diag, upper, source = _assembled(case)
    A = oracle.dense_matrix(mesh, diag, upper)
    x, st, tr = oracle.pcg(mesh.owner, mesh.neighbour, diag, upper, source, T_old, tol=1e-14,
                           trace=6)
    k = min(st.iters, 6)
    assert k >= 3
    P = tr[:k]
    G = P @ A @ P.T
    d = np.sqrt(np.diag(G))
    C = G / np.outer(d, d)
    assert np.max(np.abs(C - np.eye(k))) < 1e-8


def test_pcg_diagonal_system_one_iteration():
    # DT = 0 removes all coupling: A = diag, Jacobi-PCG is exact after one iteration
    rng = np.random.default_rng(7)
    N = 50
    diag = rng.uniform(1, 10, N)
    b = rng.uniform(-5, 5, N)
    x, st, _ = oracle.pcg(np.zeros(0, np.int32), np.zeros(0, np.int32), diag, np.zeros(0), b,
                          np.zeros(N), tol=1e-14)
    assert st.iters == 1
    assert np.max(np.abs(x - b / diag) / np.abs(b / diag)) < 4e-16 * 4


def test_pcg_zero_initial_residual_takes_no_iteration():
    # DT = 0: A = V/dt I and b = V/dt T_old, so r = 0 exactly and the convergence test
    # before the first iteration stops the solve with 0 iterations.
    case = lapcase.plain_box(4).with_(DT_uniform=0.0, T0=np.linspace(250, 300, 64))
    T, st = oracle.advance(case, n_steps=1)
    assert st[0].iters == 0 and st[0].converged and st[0].init_res == 0.0
    assert np.array_equal(T, np.linspace(250, 300, 64))


# ---------------------------------------------------------------------------------------
# Hand-worked two-cell example (tests/golden/two_cell.json)
# ---------------------------------------------------------------------------------------

def test_two_cell_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "two_cell.json")))
    case = lapcase.RawCase(xs=np.array([0.0, 0.5, 1.0]), ys=np.array([0.0, 1.0]),
                           zs=np.array([0.0, 1.0]), DT_uniform=g["DT"], dt=g["dt"],
                           patches=((lapcase.FIXED_VALUE, g["patch_x0"]),
                                    (lapcase.FIXED_VALUE, g["patch_x1"])) +
                                   ((lapcase.ZERO_GRADIENT, 0.0),) * 4,
                           T0=np.array(g["T_old"]), tol=1e-13)
    mesh, btype, bvalue, T_old, diag, upper, source = _assembled(case)
    np.testing.assert_allclose(diag, g["diag"], rtol=1e-15)
    np.testing.assert_allclose(upper, g["upper"], rtol=1e-15)
    np.testing.assert_allclose(source, g["source"], rtol=1e-15)
    x, st, _ = oracle.pcg(mesh.owner, mesh.neighbour, diag, upper, source, T_old, tol=1e-13)
    assert math.isclose(st.norm_factor, g["norm_factor"], rel_tol=1e-15)
    assert math.isclose(st.init_res, g["init_res"], rel_tol=1e-14)
    assert st.iters == g["iterations"]
    np.testing.assert_allclose(x, g["solution"], rtol=1e-13)


def test_two_cell_unequal_volumes_pins_the_plain_mean():
    # Unequal cell volumes, diagonals and row sums: normFactor uses the plain cell mean of the
    # initial guess and the row sums of the assembled matrix (63/2). Weighted means, or the
    # diagonal in place of the row sum, give other values (listed in the golden). One
    # iteration is pinned too (x, and the recurrence residual), worked by hand.
    g = json.load(open(os.path.join(GOLDEN, "two_cell_unequal.json")))
    case = lapcase.RawCase(xs=np.array([0.0, 0.5, 2.0]), ys=np.array([0.0, 1.0]),
                           zs=np.array([0.0, 1.0]), DT_uniform=g["DT"], dt=g["dt"],
                           patches=((lapcase.FIXED_VALUE, g["patch_x0"]),) +
                                   ((lapcase.ZERO_GRADIENT, 0.0),) * 5,
                           T0=np.array(g["T_old"]), tol=1e-13)
    mesh, btype, bvalue, T_old, diag, upper, source = _assembled(case)
    np.testing.assert_allclose(mesh.V, g["V"], rtol=1e-15)
    np.testing.assert_allclose(diag, g["diag"], rtol=1e-15)
    np.testing.assert_allclose(upper, g["upper"], rtol=1e-15)
    np.testing.assert_allclose(source, g["source"], rtol=1e-15)
    x, st, _ = oracle.pcg(mesh.owner, mesh.neighbour, diag, upper, source, T_old, tol=1e-13)
    assert math.isclose(st.norm_factor, g["norm_factor"], rel_tol=1e-15)
    for wrong in g["norm_factor_wrong"].values():
        assert not math.isclose(st.norm_factor, wrong, rel_tol=1e-3)
    assert math.isclose(st.init_res, g["init_res"], rel_tol=1e-15)
    assert st.iters == g["iterations"]
    np.testing.assert_allclose(x, g["solution"], rtol=1e-14)
    x1, st1, _ = oracle.pcg(mesh.owner, mesh.neighbour, diag, upper, source, T_old, tol=1e-13, max_iter=1)
    assert st1.iters == 1 and not st1.converged
    np.testing.assert_allclose(x1, g["x_after_1"], rtol=1e-14)
    assert math.isclose(st1.final_res, g["res_after_1"], rel_tol=1e-14)
    # the same system through the whole step (assembly + solve) of the advance entry point
    T, sts = oracle.advance(case, n_steps=1)
    np.testing.assert_allclose(T, g["solution"], rtol=1e-14)
    assert math.isclose(sts[0].norm_factor, g["norm_factor"], rel_tol=1e-15)


def test_convergence_test_is_strict_at_a_tie():
    # res == tol exactly must not count as converged (strict '<'), before the first iteration
    # and after one: with '<=' the solve would stop one iteration earlier.
    g = json.load(open(os.path.join(GOLDEN, "two_cell_unequal.json")))
    case = lapcase.RawCase(xs=np.array([0.0, 0.5, 2.0]), ys=np.array([0.0, 1.0]),
                           zs=np.array([0.0, 1.0]), DT_uniform=g["DT"], dt=g["dt"],
                           patches=((lapcase.FIXED_VALUE, g["patch_x0"]),) +
                                   ((lapcase.ZERO_GRADIENT, 0.0),) * 5,
                           T0=np.array(g["T_old"]))
    mesh, btype, bvalue, T_old, diag, upper, source = _assembled(case)
    args = (mesh.owner, mesh.neighbour, diag, upper, source, T_old)
    _, st0, _ = oracle.pcg(*args, tol=1e-13, max_iter=1)
    assert math.isclose(st0.init_res, 19.0 / 21.0, rel_tol=1e-15)
    _, st, _ = oracle.pcg(*args, tol=st0.init_res)           # tie before the first iteration
    assert st.iters >= 1
    _, st, _ = oracle.pcg(*args, tol=math.nextafter(st0.init_res, 1.0))
    assert st.iters == 0 and st.converged
    st1 = st0
    _, st, _ = oracle.pcg(*args, tol=st1.final_res)          # tie after the first iteration
    assert st.iters == 2 and st.final_res < st1.final_res
    _, st, _ = oracle.pcg(*args, tol=math.nextafter(st1.final_res, 1.0))
    assert st.iters == 1 and st.converged
    # relTol ties: res == relTol * initRes is not converged either
    rel = st1.final_res / st0.init_res
    if rel * st0.init_res == st1.final_res:
        _, st, _ = oracle.pcg(*args, tol=0.0, rel_tol=rel)
        assert st.iters == 2


# ---------------------------------------------------------------------------------------
# Closed forms: linear steady state and the 1D Fourier-series transient
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("axis", [0, 1, 2])
def test_linear_profile_is_steady(axis):
    # T = 373 - 100*x_a at cell centres with fixedValue 373/273 on the two faces normal to
    # axis a is an exact steady state of the discrete operator, on graded meshes too.
    n = [3, 4, 2]
    n[axis] = 7
    axes = [lapcase.uniform_axis(k) for k in n]
    axes[axis] = lapcase.graded_axis(n[axis], 1.3)
    patches = [(lapcase.ZERO_GRADIENT, 0.0)] * 6
    patches[2 * axis] = (lapcase.FIXED_VALUE, 373.0)
    patches[2 * axis + 1] = (lapcase.FIXED_VALUE, 273.0)
    c = [_centres(a) for a in axes]
    I, J, K = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    coord = [c[0][I], c[1][J], c[2][K]][axis]
    # natural order: i fastest
    T_lin = (373.0 - 100.0 * coord).transpose(2, 1, 0).reshape(-1)
    for dt in (1e-3, 1.0, 1e6):
        case = lapcase.RawCase(xs=axes[0], ys=axes[1], zs=axes[2], DT_uniform=0.7, dt=dt,
                               patches=tuple(patches), T0=T_lin, tol=1e-15, max_iter=200)
        T, st = oracle.advance(case, n_steps=2)
        assert np.max(np.abs(T - T_lin)) < 1e-9
    # and from a cold start a huge step lands on it
    case = lapcase.RawCase(xs=axes[0], ys=axes[1], zs=axes[2], DT_uniform=0.7, dt=1e12,
                           patches=tuple(patches), T0=273.0, tol=1e-15, max_iter=500)
    T, st = oracle.advance(case, n_steps=1)
    assert np.max(np.abs(T - T_lin)) < 1e-8


def _fourier(x, t, DT, nterms=4000):
    n = np.arange(1, nterms + 1)[:, None]
    return 373.0 - 100.0 * x - np.sum(200.0 / (n * np.pi) * np.sin(n * np.pi * x)
                                      * np.exp(-(n * np.pi) ** 2 * DT * t), axis=0)


def test_fourier_transient_second_order():
    # T(0)=373, T(1)=273, T(x,0)=273, DT=1e-2, t=5 s: the 1D series solution; error must
    # fall ~4x per halving of h with dt ~ h^2 (implicit Euler + central differences).
    DT, t_end = 1e-2, 5.0
    errs = []
    for nx, steps in ((10, 25), (20, 100), (40, 400)):
        xs = lapcase.uniform_axis(nx)
        three = lapcase.uniform_axis(3)
        case = lapcase.RawCase(xs=xs, ys=three, zs=three, DT_uniform=DT, dt=t_end / steps, n_steps=steps,
                               T0=273.0, tol=1e-13, max_iter=500)
        T, st = oracle.advance(case)
        T3 = T.reshape(3, 3, nx)
        # 1D reduction: all y/z slices identical
        assert np.max(np.abs(T3 - T3[0, 0])) < 1e-9
        errs.append(np.max(np.abs(T3[0, 0] - _fourier(_centres(xs), t_end, DT))))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0, errs
    assert errs[2] < 0.1


# ---------------------------------------------------------------------------------------
# Discrete conservation and relabelling invariance
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 3, 8])
def test_energy_conserved_with_insulated_walls(seed):
    case = lapcase.random_small_case(seed, nx=6, ny=5, nz=4,
                                     patch_types=[lapcase.ZERO_GRADIENT] * 6).with_(tol=1e-9)
    mesh = oracle.box_mesh(case)
    T0 = oracle.initial_field(case)
    T, st = oracle.advance(case, n_steps=1, mesh=mesh)
    # sum V (T1 - T0) = -dt * sum r, |sum r| <= finalRes * normFactor
    lhs = abs(np.sum(mesh.V * (T - T0)))
    bound = case.dt * st[0].final_res * st[0].norm_factor
    assert st[0].iters > 0
    assert lhs <= bound * (1 + 1e-9) + 1e-12 * np.sum(mesh.V * T0)


def test_energy_balance_with_fixed_value_walls():
    # Sum over cells of the assembled equations: V/dt (T1-T0) = sum_b g_b (T_b - T_P) - r,
    # with g_b read off as the excess of each boundary row over V/dt.
    case = lapcase.random_small_case(4, nx=5, ny=4, nz=3, face_dt=True,
                                     patch_types=[0, 0, 1, 1, 0, 1]).with_(tol=1e-10)
    mesh, btype, bvalue, T_old, diag, upper, source = _assembled(case)
    A = oracle.dense_matrix(mesh, diag, upper)
    x, st, _ = oracle.pcg(mesh.owner, mesh.neighbour, diag, upper, source, T_old, tol=1e-10)
    gsum = A.sum(axis=1) - mesh.V / case.dt            # total boundary conductance per cell
    inflow = np.sum(source - mesh.V / case.dt * T_old) - np.sum(gsum * x)
    storage = np.sum(mesh.V * (x - T_old)) / case.dt
    assert abs(storage - inflow) <= st.final_res * st.norm_factor * (1 + 1e-9) + 1e-9 * abs(inflow)


def test_permutation_invariance():
    nat = lapcase.permuted_box(10, n_steps=5)
    perm = nat.perm
    Tp, sp = oracle.advance(nat)
    Tn, sn = oracle.advance(nat.with_(perm=None))
    # label perm[c] in the permuted case is natural cell c
    assert np.max(np.abs(Tp[perm] - Tn) / Tn) < 1e-12
    for a, b in zip(sp, sn):
        assert abs(a.iters - b.iters) <= 1


def test_boundary_values_follow_patch_types():
    case = lapcase.random_small_case(2, patch_types=[0, 1, 0, 1, 0, 1])
    mesh = oracle.box_mesh(case)
    T = np.arange(mesh.n_cells, dtype=float)
    Tb = oracle.boundary_values(case, mesh, T)
    for b in range(mesh.n_bfaces):
        t, v = case.patches[mesh.bpatch[b]]
        assert Tb[b] == (v if t == lapcase.FIXED_VALUE else T[mesh.bcell[b]])


def test_stopping_rules():
    # relTol: stop at the first iteration with res < relTol * initRes (and not before);
    # minIter forces iterations; maxIter caps them without reporting convergence.
    case = lapcase.random_small_case(9, nx=6, ny=5, nz=4)
    mesh, btype, bvalue, T_old, diag, upper, source = _assembled(case)
    args = (mesh.owner, mesh.neighbour, diag, upper, source, T_old)
    x, st, _ = oracle.pcg(*args, tol=0.0, rel_tol=0.05)
    assert st.converged and st.final_res < 0.05 * st.init_res and st.iters >= 2
    x2, st2, _ = oracle.pcg(*args, tol=0.0, rel_tol=0.05, max_iter=st.iters - 1)
    assert not st2.converged and st2.final_res >= 0.05 * st2.init_res
    assert st2.iters == st.iters - 1
    x3, st3, _ = oracle.pcg(*args, tol=1e30, min_iter=3)
    assert st3.iters == 3 and st3.converged
    x4, st4, _ = oracle.pcg(*args, tol=1e30)
    assert st4.iters == 0
