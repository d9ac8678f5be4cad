"""Rounding bounds for the per-step solver statistics (normFactor and the initial residual).

Two implementations of one step -- the oracle and a CUDA form -- that start from the same
field assemble the same matrix (bitwise, on orthogonal meshes) but round the rest
differently: A x is a fused multiply-add chain on the GPU and separate products and sums in
the oracle; the row sum s_c of normFactor is V/dt + sum g_b on the GPU and diag + sum of
the off-diagonals in the oracle (equal in real arithmetic); the mean xRef and the global
sums are added in other orders. normFactor = sum_c (|A x_c - s_c xRef| + |b_c - s_c xRef|)
is ill-conditioned where T is nearly uniform: its terms are small differences of values of
order s_c T, so each per-cell rounding of order u |s_c T| -- and a shift of xRef, which
moves every term by s_c -- counts against a small total. The bound below adds these
contributions up from the oracle's state at the start of the step (section "Evaluation":
the PCG with the normFactor-scaled residual; the row-sum and mean readings of normFactor):

  per cell (u_c the unit roundoff of the form's per-cell arithmetic, W_c the cell's faces,
  M_c = |diag_c x_c| + sum_f |a_cf x_f|):
    e_Ax = (3 W_c + 4) u_c M_c            A x: W_c + 1 fused terms on one side, 2 W_c + 1
                                          roundings on the other, plus the field's own
                                          representation (df64: a triple-float rounded to FP64)
    e_b  = 8 (W_c + 3) u_c C_c            the explicit non-orthogonal correction (general
                                          meshes: gradient and flux weights built as operators
                                          on the GPU, face loops in the oracle; C_c the sum of
                                          its terms' magnitudes), else 0 (bitwise assembly)
    e_s  = (W_c + 3) u_c diag_c           the two row-sum formulas
    e_nf = e_Ax + e_b + 2 (e_s |xRef| + 3 u_c (|s_c xRef| + |A x_c| + |b_c|))
    e_r  = e_Ax + e_b + 2 u_c |r_c|
  the mean: |d xRef| <= |xRef_serial - xRef_exact| (the oracle's serial sum, evaluated
    exactly here) + gamma(depth_gpu, u_sum) mean|x| (the GPU's per-thread, block and team
    summation depth and the unit roundoff of its accumulator); normFactor moves by at most
    2 sum_c |s_c| |d xRef|
  the global sums (N positive terms, two orders): 2 gamma(N, u) times the sum
  so that
    |d nf| <= sum_c e_nf + 2 sum_c |s_c| |d xRef| + 2 gamma_N nf
    |d sum|r|| <= sum_c e_r + 2 gamma_N sum|r|
    |d init_res| / init_res <= |d sum|r|| / sum|r| + |d nf| / nf + 2 u
with gamma(n, u) = n u / (1 - n u). Every term is a worst case: a bar, not an estimate.
"""
from __future__ import annotations

import math
from typing import Optional, Tuple

import numpy as np

import oracle

U64 = 2.0 ** -53
UDF = 2.0 ** -47      # per operation of double-float (FP32 pair) arithmetic, with margin

# per-cell unit roundoff and per-thread accumulator unit roundoff of each form
FORMS = {"fp64": (U64, U64), "df64": (UDF, UDF), "mixed": (UDF, UDF)}


def gamma(n: float, u: float) -> float:
    return n * u / (1.0 - n * u)


def _abs_scatter(n, owner, neighbour, fo, fn, init):
    out = init.copy()
    np.add.at(out, owner, fo)
    np.add.at(out, neighbour, fn)
    return out


def _correction_magnitude(case, om, T) -> np.ndarray:
    """sum over the cell's faces of |DT_f| |S_f| |k_f| . (w |G_P| + (1 - w) |G_N|) with G the
    magnitudes of the Gauss-gradient terms, sum_f |S_f| (w |T_P| + (1 - w) |T_N|) / V_c (plus
    boundary faces): the size of the explicit correction's terms, not of its value."""
    N = om.n_cells
    aS = np.abs(om.Sf)
    Tf = om.w * np.abs(T[om.owner]) + (1.0 - om.w) * np.abs(T[om.neighbour])
    Gabs = np.zeros((N, 3))
    np.add.at(Gabs, om.owner, aS * Tf[:, None])
    np.add.at(Gabs, om.neighbour, aS * Tf[:, None])
    Tb = np.abs(oracle.boundary_values(case, om, T))
    np.add.at(Gabs, om.bcell, np.abs(om.bSf) * Tb[:, None])
    Gabs /= om.V[:, None]
    k = np.abs(om.corr)
    gam = np.abs(om.DTf) * om.magSf
    fl = gam * np.sum(k * (om.w[:, None] * Gabs[om.owner] + (1.0 - om.w[:, None]) * Gabs[om.neighbour]), axis=1)
    C = np.zeros(N)
    np.add.at(C, om.owner, fl)
    np.add.at(C, om.neighbour, fl)
    return C


def step_bounds(case, om, T: np.ndarray, form: str, launch: Tuple[int, int],
                nf: float, init_res: float) -> Tuple[float, float]:
    """Absolute bounds (normFactor, initial residual) on |GPU - oracle| for one step of
    `case` from the field T (by label), given the oracle's normFactor and initial residual
    of that step, for a CUDA form run with launch = (ctas, threads)."""
    u_c, u_sum = FORMS[form]
    N = om.n_cells
    T = np.asarray(T, dtype=np.float64)
    bt, bv = oracle.boundary_types_values(case, om)
    Su, Sp = oracle.source_arrays(case)
    d, up, b = oracle.assemble(om, bt, bv, case.dt, T, Su, Sp)
    M = _abs_scatter(N, om.owner, om.neighbour, np.abs(up * T[om.neighbour]), np.abs(up * T[om.owner]),
                     np.abs(d * T))
    Ax = _abs_scatter(N, om.owner, om.neighbour, up * T[om.neighbour], up * T[om.owner], d * T)
    s = _abs_scatter(N, om.owner, om.neighbour, up, up, d)
    nfaces = np.bincount(np.concatenate([om.owner, om.neighbour]), minlength=N).astype(np.float64)
    C = _correction_magnitude(case, om, T) if om.Sf is not None else np.zeros(N)
    r = np.abs(b - Ax) + C
    bb = np.abs(b) + C
    xb_exact = math.fsum(T) / N
    xb_serial = np.cumsum(T)[-1] / N  # the oracle's left-to-right sum
    ctas, threads = launch
    # per thread; the block (up to 4 xor levels in a warp, up to 8 partials per lane of warp 0,
    # a 5-level xor tree); the team (ranks per lane of the last arriver, a 5-level xor tree)
    depth = math.ceil(N / max(ctas * threads, 1)) + 17 + math.ceil(max(ctas, 1) / 32) + 5
    dxb = abs(xb_serial - xb_exact) + gamma(depth + 2, u_sum) * float(np.mean(np.abs(T)))
    e_ax = (3 * nfaces + 4) * u_c * M
    e_b = 8.0 * (nfaces + 3) * u_c * C
    e_s = (nfaces + 3) * u_c * d
    e_nf = e_ax + e_b + 2 * (e_s * abs(xb_exact) + 3 * u_c * (np.abs(s * xb_exact) + np.abs(Ax) + bb))
    e_r = e_ax + e_b + 2 * u_c * r
    sum_r = init_res * nf
    B_nf = float(np.sum(e_nf) + 2 * np.sum(np.abs(s)) * dxb + 2 * gamma(N, U64) * nf)
    B_r = float(np.sum(e_r) + 2 * gamma(N, U64) * sum_r)
    B_ir = init_res * ((B_r / sum_r if sum_r > 0 else 0.0) + B_nf / nf + 2 * U64) + (B_r / nf if sum_r == 0 else 0.0)
    return B_nf, B_ir


def check_step(case, om, T, form, launch, g: dict, o) -> Optional[str]:
    """None when the GPU statistics g of a step from T are within the bound of the oracle's
    o; otherwise a message with both differences and bounds."""
    B_nf, B_ir = step_bounds(case, om, T, form, launch, o.norm_factor, o.init_res)
    dnf = abs(g["norm_factor"] - o.norm_factor)
    dir_ = abs(g["init_res"] - o.init_res)
    if dnf <= B_nf and dir_ <= B_ir:
        return None
    return (f"normFactor {g['norm_factor']!r} vs {o.norm_factor!r} (diff {dnf:.3e}, bound {B_nf:.3e}); "
            f"init_res {g['init_res']!r} vs {o.init_res!r} (diff {dir_:.3e}, bound {B_ir:.3e})")


def relative_bounds(case, om, T, form, launch, o) -> Tuple[float, float]:
    """The bounds of step_bounds relative to the oracle's values (for reporting)."""
    B_nf, B_ir = step_bounds(case, om, T, form, launch, o.norm_factor, o.init_res)
    return B_nf / o.norm_factor, (B_ir / o.init_res if o.init_res > 0 else float("inf"))


def gpu_walk(case, precision: int, form: str, launch=None, n_steps: Optional[int] = None):
    """Steps a CUDA form of `case` one launch at a time (bitwise the same trajectory as one
    launch of all steps) and, for every step, runs the oracle's step from the GPU's own field
    at its start, so that only rounding separates the two. Returns (final GPU field, list of
    per-step records: GPU stats, oracle stats, |diff| / bound for normFactor and the initial
    residual, and the relative differences)."""
    from paper_2507_18268_gb300 import Solver

    om = oracle.mesh_of(case)
    n = case.n_steps if n_steps is None else n_steps
    out = []
    with Solver.from_case(case) as s:
        s.set_solver(case.tol, case.rel_tol, case.max_iter, case.min_iter, precision)
        if launch:
            s.set_launch(*launch)
        lc = s.launch()
        T = s.field()
        for _ in range(n):
            g = s.advance(1)[0]
            _, so = oracle.advance(case, n_steps=1, mesh=om, T=T)
            o = so[0]
            B_nf, B_ir = step_bounds(case, om, T, form, (lc[0], lc[1]), o.norm_factor, o.init_res)
            dnf = abs(g["norm_factor"] - o.norm_factor)
            dir_ = abs(g["init_res"] - o.init_res)
            out.append(dict(g=g, o=o, q_nf=dnf / B_nf, q_ir=(dir_ / B_ir if B_ir > 0 else (0.0 if dir_ == 0 else 1e300)),
                            rel_nf=dnf / o.norm_factor, rel_ir=(dir_ / o.init_res if o.init_res > 0 else dir_),
                            bound_rel_nf=B_nf / o.norm_factor))
            T = s.field()
    return T, out


def assert_walk(records, iters_equal: bool = True):
    """Every step within the rounding bound (and, for the FP64-class forms, the same PCG
    iteration count as the oracle's step from the same field)."""
    for k, rec in enumerate(records):
        assert rec["q_nf"] <= 1.0 and rec["q_ir"] <= 1.0, (k, rec)
        if iters_equal:
            assert rec["g"]["iters"] == rec["o"].iters, (k, rec)
