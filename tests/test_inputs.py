"""The seeded synthetic inputs (CPU): each workload generator follows the recipe stated for
it (sizes, grading, relabelling, diffusivity ranges, boundary conditions, batch and serving
distributions), and every generator is reproducible from its seed."""
import math

import numpy as np
import pytest

import lapcase


def test_plain_box_recipe():
    c = lapcase.plain_box(20)
    assert (c.nx, c.ny, c.nz) == (20, 20, 20)
    assert c.n_cells == 8000 and c.n_internal_faces == 22800 and c.n_boundary_faces == 2400
    assert c.DT_uniform == 4e-5 and c.dt == 0.005 and c.n_steps == 20 and c.tol == 1e-6 and c.rel_tol == 0.0
    assert c.patches[0] == (lapcase.FIXED_VALUE, 373.0) and c.patches[1] == (lapcase.FIXED_VALUE, 273.0)
    assert all(p[0] == lapcase.ZERO_GRADIENT for p in c.patches[2:])
    assert np.all(c.T0_natural() == 273.0)
    assert c.perm is None


def test_graded_axis_grows_by_the_ratio_per_cell():
    xs = lapcase.graded_axis(200, 1.02)
    h = np.diff(xs)
    assert xs[0] == 0.0 and xs[-1] == 1.0
    np.testing.assert_allclose(h[1:] / h[:-1], 1.02, rtol=1e-12)
    assert h[0] == pytest.approx(3.885e-4, rel=1e-3)
    assert h[-1] / h[0] == pytest.approx(1.02 ** 199, rel=1e-9)  # ratio ~51.5 end to end


def test_graded_box_recipe():
    c = lapcase.graded_box(200)
    assert c.n_cells == 8_000_000 and c.n_internal_faces == 23_880_000 and c.n_boundary_faces == 240_000
    np.testing.assert_allclose(np.diff(c.ys), 1 / 200, rtol=1e-12)
    np.testing.assert_allclose(np.diff(c.zs), 1 / 200, rtol=1e-12)
    assert c.DT_uniform == 4e-5 and c.dt == 0.005 and c.n_steps == 100 and c.tol == 1e-6


def test_permuted_box_recipe():
    c = lapcase.permuted_box(100)
    assert c.n_cells == 1_000_000 and c.dt == 0.01 and c.n_steps == 50 and c.tol == 1e-8
    assert np.array_equal(np.sort(c.perm), np.arange(c.n_cells))  # a relabelling
    assert np.mean(c.perm != np.arange(c.n_cells)) > 0.99
    # one value per geometric face, boundary faces included, log-uniform in [1e-6, 1e-4]
    assert c.DTx.shape == (100, 100, 101) and c.DTy.shape == (100, 101, 100) and c.DTz.shape == (101, 100, 100)
    logs = np.log10(np.concatenate([c.DTx.ravel(), c.DTy.ravel(), c.DTz.ravel()]))
    assert logs.min() >= -6.0 and logs.max() <= -4.0
    assert np.mean(logs) == pytest.approx(-5.0, abs=0.01)  # uniform in the exponent
    assert np.std(logs) == pytest.approx(2 / math.sqrt(12), rel=0.01)
    again = lapcase.permuted_box(100)
    assert np.array_equal(c.perm, again.perm) and np.array_equal(c.DTx, again.DTx)


def test_batch_cases_recipe():
    cases = lapcase.batch_cases(512, seed=3)
    n = np.array([c.nx for c in cases])
    assert len(cases) == 512 and n.min() >= 16 and n.max() <= 96
    assert all(c.nx == c.ny == c.nz for c in cases)
    assert np.mean(np.log(n)) == pytest.approx((math.log(16) + math.log(96)) / 2, abs=0.05)
    DT = np.array([c.DT_uniform for c in cases])
    dt = np.array([c.dt for c in cases])
    assert DT.min() >= 1e-6 and DT.max() <= 1e-4 and dt.min() >= 1e-3 and dt.max() <= 1e-1
    for c in cases:
        Ta, Tb = c.patches[0][1], c.patches[1][1]
        assert 250.0 <= Ta <= 400.0 and 250.0 <= Tb <= 400.0 and c.T0 == Tb
        assert c.n_steps == 10 and c.tol == 1e-6
    assert sum(c.n_cells for c in cases) == pytest.approx(85.8e6, rel=0.01)
    assert [c.nx for c in lapcase.batch_cases(512, seed=3)] == list(n)


def test_serving_stream_recipe():
    reqs = lapcase.serving_stream(2000, seed=4)
    t = np.array([r.arrival_s for r in reqs])
    gaps = np.diff(np.concatenate(([0.0], t)))
    assert np.all(gaps > 0)
    assert np.mean(gaps) == pytest.approx(1 / 200, rel=0.05)  # Poisson, 200 per second
    assert np.std(gaps) == pytest.approx(np.mean(gaps), rel=0.1)  # exponential gaps
    n = np.array([r.case.nx for r in reqs])
    steps = np.array([r.case.n_steps for r in reqs])
    assert n.min() >= 32 and n.max() <= 160 and steps.min() >= 1 and steps.max() <= 50
    mixed = np.mean([r.case.precision == lapcase.MIXED for r in reqs])
    assert mixed == pytest.approx(0.5, abs=0.05)
