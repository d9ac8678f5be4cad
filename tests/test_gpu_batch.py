"""Batched form against the same cases run alone and against the oracle (GPU required).

A case in a batch runs the same arithmetic as alone, with a team size set by the batch's
launch shape; FP64 results must match the single-case path and the oracle to 1e-10 with
identical iteration counts, mixed-precision results the FP64 oracle to 1e-5.
"""
import numpy as np
import pytest

import lapcase
import oracle
from paper_2507_18268_gb300 import Solver, box_mesh
from paper_2507_18268_gb300 import binding as B
from paper_2507_18268_gb300.batch import Batch

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def small_batch_cases(seed=7, n_cases=14, n_steps=4):
    cases = lapcase.batch_cases(n_cases=n_cases, seed=seed, n_min=5, n_max=28, n_steps=n_steps)
    out = []
    for i, c in enumerate(cases):
        if i % 3 == 1:
            c = c.with_(precision=lapcase.MIXED)
        if i % 4 == 2:  # a relabelled case with per-face DT
            pc = lapcase.permuted_box(c.nx, seed_perm=seed + i, seed_dt=seed + 100 + i, n_steps=n_steps)
            c = pc.with_(precision=c.precision, tol=1e-8)
        out.append(c)
    return out


def alone(case, n_steps):
    with Solver.from_case(case) as s:
        st = s.advance(n_steps)
        return s.field(), st


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("threads,cpt", [(512, (4, 8, 16)), (256, (1, 1, 1))])
def test_batch_matches_alone_and_oracle(use_graph, threads, cpt):
    n_steps = 4
    cases = small_batch_cases(n_steps=n_steps)
    with Batch() as bt:
        ids = [bt.add_case(c) for c in cases]
        bt.set_launch(threads, cpt)
        assert bt.advance(n_steps, use_graph=use_graph) == B.LFM_OK
        for cid, c in zip(ids, cases):
            T = bt.field(cid)
            st = bt.stats(cid, n_steps)
            To, so = oracle.advance(c, n_steps=n_steps)
            if c.precision == lapcase.FP64:
                Ta, sa = alone(c, n_steps)
                assert [x["iters"] for x in st] == [x["iters"] for x in sa] == [x.iters for x in so]
                assert relerr(T, Ta) <= 1e-10
                assert relerr(T, To) <= 1e-10
            else:
                assert relerr(T, To) <= 1e-5
                assert all(x["converged"] for x in st)


@pytest.mark.parametrize("use_graph", [False, True])
def test_capped_advance_runs_each_case_its_own_step_count(use_graph):
    # a capped advance of k steps: case i runs min(k, cap_i) steps and then idles, bitwise as
    # if its advance had that many steps; the bulk results report steps and iterations
    n_steps = 5
    cases = small_batch_cases(seed=13, n_cases=9, n_steps=n_steps)
    caps_list = [0, 1, 2, 5, 3, 9, 1, 4, 2]
    # reference: each case in a batch of its own, uncapped, for min(cap, k) steps
    T_ref = {}
    for cid, (c, cap) in enumerate(zip(cases, caps_list)):
        run = min(cap, n_steps)
        with Batch() as one:
            i = one.add_case(c)
            one.set_launch(256, (2, 2, 2))
            if run:
                assert one.advance(run, use_graph=use_graph) == B.LFM_OK
            T_ref[cid] = (one.field(i), one.stats(i, run) if run else [])
    with Batch() as bt:
        ids = [bt.add_case(c) for c in cases]
        bt.set_launch(256, (2, 2, 2))
        caps = dict(zip(ids, caps_list))
        B.lfm_batch_advance_capped_async(bt.handle, n_steps, [caps[i] for i in range(len(ids))], use_graph)
        assert bt.finish() == B.LFM_OK
        res = bt.results()
        for k, cid in enumerate(ids):
            run = min(caps_list[k], n_steps)
            T1, st1 = T_ref[k]
            st, steps, iters = res[cid]
            assert st == B.LFM_OK and steps == run
            assert iters == sum(x["iters"] for x in st1)
            assert np.array_equal(bt.field(cid), T1), k
    # argument checks
    with Batch() as bt:
        bt.add_case(cases[0])
        with pytest.raises(B.LfmError):
            B.lfm_batch_advance_capped_async(bt.handle, 2, [-1], False)


def test_batch_graph_and_fused_are_bitwise_equal():
    cases = small_batch_cases(seed=11, n_cases=10, n_steps=3)
    fields = []
    for use_graph in (True, False):
        with Batch() as bt:
            ids = [bt.add_case(c) for c in cases]
            bt.set_launch(256, (2, 2, 2))
            assert bt.advance(3, use_graph=use_graph) == B.LFM_OK
            fields.append([bt.field(i) for i in ids])
    for a, b in zip(*fields):
        assert np.array_equal(a, b)


def test_batch_more_jobs_than_ctas_and_repeated_advances():
    # ~700 tiny cases: the ticket queue hands out more jobs than there are CTAs
    rng = np.random.default_rng(5)
    cases = []
    for i in range(700):
        n = int(rng.integers(2, 6))
        ax = lapcase.uniform_axis(n)
        cases.append(lapcase.RawCase(xs=ax, ys=ax.copy(), zs=ax.copy(), DT_uniform=float(rng.uniform(1e-3, 1e-1)),
                                     dt=0.05, T0=300.0, n_steps=2, tol=1e-10,
                                     patches=((lapcase.FIXED_VALUE, float(rng.uniform(250, 400))),
                                              (lapcase.FIXED_VALUE, 300.0)) + ((lapcase.ZERO_GRADIENT, 0.0),) * 4))
    with Batch() as bt:
        ids = [bt.add_case(c, workspace="torch") for c in cases]
        ctas, _, _ = B.lfm_batch_get_launch(bt.handle)
        assert len(ids) > ctas
        assert bt.advance(1) == B.LFM_OK
        assert bt.advance(1) == B.LFM_OK
        for cid, c in list(zip(ids, cases))[::37]:
            To, so = oracle.advance(c, n_steps=2)
            assert relerr(bt.field(cid), To) <= 1e-10


def test_batch_remove_and_readd():
    cases = small_batch_cases(seed=3, n_cases=6, n_steps=2)
    with Batch() as bt:
        ids = [bt.add_case(c) for c in cases]
        s = bt.remove(ids[2], close=False)
        assert len(bt) == 5
        assert bt.advance(2) == B.LFM_OK
        cid = bt.add(s)
        s.set_field(oracle.initial_field(cases[2]))
        assert bt.advance(2) == B.LFM_OK
        To, _ = oracle.advance(cases[2], n_steps=2)
        tol = 1e-10 if cases[2].precision == lapcase.FP64 else 1e-5
        assert relerr(bt.field(cid), To) <= tol


def test_autotune_restores_state(tmp_path):
    cases = small_batch_cases(seed=13, n_cases=8, n_steps=2)
    with Batch() as bt:
        ids = [bt.add_case(c) for c in cases]
        before = [bt.field(i).copy() for i in ids]
        res = bt.autotune(cache=str(tmp_path / "tune.json"), force=True)
        assert res["threads"] in (256, 512) and len(res["cells_per_thread"]) == 3
        after = [bt.field(i) for i in ids]
        for a, b in zip(before, after):
            assert np.array_equal(a, b)
        # cached on the second call
        res2 = bt.autotune(cache=str(tmp_path / "tune.json"))
        assert res2["threads"] == res["threads"]


def test_batch_multi_cta_teams_match_oracle():
    # many cases, each split over several CTAs (small cells-per-thread), so team barriers
    # carry cross-CTA data every phase; every result must match the oracle to 1e-10
    cases = lapcase.batch_cases(n_cases=24, seed=21, n_min=20, n_max=36, n_steps=3)
    with Batch() as bt:
        ids = [bt.add_case(c) for c in cases]
        bt.set_launch(256, (2, 2, 2))
        for _ in range(2):
            for cid, c in zip(ids, cases):
                bt.cases[cid].set_field(oracle.initial_field(c))
            assert bt.advance(3) == B.LFM_OK
            for cid, c in zip(ids, cases):
                To, so = oracle_cached(c)
                assert relerr(bt.field(cid), To) <= 1e-10


_ORACLE = {}


def oracle_cached(c):
    key = (c.name, c.nx, c.DT_uniform, c.dt)
    if key not in _ORACLE:
        _ORACLE[key] = oracle.advance(c)
    return _ORACLE[key]


def test_batch512_full_size_sampled_against_oracle():
    # the batched workload at full size (512 cases, edge log-uniform 16..96, 10 steps, 85.8 M
    # cells), in the launch shape the bench's autotuner picks, graph-replayed steps; a seeded
    # sample of cases (the largest among them) against the oracle cell by cell
    from paper_2507_18268_gb300.mesh import box_mesh
    cases = lapcase.batch_cases(n_cases=512, seed=3, n_steps=10)
    meshes = {}
    with Batch() as bt:
        ids = []
        for c in cases:
            key = (c.nx, c.ny, c.nz)
            if key not in meshes:
                meshes[key] = box_mesh(c)
            ids.append(bt.add_case(c, mesh=meshes[key]))
        bt.autotune()
        for cid, c in zip(ids, cases):  # the autotuner advanced the cases: restart them
            bt.cases[cid].set_field(oracle.initial_field(c))
        assert bt.advance(10, use_graph=True) == B.LFM_OK
        rng = np.random.default_rng(11)
        pick = set(rng.choice(len(cases), size=6, replace=False).tolist())
        pick.add(int(np.argmax([c.n_cells for c in cases])))
        for i in sorted(pick):
            To, so = oracle.advance(cases[i])
            st = bt.stats(ids[i], 10)
            assert [x["iters"] for x in st] == [x.iters for x in so], i
            assert relerr(bt.field(ids[i]), To) <= 1e-10, i


def test_cases_sharing_a_host_mesh_keep_their_own_diffusivity():
    # one host mesh object serves several cases of the same box: each case's own DT, dt and
    # boundary values reach the device
    from paper_2507_18268_gb300.mesh import box_mesh
    cases = lapcase.batch_cases(n_cases=6, seed=17, n_min=12, n_max=12, n_steps=3)
    m = box_mesh(cases[0])
    assert len({(c.nx, c.ny, c.nz) for c in cases}) == 1 and len({c.DT_uniform for c in cases}) == 6
    with Batch() as bt:
        ids = [bt.add_case(c, mesh=m) for c in cases]
        assert bt.advance(3) == B.LFM_OK
        for cid, c in zip(ids, cases):
            To, so = oracle.advance(c)
            assert relerr(bt.field(cid), To) <= 1e-10
            assert [x["iters"] for x in bt.stats(cid, 3)] == [x.iters for x in so]
