"""The N > 1 host paths on CPU: two gloo ranks (no GPU needed).

The single-case step runs one replica per rank (it does not shard without a halo exchange);
the reported time is the maximum over ranks and the work is summed over ranks, per-rank
inputs differing only by seed. Independent cases shard: every rank computes the same plan
(shard.assign / shard.dispatch_stream) with no message, solves its own share, and the
gathered results equal those of one process solving everything.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import lapcase
    import torch.distributed as dist
    w, r, local = bench.dist_setup()
    assert (w, r) == (world, rank)
    bench.barrier(w)
    t_max = bench.reduce_max(1.0 + rank, w)
    work = bench.reduce_sum(10.0 * (rank + 1), w)
    cases = lapcase.batch_cases(n_cases=3, seed=3 + 1000 * rank)
    out.put((rank, t_max, work, [c.nx for c in cases]))
    dist.destroy_process_group()


def test_two_rank_timing_and_work_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[1] for x in res] == [2.0, 2.0]
    assert [x[2] for x in res] == [30.0, 30.0]
    assert res[0][3] != res[1][3]


def _shard_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import lapcase
    import oracle
    import torch.distributed as dist
    from paper_2507_18268_gb300 import shard
    w, r, _ = bench.dist_setup()
    cases = lapcase.batch_cases(n_cases=9, seed=3, n_min=4, n_max=9, n_steps=2)
    costs = [shard.case_cost(c) for c in cases]
    mine = shard.shard_of(costs, w, r)
    solved = {i: oracle.advance(cases[i])[0].tolist() for i in mine}
    gathered = [None] * w
    dist.all_gather_object(gathered, (mine, solved))
    reqs = lapcase.serving_stream(n_requests=50, seed=4, n_min=4, n_max=8, max_steps=3)
    plans = [None] * w
    dist.all_gather_object(plans, shard.dispatch_stream(reqs, w, rate=1e6))
    out.put((rank, gathered, plans))
    dist.destroy_process_group()


def test_two_rank_sharded_batch_equals_one_process():
    import numpy as np

    import lapcase
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    gathered = res[0][1]
    assert gathered == res[1][1]
    owned = [i for mine, _ in gathered for i in mine]
    assert sorted(owned) == list(range(9)) and len(set(owned)) == 9 and all(len(m) > 0 for m, _ in gathered)
    cases = lapcase.batch_cases(n_cases=9, seed=3, n_min=4, n_max=9, n_steps=2)
    for mine, solved in gathered:
        for i in mine:
            assert np.array_equal(np.array(solved[i]), oracle.advance(cases[i])[0])
    # both ranks computed the same dispatch of the stream, using both devices
    assert res[0][2][0] == res[0][2][1] == res[1][2][0]
    assert set(res[0][2][0]) == {0, 1}


def _dd_worker(rank, world, port, out):
    """One part of the decomposed PCG on a gloo rank: halo exchange of p by the plan (point
    to point), global sums by all_reduce -- the orchestration of the decomposed form, with
    test-only numpy arithmetic on the oracle's assembled matrix."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import numpy as np
    import torch
    import torch.distributed as dist

    import bench
    import lapcase
    import oracle
    from paper_2507_18268_gb300 import binding as B
    w, r, _ = bench.dist_setup()
    case = lapcase.permuted_box(8, n_steps=1).with_(tol=1e-12)
    m = oracle.box_mesh(case)
    bt, bv = oracle.boundary_types_values(case, m)
    T0 = oracle.initial_field(case)
    d, up, b = oracle.assemble(m, bt, bv, case.dt, T0)
    N = m.n_cells
    plans = [B.lfm_dd_plan(m.owner, m.neighbour, N, w, s) for s in range(w)]
    cnt, ghost, src, prt, slt = plans[r]
    a, n, G = cnt.first_label, cnt.n_owned, cnt.n_ghost
    loc = {lab: i for i, lab in enumerate(range(a, a + n))}
    loc.update({int(g): n + j for j, g in enumerate(ghost)})
    rows = [[] for _ in range(n)]  # (local column, coefficient)
    for f, (o, nb) in enumerate(zip(m.owner, m.neighbour)):
        if a <= o < a + n:
            rows[o - a].append((loc[int(nb)], up[f]))
        if a <= nb < a + n:
            rows[nb - a].append((loc[int(o)], up[f]))
    dl, bl = d[a:a + n], b[a:a + n]

    def exchange(v):  # push interface values to the parts that mirror them
        reqs = []
        for t in range(w):
            if t == r:
                continue
            sel = prt == t
            if sel.any():
                reqs.append(dist.isend(torch.tensor(v[src[sel]]), t))
        for t in range(w):
            pt = plans[t]
            mine = [(i, j) for i, p_, j in zip(pt[2], pt[3], pt[4]) if p_ == r]
            if t != r and mine:
                buf = torch.empty(len(mine), dtype=torch.float64)
                dist.recv(buf, t)
                for (i, j), val in zip(mine, buf.numpy()):
                    v[n + j] = val
        for q in reqs:
            q.wait()

    def allsum(*xs):
        t = torch.tensor(xs, dtype=torch.float64)
        dist.all_reduce(t)
        return t.numpy()

    def amul(v):
        return np.array([dl[i] * v[i] + sum(c * v[j] for j, c in rows[i]) for i in range(n)])

    x = np.zeros(n + G)
    x[:n] = T0[a:a + n]
    exchange(x)
    xref = allsum(x[:n].sum())[0] / N
    s_row = np.array([dl[i] + sum(c for _, c in rows[i]) for i in range(n)])
    ax = amul(x)
    rr = bl - ax
    nf, sr = allsum(np.sum(np.abs(ax - s_row * xref) + np.abs(bl - s_row * xref)), np.abs(rr).sum())
    nf += 1e-20
    init = res = sr / nf
    p = np.zeros(n + G)
    wv = rr / dl
    rho = allsum(np.dot(wv, rr))[0]
    p[:n] = wv
    it = 0
    while res >= case.tol and it < 1000:
        if it > 0:
            p[:n] = wv + beta * p[:n]
        exchange(p)
        q = amul(p)
        sigma = allsum(np.dot(q, p[:n]))[0]
        alpha = rho / sigma
        x[:n] += alpha * p[:n]
        rr -= alpha * q
        wv = rr / dl
        s2 = allsum(np.abs(rr).sum(), np.dot(wv, rr))
        res = s2[0] / nf
        beta, rho = s2[1] / rho, s2[1]
        it += 1
    full = [None] * w
    dist.all_gather_object(full, (a, x[:n].tolist()))
    out.put((rank, it, init, full))
    dist.destroy_process_group()


def test_two_rank_decomposed_pcg_equals_the_oracle():
    import numpy as np

    import lapcase
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dd_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    case = lapcase.permuted_box(8, n_steps=1).with_(tol=1e-12)
    To, so = oracle.advance(case)
    T = np.zeros(case.n_cells)
    for a, v in res[0][3]:
        T[a:a + len(v)] = v
    assert res[0][1] == res[1][1] == so[0].iters
    # the initial residual differs only by the rounding the normFactor bound allows
    import stat_bounds
    m = oracle.box_mesh(case)
    _, B_ir = stat_bounds.step_bounds(case, m, oracle.initial_field(case), "fp64", (1, 1), so[0].norm_factor,
                                      so[0].init_res)
    assert abs(res[0][2] - so[0].init_res) <= B_ir
    assert np.max(np.abs(T - To) / np.abs(To)) <= 1e-12
