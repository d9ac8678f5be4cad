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
