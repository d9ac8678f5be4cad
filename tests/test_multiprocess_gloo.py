"""The N > 1 host path of bench.py on CPU: two gloo ranks (no GPU needed).

Every rank runs its own replica (the step does not shard without a halo exchange); the
reported time is the maximum over ranks and the work is summed over ranks. Per-rank
inputs differ only by seed.
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
