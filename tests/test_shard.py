"""Spreading independent cases over several devices (host logic, no GPU needed).

The batch plan is longest processing time first: every case on exactly one device, the same
plan on every rank, and the largest device load within Graham's (4/3 - 1/(3m)) of the
lower bound max(largest case, total / m). The request dispatch joins the device with the
smallest estimated backlog: deterministic, and with a service rate above the offered load no
device's backlog grows without bound.
"""
import itertools

import numpy as np
import pytest

import lapcase
from paper_2507_18268_gb300 import shard


@pytest.mark.parametrize("m", [1, 2, 3, 4, 8])
def test_batch_plan_covers_once_and_is_balanced(m):
    cases = lapcase.batch_cases(n_cases=512, seed=3)
    costs = [shard.case_cost(c) for c in cases]
    dev = shard.assign(costs, m)
    assert dev == shard.assign(costs, m)  # deterministic
    assert sorted(itertools.chain.from_iterable(shard.shard_of(costs, m, r) for r in range(m))) == \
        list(range(len(costs)))
    load = shard.loads(costs, dev, m)
    lower = max(max(costs), sum(costs) / m)
    assert max(load) <= (4.0 / 3.0 - 1.0 / (3 * m)) * lower + 1e-9 * lower
    assert abs(sum(load) - sum(costs)) <= 1e-9 * sum(costs)


def test_batch_plan_is_optimal_on_a_small_exhaustive_case():
    rng = np.random.default_rng(0)
    costs = list(rng.integers(1, 50, 9).astype(float))
    dev = shard.assign(costs, 3)
    best = min(max(shard.loads(costs, d, 3)) for d in itertools.product(range(3), repeat=len(costs)))
    assert max(shard.loads(costs, dev, 3)) <= (4.0 / 3.0 - 1.0 / 9.0) * best + 1e-12


def test_more_devices_than_cases():
    dev = shard.assign([5.0, 1.0], 4)
    assert sorted(dev) == [0, 1]
    assert shard.shard_of([5.0, 1.0], 4, 3) == []


def test_dispatch_is_deterministic_and_bounded():
    reqs = lapcase.serving_stream(n_requests=400, seed=4)
    costs = [shard.case_cost(r.case) for r in reqs]
    span = reqs[-1].arrival_s - reqs[0].arrival_s
    offered = sum(costs) / span
    for m in (1, 2, 4):
        rate = 1.5 * offered / m  # each device serves 1.5x its share of the offered load
        a = shard.dispatch_stream(reqs, m, rate)
        assert a == shard.dispatch_stream(reqs, m, rate)
        assert set(a) <= set(range(m))
        disp = shard.Dispatcher(m, rate)
        worst = 0.0
        for r, c in zip(reqs, costs):
            disp.dispatch(r.arrival_s, c)
            worst = max(worst, max(disp.backlog))
        # a backlog never exceeds the largest request plus what arrives in a burst
        assert worst < 40 * max(costs)
        if m > 1:  # every device takes part
            assert len(set(a)) == m


def test_dispatch_prefers_the_idle_device():
    d = shard.Dispatcher(2, rate=1.0)
    assert d.dispatch(0.0, 10.0) == 0
    assert d.dispatch(0.0, 1.0) == 1
    assert d.dispatch(0.5, 1.0) == 1  # device 1 has 0.5 left, device 0 has 9.5
    assert d.dispatch(100.0, 1.0) == 0  # both idle: lowest device
