"""Independent cases spread over several GPUs.

Batched and served cases are independent problems: each device runs its own share with no
collective on the data path (one process per GPU, or one Batch per device). What has to be
shared is only the plan, and both plans here are deterministic functions of the inputs, so
every rank computes the same plan from the same list and no rank has to tell another.

* A batch (``assign``): longest processing time first -- cases in decreasing estimated cost,
  each to the device with the least cost assigned so far (ties to the lowest device). The
  cost of a case is the work its steps move: cells x (PCG iterations per step + 2) x steps,
  the estimate the batched kernel also orders its jobs by (the + 2 counts the step's row and
  sum passes). Graham (1969): the largest device load is at most (4/3 - 1/(3m)) times the
  best possible.
* A request stream (``Dispatcher``): each arriving request joins the device whose estimated
  backlog is smallest, the backlog draining at an assumed service rate between arrivals
  (join the shortest estimated queue). Arrival times and costs alone decide it, so every
  rank sees the same dispatch.
"""
from __future__ import annotations

import heapq
from typing import Iterable, List, Sequence

import lapcase


def case_cost(case: lapcase.RawCase, iters_per_step: float = 5.0) -> float:
    """Estimated work of a case: cells x (iterations per step + 2) x steps."""
    return float(case.n_cells) * (iters_per_step + 2.0) * float(case.n_steps)


def assign(costs: Sequence[float], n_devices: int) -> List[int]:
    """Device of each case (longest processing time first onto the least-loaded device)."""
    if n_devices < 1:
        raise ValueError("n_devices must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, d) for d in range(n_devices)]
    out = [0] * len(costs)
    for i in order:
        load, d = heapq.heappop(heap)
        out[i] = d
        heapq.heappush(heap, (load + float(costs[i]), d))
    return out


def shard_of(costs: Sequence[float], n_devices: int, rank: int) -> List[int]:
    """Indices of the cases device `rank` runs, in their original order."""
    dev = assign(costs, n_devices)
    return [i for i, d in enumerate(dev) if d == rank]


def loads(costs: Sequence[float], devices: Sequence[int], n_devices: int) -> List[float]:
    out = [0.0] * n_devices
    for c, d in zip(costs, devices):
        out[d] += float(c)
    return out


class Dispatcher:
    """Join-the-shortest-estimated-queue dispatch of a request stream over n devices: a
    device's backlog grows by each request's cost and drains at `rate` (cost units per
    second) while time passes; a request goes to the device with the smallest backlog at its
    arrival (ties to the lowest device)."""

    def __init__(self, n_devices: int, rate: float):
        if n_devices < 1 or not rate > 0:
            raise ValueError("need n_devices >= 1 and rate > 0")
        self.n = n_devices
        self.rate = float(rate)
        self.backlog = [0.0] * n_devices
        self.t = 0.0

    def dispatch(self, arrival_s: float, cost: float) -> int:
        dt = max(0.0, float(arrival_s) - self.t)
        self.t = max(self.t, float(arrival_s))
        self.backlog = [max(0.0, b - self.rate * dt) for b in self.backlog]
        d = min(range(self.n), key=lambda k: (self.backlog[k], k))
        self.backlog[d] += float(cost)
        return d


def dispatch_stream(requests: Iterable[lapcase.Request], n_devices: int, rate: float) -> List[int]:
    """Device of each request of a stream (in arrival order)."""
    disp = Dispatcher(n_devices, rate)
    return [disp.dispatch(r.arrival_s, case_cost(r.case)) for r in requests]
