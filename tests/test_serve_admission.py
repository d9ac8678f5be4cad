"""Serving form, host logic only (no GPU): admission under the HBM budget.

The server is driven with stand-ins for the device objects (a batch that finishes every
step at once, solvers that only report their workspace sizes, taken from the library's own
size functions), so what is checked is the scheduling: every request is served, admission
is first come first served, the bytes held never exceed the budget even when meshes have to
be evicted, a mesh is shared by every admitted request of its box size, and every request
runs exactly its own step count when a tick runs several steps.
"""
import numpy as np
import pytest

import lapcase
from paper_2507_18268_gb300 import binding as B
from paper_2507_18268_gb300 import serve


class FakeMesh:
    def __init__(self, n):
        self.n_cells = n


class FakeSolver:
    live = []

    def __init__(self, box=None, device=0, layout=B.LFM_FP64):
        nx, ny, nz = (len(a) - 1 for a in box)
        self.workspace_bytes = B.lfm_workspace_bytes_box(nx, ny, nz, B.LFM_FP64)
        self.mesh = FakeMesh(nx * ny * nz)
        self.is_mesh = True
        self.closed = False
        FakeSolver.live.append(self)

    @classmethod
    def sharing(cls, owner, case, device=0, layout=B.LFM_FP64):
        s = cls.__new__(cls)
        full = B.lfm_workspace_bytes_box(case.nx, case.ny, case.nz, layout)
        s.workspace_bytes = int(0.8 * full)  # a sharer holds no mesh arrays
        s.mesh = owner.mesh
        s.owner = owner
        s.is_mesh = False
        s.closed = False
        s.n_steps = case.n_steps
        s.steps_done = 0
        assert not owner.closed, "a case was admitted on an evicted mesh"
        FakeSolver.live.append(s)
        return s

    def field(self):
        return np.zeros(self.mesh.n_cells)

    def close(self):
        assert not self.closed
        self.closed = True


class FakeBatch:
    def __init__(self):
        self.members = {}
        self.next_id = 0
        self.admit_order = []

    def add(self, s):
        cid = self.next_id
        self.next_id += 1
        self.members[cid] = s
        self.admit_order.append(cid)
        return cid

    def advance_async(self, n, use_graph=True):
        pass

    def finish(self):
        pass

    def advance_capped_async(self, n, caps, use_graph=False):
        self.caps = dict(caps)

    def results(self):
        caps = getattr(self, "caps", {})
        out = {cid: (0, caps.get(cid, 1), 3 * caps.get(cid, 1)) for cid in self.members}
        for cid, s in self.members.items():
            s.steps_done += out[cid][1]
        self.caps = {}
        return out

    def status(self, cid):
        return 0

    def last_iters(self, cid):
        return 3

    def remove(self, cid, close=True):
        s = self.members.pop(cid)
        assert s.steps_done == s.n_steps, "a request left with another step count than it asked for"
        return s

    def close(self):
        pass


@pytest.mark.parametrize("seed,steps_per_tick", [(1, 1), (2, 4), (3, 3)])
def test_budget_is_never_exceeded_and_every_request_is_served(monkeypatch, seed, steps_per_tick):
    monkeypatch.setattr(serve, "Solver", FakeSolver)
    FakeSolver.live = []
    reqs = lapcase.serving_stream(n_requests=60, seed=seed, rate_per_s=1e6, n_min=6, n_max=16, max_steps=6)
    biggest = max(B.lfm_workspace_bytes_box(r.case.nx, r.case.ny, r.case.nz, B.LFM_BOTH) for r in reqs)
    budget = 3 * biggest
    batch = FakeBatch()
    server = serve.Server(budget_bytes=budget, batch=batch, steps_per_tick=steps_per_tick)
    rep = server.run(reqs)
    server.close()
    assert rep["requests"] == len(reqs) and rep["failed"] == 0
    assert rep["peak_hbm_bytes"] <= budget
    # first come, first served: requests (indexed in arrival order) are admitted in order
    admitted = [d.admitted_s for d in sorted(rep["done"], key=lambda d: d.index)]
    assert all(a <= b for a, b in zip(admitted, admitted[1:]))
    # every case and mesh released at the end
    assert all(s.closed for s in FakeSolver.live)
    # a case never outlives its mesh, and requests of one box size share one mesh at a time
    assert len({id(s.owner) for s in FakeSolver.live if not s.is_mesh}) < len(reqs)
