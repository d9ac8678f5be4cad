"""Serving form: continuous batching of heat-diffusion solve requests on one GPU.

Requests (a box case and a number of implicit steps, FP64 or mixed precision) arrive over
time. The server keeps every admitted case resident on the device (matrix, PCG state and
field live in its workspace) and advances all of them together: each scheduling tick is
one batched launch that moves every admitted case forward up to ``steps_per_tick`` time
steps (each request stops at its own step count; the CTAs of a finished request serve the
others' jobs in the same launch), so requests that arrive while others run join at the next
tick and their work overlaps on the device.
Admission is first-come first-served against an HBM budget (the workspaces of admitted
cases plus the shared meshes); a finished case's field is read back, its workspace is
released, and the next waiting request takes the space.

Cases with the same box share one mesh built on the device (``lfm_upload_box`` once per
size, then ``lfm_upload_mesh_shared`` per request), so admitting a request costs a
workspace allocation and a few small uploads, not a host mesh build.

The host work of a tick overlaps the device work of the previous one: once tick k is
enqueued, the server reads back and releases the cases that finished at tick k - 1, admits
waiting requests into contexts of their own (on a stream of their own, so that their
uploads do not wait for the batch), and only then waits for tick k. At the tick boundary it
removes finished cases from the batch, adds the admitted ones and enqueues tick k + 1
before any further host work.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Dict, List, Optional

import numpy as np

import lapcase

from . import binding as B
from .batch import Batch
from .solver import Solver


@dataclasses.dataclass
class Done:
    index: int
    n_cells: int
    steps: int
    precision: int
    arrival_s: float
    admitted_s: float
    finished_s: float
    cell_iterations: int
    status: int
    field: Optional[np.ndarray] = None

    @property
    def latency_s(self) -> float:
        return self.finished_s - self.arrival_s


def percentile(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=float), q)) if len(xs) else float("nan")


class Server:
    def __init__(self, device: int = 0, budget_bytes: float = 120e9, use_graph: bool = True,
                 launch: Optional[tuple] = None, batch: Optional[Batch] = None, steps_per_tick: int = 8):
        self.device = device
        self.budget = float(budget_bytes)
        self.use_graph = use_graph
        self.steps_per_tick = max(1, int(steps_per_tick))
        # admissions and read-backs run on a stream of their own, beside the batch's
        self.side = None
        if batch is None:
            import torch

            self.side = torch.cuda.Stream(device=device)
            self.stream = torch.cuda.Stream(device=device)
            batch = Batch(device=device, stream=self.stream)
        self.batch = batch
        if launch:
            self.batch.set_launch(*launch)
        self.meshes: Dict[tuple, Solver] = collections.OrderedDict()
        self.mesh_users: Dict[tuple, int] = collections.defaultdict(int)
        self.used = 0.0
        self.peak_used = 0.0

    # ---- resources -----------------------------------------------------------------------
    def _on_side(self) -> dict:
        return {} if self.side is None else {"stream": self.side}

    def _key(self, case: lapcase.RawCase):
        return (case.nx, case.ny, case.nz, case.xs.tobytes(), case.ys.tobytes(), case.zs.tobytes())

    def _mesh_for(self, case: lapcase.RawCase) -> Solver:
        key = self._key(case)
        if key in self.meshes:
            self.meshes.move_to_end(key)
            return self.meshes[key]
        owner = Solver(box=(case.xs, case.ys, case.zs), device=self.device, layout=B.LFM_FP64, **self._on_side())
        self.meshes[key] = owner
        self.used += owner.workspace_bytes
        return owner

    def _evict_idle_meshes(self, need: float, keep=None):
        """Releases least recently used meshes that no admitted case shares (never `keep`,
        the mesh of the request being admitted, which `need` assumes present) until `need`
        more bytes fit."""
        for key in list(self.meshes):
            if self.used + need <= self.budget:
                return
            if self.mesh_users[key] == 0 and key != keep:
                owner = self.meshes.pop(key)
                self.used -= owner.workspace_bytes
                owner.close()

    def _need(self, case: lapcase.RawCase) -> float:
        N, F, NB, W = B.lfm_box_counts(case.nx, case.ny, case.nz)
        per_case = B.lfm_workspace_bytes_box(case.nx, case.ny, case.nz, case.precision)
        mesh = 0 if self._key(case) in self.meshes else B.lfm_workspace_bytes_box(case.nx, case.ny, case.nz,
                                                                                   B.LFM_FP64)
        # a sharer's workspace is smaller than a full one; this bound is conservative
        return float(per_case + mesh)

    # ---- the loop ------------------------------------------------------------------------
    def run(self, requests: List[lapcase.Request], keep_fields: bool = False, time_scale: float = 1.0) -> dict:
        """Serves the requests (arrival times scaled by time_scale) and returns a report."""
        pending = collections.deque()   # arrived, not yet admitted
        ready = []                      # admitted contexts, joining the batch at the next tick
        active: Dict[int, dict] = {}    # members of the batch
        leaving = []                    # finished at the last tick: read back, then released
        done: List[Done] = []
        nxt = 0
        ticks = 0
        busy = 0.0
        in_flight = False
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0  # noqa: E731
        while nxt < len(requests) or pending or ready or active or leaving or in_flight:
            now = clock()
            while nxt < len(requests) and requests[nxt].arrival_s * time_scale <= now:
                pending.append(nxt)
                nxt += 1
            # ---- host work that overlaps the tick in flight ----------------------------------
            for a, s, st in leaving:
                r = requests[a["req"]]
                field = s.field()  # the result is served once it is on the host
                if not keep_fields:
                    field = None
                done.append(Done(a["req"], s.mesh.n_cells, r.case.n_steps, r.case.precision,
                                 r.arrival_s * time_scale, a["admitted"], clock(), a["cell_iters"], st, field))
                self.used -= s.workspace_bytes
                self.mesh_users[self._key(r.case)] -= 1
                s.close()
            leaving = []
            # admission: first come, first served, while the budget allows
            while pending:
                r = requests[pending[0]]
                need = self._need(r.case)
                if self.used + need > self.budget:
                    self._evict_idle_meshes(need, keep=self._key(r.case))
                if self.used + need > self.budget and (active or ready or in_flight):
                    break
                owner = self._mesh_for(r.case)
                s = Solver.sharing(owner, r.case, device=self.device, layout=r.case.precision, **self._on_side())
                self.mesh_users[self._key(r.case)] += 1
                self.used += s.workspace_bytes
                self.peak_used = max(self.peak_used, self.used)
                ready.append({"req": pending.popleft(), "left": r.case.n_steps, "admitted": clock(),
                              "cell_iters": 0, "solver": s})
            # ---- tick boundary -------------------------------------------------------------
            if in_flight:
                tb = time.perf_counter()
                self.batch.finish()
                busy += time.perf_counter() - tb
                in_flight = False
                ticks += 1
                res = self.batch.results()
                for cid in list(active):
                    a = active[cid]
                    st, steps, iters = res[cid]
                    a["left"] -= steps
                    a["cell_iters"] += a["solver"].mesh.n_cells * iters
                    if a["left"] <= 0 or st != 0:
                        leaving.append((a, self.batch.remove(cid, close=False), st))
                        del active[cid]
            for a in ready:
                active[self.batch.add(a["solver"])] = a
            ready = []
            if active:
                k = min(self.steps_per_tick, max(a["left"] for a in active.values()))
                if k == 1:
                    self.batch.advance_async(1, self.use_graph)
                else:  # one fused launch of k steps, each request capped at what it has left
                    self.batch.advance_capped_async(k, {cid: min(k, a["left"]) for cid, a in active.items()})
                in_flight = True
            elif not leaving and not pending and nxt < len(requests):
                time.sleep(max(0.0, requests[nxt].arrival_s * time_scale - clock()))
        makespan = clock()
        lat = [d.latency_s for d in done]
        cells_steps = sum(d.n_cells * d.steps for d in done)
        cell_iters = sum(d.cell_iterations for d in done)
        return {"requests": len(done), "makespan_s": makespan, "throughput_req_s": len(done) / makespan,
                "cell_steps_per_s": cells_steps / makespan, "cell_iterations_per_s": cell_iters / makespan,
                "p50_latency_s": percentile(lat, 50),
                "p99_latency_s": percentile(lat, 99), "mean_latency_s": float(np.mean(lat)) if lat else float("nan"),
                "ticks": ticks, "gpu_wait_s": busy, "peak_hbm_bytes": self.peak_used,
                "failed": sum(1 for d in done if d.status != 0), "done": done}

    def close(self):
        self.batch.close()
        for owner in self.meshes.values():
            owner.close()
        self.meshes.clear()


def serve_serial_fp64(requests: List[lapcase.Request], device: int = 0, keep_fields: bool = False,
                      time_scale: float = 1.0) -> dict:
    """Baseline: every request solved alone in FP64 with the single-case path, one after
    another in arrival order (meshes built on the device and shared, as in the server).
    Latency follows the queue: a request starts when it has arrived and the previous one
    has finished."""
    import torch

    meshes: Dict[tuple, Solver] = {}
    finish_prev = 0.0
    lat, done = [], []
    t_first = requests[0].arrival_s * time_scale if requests else 0.0
    cells_steps = 0
    cell_iters = 0
    for i, r in enumerate(requests):
        case = r.case.with_(precision=B.LFM_FP64)
        key = (case.nx, case.ny, case.nz)
        if key not in meshes:
            meshes[key] = Solver(box=(case.xs, case.ys, case.zs), device=device, layout=B.LFM_FP64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = Solver.sharing(meshes[key], case, device=device, layout=B.LFM_FP64)
        st = s.advance(case.n_steps)
        field = s.field()
        cell_iters += s.mesh.n_cells * sum(x["iters"] for x in st)
        s.close()
        dt = time.perf_counter() - t0
        start = max(r.arrival_s * time_scale, finish_prev)
        finish_prev = start + dt
        lat.append(finish_prev - r.arrival_s * time_scale)
        cells_steps += s.mesh.n_cells * case.n_steps
        if keep_fields:
            done.append(field)
    for m in meshes.values():
        m.close()
    makespan = finish_prev - t_first
    return {"requests": len(requests), "makespan_s": makespan, "throughput_req_s": len(requests) / makespan,
            "cell_steps_per_s": cells_steps / makespan, "cell_iterations_per_s": cell_iters / makespan,
            "p50_latency_s": percentile(lat, 50), "p99_latency_s": percentile(lat, 99),
            "mean_latency_s": float(np.mean(lat)), "latencies_s": lat, "fields": done if keep_fields else None}
