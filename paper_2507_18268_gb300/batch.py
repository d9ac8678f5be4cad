"""Batched form: many independent cases per persistent launch, with an autotuner.

A :class:`Batch` owns one ``lfm_batch`` and the :class:`Solver` contexts of its cases. One
advance runs every member case for n steps; by default one step is captured once into a
CUDA graph and the graph is replayed per step.

The autotuner picks the launch shape -- threads per CTA and cells per thread for each of the
three size classes (fewer than 32768 cells, fewer than 262144, larger), which set each
case's team size -- by timing one batch step per candidate on the batch's own cases, with
their fields saved before and restored after, so tuning leaves the batch's state unchanged.
The best shape is cached per device and per batch signature (case counts per size class)
in a JSON file (``LFM_TUNE_CACHE``, default ``~/.cache/lapfoam/tune.json``).
"""
from __future__ import annotations

import json
import os
import time
from typing import Dict, List, Optional, Sequence

import numpy as np

import lapcase

from . import binding as B
from .mesh import box_mesh
from .solver import Solver

SIZE_CLASS_BOUNDS = (32768, 262144)
DEFAULT_LAUNCH = (512, (4, 8, 16))


def size_class(n_cells: int) -> int:
    return 0 if n_cells < SIZE_CLASS_BOUNDS[0] else (1 if n_cells < SIZE_CLASS_BOUNDS[1] else 2)


class Batch:
    def __init__(self, device: int = 0, stream=None):
        self.device = device
        self.stream = stream
        handle = None if stream is None else (stream if isinstance(stream, int) else int(stream.cuda_stream))
        self.handle = B.lfm_batch_create(device, handle)
        self.cases: Dict[int, Solver] = {}
        self.launch = DEFAULT_LAUNCH

    # ---- membership ------------------------------------------------------------------
    def add(self, solver: Solver) -> int:
        cid = B.lfm_batch_add(self.handle, solver.ctx)
        self.cases[cid] = solver
        return cid

    def add_case(self, case: lapcase.RawCase, mesh=None, workspace: str = "torch") -> int:
        """Adds a case on a host-built mesh: `mesh`, else the case's box, or its general
        hexahedral mesh and geometry when the case has vertex points."""
        layout = case.precision if workspace == "torch" else B.LFM_BOTH
        s = Solver.from_case(case, mesh=mesh, device=self.device, stream=self.stream, workspace=workspace,
                             layout=layout)
        return self.add(s)

    def remove(self, cid: int, close: bool = True) -> Solver:
        B.lfm_batch_remove(self.handle, cid)
        s = self.cases.pop(cid)
        if close:
            s.close()
        return s

    def __len__(self):
        return len(self.cases)

    # ---- running ---------------------------------------------------------------------
    def set_launch(self, threads: int, cells_per_thread: Sequence[int]):
        B.lfm_batch_set_launch(self.handle, threads, list(cells_per_thread))
        self.launch = (threads, tuple(cells_per_thread))

    def advance_async(self, n_steps: int, use_graph: bool = True):
        B.lfm_batch_advance_async(self.handle, n_steps, use_graph)

    def advance_capped_async(self, n_steps: int, caps: Dict[int, int], use_graph: bool = False):
        """n_steps for every case, but case id i at most caps[i] of them (the serving form's
        multi-step ticks); fused launch by default (one launch runs all n_steps)."""
        n = max(caps) + 1 if caps else 0
        arr = [n_steps] * n
        for cid, c in caps.items():
            arr[cid] = c
        B.lfm_batch_advance_capped_async(self.handle, n_steps, arr, use_graph)

    def results(self):
        """{case id: (status, steps run, PCG iterations summed)} after the last advance."""
        n = max(self.cases) + 1 if self.cases else 0
        st, sp, it = B.lfm_batch_results(self.handle, n)
        return {cid: (st[cid], sp[cid], it[cid]) for cid in self.cases}

    def done(self) -> bool:
        return B.lfm_batch_query(self.handle) == B.LFM_OK

    def finish(self) -> int:
        return B.lfm_batch_finish(self.handle)

    def advance(self, n_steps: int, use_graph: bool = True) -> int:
        self.advance_async(n_steps, use_graph)
        return self.finish()

    def stats(self, cid: int, n: int) -> List[dict]:
        return [x.as_dict() for x in B.lfm_batch_case_stats(self.handle, cid, n)]

    def status(self, cid: int) -> int:
        return B.lfm_batch_case_status(self.handle, cid)

    def last_iters(self, cid: int) -> int:
        return B.lfm_batch_case_iters(self.handle, cid)

    def field(self, cid: int) -> np.ndarray:
        return self.cases[cid].field()

    def close(self):
        if self.handle is not None:
            for cid in list(self.cases):
                self.remove(cid, close=True)
            B.lfm_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- autotuning --------------------------------------------------------------------
    def signature(self) -> str:
        counts = [0, 0, 0]
        for s in self.cases.values():
            counts[size_class(s.mesh.n_cells)] += 1
        return "classes=" + ",".join(map(str, counts))

    def _save_fields(self):
        import torch
        saved = {}
        for cid, s in self.cases.items():
            buf = torch.empty(s.mesh.n_cells, dtype=torch.float64, device=f"cuda:{self.device}")
            _copy_device(buf.data_ptr(), s.field_device_ptr(), 8 * s.mesh.n_cells)
            saved[cid] = buf
        torch.cuda.synchronize()
        return saved

    def _restore_fields(self, saved):
        import torch
        for cid, buf in saved.items():
            self.cases[cid].set_field_device(buf.data_ptr())
        torch.cuda.synchronize()

    def _time_step(self, threads, cpt, use_graph=True) -> float:
        """Seconds per cell-iteration of one batch step with this launch shape."""
        import torch
        self.set_launch(threads, cpt)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc = self.advance(1, use_graph)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if rc != B.LFM_OK:
            return float("inf")
        work = sum(s.mesh.n_cells * (self.stats(cid, 1)[0]["iters"] + 2) for cid, s in self.cases.items())
        return dt / max(work, 1)

    def autotune(self, cache: Optional[str] = None, force: bool = False) -> dict:
        cache = cache or os.environ.get("LFM_TUNE_CACHE", os.path.expanduser("~/.cache/lapfoam/tune.json"))
        import torch
        key = f"{torch.cuda.get_device_name(self.device)}|{self.signature()}"
        table = {}
        if os.path.exists(cache):
            try:
                with open(cache) as f:
                    table = json.load(f)
            except (OSError, ValueError):
                table = {}
        if key in table and not force:
            best = table[key]
            self.set_launch(best["threads"], best["cells_per_thread"])
            return best
        saved = self._save_fields()
        trials = []
        try:
            self._time_step(512, (4, 8, 16))  # warm the graph and caches
            self._restore_fields(saved)
            best = None
            for threads in (256, 512):
                for cpt in (2, 8, 32):
                    t = self._time_step(threads, (cpt, cpt, cpt))
                    self._restore_fields(saved)
                    trials.append({"threads": threads, "cells_per_thread": [cpt] * 3, "s_per_cell_iter": t})
                    if best is None or t < best[0]:
                        best = (t, threads, [cpt] * 3)
            # refine each size class with the others fixed
            for k in range(3):
                for f in (0.25, 4.0):
                    cand = list(best[2])
                    cand[k] = max(1, int(round(cand[k] * f)))
                    t = self._time_step(best[1], cand)
                    self._restore_fields(saved)
                    trials.append({"threads": best[1], "cells_per_thread": cand, "s_per_cell_iter": t})
                    if t < best[0]:
                        best = (t, best[1], cand)
        finally:
            self._restore_fields(saved)
        result = {"threads": best[1], "cells_per_thread": best[2], "s_per_cell_iter": best[0], "trials": trials}
        self.set_launch(best[1], best[2])
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        table[key] = result
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1)
        os.replace(tmp, cache)
        return result


def _copy_device(dst: int, src: int, nbytes: int):
    """Device-to-device copy on the current torch stream."""
    import torch
    src_t = _wrap(src, nbytes)
    dst_t = _wrap(dst, nbytes)
    dst_t.copy_(src_t)


def _wrap(ptr: int, nbytes: int):
    import torch
    class _Holder:
        pass
    h = _Holder()
    h.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False), "version": 3}
    return torch.as_tensor(h, device="cuda")
