"""One case decomposed into parts (the paper's multi-GPU data flow, emulated on one GPU).

``Decomposed`` wraps an ``lfm_dd``: the parts of a configured single case (a
:class:`Solver`), each with its own vectors and ghost slots, exchanging interface values of
T once per step and of p once per PCG iteration, with the global sums over all parts. See
``lfm_dd_create`` in include/lapfoam.h.
"""
from __future__ import annotations

from typing import List

import numpy as np

from . import binding as B
from .solver import Solver


class Decomposed:
    def __init__(self, solver: Solver, n_parts: int):
        self.solver = solver
        self.n_parts = int(n_parts)
        self.handle = B.lfm_dd_create(solver.ctx, self.n_parts)

    def counts(self) -> List[B.lfm_dd_counts]:
        return [B.lfm_dd_part_counts(self.handle, s) for s in range(self.n_parts)]

    def set_field(self, T: np.ndarray):
        B.lfm_dd_set_field(self.handle, T)

    def field(self) -> np.ndarray:
        return B.lfm_dd_get_field(self.handle, self.solver.mesh.n_cells)

    def advance(self, n_steps: int) -> List[dict]:
        return [s.as_dict() for s in B.lfm_dd_advance(self.handle, n_steps)]

    def close(self):
        if self.handle is not None:
            B.lfm_dd_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
