"""A case on the GPU: one ``lfm_ctx`` with its mesh, properties, controls and field.

PyTorch supplies device memory (the workspace tensor) and the CUDA stream; the library does
all the work.
"""
from __future__ import annotations

from typing import List, Optional

import numpy as np

import lapcase

from . import binding as B
from .mesh import HexGeometry, LduMesh, box_mesh, field_by_label, hex_mesh


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def solver_log(stats: List[dict], field: str = "T", dt: Optional[float] = None, t0: float = 0.0,
               mixed: bool = False) -> str:
    """The per-step statistics as a solver log in the layout laplacianFoam prints: with dt, a
    "Time = t" line per step, then the solve line with the solver (diagonal-preconditioned
    CG), the field, the initial and final normFactor-scaled residuals and the iteration count.
    mixed: the steps ran the mixed form; its defect-correction sweeps are added. A step that
    stopped on an error status shows the status."""
    lines = []
    for k, s in enumerate(stats):
        if dt is not None:
            lines.append(f"Time = {t0 + (k + 1) * dt:g}")
            lines.append("")
        line = (f"diagonalPCG:  Solving for {field}, Initial residual = {s['init_res']:.6g}, "
                f"Final residual = {s['final_res']:.6g}, No Iterations {s['iters']}")
        if mixed:
            line += f", sweeps {s['sweeps']}"
        if s.get("status", 0) != 0:
            line += f", status {B._NAMES.get(s['status'], s['status'])}"
        lines.append(line)
    return "\n".join(lines)


class BoxInfo:
    """Sizes of a mesh that was built on the device or is shared (no host arrays)."""

    def __init__(self, n_cells: int, n_faces: int, n_bfaces: int):
        self.n_cells, self.n_faces, self.n_bfaces = n_cells, n_faces, n_bfaces
        self.DT_faces = self.DT_bfaces = None
        self.cell_of_label = None


class Solver:
    """One case: exactly one of ``mesh`` (host LDU arrays, uploaded), ``box`` ((xs, ys, zs)
    vertex coordinates of a naturally numbered box, built on the device) or ``share``
    (another Solver whose uploaded mesh this one uses) gives the mesh."""

    def __init__(self, mesh: Optional[LduMesh] = None, device: int = 0, stream=None, workspace: str = "torch",
                 layout: int = B.LFM_BOTH, box=None, share: Optional["Solver"] = None,
                 geometry: Optional[HexGeometry] = None):
        assert (mesh is not None) + (box is not None) + (share is not None) == 1
        self.device = device
        self.stream = stream
        self._ws = None
        self._share = share
        self.geometry = geometry
        self.ctx = B.lfm_create(device, _stream_handle(stream))
        try:
            if mesh is not None:
                self.mesh = mesh
                nbytes = (B.lfm_workspace_bytes(mesh, layout) if geometry is None
                          else B.lfm_workspace_bytes_geometry(mesh, layout))
            elif box is not None:
                xs, ys, zs = box
                n, f, nb, _ = B.lfm_box_counts(len(xs) - 1, len(ys) - 1, len(zs) - 1)
                self.mesh = BoxInfo(n, f, nb)
                nbytes = B.lfm_workspace_bytes_box(len(xs) - 1, len(ys) - 1, len(zs) - 1, layout)
            else:
                # a host mesh's arrays (per-face DT, labels, weights) serve the sharer too
                self.mesh = (share.mesh if isinstance(share.mesh, LduMesh)
                             else BoxInfo(share.mesh.n_cells, share.mesh.n_faces, share.mesh.n_bfaces))
                self.geometry = share.geometry
                nbytes = B.lfm_workspace_bytes_shared(share.ctx, layout)
            self.workspace_bytes = nbytes
            if workspace == "torch":
                import torch

                self._ws = torch.empty(nbytes, dtype=torch.uint8, device=f"cuda:{device}")
                B.lfm_bind_workspace(self.ctx, self._ws.data_ptr(), nbytes, layout)
            if mesh is not None and geometry is not None:
                B.lfm_upload_mesh_geometry(self.ctx, mesh, geometry)
            elif mesh is not None:
                B.lfm_upload_mesh(self.ctx, mesh)
            elif box is not None:
                B.lfm_upload_box(self.ctx, *box)
            else:
                B.lfm_upload_mesh_shared(self.ctx, share.ctx)
        except Exception:
            B.lfm_destroy(self.ctx)
            self.ctx = None
            raise

    # ---- configuration ---------------------------------------------------------------
    @classmethod
    def from_case(cls, case: lapcase.RawCase, mesh: Optional[LduMesh] = None,
                  geometry: Optional[HexGeometry] = None, **kw) -> "Solver":
        """A case on a host-built mesh: the rectilinear box, or with ``case.points`` the
        general hexahedral mesh and its geometry (corrected laplacian; the face weights and
        coefficients computed on the solver's GPU)."""
        if mesh is None and case.points is not None:
            mesh, geometry = hex_mesh(case, device=kw.get("device", 0))
        mesh = mesh or box_mesh(case)
        s = cls(mesh, geometry=geometry, **kw)
        s.configure(case)
        return s

    @classmethod
    def from_box_case(cls, case: lapcase.RawCase, **kw) -> "Solver":
        """A naturally numbered box case with its mesh built on the device."""
        assert case.perm is None
        s = cls(box=(case.xs, case.ys, case.zs), **kw)
        s.configure(case)
        return s

    @classmethod
    def sharing(cls, src: "Solver", case: lapcase.RawCase, **kw) -> "Solver":
        """A case on the mesh already uploaded by ``src``."""
        s = cls(share=src, **kw)
        s.configure(case)
        return s

    def configure(self, case: lapcase.RawCase, field: bool = True):
        m = self.mesh
        if case.DTx is None and case.DTy is None and case.DTz is None:
            # the case's own uniform DT (a host mesh shared between cases carries the
            # diffusivity of the case it was built from)
            B.lfm_set_diffusivity(self.ctx, float(case.DT_uniform), None, None)
        elif m.DT_faces is None:
            raise ValueError("per-face DT needs a host mesh built from the case (Solver(mesh=...))")
        else:
            B.lfm_set_diffusivity(self.ctx, 0.0, m.DT_faces, m.DT_bfaces)
        for p, (ptype, value) in enumerate(case.patches):
            B.lfm_set_patch(self.ctx, p, int(ptype), None, float(value))
        B.lfm_set_time_step(self.ctx, case.dt)
        B.lfm_set_solver(self.ctx, case.tol, case.rel_tol, case.max_iter, case.min_iter, case.precision)
        B.lfm_set_nonorth_correctors(self.ctx, int(case.n_nonorth_corr))
        if case.DT_cells is not None:
            if m.cell_of_label is None:
                raise ValueError("a cell-field DT needs a host mesh")
            w = None if self.geometry is not None else m.weights
            B.lfm_set_diffusivity_cells(self.ctx, case.cell_array(case.DT_cells)[m.cell_of_label], w)
        if case.Su is not None or case.Sp is not None:
            if m.cell_of_label is None and case.perm is not None:
                raise ValueError("sources on a relabelled mesh need a host mesh")
            order = m.cell_of_label if m.cell_of_label is not None else slice(None)
            Su = case.cell_array(case.Su)
            Sp = case.cell_array(case.Sp)
            B.lfm_set_source(self.ctx, None if Su is None else Su[order], None if Sp is None else Sp[order])
        if field:
            if np.isscalar(case.T0):
                B.lfm_fill_field(self.ctx, float(case.T0))
            elif m.cell_of_label is None:
                B.lfm_set_field(self.ctx, case.T0_natural())
            else:
                B.lfm_set_field(self.ctx, field_by_label(case, m))

    def set_solver(self, tol, rel_tol=0.0, max_iter=1000, min_iter=0, precision=B.LFM_FP64):
        B.lfm_set_solver(self.ctx, tol, rel_tol, max_iter, min_iter, precision)

    def grad(self, boundary: bool = True):
        """Gauss linear gradient of the current T: (cells [N, 3], boundary faces [NB, 3])."""
        return B.lfm_grad(self.ctx, self.mesh.n_cells, self.mesh.n_bfaces, boundary)

    def set_field(self, T: np.ndarray):
        B.lfm_set_field(self.ctx, T)

    def set_field_device(self, ptr: int):
        B.lfm_set_field_device(self.ctx, ptr)

    # ---- running ---------------------------------------------------------------------
    def advance(self, n_steps: int) -> List[dict]:
        return [s.as_dict() for s in B.lfm_advance(self.ctx, n_steps)]

    def advance_async(self, n_steps: int):
        B.lfm_advance_async(self.ctx, n_steps)

    def done(self) -> bool:
        return B.lfm_query(self.ctx) == B.LFM_OK

    def finish(self, n: int) -> List[dict]:
        return [s.as_dict() for s in B.lfm_finish(self.ctx, n)]

    # ---- results ---------------------------------------------------------------------
    def field(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        return B.lfm_get_field(self.ctx, self.mesh.n_cells, out=out)

    def fields(self):
        return B.lfm_get_field(self.ctx, self.mesh.n_cells, self.mesh.n_bfaces, boundary=True)

    def field_device_ptr(self) -> int:
        return B.lfm_field_device_ptr(self.ctx)

    def matrix(self):
        return B.lfm_get_matrix(self.ctx, self.mesh.n_cells, self.mesh.n_faces)

    def launch(self):
        return B.lfm_get_launch(self.ctx)

    def phase_times(self) -> dict:
        """Device milliseconds per phase kind of the last advance."""
        return B.lfm_get_phase_times(self.ctx)

    def set_launch(self, ctas: int, threads: int):
        B.lfm_set_launch(self.ctx, ctas, threads)

    def close(self):
        if self.ctx is not None:
            B.lfm_destroy(self.ctx)
            self.ctx = None
        self._ws = None
        self._share = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
