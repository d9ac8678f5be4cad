"""GB300-native implicit time step of laplacianFoam (arXiv 2507.18268).

Each step assembles fvm::ddt(T) - fvm::laplacian(DT, T) in LDU face-addressed form and
solves it with diagonal-preconditioned CG (normFactor residual), all in hand-written CUDA
for sm_103a behind the C ABI of ``include/lapfoam.h``:

* :mod:`.binding`  -- ctypes binding with the C names (marshalling only);
* :mod:`.mesh`     -- box meshes in LDU addressing (the blockMesh role);
* :mod:`.solver`   -- one case on the GPU (torch supplies workspace memory and stream).
"""
from . import binding
from .binding import LfmError, load
from .mesh import LduMesh, box_mesh, field_by_label
from .solver import Solver, solver_log

__all__ = ["binding", "LfmError", "load", "LduMesh", "box_mesh", "field_by_label", "Solver", "solver_log"]
