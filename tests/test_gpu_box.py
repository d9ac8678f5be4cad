"""Device-built box meshes and mesh sharing against the host upload path (GPU required)."""
import numpy as np
import pytest

import lapcase
from paper_2507_18268_gb300 import Solver
from paper_2507_18268_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", [lapcase.plain_box(9), lapcase.graded_box(12, n_steps=4),
                                  lapcase.RawCase(xs=lapcase.graded_axis(7, 1.2), ys=lapcase.uniform_axis(1),
                                                  zs=lapcase.uniform_axis(3), DT_uniform=1e-2, dt=0.1,
                                                  n_steps=3, tol=1e-12)])
def test_device_box_equals_host_upload_bitwise(case):
    with Solver.from_case(case) as host, Solver.from_box_case(case) as dev:
        for a, b in zip(host.matrix(), dev.matrix()):
            assert np.array_equal(a, b)
        sa, sb = host.advance(case.n_steps), dev.advance(case.n_steps)
        assert np.array_equal(host.field(), dev.field())
        assert sa == sb


def test_shared_mesh_cases_are_independent():
    base = lapcase.plain_box(10)
    c1 = base.with_(DT_uniform=1e-3, dt=0.05, n_steps=3)
    c2 = base.with_(DT_uniform=5e-4, dt=0.02, n_steps=3, precision=B.LFM_MIXED,
                    patches=((0, 300.0), (0, 320.0)) + ((1, 0.0),) * 4, T0=310.0)
    with Solver(box=(base.xs, base.ys, base.zs)) as owner:
        a = Solver.sharing(owner, c1)
        b = Solver.sharing(owner, c2)
        a.advance(3)
        b.advance(3)
        with Solver.from_box_case(c1) as ra, Solver.from_box_case(c2) as rb:
            ra.advance(3)
            rb.advance(3)
            assert np.array_equal(a.field(), ra.field())
            assert np.array_equal(b.field(), rb.field())
        # the mesh owner cannot go while cases use its mesh
        assert B.load().lfm_destroy(owner.ctx) == B.LFM_ESTATE
        a.close()
        b.close()
