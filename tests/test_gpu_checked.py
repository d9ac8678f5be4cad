"""The checked build against the normal build (GPU required).

The checked build (liblapfoam_checked.so, loaded when LFM_CHECKED=1) tests every index a
kernel reads from the mesh addressing before using it as an address: a slot's neighbour
cell, a face's slot positions and a slot's face, a cell's boundary faces and a boundary
face's cell. compute-sanitizer is closed on this machine, so this build stands in for its
memory checker. On the cases below no index check fails, and every result equals the
normal build's bit for bit. The cases cover the FP64, df64 and mixed forms, relabelled and
ragged meshes, general geometry with correctors and per-face DT, volumetric sources, a
batch, and matrix and boundary read-back. The test hook then makes one check site report
as failing, with no bad index: the advance returns LFM_EINVAL naming the site, and the
context keeps working. Each build runs in a child process, since a process loads one
library.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2507_18268_gb300 import binding as B

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
sys.path.insert(0, "tests")
import lapcase
from paper_2507_18268_gb300 import Solver
from paper_2507_18268_gb300 import binding as B
from paper_2507_18268_gb300.batch import Batch
from test_gpu_parity import CASES
from test_gpu_nonorth import CASES as GEO

out = {"checked": np.array([int(B.lfm_checked_build())])}


def run(tag, case, prec=None, readback=False):
    with Solver.from_case(case) as s:
        if prec is not None:
            s.set_solver(case.tol, case.rel_tol, case.max_iter, case.min_iter, prec)
        st = s.advance(case.n_steps)
        out[tag + "_T"] = s.field()
        out[tag + "_iters"] = np.array([x["iters"] for x in st])
        out[tag + "_res"] = np.array([x["final_res"] for x in st])
        if readback:
            T, Tb = s.fields()
            out[tag + "_Tb"] = Tb
            d, u, src = s.matrix()
            out[tag + "_diag"], out[tag + "_upper"], out[tag + "_src"] = d, u, src


for prec, name in ((B.LFM_FP64, "fp64"), (B.LFM_DF64, "df64"), (B.LFM_MIXED, "mixed")):
    run(name + "_permuted20", CASES["permuted20"](), prec, readback=(name == "fp64"))
    run(name + "_ragged", CASES["ragged"](), prec)
    run(name + "_geo", GEO["perturbed_corr2_facedt"](), prec)
src = lapcase.random_small_case(33, nx=7, ny=6, nz=5, permute=False).with_(Su=150.0, Sp=-0.3, tol=1e-10, n_steps=3)
run("fp64_sources", src)
run("df64_sources", src, B.LFM_DF64)

cases = [CASES["plain7"](), CASES["ragged"](), GEO["perturbed_corr0"](),
         CASES["permuted20"]().with_(precision=lapcase.MIXED), CASES["ragged"]().with_(precision=lapcase.DF64)]
solvers = [Solver.from_case(c) for c in cases]
bt = Batch()
for s in solvers:
    bt.add(s)
bt.advance(3)
for i, s in enumerate(solvers):
    out["batch%d_T" % i] = s.field()
bt.close()
for s in solvers:
    s.close()

case = CASES["permuted20"]()
with Solver.from_case(case) as s:
    try:
        B.lfm_debug_check_inject(s.ctx, 1)
        s.advance(1)
        out["inject_rc"] = np.array([0])
    except B.LfmError as e:
        out["inject_rc"] = np.array([e.code])
        out["inject_msg"] = np.array([str(e)])
    st = s.advance(2)
    out["after_ok"] = np.array([int(all(x["status"] == 0 for x in st))])
np.savez(sys.argv[1], **out)
'''


def _run(path, checked):
    env = dict(os.environ, LFM_CHECKED="1" if checked else "0")
    r = subprocess.run([sys.executable, "-c", SCRIPT, path], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1800)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    with np.load(path) as z:
        return {k: z[k] for k in z.files}


def test_checked_build_equals_normal_build_and_reports_failures(tmp_path):
    a = _run(str(tmp_path / "normal.npz"), False)
    b = _run(str(tmp_path / "checked.npz"), True)
    assert a["checked"][0] == 0 and b["checked"][0] == 1
    results = [k for k in a if k not in ("checked", "inject_rc", "inject_msg", "after_ok")]
    assert len(results) > 40
    for k in results:
        assert np.array_equal(a[k], b[k], equal_nan=True), k
    # the hook exists only in the checked build; there it is reported, once
    assert a["inject_rc"][0] == B.LFM_ESTATE
    assert b["inject_rc"][0] == B.LFM_EINVAL and "check site 1" in str(b["inject_msg"][0])
    assert a["after_ok"][0] == 1 and b["after_ok"][0] == 1
