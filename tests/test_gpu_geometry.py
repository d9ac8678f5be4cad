"""Face coefficients of general meshes computed on the GPU (lfm_face_coeffs_device: the
interpolation weights of the paper's "weights" loop, |Sf|, the non-orthogonal implicit
coefficients and correction vectors, the boundary |Sf| and inverse distances) against the
oracle's ora_hex_coeffs on the oracle's own geometry (GPU required).

Both evaluate the same formulas with every operation rounded on its own in the same order
(the oracle is compiled without fused multiply-adds, the kernel uses explicitly rounded
intrinsics), so the results must be equal bit for bit; the host path of mesh.hex_mesh must
give the same arrays as its device path.
"""
import numpy as np
import pytest
import torch

import lapcase
import oracle
from paper_2507_18268_gb300 import binding as B
from paper_2507_18268_gb300.mesh import hex_mesh

from test_gpu_nonorth import CASES

pytestmark = pytest.mark.gpu


def device_coeffs(N, owner, neighbour, Sf, Cf, C, bcell, bSf, bCf):
    dev = torch.device("cuda", 0)

    def up(a, dtype):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).to(dev)

    F, NB = len(owner), len(bcell)
    args = [up(owner, np.int32), up(neighbour, np.int32), up(Sf, np.float64), up(Cf, np.float64),
            up(C, np.float64), up(bcell, np.int32), up(bSf, np.float64), up(bCf, np.float64)]
    outs = [torch.empty(F, dtype=torch.float64, device=dev) for _ in range(3)]
    outs.append(torch.empty((F, 3), dtype=torch.float64, device=dev))
    outs += [torch.empty(NB, dtype=torch.float64, device=dev) for _ in range(2)]
    B.lfm_face_coeffs_device(N, F, NB, *[t.data_ptr() for t in args + outs], torch.cuda.current_stream().cuda_stream)
    return [t.cpu().numpy() for t in outs]


@pytest.mark.parametrize("name", list(CASES))
def test_face_coeffs_bitwise_equal_to_the_oracle(name):
    case = CASES[name]()
    om = oracle.hex_mesh(case)
    w, mag, delta, corr, bmag, bdelta = device_coeffs(om.n_cells, om.owner, om.neighbour, om.Sf, om.Cf, om.C,
                                                      om.bcell, om.bSf, om.bCf)
    for got, want in [(w, om.w), (mag, om.magSf), (delta, om.delta), (corr, om.corr), (bmag, om.bmagSf),
                      (bdelta, om.bdelta)]:
        assert np.array_equal(got, np.asarray(want).reshape(got.shape))


def test_degenerate_face_takes_the_half_weight():
    # a face whose area vector is orthogonal to both centre offsets: weight 0.5 (as the oracle)
    C = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    Cf = np.array([[0.5, 0.0, 0.0]])
    Sf = np.array([[0.0, 1.0, 0.0]])
    w, mag, delta, corr, _, _ = device_coeffs(2, np.array([0]), np.array([1]), Sf, Cf, C, np.zeros(0, np.int32),
                                             np.zeros((0, 3)), np.zeros((0, 3)))
    assert w[0] == 0.5 and mag[0] == 1.0
    assert delta[0] == 1.0 / 0.05  # n.d = 0, so the floor 0.05 |d| sets it
    assert np.array_equal(corr[0], np.array([0.0, 1.0, 0.0]) - np.array([1.0, 0.0, 0.0]) * delta[0])


@pytest.mark.parametrize("name", ["perturbed_corr1", "mapped24", "perturbed40"])
def test_host_and_device_paths_of_hex_mesh_agree(name):
    case = CASES[name]()
    mh, gh = hex_mesh(case)
    md, gd = hex_mesh(case, device=0)
    for a, b in [(mh.magSf, md.magSf), (mh.deltaCoeffs, md.deltaCoeffs), (mh.bmagSf, md.bmagSf),
                 (mh.bdeltaCoeffs, md.bdeltaCoeffs), (gh.weights, gd.weights), (gh.corr_vec, gd.corr_vec)]:
        assert np.array_equal(a, b)


def test_out_of_range_cell_index_is_rejected():
    case = CASES["perturbed_corr0"]()
    om = oracle.hex_mesh(case)
    owner = np.array(om.owner, copy=True)
    owner[3] = om.n_cells  # out of range: reported, never read through
    with pytest.raises(B.LfmError) as e:
        device_coeffs(om.n_cells, owner, om.neighbour, om.Sf, om.Cf, om.C, om.bcell, om.bSf, om.bCf)
    assert e.value.code == B.LFM_EINVAL
