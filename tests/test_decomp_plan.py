"""The decomposition plan of a mesh into label ranges (host only, no GPU): the paper's
multi-GPU runs decompose the mesh and exchange halo values every PCG iteration (section
"Evaluation"). Checked against brute force: every part's ghosts are exactly the outside
neighbours of its cells; what a part pushes to another is exactly the other's ghosts that it
owns, at the right slots; the parts cover the labels once; and a rank-by-rank exchange over
the plans (simulated here with numpy arrays, one per part) reproduces the neighbour values
every part needs."""
import numpy as np
import pytest

import lapcase
import oracle
from paper_2507_18268_gb300 import binding as B


def _mesh(name):
    case = {"plain12": lambda: lapcase.plain_box(12),
            "permuted9": lambda: lapcase.permuted_box(9, n_steps=1),
            "ragged": lambda: lapcase.random_small_case(3, nx=7, ny=5, nz=3)}[name]()
    return oracle.box_mesh(case)


@pytest.mark.parametrize("name", ["plain12", "permuted9", "ragged"])
@pytest.mark.parametrize("P", [1, 2, 3, 5])
def test_plan_matches_brute_force(name, P):
    m = _mesh(name)
    N = m.n_cells
    nbrs = [set() for _ in range(N)]
    for o, n in zip(m.owner, m.neighbour):
        nbrs[o].add(int(n))
        nbrs[n].add(int(o))
    plans = [B.lfm_dd_plan(m.owner, m.neighbour, N, P, s) for s in range(P)]
    firsts = [p[0].first_label for p in plans] + [N]
    assert firsts[0] == 0 and all(firsts[s] <= firsts[s + 1] for s in range(P))
    assert sum(p[0].n_owned for p in plans) == N
    for s, (cnt, ghost, src, prt, slt) in enumerate(plans):
        a, b = firsts[s], firsts[s + 1]
        assert cnt.n_owned == b - a
        want = sorted({o for c in range(a, b) for o in nbrs[c] if not a <= o < b})
        assert list(ghost) == want
        # pushes: exactly the other parts' ghosts that s owns, sorted by source
        exp = sorted((g - a, t, j) for t, pl in enumerate(plans) if t != s
                     for j, g in enumerate(pl[1]) if a <= g < b)
        assert list(zip(src, prt, slt)) == exp


@pytest.mark.parametrize("P", [2, 4])
def test_exchange_over_the_plans_fills_every_ghost(P):
    # one array per part (owned values, then ghost slots); each part pushes its interface
    # values by its plan; afterwards every ghost slot holds its label's value
    m = _mesh("permuted9")
    N = m.n_cells
    T = np.random.default_rng(0).normal(size=N)
    plans = [B.lfm_dd_plan(m.owner, m.neighbour, N, P, s) for s in range(P)]
    parts = []
    for cnt, ghost, *_ in plans:
        v = np.full(cnt.n_owned + cnt.n_ghost, np.nan)
        v[:cnt.n_owned] = T[cnt.first_label:cnt.first_label + cnt.n_owned]
        parts.append(v)
    for s, (cnt, ghost, src, prt, slt) in enumerate(plans):
        for i, t, j in zip(src, prt, slt):
            parts[t][plans[t][0].n_owned + j] = parts[s][i]
    for (cnt, ghost, *_), v in zip(plans, parts):
        assert np.array_equal(v[cnt.n_owned:], T[ghost])


def test_plan_rejects_bad_input():
    m = _mesh("plain12")
    with pytest.raises(B.LfmError):
        B.lfm_dd_plan(m.owner, m.neighbour, m.n_cells, 0, 0)
    with pytest.raises(B.LfmError):
        B.lfm_dd_plan(m.neighbour, m.owner, m.n_cells, 2, 0)  # owner > neighbour
