"""Geometric-multigrid ablation (Sec. 3.3): cells with children rediscretised from the grid
at their own resolution instead of Alg. 3's algebraically consistent coarsening.

Pins: in fluid-only systems the two constructions give the same matrices (the paper's
worked values -2h / 12h with alpha = 2: the Galerkin product equals the direct
discretisation), entry for entry on every level, Dirichlet and Neumann, with T-junctions;
on a cut-cell tree the geometric hierarchy loses the grid-independent iteration count
(the paper's static-tank comparison: many more iterations than the consistent one).
"""
import numpy as np
import pytest

from oracle import mg
from oracle import octree as O
from oracle import operator as OP
from oracle import pcg
from paper_2604_18886_b300 import problems as P


def coarse_beta_of(p):
    """beta of the - faces of coarse cells, from the input generator's geometry."""
    def f(m, a, i, j, k):
        faces = {"axis": np.full(len(i), a), "depth": np.full(len(i), m), "i": i, "j": j, "k": k}
        return P.face_beta(p, faces)
    return f


@pytest.mark.parametrize("bc", [P.DIRICHLET, P.NEUMANN])
@pytest.mark.parametrize("kind", ["ball", "band"])
def test_fluid_only_geometric_equals_algebraic(kind, bc):
    p = P.laplacian_problem(kind, 8)
    p.bc = (bc,) * 6
    t = O.Octree(p.desc)
    f = t.faces()
    beta = P.face_beta(p, f)                       # beta = 1 everywhere
    Ha = OP.Hierarchy(t, beta, p.bc)
    Hg = OP.Hierarchy(t, beta, p.bc, coarse_beta=lambda m, a, i, j, k: np.ones(len(i)))
    for m in range(Ha.mc, Ha.D + 1):
        La, Lg = Ha.levels[m], Hg.levels[m]
        assert np.array_equal(La.c, Lg.c), m
        assert np.array_equal(La.cm, Lg.cm), m
    # the worked coarse values of Sec. 3.3 on an interior cell of the root grid's first
    # coarsening: off-diagonal -2h, diagonal 12h (h = fine cell size, alpha = 2)
    L = Ha.levels[-1]
    h = 1.0 / 8
    inner = (L.i > 0) & (L.j > 0) & (L.k > 0) & (L.i < L.N - 1) & (L.j < L.N - 1) & (L.k < L.N - 1)
    assert np.all(L.c[inner] == 12 * h) and np.all(L.cm[:, inner] == -2 * h)


def test_cut_cell_geometric_coarsening_loses_grid_independence():
    its = {}
    for n0 in (8, 16):
        p = P.cut_cell(n0, 2)
        t = O.Octree(p.desc)
        f = t.faces()
        beta = P.face_beta(p, f)
        b = P.rhs(p, t.leaves, f, beta)
        Ha = OP.Hierarchy(t, beta, p.bc)
        Hg = OP.Hierarchy(t, beta, p.bc, coarse_beta=coarse_beta_of(p))
        its[n0] = (pcg.pcg(Ha, b, tol=1e-6)[1], pcg.pcg(Hg, b, tol=1e-6, max_iter=300)[1])
        # both preconditioners give the same solution
        xa = pcg.pcg(Ha, b, tol=1e-10)[0]
        xg = pcg.pcg(Hg, b, tol=1e-10, max_iter=300)[0]
        xa, xg = xa - xa.mean(), xg - xg.mean()
        assert np.abs(xa - xg).max() <= 1e-7 * np.abs(xa).max()
    assert its[16][1] >= 2 * its[16][0], its
    assert its[16][1] > its[8][1] and its[16][0] <= its[8][0] + 1, its
