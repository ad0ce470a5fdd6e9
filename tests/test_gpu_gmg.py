"""Geometric-multigrid ablation (Sec. 3.3) through the library against the oracle's
geometric hierarchy: coefficients (FP64, 1e-13 of the level's largest diagonal: the library
computes the coarse face fractions itself, from the description's solids), the FP64 cycle
(1e-10), PCG iterates, and at the full cut-cell size the iteration count: several times
Alg. 3's, whose count stays the same when the tree doubles.
"""
import numpy as np
import pytest

from oracle import mg
from oracle import octree as O
from oracle import operator as OP
from oracle import pcg
from paper_2604_18886_b300 import _lib as L
from paper_2604_18886_b300 import problems as P
from paper_2604_18886_b300 import solver as S

from test_oracle_gmg import coarse_beta_of

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _cuda(x, dt=None):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype=dt or torch.float64, device="cuda")


def _pair(p, coef="f64", mu=1):
    t = O.Octree(p.desc)
    f = t.faces()
    beta = P.face_beta(p, f)
    Hg = OP.Hierarchy(t, beta, p.bc, coarse_beta=coarse_beta_of(p))
    g = S.Octree(p.desc)
    hg = S.Hierarchy(g, beta, p.bc, S.mg_params(coef=coef, mu=mu, coarsening="geometric"))
    return t, f, beta, Hg, g, hg


@pytest.mark.parametrize("make", [lambda: P.cut_cell(16, 2), lambda: P.batch_tree(1), lambda: P.cut_cell(12, 2)])
def test_geometric_coefficients_match_oracle(make):
    t, f, beta, Hg, g, hg = _pair(make())
    for m in range(Hg.mc, Hg.D + 1):
        c, cx, cy, cz = hg.coefs(m)
        Lv = Hg.levels[m]
        scale = np.abs(Lv.c).max()
        assert np.abs(c - Lv.c).max() <= 1e-13 * scale, m
        for a, v in enumerate((cx, cy, cz)):
            assert np.abs(v - Lv.cm[a]).max() <= 1e-13 * scale, (m, a)


@pytest.mark.parametrize("mu", [1, 2])
def test_geometric_vcycle_and_pcg_match_oracle(mu):
    p = P.cut_cell(16, 2)
    t, f, beta, Hg, g, hg = _pair(p, mu=mu)
    r = P.random_vector(t.n_leaves, 70)
    z = hg.vcycle(_cuda(r)).cpu().numpy()
    zo = mg.vcycle(Hg, r, mg.CycleParams(mu=mu))
    assert np.abs(z - zo).max() <= 1e-10 * np.abs(zo).max()
    b = P.rhs(p, t.leaves, f, beta)
    xo, ko, ho = pcg.pcg(Hg, b, tol=1e-8, prm=mg.CycleParams(mu=mu), max_iter=300)
    x, st = hg.solve(_cuda(b), tol=1e-8, precision="fp64", max_iter=300)
    assert st.converged and st.iterations == ko
    xo = xo - xo.mean()
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-8 * np.abs(xo).max()


def test_geometric_coarsening_needs_a_sdf_description():
    p = P.two_level_ball(16)
    g = S.Octree(p.desc)
    beta = P.face_beta(p, g.faces())
    with pytest.raises(RuntimeError):
        S.Hierarchy(g, beta, p.bc, S.mg_params(coarsening="geometric"))


def test_full_size_cut_cell_geometric_needs_several_times_the_iterations():
    # the cut-cell workload (64^3 root, 2 levels) and its half-size tree: Alg. 3 keeps the
    # iteration count, the geometric hierarchy needs several times more at both sizes
    # (measured 18 and 14 against 5 and 5)
    its = {}
    for n0 in (32, 64):
        p = P.cut_cell(n0, 2)
        g = S.Octree(p.desc)
        f = g.faces()
        beta = P.face_beta(p, f)
        b = _cuda(P.rhs(p, g.leaves(), f, beta))
        row = []
        for co in ("algebraic", "geometric"):
            h = S.Hierarchy(g, beta, p.bc, S.mg_params(coef="f32", coarsening=co))
            _, st = h.solve(b, tol=1e-6, precision="mixed", max_iter=400)
            assert st.converged and st.true_rel_res <= 1.5e-6
            row.append(st.iterations)
            del h
        its[n0] = row
    assert all(its[n][1] >= 2.5 * its[n][0] for n in its), its
    assert abs(its[64][0] - its[32][0]) <= 1, its
