"""Pins for the oracle cycles (Alg. 2, Alg. 4) and PCG (Alg. 1)."""
import math

import numpy as np
import pytest

from oracle import mg
from oracle import octree as O
from oracle import operator as OP
from oracle import pcg
from paper_2604_18886_b300 import problems as P


def _hier(p):
    t = O.Octree(p.desc)
    f = t.faces()
    beta = P.face_beta(p, f)
    return OP.Hierarchy(t, beta, p.bc), f, beta


def _uniform_cut(n=16, bc=P.NEUMANN):
    p = P.uniform(n)
    p.bc = (bc,) * 6
    t = O.Octree(p.desc)
    f = t.faces()
    beta = np.random.default_rng(3).uniform(1e-3, 1.0, len(f["axis"]))
    return OP.Hierarchy(t, beta, p.bc)


@pytest.mark.parametrize("bc", [P.DIRICHLET, P.NEUMANN])
@pytest.mark.parametrize("mu", [1, 2])
def test_fas_equals_plain_cycle_on_uniform_grid(bc, mu):
    # Sec. 3.3: without leaves below the finest level, beta on the restriction of the
    # FAS-style cycle equals beta on the prolongation of Alg. 2
    H = _uniform_cut(16, bc)
    r = np.random.default_rng(7).standard_normal(H.A.shape[0])
    prm = mg.CycleParams(mu=mu)
    z1 = mg.vcycle(H, r, prm)
    z2 = mg.plain_vcycle(H, r, prm)
    assert np.abs(z1 - z2).max() <= 1e-11 * np.abs(z2).max()


@pytest.mark.parametrize("mu", [1, 2])
def test_cycle_is_linear(mu):
    H, _, _ = _hier(P.cut_cell(8, 2))
    rng = np.random.default_rng(11)
    n = H.A.shape[0]
    r1, r2 = rng.standard_normal(n), rng.standard_normal(n)
    prm = mg.CycleParams(mu=mu)
    z = mg.vcycle(H, 0.7 * r1 - 1.9 * r2, prm)
    zl = 0.7 * mg.vcycle(H, r1, prm) - 1.9 * mg.vcycle(H, r2, prm)
    assert np.abs(z - zl).max() <= 1e-12 * np.abs(z).max()


def test_mean_of_children_equals_parent_after_prolongation():
    # Sec. 3.3, Eq. fas-flux-conservation
    H, _, _ = _hier(P.two_level_ball(8))
    seen = []

    def hook(m, u):
        C, F = H.levels[m - 1], H.levels[m]
        I = np.nonzero(C.children[:, 0] >= 0)[0]
        mean = u[m][C.children[I]].mean(axis=1)
        seen.append(np.abs(mean - u[m - 1][I]).max() / max(1e-300, np.abs(u[m - 1][I]).max()))

    r = np.random.default_rng(2).standard_normal(H.A.shape[0])
    mg.vcycle(H, r, mg.CycleParams(mu=2), hook=hook)
    assert len(seen) > 0 and max(seen) < 1e-13


def test_colour_sweep_zeroes_residual_of_updated_cells():
    # Gauss-Seidel property of one colour sweep where no same-colour coupling exists
    H = _uniform_cut(8, P.DIRICHLET)
    L = H.levels[0]
    rng = np.random.default_rng(5)
    u = {m: rng.standard_normal(H.levels[m].n) for m in H.levels}
    b = {m: rng.standard_normal(H.levels[m].n) for m in H.levels}
    mg.colour_sweep(H, 0, u, b, 0)
    r = mg.level_residual(H, 0, u, b)
    assert np.abs(r[L.colour == 0]).max() < 1e-12
    assert np.abs(r[L.colour == 1]).max() > 1e-3


def test_cycle_converges_as_standalone_iteration():
    H, _, _ = _hier(P.two_level_ball(8))
    rng = np.random.default_rng(9)
    n = H.A.shape[0]
    b = rng.standard_normal(n)
    x = np.zeros(n)
    res = []
    for _ in range(8):
        r = b - H.A @ x
        res.append(np.linalg.norm(r))
        x = x + mg.vcycle(H, r, mg.CycleParams(beta=1.0))   # standalone solver: beta = 1
    assert res[-1] < 1e-3 * res[0]
    assert all(res[i + 1] < 0.5 * res[i] for i in range(len(res) - 1))


@pytest.mark.parametrize("name", ["dirichlet", "neumann", "cut"])
def test_pcg_matches_dense_solve_on_tiny_octrees(name):
    if name == "dirichlet":
        p = P.two_level_ball(6)
    elif name == "neumann":
        p = P.two_level_ball(6)
        p.bc = (P.NEUMANN,) * 6
        p.rhs = "normal"
    else:
        p = P.cut_cell(6, 2)
    H, f, beta = _hier(p)
    assert H.A.shape[0] < 6000
    b = P.rhs(p, H.tree.leaves, f, beta)
    x, k, hist = pcg.pcg(H, b, tol=1e-13, max_iter=100)
    xd = pcg.direct_solve(H, b)
    if H.nullspace:
        x = x - x.mean()
    assert np.abs(x - xd).max() <= 1e-10 * np.abs(xd).max()
    assert k < 30


def test_closed_form_uniform_dirichlet():
    # sin(pi x) sin(pi y) sin(pi z) is an exact eigenvector with face-Dirichlet walls, so
    # the discrete solution of the manufactured rhs is that function times
    # 3 pi^2 h^2 / (12 sin^2(pi h / 2))
    n = 16
    p = P.uniform(n)
    H, f, beta = _hier(p)
    b = P.rhs(p, H.tree.leaves, f, beta)
    x, k, hist = pcg.pcg(H, b, tol=1e-12, max_iter=100)
    L = H.tree.leaves
    h = 1.0 / n
    s = np.sin(math.pi * (L["i"] + 0.5) * h) * np.sin(math.pi * (L["j"] + 0.5) * h) * \
        np.sin(math.pi * (L["k"] + 0.5) * h)
    scale = 3 * math.pi ** 2 * h ** 2 / (12 * math.sin(math.pi * h / 2) ** 2)
    assert np.abs(x - scale * s).max() < 1e-10


def test_second_order_solution_error():
    # Sec. 4.3 (Fig. athena-sin-grid-convergence): close to second order on octrees
    errs = []
    for n0 in (8, 16, 32):
        p = P.two_level_ball(n0)
        H, f, beta = _hier(p)
        L = H.tree.leaves
        b = P.rhs(p, L, f, beta)
        x, k, _ = pcg.pcg(H, b, tol=1e-11)
        h = 1.0 / (n0 * 2.0 ** L["depth"])
        xe = P.exact_solution(p, (L["i"] + .5) * h, (L["j"] + .5) * h, (L["k"] + .5) * h)
        V = h ** 3
        errs.append(math.sqrt(np.sum(V * (x - xe) ** 2) / np.sum(V)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 1.6, (errs, rates)


def test_grid_independent_iterations_and_reduction():
    # Sec. 4.3 / Table 1: about 6 iterations to 1e-6 with ~1/20 reduction per iteration,
    # independent of the resolution
    its = []
    for n0 in (16, 32):
        p = P.two_level_ball(n0)
        H, f, beta = _hier(p)
        b = P.rhs(p, H.tree.leaves, f, beta)
        x, k, hist = pcg.pcg(H, b, tol=1e-6)
        its.append(k)
        red = (hist[0] / hist[-1]) ** (1.0 / k)
        assert red > 10
    assert abs(its[0] - its[1]) <= 1 and max(its) <= 8


def test_mu_min_cells_runs_w_above_and_v_below():
    """The minimum level size of the mu-recursion (an extension of Alg. 4): 0 reproduces
    the W-cycle bit for bit, a threshold above every level the V-cycle bit for bit, and a
    threshold between the level sizes a cycle that differs from both but converges no
    slower than V as a preconditioner."""
    p = P.two_level_ball(16)
    t = O.Octree(p.desc)
    H = OP.Hierarchy(t, P.face_beta(p, t.faces()), p.bc)
    r = P.random_vector(t.n_leaves, 41)
    z_w = mg.vcycle(H, r, mg.CycleParams(mu=2))
    z_v = mg.vcycle(H, r, mg.CycleParams(mu=1))
    assert np.array_equal(mg.vcycle(H, r, mg.CycleParams(mu=2, mu_min_cells=0)), z_w)
    assert np.array_equal(mg.vcycle(H, r, mg.CycleParams(mu=2, mu_min_cells=10 ** 9)), z_v)
    sizes = sorted(H.levels[m].n for m in H.levels)
    mid = sizes[len(sizes) // 2]
    z_m = mg.vcycle(H, r, mg.CycleParams(mu=2, mu_min_cells=mid))
    assert not np.array_equal(z_m, z_w) and not np.array_equal(z_m, z_v)
    b = P.rhs(p, t.leaves, t.faces(), P.face_beta(p, t.faces()))
    _, kv, _ = pcg.pcg(H, b, tol=1e-8, prm=mg.CycleParams(mu=1))
    _, km, _ = pcg.pcg(H, b, tol=1e-8, prm=mg.CycleParams(mu=2, mu_min_cells=mid))
    assert km <= kv
