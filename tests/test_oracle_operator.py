"""Pins for the oracle operator (Sec. 2.1, 2.4, 2.5, 3.1, 3.3)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import octree as O
from oracle import operator as OP
from paper_2604_18886_b300 import problems as P

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_worked_values.json")))


def _hier(p, beta=None):
    t = O.Octree(p.desc)
    f = t.faces()
    if beta is None:
        beta = P.face_beta(p, f)
    return OP.Hierarchy(t, beta, p.bc), f


def _neumann(p):
    p.bc = (P.NEUMANN,) * 6
    return p


def test_uniform_fluid_coefficients():
    # Sec. 2.1: fluid cell c_{x-} = -h, c = 6h
    H, _ = _hier(_neumann(P.uniform(8)))
    L = H.levels[0]
    h = 1.0 / 8
    interior = (L.i > 0) & (L.i < 7) & (L.j > 0) & (L.j < 7) & (L.k > 0) & (L.k < 7)
    g = GOLD["galerkin_alpha2"]
    assert np.allclose(L.c[interior], g["fine_diag_over_h"] * h, rtol=0, atol=1e-15)
    assert np.allclose(L.cm[:, interior], g["fine_offdiag_over_h"] * h, rtol=0, atol=1e-15)


def test_galerkin_worked_values_alpha2():
    # Sec. 2.4: coarse off-diagonal -4h/alpha, diagonal 24h/alpha, i.e. -2h and 12h
    H, _ = _hier(_neumann(P.uniform(16)))
    g = GOLD["galerkin_alpha2"]
    h = 1.0 / 16
    C = H.levels[-1]
    interior = (C.i > 0) & (C.i < 7) & (C.j > 0) & (C.j < 7) & (C.k > 0) & (C.k < 7)
    assert np.allclose(C.c[interior], g["coarse_diag_over_h_fine"] * h, atol=1e-15)
    assert np.allclose(C.cm[:, interior & (C.i > 0)], g["coarse_offdiag_over_h_fine"] * h, atol=1e-15)
    assert g["coarse_diag_over_h_fine"] == g["coarse_diag_over_h_fine_times_alpha"] / g["alpha"]


@pytest.mark.parametrize("bc", [P.DIRICHLET, P.NEUMANN])
def test_coarse_equals_geometric_alpha2(bc):
    # Sec. 3.3: with alpha = 2 coarsened inner coefficients equal the leaf coefficients
    # the discretisation gives directly at that cell size (including Dirichlet walls)
    p = P.two_level_ball(8)
    p.bc = (bc,) * 6
    H, _ = _hier(p)
    for m in range(H.mc, H.D):
        L = H.levels[m]
        h = 1.0 / L.N
        n = L.N
        exp_c = np.zeros(L.n)
        exp_cm = np.zeros((3, L.n))
        coords = (L.i, L.j, L.k)
        for q, (a, s) in enumerate(O.DIRS):
            wall = coords[a] == (0 if s < 0 else n - 1)
            w = np.where(wall, 2 * h if bc == P.DIRICHLET else 0.0, h)
            exp_c += w
            if s < 0:
                exp_cm[a] = -w
        inner = L.children[:, 0] >= 0
        assert np.allclose(L.c[inner], exp_c[inner], rtol=1e-14, atol=0)
        assert np.allclose(L.cm[:, inner], exp_cm[:, inner], rtol=1e-14, atol=1e-18)


def test_alg3_equals_rap_on_uniform_cut_cells():
    # Alg. 3 equals R A P (Eq. galerkin-mat-coarsen) where there are no T-junctions, for
    # arbitrary face beta including zero faces that deactivate cells (active_cnt branch)
    p = P.uniform(8)
    p.bc = (P.NEUMANN, P.DIRICHLET, P.NEUMANN, P.NEUMANN, P.NEUMANN, P.DIRICHLET)
    t = O.Octree(p.desc)
    f = t.faces()
    rng = np.random.default_rng(0)
    beta = rng.uniform(0.0, 1.0, len(f["axis"]))
    # cells (0..1)^3 become inactive: all their faces get beta = 0
    dead = np.zeros(len(beta), bool)
    for a in range(3):
        sel = f["axis"] == a
        ijk = np.stack([f["i"], f["j"], f["k"]], 1)
        minus = ijk.copy(); minus[:, a] -= 1
        in_plus = np.all(ijk <= 1, 1) & np.all(ijk >= 0, 1)
        in_minus = np.all(minus <= 1, 1) & np.all(minus >= 0, 1)
        dead |= sel & (in_plus | in_minus)
    beta[dead] = 0.0
    H = OP.Hierarchy(t, beta, p.bc)
    L0 = H.levels[0]
    assert np.sum(L0.c == 0.0) == 8
    for m in range(H.D, H.mc, -1):
        inner, rap = H.rap_inner_block(m)
        dense = H.level_dense(m - 1)[np.ix_(inner, inner)]
        assert np.allclose(rap, dense, rtol=0, atol=1e-14 * np.abs(dense).max())
    # one coarse cell with no active child
    C = H.levels[-1]
    assert np.sum(C.c == 0.0) == 1


def test_alg3_literal_equals_vectorised():
    H, _ = _hier(P.cut_cell(8, 2))
    for m in range(H.D, H.mc, -1):
        C = H.levels[m - 1]
        for I in np.nonzero(C.children[:, 0] >= 0)[0][:200]:
            c, x, y, z = H.coarsen_cell(m, C.children[I])
            assert c == C.c[I] and (x, y, z) == tuple(C.cm[:, I])


def test_alg3_equals_rap_away_from_t_junctions():
    H, _ = _hier(P.two_level_ball(8))
    m = 1
    inner, rap = H.rap_inner_block(m)
    dense = H.level_dense(0)[np.ix_(inner, inner)]
    # rows of parents none of whose children has a T face
    L = H.levels[1]
    has_t = np.zeros(H.levels[0].n, bool)
    tchild = np.nonzero((L.tK >= 0).any(axis=1))[0]
    has_t[L.parent[tchild]] = True
    ok = ~has_t[inner]
    assert ok.sum() > 0 and (~ok).sum() > 0
    assert np.allclose(rap[ok][:, ok], dense[ok][:, ok], atol=1e-15)


def test_t_junction_coefficient_and_ghost_2d_worked_values():
    # Sec. 3.1: c_{4,x-} = (S1 + S3) / (2h) = (c_{6,x-} + c_{7,x-}) / 2
    g = GOLD["t_junction_2d"]
    assert abs(g["c4_xm"] - 0.5 * (g["c6_xm"] + g["c7_xm"])) < 1e-15
    assert abs(g["c6_xm"] - g["S1"] / g["h"]) < 1e-15
    # 3-D: the coarse leaf's face weight is half the sum of its four sub-face weights
    p = P.cut_cell(8, 1)
    H, f = _hier(p)
    t = H.tree
    kind, rank = t.neighbour_table()
    Lf = t.leaves
    checked = 0
    for r in np.nonzero((kind == O.FINER).any(axis=1))[0][:50]:
        d = Lf["depth"][r]
        L = H.levels[d]
        idx = L.index(Lf["i"][r], Lf["j"][r], Lf["k"][r])
        for q in np.nonzero(kind[r] == O.FINER)[0]:
            a, s = O.DIRS[q]
            if s > 0:
                continue
            base = [Lf["i"][r], Lf["j"][r], Lf["k"][r]]
            acc = 0.0
            o1, o2 = [b for b in range(3) if b != a]
            for u in (0, 1):
                for v in (0, 1):
                    cc = [2 * base[0], 2 * base[1], 2 * base[2]]
                    cc[o1] += u
                    cc[o2] += v
                    acc += H.face_beta(a, d + 1, *cc) * t.h(d + 1)
            assert abs(-L.cm[a, idx] - 0.5 * acc) < 1e-15
            checked += 1
    assert checked > 0


def _t_free(p):
    H, _ = _hier(p)
    return H


def test_constant_nullspace_and_conservation():
    # Sec. 2.2: pure Neumann -> A 1 = 0; flux conservation (f1 + f3 = f4, Eq.
    # flux-conservation) -> every column sums to zero as well
    for p in (_neumann(P.two_level_ball(8)), P.cut_cell(8, 2)):
        H, _ = _hier(p)
        one = np.ones(H.A.shape[0])
        assert np.abs(H.A @ one).max() < 1e-14
        assert np.abs(H.A.T @ one).max() < 1e-14


def test_symmetric_psd_without_t_junctions():
    # Sec. 2.1: the seven-point system is symmetric and positive semi-definite
    p = P.uniform(6)
    t = O.Octree(p.desc)
    f = t.faces()
    beta = np.random.default_rng(1).uniform(1e-3, 1.0, len(f["axis"]))
    for bc in ((P.NEUMANN,) * 6, (P.DIRICHLET,) * 6):
        H = OP.Hierarchy(t, beta, bc)
        A = H.A.toarray()
        assert np.abs(A - A.T).max() < 1e-16
        ev = np.linalg.eigvalsh(A)
        assert ev.min() > -1e-13
        if bc[0] == P.DIRICHLET:
            assert ev.min() > 0


def test_t_junction_asymmetry_closed_form():
    # Literal T operator: A[i,K] = -w_f/2 per T face of fine leaf i, A[K,i] = -w_KP/8;
    # with full faces w_f = h, w_KP = 2h -> -h/2 vs -h/4; A - A^T vanishes elsewhere
    p = _neumann(P.two_level_ball(8))
    H, _ = _hier(p)
    A = H.A.toarray()
    t = H.tree
    kind, rank = t.neighbour_table()
    Lf = t.leaves
    trow = np.nonzero((kind == O.COARSER).any(axis=1))[0]
    tcol = set()
    for r in trow:
        h = t.h(Lf["depth"][r])
        for q in np.nonzero(kind[r] == O.COARSER)[0]:
            K = rank[r, q]
            nT = np.sum((kind[r] == O.COARSER) & (rank[r] == K))
            assert abs(A[r, K] - (-0.5 * h * nT)) < 1e-15
            assert abs(A[K, r] - (-0.25 * h)) < 1e-15
            tcol.add(K)
    Dm = A - A.T
    mask = np.zeros_like(Dm, bool)
    # rows/cols of fine T leaves, their siblings, and coarse K leaves
    t_related = set(trow.tolist()) | tcol
    sib = set()
    L1 = H.levels[1]
    for r in trow:
        idx = L1.index(Lf["i"][r], Lf["j"][r], Lf["k"][r])
        for s in H.levels[0].children[L1.parent[idx]]:
            sib.add(int(L1.rank[s]))
    t_related |= sib
    rel = np.array(sorted(t_related))
    mask[np.ix_(rel, np.arange(len(A)))] = True
    mask[np.ix_(np.arange(len(A)), rel)] = True
    assert np.abs(Dm[~mask]).max() < 1e-16
    assert np.abs(Dm).max() > 1e-4


def test_dirichlet_sine_is_exact_eigenvector():
    # face-Dirichlet walls: sin(pi x_i) sin(pi y_j) sin(pi z_k) is an eigenvector of the
    # uniform operator, eigenvalue h^3 * 3 * 4 sin^2(pi h / 2) / h^2
    n = 12
    p = P.uniform(n)
    H, _ = _hier(p)
    L = H.tree.leaves
    h = 1.0 / n
    x = (L["i"] + 0.5) * h; y = (L["j"] + 0.5) * h; z = (L["k"] + 0.5) * h
    v = np.sin(math.pi * x) * np.sin(math.pi * y) * np.sin(math.pi * z)
    lam = h ** 3 * 3 * 4 * math.sin(math.pi * h / 2) ** 2 / h ** 2
    assert np.abs(H.A @ v - lam * v).max() < 1e-15


def test_laplacian_accuracy_on_octree():
    # Sec. 4.2 test function f = (x^2+y^2+z^2) exp(-xyz).  Away from refinement
    # boundaries the per-volume operator error is second order; on cells touching a
    # T-junction the flux uses the coarse-level gradient (Eq. t-junction-ghost-values) at
    # an offset fine face, so the per-volume error stays O(1) but must not grow as h
    # shrinks (a wrong ghost weight grows like 1/h there)
    reg_err, t_max = [], []
    for n0 in (8, 16, 32):
        p = _neumann(P.two_level_ball(n0))
        H, _ = _hier(p)
        t = H.tree
        L = t.leaves
        h = 1.0 / (n0 * 2.0 ** L["depth"])
        x = (L["i"] + 0.5) * h; y = (L["j"] + 0.5) * h; z = (L["k"] + 0.5) * h
        r2 = x * x + y * y + z * z
        f = r2 * np.exp(-x * y * z)
        lap = np.exp(-x * y * z) * (6 - 12 * x * y * z + r2 * (y * y * z * z + x * x * z * z + x * x * y * y))
        e = (H.A @ f) / h ** 3 + lap
        kind, _ = t.neighbour_table()
        tcell = ((kind == O.COARSER) | (kind == O.FINER)).any(axis=1)
        inside = (x > 0.1) & (x < 0.9) & (y > 0.1) & (y < 0.9) & (z > 0.1) & (z < 0.9)
        reg = inside & ~tcell
        V = h ** 3
        reg_err.append(math.sqrt(np.sum(V[reg] * e[reg] ** 2) / np.sum(V[reg])))
        t_max.append(np.abs(e[tcell]).max())
    rates = [math.log2(reg_err[i] / reg_err[i + 1]) for i in range(2)]
    assert min(rates) > 1.8, reg_err
    assert t_max[2] < 1.2 * t_max[1] and t_max[1] < 1.2 * t_max[0], t_max
