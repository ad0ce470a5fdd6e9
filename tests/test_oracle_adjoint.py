"""Pins for the oracle adjoint (oracle/adjoint.py): the per-face gradient formula against
the beta-derivative of the assembled composite operator, and the full gradients against
central finite differences of dense solves."""
import numpy as np
import pytest

from oracle import adjoint as ADJ
from oracle import mg
from oracle import octree as O
from oracle import operator as OP
from oracle import pcg
from paper_2604_18886_b300 import problems as P


def _tree(p):
    t = O.Octree(p.desc)
    f = t.faces()
    return t, f, P.face_beta(p, f)


def _face_classes(H):
    """Indices of regular faces, T faces with the fine leaf on the - side and on the +
    side, and T faces whose fine leaf has a refined sibling (a_P reaches deeper)."""
    f, L = H.faces, H.tree.leaves
    dm, dp = L["depth"][f["minus"]], L["depth"][f["plus"]]
    reg = np.nonzero(dm == dp)[0]
    tm = np.nonzero((dm != dp) & (dm == f["depth"]))[0]
    tp = np.nonzero((dm != dp) & (dp == f["depth"]))[0]
    deep = []
    for q in np.concatenate([tm, tp]):
        fine = f["minus"][q] if dm[q] == f["depth"][q] else f["plus"][q]
        lv = H.levels[f["depth"][q] - 1]
        Pi = lv.index(L["i"][fine] // 2, L["j"][fine] // 2, L["k"][fine] // 2)
        if np.any(~H.levels[f["depth"][q]].leaf[lv.children[Pi]]):
            deep.append(q)
    return reg, tm, tp, np.asarray(deep, np.int64)


@pytest.mark.parametrize("name", ["ball_dirichlet", "cut_neumann"])
def test_face_grad_equals_assembled_beta_derivative(name):
    # A is affine in beta with a fixed active set, so (A(beta + e_f / 2) - A(beta)) * 2 is
    # dA/dbeta_f up to rounding; -lambda^T (that matrix) p must equal the closed form.
    p = P.two_level_ball(6) if name == "ball_dirichlet" else P.cut_cell(6, 2)
    t, f, beta = _tree(p)
    if name == "ball_dirichlet":
        beta = np.random.default_rng(11).uniform(0.2, 1.0, len(beta)).astype(np.float32)
    H = OP.Hierarchy(t, beta, p.bc)
    rng = np.random.default_rng(12)
    pv = rng.normal(size=t.n_leaves)
    lam = rng.normal(size=t.n_leaves)
    g = ADJ.face_grad(H, pv, lam)
    reg, tm, tp, deep = _face_classes(H)
    assert len(tm) and len(tp)
    if name == "cut_neumann":
        assert len(deep)
    pick = []
    for cls in (reg, tm, tp, deep):
        if len(cls):
            pick.extend(rng.choice(cls, size=min(8, len(cls)), replace=False).tolist())
    scale = np.abs(g).max()
    for q in pick:
        b2 = np.asarray(beta, np.float64).copy()
        b2[q] += 0.5
        dA = (OP.Hierarchy(t, b2, p.bc).A - H.A) * 2.0
        ref = -(lam @ (dA @ pv))
        assert abs(ref - g[q]) <= 1e-12 * scale, (q, ref, g[q])


def _fd_problem(name):
    if name == "dirichlet":
        p = P.two_level_ball(4)
    else:
        p = P.cut_cell(4, 1)
    t, f, beta = _tree(p)
    H = OP.Hierarchy(t, beta, p.bc)
    b = P.rhs(p, t.leaves, f, beta)
    pt = np.random.default_rng(2).normal(size=t.n_leaves)
    return p, t, beta, H, b, pt


@pytest.mark.parametrize("name", ["dirichlet", "neumann"])
def test_gradients_match_central_differences(name):
    p, t, beta, H, b, pt = _fd_problem(name)
    x, lam, gb, gbeta = ADJ.gradients(H, b, pt, method="direct")
    rng = np.random.default_rng(3)
    # dL/dbeta: central differences with eps = 1e-3 beta_f; L+ - L- evaluated as
    # 1/2 <p+ - p-, p+ + p- - 2 p_t> so that the large common part cancels exactly
    reg, tm, tp, _ = _face_classes(H)
    faces = np.concatenate([rng.choice(c, size=min(6, len(c)), replace=False) for c in (reg, tm, tp)])
    scale = np.abs(gbeta).max()
    for q in faces:
        eps = 1e-3 * float(beta[q])
        sols = []
        for s in (+1.0, -1.0):
            b2 = np.asarray(beta, np.float64).copy()
            b2[q] += s * eps
            H2 = OP.Hierarchy(t, b2, p.bc)
            sols.append(ADJ.solve(H2, b, method="direct"))
        dl = 0.5 * (sols[0] - sols[1]) @ (sols[0] + sols[1] - 2.0 * pt)
        fd = dl / (2.0 * eps)
        assert abs(fd - gbeta[q]) <= 1e-6 * scale + 1e-4 * abs(gbeta[q]), (q, fd, gbeta[q])
    # dL/db: L is quadratic in b, so central differences are exact up to rounding
    for j in rng.choice(t.n_leaves, size=6, replace=False):
        e = np.zeros(t.n_leaves)
        e[j] = 1e-3
        pp = ADJ.solve(H, b + e, method="direct")
        pm = ADJ.solve(H, b - e, method="direct")
        fd = 0.5 * (pp - pm) @ (pp + pm - 2.0 * pt) / 2e-3
        assert abs(fd - gb[j]) <= 1e-8 * np.abs(gb).max(), (j, fd, gb[j])


def test_adjoint_is_the_transpose_solve():
    # <g, A^{-1} b> = <A^{-T} g, b>: the adjoint identity with a non-symmetric A
    p, t, beta, H, b, pt = _fd_problem("dirichlet")
    A = H.A.toarray()
    assert np.abs(A - A.T).max() > 1e-3          # T junctions make A non-symmetric
    g = np.random.default_rng(4).normal(size=t.n_leaves)
    x = ADJ.solve(H, b, method="direct")
    lam = ADJ.solve(H, g, transpose=True, method="direct")
    assert abs(g @ x - lam @ b) <= 1e-11 * np.abs(g).sum() * np.abs(x).max()
    # preconditioned BiCGStab with the forward cycle reaches the transpose solution
    lam_k, k, _ = pcg.bicgstab(H, g, tol=1e-12, max_iter=200, transpose=True)
    assert np.abs(lam_k - lam).max() <= 1e-9 * np.abs(lam).max()
    assert k < 20
    # ... while Alg. 1 with that cycle stagnates on A^T (the reason for BiCGStab)
    _, k_cg, hist = pcg.pcg(H, g, tol=1e-12, max_iter=60, transpose=True)
    assert k_cg == 60 and hist[-1] > 1e-6


@pytest.mark.parametrize("name", ["dirichlet", "neumann", "cut"])
def test_bicgstab_matches_dense_solve(name):
    if name == "dirichlet":
        p = P.two_level_ball(6)
    elif name == "neumann":
        p = P.two_level_ball(6)
        p.bc = (P.NEUMANN,) * 6
    else:
        p = P.cut_cell(6, 2)
    t, f, beta = _tree(p)
    H = OP.Hierarchy(t, beta, p.bc)
    g = np.random.default_rng(6).normal(size=t.n_leaves)
    for transpose in (False, True):
        x, k, hist = pcg.bicgstab(H, g, tol=1e-12, max_iter=100, transpose=transpose)
        xd = pcg.direct_solve(H, g, transpose=transpose)
        if H.nullspace:
            x = x - x.mean()
        assert np.abs(x - xd).max() <= 1e-9 * np.abs(xd).max()
        assert k < 20 and hist[-1] <= 1e-12


def test_neumann_gradients_ignore_constants():
    # adding a constant to p or lambda leaves every face gradient unchanged
    p, t, beta, H, b, pt = _fd_problem("neumann")
    rng = np.random.default_rng(5)
    pv, lam = rng.normal(size=t.n_leaves), rng.normal(size=t.n_leaves)
    g0 = ADJ.face_grad(H, pv, lam)
    g1 = ADJ.face_grad(H, pv + 3.0, lam - 2.0)
    assert np.abs(g0 - g1).max() <= 1e-12 * np.abs(g0).max()


@pytest.mark.parametrize("mu", [1, 2])
@pytest.mark.parametrize("make", [lambda: P.two_level_ball(8), lambda: P.cut_cell(8, 2), lambda: P.sine_band(8, 2)])
def test_transposed_cycle_is_the_transpose(make, mu):
    """mg.vcycle_T is the exact transpose of the cycle: <M r1, r2> = <r1, M^T r2>."""
    p = make()
    t = O.Octree(p.desc)
    f = t.faces()
    H = OP.Hierarchy(t, P.face_beta(p, f), p.bc)
    prm = mg.CycleParams(mu=mu)
    for s in range(3):
        r1 = P.random_vector(t.n_leaves, 50 + s)
        r2 = P.random_vector(t.n_leaves, 60 + s)
        a = mg.vcycle(H, r1, prm) @ r2
        b = r1 @ mg.vcycle_T(H, r2, prm)
        assert abs(a - b) <= 1e-12 * abs(a) * 10, (a, b)


def _bordered_transpose_solve(H, g):
    """Zero-mean solution of A^T x = g (g shifted to zero mean) by a sparse direct solve of
    the system bordered with the constant null vector."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    n = H.A.shape[0]
    one = sp.csr_matrix(np.ones((n, 1)))
    K = sp.bmat([[H.A.T.tocsr(), one], [one.T, None]]).tocsc()
    rhs = np.concatenate([g - g.mean(), [0.0]])
    return sla.spsolve(K, rhs)[:n]


def test_transposed_cycle_rescues_the_high_contrast_adjoint():
    """On an under-resolved sine-band tree (beta clamped at 1e-3 on a third of the faces)
    BiCGStab on A^T preconditioned by the forward cycle diverges; with the transposed
    cycle it converges to the direct solution."""
    p = P.sine_band(8, 2)
    t = O.Octree(p.desc)
    H = OP.Hierarchy(t, P.face_beta(p, t.faces()), p.bc)
    g = P.random_vector(t.n_leaves, 23)
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        _, kf, hf = pcg.bicgstab(H, g, tol=1e-6, transpose=True, max_iter=60)
    assert not (hf[-1] <= 1e-6)
    x, k, h = pcg.bicgstab(H, g, tol=1e-10, transpose=True, precond="transposed", max_iter=60)
    assert h[-1] <= 1e-10 and k <= 25
    ref = _bordered_transpose_solve(H, g)
    assert np.abs((x - x.mean()) - ref).max() <= 1e-7 * np.abs(ref).max()


@pytest.mark.parametrize("make", [lambda: P.sine_band(8, 2), lambda: P.cut_cell(8, 2), lambda: P.two_level_ball(8)])
def test_alg1_on_the_transpose_with_the_transposed_cycle(make):
    """Alg. 1 on A^T preconditioned by M^T reaches the direct transpose solution, in about
    as many iterations as BiCGStab with M^T needs preconditioner applications or fewer."""
    p = make()
    t = O.Octree(p.desc)
    H = OP.Hierarchy(t, P.face_beta(p, t.faces()), p.bc)
    g = P.random_vector(t.n_leaves, 23)
    x, k, h = pcg.pcg(H, g, tol=1e-10, transpose=True, precond="transposed", max_iter=60)
    assert h[-1] <= 1e-10 and k <= 30
    if H.nullspace:
        ref = _bordered_transpose_solve(H, g)
        x = x - x.mean()
    else:
        import scipy.sparse.linalg as sla
        ref = sla.spsolve(H.A.T.tocsc(), g)
    assert np.abs(x - ref).max() <= 1e-7 * np.abs(ref).max()
    _, kb, _ = pcg.bicgstab(H, g, tol=1e-6, transpose=True, precond="transposed", max_iter=60)
    _, kp, _ = pcg.pcg(H, g, tol=1e-6, transpose=True, precond="transposed", max_iter=60)
    assert kp <= 2 * kb
