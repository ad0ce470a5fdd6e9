"""In-place refresh of a hierarchy for new face fractions (ocg_hier_update_beta): the
refreshed hierarchy equals one set up from scratch for the new beta, bit for bit, and the
CUDA graph captured by a solve before the refresh runs on the new coefficients.
"""
import numpy as np
import pytest

from paper_2604_18886_b300 import problems as P
from paper_2604_18886_b300 import solver as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _betas(p, g):
    f = g.faces()
    b1 = P.face_beta(p, f)
    rng = np.random.default_rng(80)
    b2 = np.clip(b1 * rng.uniform(0.5, 1.5, len(b1)), 1e-3, 1.0).astype(np.float32)
    return f, b1, b2


@pytest.mark.parametrize("coarsening", ["algebraic", "geometric"])
def test_refreshed_coefficients_equal_a_fresh_set_up(coarsening):
    p = P.cut_cell(16, 2)
    g = S.Octree(p.desc)
    f, b1, b2 = _betas(p, g)
    prm = S.mg_params(coef="f64", sweep="octet", coarsening=coarsening)
    h = S.Hierarchy(g, b1, p.bc, prm)
    h.update_beta(b2)
    fresh = S.Hierarchy(g, b2, p.bc, prm)
    for m in range(g.mc, g.D + 1):
        for a, b in zip(h.coefs(m), fresh.coefs(m)):
            assert np.array_equal(a, b), m


@pytest.mark.parametrize("coef, precision, bf16", [("f64", "fp64", False), ("f32", "mixed", False),
                                                   ("f32", "mixed", True)])
def test_graph_captured_before_the_refresh_solves_the_new_system(coef, precision, bf16):
    p = P.cut_cell(16, 2)
    g = S.Octree(p.desc)
    f, b1, b2 = _betas(p, g)
    b = torch.from_numpy(P.rhs(p, g.leaves(), f, b2)).cuda()
    prm = S.mg_params(coef=coef, sweep="octet", bf16_coarse=bf16)
    h = S.Hierarchy(g, b1, p.bc, prm)
    x1, s1 = h.solve(b, tol=1e-8, precision=precision)     # captures the graph on beta1
    h.update_beta(b2)
    x2, s2 = h.solve(b, tol=1e-8, precision=precision)     # the same graph, beta2
    fresh = S.Hierarchy(g, b2, p.bc, prm)
    x3, s3 = fresh.solve(b, tol=1e-8, precision=precision)
    assert s2.converged and s2.iterations == s3.iterations
    assert torch.equal(x2, x3)
    assert not torch.equal(x1, x2)


def test_rejected_refresh_then_a_valid_one():
    p = P.cut_cell(12, 2)
    g = S.Octree(p.desc)
    f, b1, b2 = _betas(p, g)
    prm = S.mg_params(coef="f64", sweep="octet")
    h = S.Hierarchy(g, b1, p.bc, prm)
    bad = b2.copy()
    bad[3] = -1.0
    with pytest.raises(RuntimeError):
        h.update_beta(bad)
    h.update_beta(b2)
    fresh = S.Hierarchy(g, b2, p.bc, prm)
    for m in range(g.mc, g.D + 1):
        for a, c in zip(h.coefs(m), fresh.coefs(m)):
            assert np.array_equal(a, c), m


def test_autograd_with_a_refreshed_hierarchy_matches_fresh_set_ups():
    from paper_2604_18886_b300.autograd import poisson_solve
    p = P.cut_cell(12, 2)
    g = S.Octree(p.desc)
    f, b1, b2 = _betas(p, g)
    prm = S.mg_params(coef="f32", sweep="octet")
    reuse = S.Hierarchy(g, b1, p.bc, prm)
    pt = torch.from_numpy(P.random_vector(g.n_leaves, 81)).cuda()
    for beta in (b1, b2, b1):
        b = torch.from_numpy(P.rhs(p, g.leaves(), f, beta)).cuda()
        grads = []
        for hier in (None, reuse):
            bt = b.clone().requires_grad_(True)
            betat = torch.from_numpy(beta).cuda().requires_grad_(True)
            x = poisson_solve(bt, betat, g, p.bc, tol=1e-8, precision="mixed", mg=prm, hierarchy=hier)
            (0.5 * ((x - pt) ** 2).sum()).backward()
            grads.append((x.detach(), bt.grad, betat.grad))
        for u, v in zip(grads[0], grads[1]):
            assert torch.equal(u, v)
