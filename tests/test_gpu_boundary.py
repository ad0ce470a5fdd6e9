"""Boundary features of the C ABI: warm start (OCG_SOLVE_WARM) and the device-allocation
hooks (ocg_set_allocator) with torch's caching allocator."""
import numpy as np
import pytest

from paper_2604_18886_b300 import problems as P
from paper_2604_18886_b300 import solver as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _c3():
    p = P.cut_cell(16, 2)
    g = S.Octree(p.desc)
    f = g.faces()
    beta = P.face_beta(p, f)
    b = torch.from_numpy(P.rhs(p, g.leaves(), f, beta)).cuda()
    return p, g, beta, b


@pytest.mark.parametrize("transpose, method", [(False, "pcg"), (True, "pcg"), (True, "bicgstab")])
@pytest.mark.parametrize("eager", [False, True])
def test_warm_start(transpose, method, eager):
    p, g, beta, b = _c3()
    h = S.Hierarchy(g, beta, p.bc, S.mg_params(coef="f32", sweep="octet"))
    kw = dict(precision="mixed", transpose=transpose, method=method, eager=eager, max_iter=100)
    x_ref, s_ref = h.solve(b, tol=1e-10, **kw)
    # from a rough iterate: fewer iterations to the same tolerance, the same solution
    x0, s0 = h.solve(b, tol=1e-3, **kw)
    x = x0.clone()
    _, sw = h.solve(b, x, tol=1e-10, warm=True, **kw)
    assert sw.converged and sw.true_rel_res <= 2e-10
    assert sw.iterations < s_ref.iterations
    # two solutions to relative residual 1e-10 of a cut-cell system (beta down to 1e-3):
    # they agree to the conditioning times the tolerance (measured 1.1e-8)
    assert (x - x_ref).abs().max().item() <= 1e-7 * x_ref.abs().max().item()
    # from the converged solution: one iteration suffices
    x = x_ref.clone()
    _, s1 = h.solve(b, x, tol=1e-9, warm=True, **kw)
    assert s1.converged and s1.iterations <= 1


def test_torch_allocator_hooks():
    p, g0, beta, b = _c3()
    ref = S.Hierarchy(g0, beta, p.bc, S.mg_params(coef="f32", sweep="octet"))
    x_ref, _ = ref.solve(b, tol=1e-8)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    S.use_torch_allocator(True)
    try:
        g = S.Octree(p.desc)
        h = S.Hierarchy(g, beta, p.bc, S.mg_params(coef="f32", sweep="octet"))
        x, st = h.solve(b, tol=1e-8)
        torch.cuda.synchronize()
        held = torch.cuda.memory_allocated() - base
        assert held > 8 * g.n_cells          # the hierarchy's buffers came from torch
        assert torch.equal(x, x_ref)
        del h, g
        import gc
        gc.collect()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() - base <= x.numel() * 8 + 4096
    finally:
        S.use_torch_allocator(False)
    # blocks made by cudaMalloc before and after the hooks are unaffected
    h2 = S.Hierarchy(g0, beta, p.bc, S.mg_params(coef="f32", sweep="octet"))
    x2, _ = h2.solve(b, tol=1e-8)
    assert torch.equal(x2, x_ref)
