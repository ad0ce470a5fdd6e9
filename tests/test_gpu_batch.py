"""GPU parity of the batched solve (ocg_pcg_solve_batched): every problem of a batch
against the FP64 oracle (same bar as the single solves) and against its own single
mixed solve, with V- and W-cycles; converged problems are frozen; incompatible
hierarchies are refused; the 64-tree batched workload at full size against single solves.

Tolerances: the batched solve runs the single solve's arithmetic per problem, but its
reductions sum in another block order and the tail kernel may pick the other sweep form
(different summation order), so results agree to rounding: 1e-6 relative at tol 1e-9.
"""
import numpy as np
import pytest

from oracle import pcg
from paper_2604_18886_b300 import problems as P
from paper_2604_18886_b300 import solver as S

from test_gpu_parity import CASES, build, cuda, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MIX = ["uniform_16", "ball_16", "ball_16_neumann", "cut_16_d2", "batch_t1", "band_12_d2"]


def _rhs(name, t, f, beta):
    p = CASES[name]()
    return P.rhs(p, t.leaves, f, beta)


def _batch(names):
    items = [build(CASES[n](), "f32") for n in names]
    hs = [it[3] for it in items]
    return items, S.Batch(hs)


def test_batched_solutions_match_oracle_and_single_solves():
    items, bt = _batch(MIX)
    bs = [cuda(_rhs(n, it[0], it[4], it[5])) for n, it in zip(MIX, items)]
    xs, stats = bt.solve(bs, tol=1e-6)
    for n, it, b, x, st in zip(MIX, items, bs, xs, stats):
        t, H, g, gh, f, beta = it
        bn = b.cpu().numpy()
        ref, _, _ = pcg.pcg(H, bn, tol=1e-12, max_iter=200)
        xo, ko, _ = pcg.pcg(H, bn, tol=1e-6)
        if H.nullspace:
            ref = ref - ref.mean()
            xo = xo - xo.mean()
        xb = x.cpu().numpy()
        assert st.converged and st.rel_res <= 1e-6 and st.true_rel_res <= 1.5e-6, n
        assert abs(st.iterations - ko) <= 1, (n, st.iterations, ko)
        assert rel(xb, ref) <= 1.5 * rel(xo, ref) + 1e-5, (n, rel(xb, ref), rel(xo, ref))
        xs1, s1 = gh.solve(b, tol=1e-6, precision="mixed")
        assert abs(s1.iterations - st.iterations) <= 1, n
    # tight tolerance: the batched and single solves agree to rounding
    xs9, st9 = bt.solve(bs, tol=1e-9)
    for n, it, b, x, st in zip(MIX, items, bs, xs9, st9):
        x1, s1 = it[3].solve(b, tol=1e-9, precision="mixed")
        assert st.converged and abs(st.iterations - s1.iterations) <= 1, n
        assert rel(x.cpu().numpy(), x1.cpu().numpy()) <= 1e-6, n


def test_converged_problems_are_frozen():
    names = ["ball_16", "cut_16_d2"]
    items, bt = _batch(names)
    b0 = cuda(np.zeros(items[0][0].n_leaves))          # converged before the first iteration
    b1 = cuda(_rhs(names[1], items[1][0], items[1][4], items[1][5]))
    xs, stats = bt.solve([b0, b1], tol=1e-8)
    assert stats[0].converged and stats[0].iterations <= 1
    assert torch.count_nonzero(xs[0]).item() == 0
    x1, s1 = items[1][3].solve(b1, tol=1e-8, precision="mixed")
    assert stats[1].converged and abs(stats[1].iterations - s1.iterations) <= 1
    assert stats[1].iterations > stats[0].iterations
    assert rel(xs[1].cpu().numpy(), x1.cpu().numpy()) <= 1e-6


def test_batched_w_cycles_match_oracle_and_single_solves():
    # mu = 2 for every problem: the batch's schedule, aligned at the finest levels, visits
    # each problem's coarser levels as its own W-cycle does (Alg. 4)
    from oracle import mg
    items = [build(CASES[n](), "f32", mu=2) for n in MIX]
    bt = S.Batch([it[3] for it in items])
    bs = [cuda(_rhs(n, it[0], it[4], it[5])) for n, it in zip(MIX, items)]
    xs, stats = bt.solve(bs, tol=1e-6)
    for n, it, b, x, st in zip(MIX, items, bs, xs, stats):
        t, H, g, gh, f, beta = it
        bn = b.cpu().numpy()
        ref, _, _ = pcg.pcg(H, bn, tol=1e-12, max_iter=200, prm=mg.CycleParams(mu=2))
        xo, ko, _ = pcg.pcg(H, bn, tol=1e-6, prm=mg.CycleParams(mu=2))
        if H.nullspace:
            ref = ref - ref.mean()
            xo = xo - xo.mean()
        assert st.converged and st.true_rel_res <= 1.5e-6, n
        assert abs(st.iterations - ko) <= 1, (n, st.iterations, ko)
        assert rel(x.cpu().numpy(), ref) <= 1.5 * rel(xo, ref) + 1e-5, n
    xs9, st9 = bt.solve(bs, tol=1e-9)
    for n, it, b, x, st in zip(MIX, items, bs, xs9, st9):
        x1, s1 = it[3].solve(b, tol=1e-9, precision="mixed")
        assert st.converged and abs(st.iterations - s1.iterations) <= 1, (n, st.iterations, s1.iterations)
        assert rel(x.cpu().numpy(), x1.cpu().numpy()) <= 1e-6, n


def test_batch_refuses_incompatible_hierarchies():
    from paper_2604_18886_b300 import _lib
    p = CASES["ball_16"]()
    g = S.Octree(p.desc)
    beta = P.face_beta(p, g.faces())
    ok = S.Hierarchy(g, beta, p.bc, S.mg_params(coef="f32"))
    for bad in (S.mg_params(coef="f32", mu=2), S.mg_params(coef="f32", bf16_coarse=True), S.mg_params(coef="f64"),
                S.mg_params(coef="f32", mu=2, mu_min_cells=4096)):
        h = S.Hierarchy(g, beta, p.bc, bad)
        with pytest.raises(_lib.OcgError) as e:
            S.Batch([ok, h])
        assert e.value.code == _lib.OCG_EINVAL
    with pytest.raises(_lib.OcgError):
        S.Batch([ok, ok])


def test_batched_64_trees_full_size():
    # the batched workload: 64 trees (effective 64/96/128, 2-3 levels, random sphere
    # band; even k Dirichlet beta = 1, odd k cut-cell Neumann), rhs N(0,1)
    hs, bs, leaves = [], [], 0
    for k in range(64):
        p = P.batch_tree(k)
        g = S.Octree(p.desc)
        f = g.faces()
        beta = P.face_beta(p, f)
        hs.append(S.Hierarchy(g, beta, p.bc, S.mg_params(coef="f32")))
        bs.append(cuda(P.rhs(p, g.leaves(), f, beta)))
        leaves += g.n_leaves
    bt = S.Batch(hs)
    xs, stats = bt.solve(bs, tol=1e-6)
    for k in range(64):
        st = stats[k]
        assert st.converged and st.true_rel_res <= 1.5e-6, (k, st.rel_res, st.true_rel_res)
    for k in (0, 1, 17, 42, 63):
        x1, s1 = hs[k].solve(bs[k], tol=1e-6, precision="mixed")
        assert abs(s1.iterations - stats[k].iterations) <= 1, k
        assert rel(xs[k].cpu().numpy(), x1.cpu().numpy()) <= 1e-4, k
    assert leaves > 5_000_000
