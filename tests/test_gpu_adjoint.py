"""GPU parity of the adjoint path (transposed operator, BiCGStab transpose solve, face
gradient, autograd wrapper) against the FP64 oracle, and the gradient against central
finite differences at the full two-level workload size.

Tolerances as in test_gpu_parity: FP64 applies 1e-12, FP32 applies 1e-6 relative to the
vector's max norm; the transposed cycle M^T as the forward cycle (FP64 1e-10, FP32 1e-5);
FP64 Krylov iterates 1e-8 (BiCGStab's two-sided recurrences amplify rounding-order
differences more than CG's).  Gradients face by face: against the oracle's gradient
within the change that the measured entry errors of p and lambda can cause (grad_bound);
against central finite differences within 1e-4 of each face's own finite difference, plus
that difference's derived solver-error bound (fd_check).  The adjoint solves are preconditioned by M^T (Alg. 1 on A^T by default,
BiCGStab on request), so the oracle's solvers run with precond="transposed".
"""
import numpy as np
import pytest

from oracle import adjoint as ADJ
from oracle import pcg
from paper_2604_18886_b300 import problems as P
from paper_2604_18886_b300 import solver as S

from test_gpu_parity import CASES, build, cuda, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NAMES = ["ball_16", "ball_16_neumann", "cut_16_d2", "batch_t1", "band_12_d2", "sine_8_d2"]


@pytest.mark.parametrize("name", NAMES)
def test_transposed_apply_matches_oracle(name):
    t, H, g, gh, f, beta = build(CASES[name](), "f64")
    x = P.random_vector(t.n_leaves, 21)
    AT = H.A.T.tocsr()
    y = gh.apply_A(cuda(x), transpose=True).cpu().numpy()
    assert rel(y, AT @ x) <= 1e-12
    # A^T differs from A exactly where T-junctions are
    yf = gh.apply_A(cuda(x)).cpu().numpy()
    assert rel(yf, H.A @ x) <= 1e-12
    t, H, g, gh, f, beta = build(CASES[name](), "f32")
    x32 = x.astype(np.float32)
    y32 = gh.apply_A(cuda(x32, torch.float32), transpose=True).double().cpu().numpy()
    assert rel(y32, AT @ x32.astype(np.float64)) <= 1e-6


@pytest.mark.parametrize("mu", [1, 2])
@pytest.mark.parametrize("name", NAMES)
def test_vcycle_transpose_fp64_matches_oracle(name, mu):
    from oracle import mg
    t, H, g, gh, f, beta = build(CASES[name](), "f64", mu=mu)
    z = P.random_vector(t.n_leaves, 30)
    r = gh.vcycle_transpose(cuda(z)).cpu().numpy()
    assert rel(r, mg.vcycle_T(H, z, mg.CycleParams(mu=mu))) <= 1e-10


@pytest.mark.parametrize("name", NAMES)
def test_vcycle_transpose_fp32_matches_oracle(name):
    from oracle import mg
    t, H, g, gh, f, beta = build(CASES[name](), "f32")
    z = P.random_vector(t.n_leaves, 31).astype(np.float32)
    r = gh.vcycle_transpose(cuda(z, torch.float32)).double().cpu().numpy()
    assert rel(r, mg.vcycle_T(H, z.astype(np.float64))) <= 1e-5


@pytest.mark.parametrize("name", ["cut_16_d2", "band_12_d2", "sine_8_d2"])
def test_vcycle_transpose_hybrid_matches_oracle(name):
    from oracle import mg
    t, H, g, gh, f, beta = build(CASES[name](), "f64", mu=2, mu_min=4096)
    z = P.random_vector(t.n_leaves, 32)
    r = gh.vcycle_transpose(cuda(z)).cpu().numpy()
    assert rel(r, mg.vcycle_T(H, z, mg.CycleParams(mu=2, mu_min_cells=4096))) <= 1e-10


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("name", ["cut_16_d2", "sine_8_d2"])
def test_vcycle_transpose_is_the_adjoint_of_the_gpu_cycle(name, bf16):
    # (M^T z, r) = (z, M r) for the library's own M, in FP64 and in FP32 (also with the
    # BF16 coarse coefficients, where no oracle cycle exists)
    t, H, g, gh, f, beta = build(CASES[name](), "f64")
    r = P.random_vector(t.n_leaves, 33)
    z = P.random_vector(t.n_leaves, 34)
    lhs = float(np.dot(gh.vcycle_transpose(cuda(z)).cpu().numpy(), r))
    rhs = float(np.dot(z, gh.vcycle(cuda(r)).cpu().numpy()))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-300) * t.n_leaves ** 0.5
    t, H, g, gh, f, beta = build(CASES[name](), "f32", bf16=bf16)
    r32 = cuda(r, torch.float32)
    z32 = cuda(z, torch.float32)
    lhs = torch.dot(gh.vcycle_transpose(z32).double(), r32.double()).item()
    rhs = torch.dot(z32.double(), gh.vcycle(r32).double()).item()
    scale = gh.vcycle_transpose(z32).double().norm().item() * r32.double().norm().item()
    assert abs(lhs - rhs) <= 1e-5 * scale


@pytest.mark.parametrize("name", ["ball_16", "ball_16_neumann", "cut_16_d2", "batch_t1", "sine_8_d2"])
def test_alg1_transpose_fp64_follows_oracle_iterates(name):
    # Alg. 1 on A^T with M^T (the default adjoint method)
    t, H, g, gh, f, beta = build(CASES[name](), "f64")
    rhs = P.random_vector(t.n_leaves, 22)
    xo, ko, ho = pcg.pcg(H, rhs, tol=1e-8, transpose=True, precond="transposed")
    x, st = gh.solve(cuda(rhs), tol=1e-8, precision="fp64", transpose=True)
    assert st.converged and st.iterations == ko
    hist = [st.hist[i] for i in range(st.iterations + 1)]
    assert np.allclose(hist, ho, rtol=1e-7, atol=0)
    if H.nullspace:
        assert abs(x.mean().item()) <= 1e-12 * x.abs().max().item()
        xo = xo - xo.mean()
    assert rel(x.cpu().numpy(), xo) <= 1e-9


@pytest.mark.parametrize("name", ["ball_16", "ball_16_neumann", "cut_16_d2", "batch_t1", "sine_8_d2"])
def test_bicgstab_fp64_follows_oracle_iterates(name):
    t, H, g, gh, f, beta = build(CASES[name](), "f64")
    rhs = P.random_vector(t.n_leaves, 22)
    xo, ko, ho = pcg.bicgstab(H, rhs, tol=1e-8, transpose=True, precond="transposed")
    x, st = gh.solve(cuda(rhs), tol=1e-8, precision="fp64", transpose=True, method="bicgstab")
    assert st.converged and st.iterations == ko
    hist = [st.hist[i] for i in range(st.iterations + 1)]
    assert np.allclose(hist, ho, rtol=1e-6, atol=0)
    if H.nullspace:
        xo = xo - xo.mean()
    assert rel(x.cpu().numpy(), xo) <= 1e-8


@pytest.mark.parametrize("method", ["pcg", "bicgstab"])
@pytest.mark.parametrize("precision", ["mixed", "fp32"])
@pytest.mark.parametrize("name", ["ball_16", "ball_16_neumann", "cut_16_d2", "batch_t1", "sine_8_d2"])
def test_transpose_solution_within_1e5(name, precision, method):
    t, H, g, gh, f, beta = build(CASES[name](), "f32")
    rhs = P.random_vector(t.n_leaves, 23)
    ref = ADJ.solve(H, rhs, transpose=True, tol=1e-12)
    if method == "pcg":
        xo, ko, _ = pcg.pcg(H, rhs, tol=1e-6, transpose=True, precond="transposed")
    else:
        xo, ko, _ = pcg.bicgstab(H, rhs, tol=1e-6, transpose=True, precond="transposed")
    if H.nullspace:
        xo = xo - xo.mean()
    x, st = gh.solve(cuda(rhs), tol=1e-6, precision=precision, transpose=True, method=method)
    x = x.cpu().numpy()
    assert st.converged and st.rel_res <= 1e-6 and abs(st.iterations - ko) <= 1
    if H.nullspace:
        assert abs(x.mean()) <= 1e-12 * np.abs(x).max()
    assert rel(x, ref) <= 1.5 * rel(xo, ref) + 1e-5, (rel(x, ref), rel(xo, ref))
    if precision == "mixed":
        assert st.true_rel_res <= 1.5e-6
        x9, st9 = gh.solve(cuda(rhs), tol=1e-9, precision="mixed", transpose=True, method=method)
        assert st9.converged and st9.true_rel_res <= 2e-9
        assert rel(x9.cpu().numpy(), ref) <= 1e-5


@pytest.mark.parametrize("name", NAMES)
def test_face_grad_matches_oracle(name):
    t, H, g, gh, f, beta = build(CASES[name](), "f32")
    p = P.random_vector(t.n_leaves, 24)
    lam = P.random_vector(t.n_leaves, 25)
    ref = ADJ.face_grad(H, p, lam)
    out = gh.face_grad(cuda(p), cuda(lam)).cpu().numpy()
    assert out.shape == ref.shape
    assert rel(out, ref) <= 1e-12


@pytest.mark.parametrize("method", ["pcg", "bicgstab"])
def test_graph_and_eager_transpose_solves_agree(method):
    t, H, g, gh, f, beta = build(CASES["cut_16_d2"](), "f32")
    rhs = cuda(P.random_vector(t.n_leaves, 26))
    xg, sg = gh.solve(rhs, tol=1e-6, precision="mixed", transpose=True, method=method)
    xe, se = gh.solve(rhs, tol=1e-6, precision="mixed", transpose=True, eager=True, method=method)
    assert torch.equal(xg, xe) and sg.iterations == se.iterations and sg.kernels == se.kernels


def grad_bound(coef, dlam, dp, e_p, e_lam):
    """Largest change of -coef * dlam * dp per face when every entry of p moves by at most
    e_p and every entry of lambda by at most e_lam: each face factor is a difference of two
    values (dp of a T sub-face: a mean of children minus a value), so it moves by at most
    twice the entry bound.  Rounding of the FP64 products is added at 1e-13 relative."""
    a = np.abs(coef)
    return a * (np.abs(dlam) * 2 * e_p + np.abs(dp) * 2 * e_lam + 4 * e_p * e_lam) + \
        1e-13 * a * (np.abs(dlam) + 2 * e_lam) * (np.abs(dp) + 2 * e_p)


@pytest.mark.parametrize("name", ["ball_16", "cut_16_d2"])
def test_autograd_matches_oracle_gradients(name):
    # per element: the solution p and dL/db = lambda against the oracle within the solve's
    # 1e-5 bar (max norm); dL/dbeta face by face within the change that the measured
    # entry errors of p and lambda can cause through the face formula (grad_bound), which
    # is far below 1e-4 of each face's gradient unless the face's gradient nearly vanishes
    from paper_2604_18886_b300.autograd import poisson_solve
    p = CASES[name]()
    t, H, g, gh, f, beta = build(p, "f32")
    b = P.rhs(p, t.leaves, f, beta)
    pt = P.random_vector(t.n_leaves, 2)
    x_o, lam_o, gb_o, gbeta_o = ADJ.gradients(H, b, pt)
    bt = cuda(b).requires_grad_(True)
    betat = cuda(beta, torch.float32).requires_grad_(True)
    x = poisson_solve(bt, betat, g, p.bc, tol=1e-12, precision="mixed", max_iter=400)
    loss = 0.5 * ((x - cuda(pt)) ** 2).sum()
    loss.backward()
    xg = x.detach().cpu().numpy()
    lg = bt.grad.cpu().numpy()
    assert rel(xg, x_o) <= 1e-5
    assert rel(lg, gb_o) <= 1e-5
    e_p = np.abs(xg - x_o).max()
    e_l = np.abs(lg - lam_o).max()
    coef, dlam, dp = ADJ.face_factors(H, x_o, lam_o)
    got = betat.grad.double().cpu().numpy()
    err = np.abs(got - gbeta_o)
    # dL/dbeta comes back in beta's dtype (float32): one rounding to 24 bits on top
    bound = grad_bound(coef, dlam, dp, e_p, e_l)
    bound = bound + 2.0 ** -24 * (np.abs(gbeta_o) + bound)
    gmag = np.maximum(np.abs(gbeta_o), 1e-300)  # faces with no gradient at all divide by a tiny floor
    worst = np.argsort(err / gmag)[-5:]
    print("faces %d, e_p %.2e, e_lambda %.2e; largest per-face relative errors:" % (len(got), e_p, e_l),
          ["%.2e (bound %.2e, |g| %.2e)" % (err[q] / gmag[q], bound[q] / gmag[q], abs(gbeta_o[q]))
           for q in worst])
    assert np.all(err <= bound), (err - bound).max()
    # the bound is tight enough to mean something: 1e-4 of the face's gradient or better on
    # nearly every face (it exceeds that only where a face's difference of p or lambda
    # nearly vanishes)
    tight = np.mean(bound <= 1e-4 * np.abs(gbeta_o))
    print("faces with a bound within 1e-4 of their gradient: %.4f" % tight)
    assert tight >= 0.95


def _difference_fd(hs, beta, fi, x0, Ax0, g0, lam_norm, eps_rel, tol=1e-12):
    """Central finite difference of L = 1/2 ||p - p_t||^2 in beta_f (face fi) at step
    eps_rel * beta_f, and a bound on its solver error.

    p(beta +- eps) - p(beta) is solved for directly, A(beta +- eps) dp = A(beta) p -
    A(beta +- eps) p (an identity, not a linearisation), so the difference carries the
    solver's relative accuracy instead of the cancellation of two full solutions, and
        L+ - L- = <dp+ - dp-, g0 + (dp+ + dp-)/2>,   g0 = p - p_t.
    A dp solve that stops at residual res moves L by <A'^{-1} res, g0 + dp> =
    <res, A'^{-T}(p' - p_t)>, at most ||res|| ||lambda'|| (lambda' the perturbed system's
    adjoint solution, within a few eps of lambda); hence the bound
    (||res+|| + ||res-||) * 1.01 ||lambda|| / (eps+ + eps-)."""
    b0 = float(beta[fi])
    eps = eps_rel * b0
    dps, epss, noise = [], [], 0.0
    for sgn in (1.0, -1.0):
        bb = beta.clone()
        bb[fi] = float(np.float32(b0 + sgn * eps))
        epss.append(abs(float(bb[fi]) - b0))
        hs.update_beta(bb)
        rhs = Ax0 - hs.apply_A(x0)
        dp, st = hs.solve(rhs, tol=tol, precision="fp64", max_iter=300)
        assert st.converged
        noise += st.true_rel_res * rhs.norm().item()
        dps.append(dp)
    dl = torch.dot(dps[0] - dps[1], g0 + 0.5 * (dps[0] + dps[1])).item()
    den = epss[0] + epss[1]
    return dl / den, noise * 1.01 * lam_norm / den


def fd_check(g, beta, bc, b, pt, faces, kinds, prm):
    """Gradient of L = 1/2 ||p - p_t||^2 with respect to the face fractions of `faces`
    against central finite differences, face by face: Richardson's combination of the
    steps 1e-3 beta_f and 5e-4 beta_f (its truncation error is O(eps^4)) must agree with
    the adjoint gradient within 1e-4 of its own magnitude, plus the finite difference's
    solver-error bound (_difference_fd).  Returns the per-face table."""
    h0 = S.Hierarchy(g, beta, bc, prm)
    x0, st = h0.solve(b, tol=1e-12, precision="fp64", max_iter=300)
    assert st.converged
    g0 = x0 - pt
    if h0.nullspace:
        g0 = g0 - g0.mean()
    lam, st = h0.solve(g0, tol=1e-12, precision="fp64", max_iter=300, transpose=True)
    assert st.converged
    grad = h0.face_grad(x0, lam)[torch.from_numpy(np.asarray(faces)).cuda()].cpu().numpy()
    Ax0 = h0.apply_A(x0)
    hs = S.Hierarchy(g, beta, bc, prm)
    lam_norm = lam.norm().item()
    rows = []
    for q, fi in enumerate(faces):
        f1, n1 = _difference_fd(hs, beta, int(fi), x0, Ax0, g0, lam_norm, 1e-3)
        f2, n2 = _difference_fd(hs, beta, int(fi), x0, Ax0, g0, lam_norm, 5e-4)
        fdr = (4.0 * f2 - f1) / 3.0
        noise = (4.0 * n2 + n1) / 3.0
        err = abs(fdr - grad[q])
        rows.append((int(fi), kinds[q], float(beta[int(fi)]), grad[q], fdr, err / abs(fdr), noise / abs(fdr),
                     abs(f1 - fdr) / abs(fdr)))
    print("face kind beta grad fd rel_err noise_bound/|fd| O(eps^2)_term/|fd|")
    for r in rows:
        print("%d %s %.4g %.6e %.6e %.2e %.2e %.2e" % r)
    for r in rows:
        assert abs(r[3] - r[4]) <= 1e-4 * abs(r[4]) + r[6] * abs(r[4]), r
    return rows


def test_gradient_matches_central_differences_full_size():
    # the two-level workload (64^3 root, ball r = 0.25 refined once): L = 1/2 ||p - p_t||^2,
    # p_t ~ N(0,1) (seed 2); 64 interior faces drawn with seed 3, 48 between equal-depth
    # leaves and 16 T sub-faces; FP64 solves to 1e-12
    p = P.two_level_ball(64)
    g = S.Octree(p.desc)
    fc = g.faces()
    beta = cuda(P.face_beta(p, fc), torch.float32)
    lv = g.leaves()
    b = cuda(P.rhs(p, lv, fc, beta.cpu().numpy()))
    pt = cuda(P.random_vector(g.n_leaves, 2))
    dm = lv["depth"][fc["minus"]]
    dp = lv["depth"][fc["plus"]]
    rng = np.random.default_rng(3)
    reg = np.nonzero(dm == dp)[0]
    tf = np.nonzero(dm != dp)[0]
    faces = np.concatenate([rng.choice(reg, 48, replace=False), rng.choice(tf, 16, replace=False)])
    kinds = ["regular"] * 48 + ["T"] * 16
    fd_check(g, beta, p.bc, b, pt, faces, kinds, S.mg_params(coef="f64", sweep="octet"))
