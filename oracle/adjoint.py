"""Oracle adjoint of the composite octree solve (TEST INFRASTRUCTURE).

The paper solves A p = b (Sec. 2.1, Eq. projection-poisson-system, with the T-junction
ghost of Sec. 3.1) but differentiates nothing; the gradients here follow from that
operator alone.  For a loss L(p) with p = A^{-1} b:

    lambda      = A^{-T} dL/dp                     (one solve with the transpose;
                                                    BiCGStab with the same mu-cycle)
    dL/db       = lambda
    dL/dbeta_f  = -lambda^T (dA/dbeta_f) p

A depends linearly on the face fractions beta_f (every face weight is w_f = beta_f h_f;
Dirichlet walls carry beta = 1 and are not inputs), so dA/dbeta_f is the operator of
face f alone with w_f replaced by h_f:

  * a face between two leaves i, j of the same depth adds h (e_i - e_j)(e_i - e_j)^T, so
        dL/dbeta_f = -h (lambda_i - lambda_j)(p_i - p_j);
  * a T sub-face of the fine leaf i against the coarser leaf K adds
    (h/2)(e_i - e_K)(a_P - e_K)^T, where a_P averages the leaves under i's parent P
    (row i gets (w/2)(pbar_P - p_K), row K the opposite), so
        dL/dbeta_f = -(h/2)(lambda_i - lambda_K)(pbar_P - p_K).

With the constant null space (all walls Neumann) p is reported with zero mean, the
adjoint right-hand side is projected to zero mean, and lambda is reported with zero mean.
"""
from __future__ import annotations

import numpy as np

from . import pcg


def _project(v):
    return v - v.mean()


def face_factors(H, p, lam):
    """The three factors of dL/dbeta_f = -coef_f * dlam_f * dp_f for every canonical face
    (order of H.faces), from the per-face closed forms in the module docstring:
    regular faces coef = h, dlam = lambda_i - lambda_j, dp = p_i - p_j; T sub-faces
    coef = h/2, dlam = lambda_i - lambda_K, dp = pbar_P - p_K."""
    t = H.tree
    f = H.faces
    L = t.leaves
    p = np.asarray(p, np.float64)
    lam = np.asarray(lam, np.float64)
    mi, pl = f["minus"], f["plus"]
    d = f["depth"]
    h = 1.0 / (t.n0 * (2.0 ** d))
    dm, dp = L["depth"][mi], L["depth"][pl]
    coef = h.astype(np.float64).copy()
    dlam = np.zeros(len(mi))
    dpv = np.zeros(len(mi))
    reg = dm == dp
    dlam[reg] = lam[mi[reg]] - lam[pl[reg]]
    dpv[reg] = p[mi[reg]] - p[pl[reg]]
    tf = np.nonzero(~reg)[0]
    if len(tf):
        fine = np.where(dm[tf] == d[tf], mi[tf], pl[tf])
        coarse = np.where(dm[tf] == d[tf], pl[tf], mi[tf])
        pbar = np.empty(len(tf))
        for dd in np.unique(d[tf]):
            sel = np.nonzero(d[tf] == dd)[0]
            lv = H.levels[dd - 1]
            fi = fine[sel]
            P = lv.index(L["i"][fi] // 2, L["j"][fi] // 2, L["k"][fi] // 2)
            assert np.all(P >= 0)
            pbar[sel] = H.leaves_to_level(dd - 1, p)[P]
        coef[tf] = h[tf] / 2.0
        dlam[tf] = lam[fine] - lam[coarse]
        dpv[tf] = pbar - p[coarse]
    return coef, dlam, dpv


def face_grad(H, p, lam):
    """dL/dbeta_f = -lambda^T (dA/dbeta_f) p for every canonical face (order of
    H.faces), from the per-face closed forms in the module docstring."""
    coef, dlam, dpv = face_factors(H, p, lam)
    return -coef * dlam * dpv


def solve(H, rhs, transpose=False, tol=1e-13, method="krylov", prm=None):
    """A x = rhs (or A^T x = rhs): oracle Krylov solve to a tight tolerance (PCG, Alg. 1,
    for A; BiCGStab preconditioned by the transposed cycle M^T for A^T, which converges
    where the forward cycle diverges at high coefficient contrast), or the dense solve;
    zero mean under the constant null space."""
    if method == "direct":
        x = pcg.direct_solve(H, rhs, transpose=transpose)
    elif transpose:
        x, _, _ = pcg.bicgstab(H, rhs, tol=tol, max_iter=500, prm=prm, transpose=True, precond="transposed")
    else:
        x, _, _ = pcg.pcg(H, rhs, tol=tol, max_iter=500, prm=prm)
    return _project(x) if H.nullspace else x


def loss(p, p_target):
    """L = 1/2 ||p - p_target||^2."""
    e = np.asarray(p) - np.asarray(p_target)
    return 0.5 * float(e @ e)


def gradients(H, b, p_target, method="krylov", tol=1e-13):
    """Forward solve, adjoint solve and both gradients of L = 1/2 ||p - p_target||^2.
    Returns (p, lambda, dL/db, dL/dbeta)."""
    p = solve(H, b, tol=tol, method=method)
    g = p - np.asarray(p_target, np.float64)
    if H.nullspace:
        g = _project(g)
    lam = solve(H, g, transpose=True, tol=tol, method=method)
    return p, lam, lam.copy(), face_grad(H, p, lam)
