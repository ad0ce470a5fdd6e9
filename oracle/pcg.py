"""Oracle preconditioned conjugate gradient, Alg. 1 (Sec. 2.2), and the BiCGStab used
for the adjoint system (TEST INFRASTRUCTURE).

x0 = 0, r0 = b; under pure Neumann walls the residual is shifted to zero mean after it
is formed (Sec. 2.2, the null-space remark); the loop runs while ||r||_2 > tol ||b||_2
(relative residual, b after the mean shift), the preconditioner is one FAS-style
mu-cycle (oracle.mg.vcycle).  Returns (x, iterations, history of ||r||/||b||).
"""
from __future__ import annotations

import numpy as np

from . import mg


def pcg(H, b, tol=1e-6, max_iter=200, prm=None, precond=True, transpose=False):
    """Alg. 1 on A x = b, or on A^T x = b with transpose=True.  precond: True (the
    mu-cycle M), False (none) or "transposed" (M^T, mg.vcycle_T: the preconditioner of the
    adjoint system, whose scalars (r, M^T r) = (M r, r) and (p, A^T p) = (A p, p) are the
    forward method's quadratic forms)."""
    A = H.A.T.tocsr() if transpose else H.A
    b = np.asarray(b, np.float64).copy()
    ns = H.nullspace
    if ns:
        b = b - b.mean()
    x = np.zeros_like(b)
    r = b.copy()
    bn = np.linalg.norm(b)
    hist = [1.0]
    if bn == 0.0:
        return x, 0, hist
    if precond == "transposed":
        M = lambda v: mg.vcycle_T(H, v, prm)
    elif precond:
        M = lambda v: mg.vcycle(H, v, prm)
    else:
        M = lambda v: v.copy()
    z = M(r)
    p = z.copy()
    rz = r @ z
    k = 0
    while np.linalg.norm(r) > tol * bn and k < max_iter:
        Ap = A @ p
        alpha = rz / (Ap @ p)
        x = x + alpha * p
        r = r - alpha * Ap
        if ns:
            r = r - r.mean()
        k += 1
        hist.append(np.linalg.norm(r) / bn)
        if np.linalg.norm(r) <= tol * bn:
            break
        z = M(r)
        rz_new = r @ z
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    return x, k, hist


def direct_solve(H, b, transpose=False):
    """Dense reference solution (tiny problems): numpy solve, or least squares with the
    zero-mean normalisation when the operator has the constant null space."""
    A = H.A.toarray()
    if transpose:
        A = A.T
    b = np.asarray(b, np.float64)
    if H.nullspace:
        b = b - b.mean()
        x = np.linalg.lstsq(A, b, rcond=None)[0]
        return x - x.mean()
    return np.linalg.solve(A, b)


def bicgstab(H, b, tol=1e-6, max_iter=200, prm=None, transpose=False, precond=None):
    """Right-preconditioned BiCGStab (H. A. van der Vorst, SIAM J. Sci. Stat. Comput. 13,
    1992) with one mu-cycle as the preconditioner M; the solver of the adjoint system
    A^T lambda = g.  Alg. 1 with the same cycle stagnates there (M approximates A^{-1},
    and A is not symmetric at T-junctions), BiCGStab does not.  Stopping rule, zero start
    and null-space shift of the residual as in `pcg`.  Returns (x, iterations, history)."""
    A = H.A.T.tocsr() if transpose else H.A
    b = np.asarray(b, np.float64).copy()
    ns = H.nullspace
    if ns:
        b = b - b.mean()
    x = np.zeros_like(b)
    r = b.copy()
    rhat = b.copy()
    bn = np.linalg.norm(b)
    hist = [1.0]
    if bn == 0.0:
        return x, 0, hist
    # precond: "forward" (the mu-cycle M) or "transposed" (M^T, mg.vcycle_T); default:
    # the forward cycle
    if precond == "transposed":
        M = lambda v: mg.vcycle_T(H, v, prm)
    else:
        M = lambda v: mg.vcycle(H, v, prm)
    rho = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    k = 0
    while np.linalg.norm(r) > tol * bn and k < max_iter:
        rho_new = rhat @ r
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = M(p)
        v = A @ ph
        alpha = rho_new / (rhat @ v)
        s = r - alpha * v
        sh = M(s)
        t = A @ sh
        omega = (t @ s) / (t @ t)
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        if ns:
            r = r - r.mean()
        rho = rho_new
        k += 1
        hist.append(np.linalg.norm(r) / bn)
    return x, k, hist
