"""Oracle multigrid cycles (TEST INFRASTRUCTURE).

fas_cycle   - the FAS-style mu-cycle of Alg. 4 (Sec. 3.2) on the octree levels
plain_cycle - the mu-cycle of Alg. 2 (Sec. 2.3), beta on prolongation; used only to
              check that Alg. 4 reduces to it where no leaves live below the finest level

Smoother (Sec. 2.3): red-black Gauss-Seidel, colour = (i+j+k) mod 2 on the level's own
integer grid.  One colour sweep updates u_i += r_i / c_i on the active cells of that
colour, r = b - A^m u - B^m u^{m-1} evaluated from the state at the start of the sweep
(the T-junction ghosts couple same-colour siblings through pbar_P, so every read uses
the sweep-start state), c_i the stored diagonal.  nu_l iterations before (red then
black) and after (black then red) the coarse correction; nu_b at the coarsest level,
half red-then-black and half black-then-red.

Level layout: u[m], b[m] arrays per level.  Leaves at level m < D carry the rhs of the
preconditioned system and their current value; inner cells carry the FAS full
approximation.  Restriction (Alg. 4): u*_{m-1} = Avg(u^m) (mean over active children),
b^{m-1} = beta R r^m + A^{m-1} u*_{m-1} on the cells with children, the leaves of level
m-1 keep their b and u.  Prolongation: u^m += P (u^{m-1} - u*), no beta.
"""
from __future__ import annotations

import numpy as np


class CycleParams:
    """mu_min_cells (an extension, not in the paper; 0 = the paper's cycle): the recursion
    into a coarser level is repeated mu times only when that level has at least this many
    cells (leaves and inner, padding excluded); smaller levels are visited once per visit of
    their parent, i.e. a W-cycle on the large levels and a V-cycle below."""

    def __init__(self, mu=1, nu_pre=2, nu_post=2, nu_coarsest=10, beta=2.0, mu_min_cells=0):
        self.mu = mu
        self.nu_pre = nu_pre
        self.nu_post = nu_post
        self.nu_coarsest = nu_coarsest
        self.beta = beta
        self.mu_min_cells = mu_min_cells


def level_residual(H, m, u, b):
    L = H.levels[m]
    r = b[m] - L.A @ u[m]
    if m > H.mc and L.B is not None and L.B.nnz:
        r = r - L.B @ u[m - 1]
    r[~L.active] = 0.0
    return r


def colour_sweep(H, m, u, b, colour):
    L = H.levels[m]
    r = level_residual(H, m, u, b)
    sel = (L.colour == colour) & L.active
    u[m][sel] += r[sel] / L.c[sel]


def smooth(H, m, u, b, iters, first_colour):
    for _ in range(iters):
        colour_sweep(H, m, u, b, first_colour)
        colour_sweep(H, m, u, b, 1 - first_colour)


def avg_children(H, m, u):
    """Avg(u^m) on the cells of level m-1 that have children: mean over active children
    (0 if none)."""
    C, F = H.levels[m - 1], H.levels[m]
    I = np.nonzero(C.children[:, 0] >= 0)[0]
    ch = C.children[I]
    act = F.active[ch]
    s = np.where(act, u[m][ch], 0.0).sum(axis=1)
    n = act.sum(axis=1)
    out = np.zeros(len(I))
    nz = n > 0
    out[nz] = s[nz] / n[nz]
    return I, out


def fas_cycle(H, m, u, b, prm, hook=None):
    """Alg. 4 at level m: updates u in place (u, b are dicts of per-level arrays)."""
    if m == H.mc:
        half = prm.nu_coarsest // 2
        smooth(H, m, u, b, half, 0)
        smooth(H, m, u, b, prm.nu_coarsest - half, 1)
        return
    smooth(H, m, u, b, prm.nu_pre, 0)                       # pre-smoothing
    r = level_residual(H, m, u, b)                           # residual
    C = H.levels[m - 1]
    L = H.levels[m]
    I, ustar = avg_children(H, m, u)                         # u* = Avg(u^m)
    v = u[m - 1].copy()
    v[I] = ustar
    Av = C.A @ v                                             # rows with children have no ghosts
    Rr = L.R @ r
    b[m - 1][I] = prm.beta * Rr[I] + Av[I]                   # restriction
    u[m - 1][I] = ustar                                      # u^{m-1} <- u*
    mu = prm.mu if C.n >= getattr(prm, "mu_min_cells", 0) else 1
    for _ in range(mu):
        fas_cycle(H, m - 1, u, b, prm, hook)                 # recursive solve
    corr = np.zeros(C.n)
    corr[I] = u[m - 1][I] - ustar
    u[m] = u[m] + np.where(L.active, L.P @ corr, 0.0)       # prolongation
    if hook is not None:
        hook(m, u)
    smooth(H, m, u, b, prm.nu_post, 1)                       # post-smoothing


def _leaf_slots(H, m):
    L = H.levels[m]
    return np.nonzero(L.leaf)[0], L.rank[L.leaf]


def vcycle(H, r_leaf, prm=None, hook=None):
    """One mu-cycle from zero for the composite system A z = r (preconditioner)."""
    prm = prm or CycleParams()
    u = {m: np.zeros(H.levels[m].n) for m in H.levels}
    b = {m: np.zeros(H.levels[m].n) for m in H.levels}
    for m in range(0, H.D + 1):
        idx, rk = _leaf_slots(H, m)
        b[m][idx] = r_leaf[rk]
    fas_cycle(H, H.D, u, b, prm, hook)
    z = np.zeros(len(r_leaf))
    for m in range(0, H.D + 1):
        idx, rk = _leaf_slots(H, m)
        z[rk] = u[m][idx]
    return z


def plain_cycle(H, m, u, b, prm):
    """Alg. 2 at level m (no leaves below the finest level are allowed here): residual
    equation on the coarse level from zero, u^m += beta P u^{m-1}."""
    if m == H.mc:
        half = prm.nu_coarsest // 2
        smooth(H, m, u, b, half, 0)
        smooth(H, m, u, b, prm.nu_coarsest - half, 1)
        return
    smooth(H, m, u, b, prm.nu_pre, 0)
    r = level_residual(H, m, u, b)
    L = H.levels[m]
    b[m - 1] = L.R @ r
    u[m - 1] = np.zeros(H.levels[m - 1].n)
    for _ in range(prm.mu):
        plain_cycle(H, m - 1, u, b, prm)
    u[m] = u[m] + prm.beta * (L.P @ u[m - 1])
    smooth(H, m, u, b, prm.nu_post, 1)


def plain_vcycle(H, r_leaf, prm=None):
    prm = prm or CycleParams()
    assert all(not np.any(H.levels[m].leaf) for m in range(H.mc, H.D)), \
        "plain cycle comparison needs a tree without leaves below the finest level"
    u = {m: np.zeros(H.levels[m].n) for m in H.levels}
    b = {m: np.zeros(H.levels[m].n) for m in H.levels}
    idx, rk = _leaf_slots(H, H.D)
    b[H.D][idx] = r_leaf[rk]
    plain_cycle(H, H.D, u, b, prm)
    z = np.zeros(len(r_leaf))
    z[rk] = u[H.D][idx]
    return z


# ----------------------------------------------------------------------------------
# Transposed cycle (for the adjoint system; no counterpart in the paper).  The cycle from
# zero is a linear map M: r -> z.  Its transpose M^T applies the transposes of the cycle's
# steps in reverse order to adjoint states (ubar[m], bbar[m]).  Preconditioning A^T by
# M^T gives A^T M^T = (M A)^T, which has the spectrum of A M, so a Krylov method on the
# adjoint system converges as the forward one does.

def _avg_matrix(H, m):
    """(I, G): rows I of level m-1 with children and G (len(I) x n_m) with
    Avg(u^m)[I] = G @ u^m (mean over active children, 0 rows where none is active)."""
    import scipy.sparse as sp
    C, F = H.levels[m - 1], H.levels[m]
    I = np.nonzero(C.children[:, 0] >= 0)[0]
    ch = C.children[I]
    act = F.active[ch]
    n = act.sum(axis=1)
    rows = np.repeat(np.arange(len(I)), 8)
    vals = np.where(act, 1.0 / np.maximum(n, 1)[:, None], 0.0).ravel()
    G = sp.csr_matrix((vals, (rows, ch.ravel())), shape=(len(I), F.n))
    return I, G


def colour_sweep_T(H, m, ub, bb, colour):
    """Transpose of colour_sweep: u_C += (b - A u - B u^{m-1})_C / c_C."""
    L = H.levels[m]
    sel = (L.colour == colour) & L.active
    v = np.zeros(L.n)
    v[sel] = ub[m][sel] / L.c[sel]
    bb[m] += v
    ub[m] -= L.A.T @ v
    if m > H.mc and L.B is not None and L.B.nnz:
        ub[m - 1] -= L.B.T @ v


def smooth_T(H, m, ub, bb, iters, first_colour):
    """Transpose of smooth(iters, first_colour): the sweeps in reverse order."""
    for _ in range(iters):
        colour_sweep_T(H, m, ub, bb, 1 - first_colour)
        colour_sweep_T(H, m, ub, bb, first_colour)


def fas_cycle_T(H, m, ub, bb, prm):
    """Transpose of fas_cycle at level m on the adjoint state (ub, bb), in place."""
    if m == H.mc:
        half = prm.nu_coarsest // 2
        smooth_T(H, m, ub, bb, prm.nu_coarsest - half, 1)
        smooth_T(H, m, ub, bb, half, 0)
        return
    L, C = H.levels[m], H.levels[m - 1]
    I, G = _avg_matrix(H, m)
    smooth_T(H, m, ub, bb, prm.nu_post, 1)                   # post-smoothing
    corr_b = L.P.T @ np.where(L.active, ub[m], 0.0)          # prolongation u^m += P corr
    ustar_b = np.zeros(len(I))
    ub[m - 1][I] += corr_b[I]                                # corr = u^{m-1}[I] - u*
    ustar_b -= corr_b[I]
    mu = prm.mu if C.n >= getattr(prm, "mu_min_cells", 0) else 1
    for _ in range(mu):
        fas_cycle_T(H, m - 1, ub, bb, prm)                   # recursive solves
    ustar_b += ub[m - 1][I]                                  # u^{m-1}[I] <- u*
    ub[m - 1][I] = 0.0
    g = np.zeros(C.n)                                        # b^{m-1}[I] <- beta R r + A v
    g[I] = bb[m - 1][I]
    bb[m - 1][I] = 0.0
    r_b = prm.beta * (L.R.T @ g)
    v_b = C.A.T @ g                                          # v = u^{m-1}, v[I] = u*
    ustar_b += v_b[I]
    v_b[I] = 0.0
    ub[m - 1] += v_b
    ub[m] += G.T @ ustar_b                                   # u* = Avg(u^m)
    r_b = np.where(L.active, r_b, 0.0)                       # r = b - A u - B u^{m-1}
    bb[m] += r_b
    ub[m] -= L.A.T @ r_b
    if L.B is not None and L.B.nnz:
        ub[m - 1] -= L.B.T @ r_b
    smooth_T(H, m, ub, bb, prm.nu_pre, 0)                    # pre-smoothing


def vcycle_T(H, z_leaf, prm=None):
    """M^T z: the transpose of vcycle (one mu-cycle from zero)."""
    prm = prm or CycleParams()
    ub = {m: np.zeros(H.levels[m].n) for m in H.levels}
    bb = {m: np.zeros(H.levels[m].n) for m in H.levels}
    for m in range(0, H.D + 1):
        idx, rk = _leaf_slots(H, m)
        ub[m][idx] = z_leaf[rk]
    fas_cycle_T(H, H.D, ub, bb, prm)
    r = np.zeros(len(z_leaf))
    for m in range(0, H.D + 1):
        idx, rk = _leaf_slots(H, m)
        r[rk] = bb[m][idx]
    return r
