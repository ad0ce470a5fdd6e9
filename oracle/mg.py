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
