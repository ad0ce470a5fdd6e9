"""Oracle operators: coefficients, coarsening and explicit matrices (TEST INFRASTRUCTURE).

Discretisation (Sec. 2.1, Eqs. discretized-flux-integration and projection-poisson-
system): every cell stores a diagonal c and the coefficients c_{x-}, c_{y-}, c_{z-} of
its three negative faces, c_face = -S/h = -beta*h for a face of fluid area beta*h^2;
the diagonal is the sum of the six face magnitudes.  Domain walls: Neumann faces
contribute nothing; Dirichlet faces hold the value at the wall face (half a cell away),
weight 2*beta*h with beta = 1, and are stored as the negative-face coefficient of the
cell on the - wall and in the diagonal only on the + wall.

T-junctions (Sec. 3.1, Eqs. flux-conservation and t-junction-ghost-values): a fine leaf
i whose face touches a leaf K one depth coarser sees a ghost value
    g = p_i + (p_K - pbar_P) / 2,   pbar_P = mean of the children of i's parent P,
so the face adds w_f (p_i - g) = (w_f/2)(pbar_P - p_K) to row i; the coarse leaf's
face towards P carries the weight (1/2) sum_f w_f of the fine sub-faces (the paper's
c_{4,x-} = (S1+S3)/(2h)) and couples to the value of P, the average of its children.

Coarsening (Sec. 2.5, Alg. 3) with alpha = 2 builds each inner cell from its eight
children; it equals the Galerkin product R A P on T-free regions (Sec. 2.4,
Eq. galerkin-mat-coarsen), which `rap_inner_block` forms explicitly for the check.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import octree as O


def _gkey(i, j, k, n):
    return (np.asarray(k, np.int64) * n + j) * n + i


class Level:
    """One multigrid level: cells, stored coefficients, matrices."""

    def __init__(self, m, N, i, j, k, leaf):
        self.m = m
        self.N = N                # cells per axis of the level's grid
        self.i, self.j, self.k = i, j, k
        self.leaf = leaf
        self.n = len(i)
        key = _gkey(i, j, k, N)
        self._order = np.argsort(key)
        self._skey = key[self._order]
        self.colour = ((i + j + k) & 1).astype(np.int8)
        self.c = np.zeros(self.n)
        self.cm = np.zeros((3, self.n))     # c_{x-}, c_{y-}, c_{z-}
        self.tK = np.full((self.n, 6), -1, np.int64)   # coarse leaf index at level m-1
        self.tw = np.zeros((self.n, 6))                # fine T-face weight w_f >= 0
        self.parent = None
        self.children = None                # (n, 8) child indices at m+1, -1 if none
        self.rank = np.full(self.n, -1, np.int64)

    def index(self, i, j, k):
        """Index of the cell at (i,j,k) on this level, -1 if absent or outside."""
        i = np.asarray(i, np.int64); j = np.asarray(j, np.int64); k = np.asarray(k, np.int64)
        N = self.N
        inside = (i >= 0) & (i < N) & (j >= 0) & (j < N) & (k >= 0) & (k < N)
        key = _gkey(np.clip(i, 0, N - 1), np.clip(j, 0, N - 1), np.clip(k, 0, N - 1), N)
        if self.n == 0:
            return np.full(key.shape, -1, np.int64)
        pos = np.minimum(np.searchsorted(self._skey, key), self.n - 1)
        hit = inside & (self._skey[pos] == key)
        return np.where(hit, self._order[pos], -1)

    @property
    def active(self):
        return self.c != 0.0


class Hierarchy:
    """All levels m = D (finest) .. mc (coarsest) of the octree multigrid.

    Parameters: tree (oracle.octree.Octree), beta per canonical face, bc (6 wall codes),
    alpha (restriction scaling, Sec. 3.3: alpha = 2), coarse_beta: None for the
    algebraically consistent coarsening of Alg. 3 (the paper's method); for the
    geometric-multigrid ablation of Sec. 3.3, a function (m, axis, i, j, k) -> beta of
    the - face of cells (i, j, k) of level m along axis, with which every cell that has
    children is rediscretised at its own resolution (`_rediscretise`)."""

    def __init__(self, tree, beta, bc, alpha=2.0, coarse_beta=None):
        self.tree = tree
        self.D = tree.D
        self.mc = tree.min_level()
        self.alpha = float(alpha)
        self.bc = tuple(bc)
        self.beta = np.asarray(beta, np.float64)
        self.faces = tree.faces()
        self.levels = {}
        for m in range(self.mc, self.D + 1):
            i, j, k, leaf = tree.level_cells(m)
            N = tree.nd(m) if m >= 0 else tree.n0 >> (-m)
            self.levels[m] = Level(m, N, i, j, k, leaf)
        for m in range(0, self.D + 1):
            L = self.levels[m]
            L.rank[L.leaf] = tree.leaf_rank(m, L.i[L.leaf], L.j[L.leaf], L.k[L.leaf])
        self._link_levels()
        self._face_lookup()
        self._fill_leaves()
        self._coarsen_all()
        if coarse_beta is not None:
            self._rediscretise(coarse_beta)
        self._assemble_all()
        self._composite()

    # ------------------------------------------------------------------ structure
    def _link_levels(self):
        for m in range(self.mc + 1, self.D + 1):
            L, Pl = self.levels[m], self.levels[m - 1]
            L.parent = Pl.index(L.i // 2, L.j // 2, L.k // 2)
            assert np.all(L.parent >= 0)
        for m in range(self.mc, self.D + 1):
            L = self.levels[m]
            L.children = np.full((L.n, 8), -1, np.int64)
            if m == self.D:
                continue
            F = self.levels[m + 1]
            for s in range(8):
                dx, dy, dz = s & 1, (s >> 1) & 1, (s >> 2) & 1
                L.children[:, s] = F.index(2 * L.i + dx, 2 * L.j + dy, 2 * L.k + dz)

    def _face_lookup(self):
        f = self.faces
        self._fkeys = {}
        mk = O.morton(f["i"], f["j"], f["k"])
        for a in range(3):
            for d in range(self.D + 1):
                sel = np.nonzero((f["axis"] == a) & (f["depth"] == d))[0]
                o = np.argsort(mk[sel])
                self._fkeys[(a, d)] = (mk[sel][o], sel[o])

    def face_beta(self, a, d, i, j, k):
        """beta of the face named (axis a, depth d, + cell (i,j,k)); KeyError if absent."""
        keys, idx = self._fkeys[(a, d)]
        q = O.morton(i, j, k)
        pos = np.minimum(np.searchsorted(keys, q), len(keys) - 1)
        if len(keys) == 0 or np.any(keys[pos] != q):
            raise KeyError("face not in canonical list")
        return self.beta[idx[pos]]

    # ------------------------------------------------------------------ Sec. 2.1
    def _fill_leaves(self):
        """Leaf coefficients from face beta and wall conditions (Eq. projection-poisson-
        system with c_face = -beta*h; T sub-faces per Sec. 3.1)."""
        t = self.tree
        for m in range(0, self.D + 1):
            L = self.levels[m]
            sel = np.nonzero(L.leaf)[0]
            if len(sel) == 0:
                continue
            h = t.h(m)
            ci, cj, ck = L.i[sel], L.j[sel], L.k[sel]
            w_all = np.zeros((len(sel), 6))
            for q, (a, s) in enumerate(O.DIRS):
                c = [ci.copy(), cj.copy(), ck.copy()]
                c[a] = c[a] + s
                inside = (c[a] >= 0) & (c[a] < L.N)
                nb = L.index(*c)
                w = np.zeros(len(sel))
                # wall
                wall = ~inside
                if self.bc[q] == 1:
                    w[wall] = 2.0 * h
                # same-depth neighbour (leaf or inner)
                same = nb >= 0
                if np.any(same):
                    plus = [v[same] for v in c] if s > 0 else [ci[same], cj[same], ck[same]]
                    is_leaf_nb = L.leaf[nb[same]]
                    wl = np.zeros(same.sum())
                    # leaf-leaf regular face
                    if np.any(is_leaf_nb):
                        pp = [v[is_leaf_nb] for v in plus]
                        wl[is_leaf_nb] = self.face_beta(a, m, *pp) * h
                    # coarse side of a T-junction: neighbour is an inner cell; its four
                    # sub-faces live at depth m+1
                    inner = ~is_leaf_nb
                    if np.any(inner):
                        hf = t.h(m + 1)
                        # + cells of the sub-faces at depth m+1 (bit a = 0 children of the
                        # + side cell at depth m)
                        base = [v[inner] for v in plus]
                        acc = np.zeros(inner.sum())
                        for u in (0, 1):
                            for v in (0, 1):
                                cc = [2 * base[0], 2 * base[1], 2 * base[2]]
                                o1, o2 = [b for b in range(3) if b != a]
                                cc[o1] = cc[o1] + u
                                cc[o2] = cc[o2] + v
                                acc += self.face_beta(a, m + 1, *cc) * hf
                        wl[inner] = 0.5 * acc
                    w[same] = wl
                # fine side of a T-junction: region covered by a coarser leaf
                tj = inside & (nb < 0)
                if np.any(tj):
                    assert m >= 1
                    plus = [v[tj] for v in c] if s > 0 else [ci[tj], cj[tj], ck[tj]]
                    wf = self.face_beta(a, m, *plus) * h
                    w[tj] = wf
                    Lc = self.levels[m - 1]
                    K = Lc.index(c[0][tj] // 2, c[1][tj] // 2, c[2][tj] // 2)
                    assert np.all(K >= 0) and np.all(Lc.leaf[K])
                    L.tK[sel[tj], q] = K
                    L.tw[sel[tj], q] = wf
                w_all[:, q] = w
            for a in range(3):
                L.cm[a, sel] = -w_all[:, 2 * a]
            L.c[sel] = w_all.sum(axis=1)

    # ------------------------------------------------------------------ Alg. 3
    def coarsen_cell(self, m, child_idx):
        """Alg. 3 for one coarse cell: child_idx[s], s = di + 2 dj + 4 dk, indices at
        level m (the fine level).  Returns (c, cx-, cy-, cz-) of the parent."""
        F = self.levels[m]
        a = self.alpha
        c = 0.0
        cm = [0.0, 0.0, 0.0]
        active = 0
        for s in range(8):
            ch = child_idx[s]
            cc = F.c[ch]
            if cc != 0.0:
                active += 1
                c += cc / a
            for ax in range(3):
                bit = 1 << ax
                if s & bit:
                    sib = child_idx[s ^ bit]
                    if cc != 0.0 and F.c[sib] != 0.0:
                        c += (2.0 / a) * F.cm[ax, ch]
                else:
                    cm[ax] += F.cm[ax, ch] / a
        if active == 0:
            c = 0.0
        return c, cm[0], cm[1], cm[2]

    def coarsen_level(self, m):
        """Alg. 3 for every cell of level m-1 that has children, vectorised over those
        cells; the loop over the eight children and the order of the additions are those
        of `coarsen_cell`, so both give identical bits."""
        C, F = self.levels[m - 1], self.levels[m]
        a = self.alpha
        I = np.nonzero(C.children[:, 0] >= 0)[0]
        ch = C.children[I]
        c = np.zeros(len(I))
        cm = np.zeros((3, len(I)))
        active = np.zeros(len(I), np.int64)
        for s in range(8):
            cc = F.c[ch[:, s]]
            act = cc != 0.0
            active += act
            c = np.where(act, c + cc / a, c)
            for ax in range(3):
                bit = 1 << ax
                if s & bit:
                    both = act & (F.c[ch[:, s ^ bit]] != 0.0)
                    c = np.where(both, c + (2.0 / a) * F.cm[ax, ch[:, s]], c)
                else:
                    cm[ax] = cm[ax] + F.cm[ax, ch[:, s]] / a
        c[active == 0] = 0.0
        C.c[I] = c
        C.cm[:, I] = cm

    def _coarsen_all(self):
        """Every cell with children gets Alg. 3 of its children, finest first."""
        for m in range(self.D, self.mc, -1):
            self.coarsen_level(m)

    def _rediscretise(self, coarse_beta):
        """Geometric multigrid (Sec. 3.3): each cell with children takes the coefficients
        the grid discretisation gives it directly at its size H, without reference to the
        finer operator: w = beta_face H on each face (beta_face from coarse_beta), the
        wall weight on a wall face (0 Neumann, 2H Dirichlet, as for leaves), c = the sum
        of its six face weights (0 kept for a cell without active children).  Leaves keep
        their coefficients; the - face coefficient of a leaf beside such a cell is the same
        face's weight, so each face keeps one value."""
        for m in range(self.D - 1, self.mc - 1, -1):
            L = self.levels[m]
            I = np.nonzero(L.children[:, 0] >= 0)[0]
            if len(I) == 0:
                continue
            H = 1.0 / (self.tree.n0 * 2.0 ** m)
            crd = (L.i[I], L.j[I], L.k[I])
            total = np.zeros(len(I))
            for a in range(3):
                for side in (0, 1):
                    c = [crd[0].copy(), crd[1].copy(), crd[2].copy()]
                    if side:
                        c[a] = c[a] + 1          # the + face is the - face of (i + e_a)
                    wall = (c[a] - 1 < 0) if side == 0 else (c[a] >= L.N)
                    wb = 2.0 * H if self.bc[2 * a + side] == 1 else 0.0     # 1: Dirichlet
                    beta = np.asarray(coarse_beta(m, a, c[0], c[1], c[2]), np.float64)
                    w = np.where(wall, wb, beta * H)
                    total += w
                    if side == 0:
                        L.cm[a, I] = -w
            L.c[I] = np.where(L.c[I] != 0.0, total, 0.0)

    # ------------------------------------------------------------------ matrices
    def _assemble_all(self):
        for m in range(self.mc, self.D + 1):
            self._assemble(m)

    def _assemble(self, m):
        """Level operator A^m (cells of level m) and ghost-source matrix B^m (columns are
        level m-1 cells).  Row i: c_i u_i + sum over faces of c_face u_nb; a T face
        replaces u_nb by the ghost g = u_i + (u_K - ubar_P)/2."""
        L = self.levels[m]
        rows, cols, vals = [np.arange(L.n)], [np.arange(L.n)], [L.c.copy()]
        brow, bcol, bval = [], [], []
        for q, (a, s) in enumerate(O.DIRS):
            c = [L.i.copy(), L.j.copy(), L.k.copy()]
            c[a] = c[a] + s
            nb = L.index(*c)
            reg = np.nonzero(nb >= 0)[0]
            coef = L.cm[a, reg] if s < 0 else L.cm[a, nb[reg]]
            rows.append(reg); cols.append(nb[reg]); vals.append(coef)
            tj = np.nonzero(L.tK[:, q] >= 0)[0]
            if len(tj):
                wf = L.tw[tj, q]
                # -w_f * g = -w_f u_i - (w_f/2) u_K + (w_f/2) ubar_P
                rows.append(tj); cols.append(tj); vals.append(-wf)
                brow.append(tj); bcol.append(L.tK[tj, q]); bval.append(-0.5 * wf)
                P = self.levels[m - 1]
                par = L.parent[tj]
                sibs = P.children[par]                  # (len, 8) indices at level m
                act = L.active[sibs]
                nact = np.maximum(act.sum(axis=1), 1)
                for sl in range(8):
                    ok = act[:, sl]
                    rows.append(tj[ok]); cols.append(sibs[ok, sl])
                    vals.append(0.5 * wf[ok] / nact[ok])
        L.A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                            shape=(L.n, L.n))
        if m > self.mc:
            nP = self.levels[m - 1].n
            if brow:
                L.B = sp.csr_matrix((np.concatenate(bval), (np.concatenate(brow), np.concatenate(bcol))),
                                    shape=(L.n, nP))
            else:
                L.B = sp.csr_matrix((L.n, nP))
            # P^m: copy parent value to each child (Sec. 2.3); R^m = P^T / alpha
            L.P = sp.csr_matrix((np.ones(L.n), (np.arange(L.n), L.parent)), shape=(L.n, nP))
            L.R = (L.P.T / self.alpha).tocsr()
        else:
            L.B = None
            L.P = L.R = None

    def _composite(self):
        """Composite leaf operator: rows of the leaves of every level, with inner values
        replaced by the mean of their active children (recursively) and ghost sources
        (coarse leaves) read from the leaf vector."""
        nl = self.tree.n_leaves
        Q = {}
        for m in range(self.D, -1, -1):
            L = self.levels[m]
            rows_leaf = np.nonzero(L.leaf)[0]
            Ql = sp.csr_matrix((np.ones(len(rows_leaf)), (rows_leaf, L.rank[rows_leaf])),
                               shape=(L.n, nl))
            if m < self.D:
                F = self.levels[m + 1]
                inner = np.nonzero(~L.leaf)[0]
                ch = L.children[inner]
                act = F.active[ch]
                nact = np.maximum(act.sum(axis=1), 1)
                r, cidx, v = [], [], []
                for sl in range(8):
                    ok = act[:, sl]
                    r.append(inner[ok]); cidx.append(ch[ok, sl]); v.append(1.0 / nact[ok])
                Cm = sp.csr_matrix((np.concatenate(v), (np.concatenate(r), np.concatenate(cidx))),
                                   shape=(L.n, F.n))
                Ql = Ql + Cm @ Q[m + 1]
            Q[m] = Ql.tocsr()
        self.Q = Q
        parts = []
        for m in range(0, self.D + 1):
            L = self.levels[m]
            Am = L.A @ Q[m]
            if m > 0 and L.B is not None:
                Am = Am + L.B @ Q[m - 1]
            leaf_rows = np.nonzero(L.leaf)[0]
            Sel = sp.csr_matrix((np.ones(len(leaf_rows)), (L.rank[leaf_rows], leaf_rows)),
                                shape=(nl, L.n))
            parts.append(Sel @ Am)
        self.A = sp.csr_matrix(sum(parts)).tocsr()
        self.A.eliminate_zeros()

    # ------------------------------------------------------------------ helpers
    def apply_A(self, p):
        """Composite leaf operator applied to p (canonical leaf order)."""
        return self.A @ p

    def leaves_to_level(self, m, p):
        """Values of all level-m cells (m >= 0) from a leaf vector (inner = Avg)."""
        return self.Q[m] @ p

    def rap_inner_block(self, m):
        """Explicit Galerkin product R^m A^m P^m restricted to rows and columns of the
        cells of level m-1 that have children (Sec. 2.3, Eq. galerkin-principle)."""
        L = self.levels[m]
        C = self.levels[m - 1]
        inner = np.nonzero(C.children[:, 0] >= 0)[0]
        Pm = L.P[:, inner]
        return inner, (L.R[inner, :] @ L.A @ Pm).toarray()

    def level_dense(self, m):
        """Stored-coefficient 7-point operator of level m as a dense matrix (regular part
        only, T ghosts excluded): diag c, off-diagonals from the shared face coefficient."""
        L = self.levels[m]
        A = np.diag(L.c.copy())
        for q, (a, s) in enumerate(O.DIRS):
            c = [L.i.copy(), L.j.copy(), L.k.copy()]
            c[a] = c[a] + s
            nb = L.index(*c)
            reg = np.nonzero(nb >= 0)[0]
            coef = L.cm[a, reg] if s < 0 else L.cm[a, nb[reg]]
            A[reg, nb[reg]] += coef
        return A

    @property
    def nullspace(self):
        return all(b == 0 for b in self.bc)
