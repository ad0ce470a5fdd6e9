"""Oracle octree: refinement, face 2:1 balance and canonical tables (TEST INFRASTRUCTURE).

Follows Sec. 3 of the paper: leaf cells carry the unknowns, an inner cell has 8
children one depth finer, and two face-neighbouring leaves differ by at
most one depth.  Refinement is top-down from the root grid by the predicate of the
problem description (Sec. 4.1 grids); the 2:1 rule is then enforced by the minimal
extra refinement, processed from the deepest inner cells upward: every inner cell at
depth e needs all six face neighbours at depth e to exist, i.e. their parents at
depth e-1 must be refined.

Independent of the CUDA library's builder: cells are held as sorted int64 key sets per
depth (key = (k*n + j)*n + i at that depth) and combined with numpy set operations.
Predicate arithmetic is IEEE float64 evaluated in the fixed operation order stated in
`refine_predicate` so that both builders make identical decisions.
"""
from __future__ import annotations

import math

import numpy as np

WALL, SAME, COARSER, FINER = 0, 1, 2, 3

DIRS = [(0, -1), (0, +1), (1, -1), (1, +1), (2, -1), (2, +1)]  # (axis, sign)


def _key(i, j, k, n):
    return (np.asarray(k, np.int64) * n + j) * n + i


def _unkey(key, n):
    key = np.asarray(key, np.int64)
    i = key % n
    j = (key // n) % n
    k = key // (n * n)
    return i, j, k


def morton(i, j, k):
    """Bit-interleaved key with x in bit 0, y in bit 1, z in bit 2 (plain bit loop)."""
    i = np.asarray(i, np.int64)
    j = np.asarray(j, np.int64)
    k = np.asarray(k, np.int64)
    out = np.zeros(np.broadcast(i, j, k).shape, np.int64)
    for b in range(20):
        out |= ((i >> b) & 1) << (3 * b)
        out |= ((j >> b) & 1) << (3 * b + 1)
        out |= ((k >> b) & 1) << (3 * b + 2)
    return out


def _box_sdf(box, x, y, z):
    """Signed distance to the axis-aligned box (lo, hi): positive outside."""
    lx, ly, lz, hx, hy, hz = box
    qx = np.abs(x - 0.5 * (lx + hx)) - 0.5 * (hx - lx)
    qy = np.abs(y - 0.5 * (ly + hy)) - 0.5 * (hy - ly)
    qz = np.abs(z - 0.5 * (lz + hz)) - 0.5 * (hz - lz)
    mx, my, mz = np.maximum(qx, 0.0), np.maximum(qy, 0.0), np.maximum(qz, 0.0)
    outside = np.sqrt(mx * mx + my * my + mz * mz)
    inside = np.minimum(np.maximum(qx, np.maximum(qy, qz)), 0.0)
    return outside + inside


def _star_phi(desc, x, y, z):
    """Sec. 4.1 star surface r = r0 + a cos(k theta) cos(k phi) about the first sphere's
    centre: r - (r0 + (a T_k(dz/r)) T_k(dx/rho)), the cosines of multiple angles as
    Chebyshev polynomials of cos(theta) = dz / r and cos(phi) = dx / rho."""
    (cx, cy, cz, r0), (a, kk, _, _) = desc.spheres[0], desc.spheres[1]
    dx, dy, dz = x - cx, y - cy, z - cz
    rho2 = dx * dx + dy * dy
    r = np.sqrt(rho2 + dz * dz)
    rho = np.sqrt(rho2)
    with np.errstate(divide="ignore", invalid="ignore"):
        u = np.where(r > 0.0, dz / r, 1.0)
        v = np.where(rho > 0.0, dx / rho, 1.0)

    def cheb(w):
        t0, t1 = np.ones_like(w), w
        if int(kk) == 0:
            return t0
        for _ in range(2, int(kk) + 1):
            t0, t1 = t1, (2.0 * w) * t1 - t0
        return t1
    return r - (r0 + (a * cheb(u)) * cheb(v))


def refine_predicate(desc, d, i, j, k):
    """Refinement decision for depth-d cells (d < max_depth), Sec. 4.1.

    Centre x = (i + 0.5) / n_d in one IEEE division, n_d = n0 * 2^d.
      ball centre : dx*dx + dy*dy + dz*dz  <  r*r           (sum left to right)
      SDF band    : |phi| < band + (0.5*sqrt(3)) * (1/n_d),  phi = min over primitives of
                    sphere  sqrt(dx*dx + dy*dy + dz*dz) - r
                    box     q = |x - 0.5*(lo+hi)| - 0.5*(hi-lo) per axis;
                            sqrt(mx*mx + my*my + mz*mz) + min(max(qx, max(qy, qz)), 0)
                            with m = max(q, 0)
      sine band   : |phi| < band + (|grad phi| * (0.5*sqrt(3))) * (1/n_d) with
                    phi = s/n, |grad phi| = sqrt(gx*gx + gy*gy + gz*gz)/n over the n waves
                    (kappa, dx, dy, dz, theta), accumulated wave by wave from 0:
                    w = 2pi*kappa, a = w*(dx*x + dy*y + dz*z) + theta, s += sin a,
                    g += (w cos a) * (dx, dy, dz); sin and cos from oracle.trig
      star band   : |phi| < band + (L * (0.5*sqrt(3))) * (1/n_d), phi = r - (r0 +
                    (a * T_k(dz/r)) * T_k(dx/rho)) about the first sphere's centre, T_k
                    by the Chebyshev recurrence (Sec. 4.1's star surface)
    Ties count as not refined.
    Tiles (desc.tile_log2 = t > 0; Sec. 4.1 refines the 8^3 tiles that meet the surface):
    the aligned block of 2^t cells per axis around (i, j, k) decides as one cell of that
    size, i.e. the rule above for the block (i // 2^t, j // 2^t, k // 2^t) on a grid of
    n_d / 2^t blocks per axis.
    """
    from paper_2604_18886_b300 import problems as P

    t = int(getattr(desc, "tile_log2", 0))
    i = np.asarray(i, np.int64) >> t
    j = np.asarray(j, np.int64) >> t
    k = np.asarray(k, np.int64) >> t
    nd = float((desc.n0 * 2 ** d) >> t)
    x = (np.asarray(i, np.float64) + 0.5) / nd
    y = (np.asarray(j, np.float64) + 0.5) / nd
    z = (np.asarray(k, np.float64) + 0.5) / nd
    if desc.refine == P.REFINE_NONE:
        return np.zeros(x.shape, bool)
    if desc.refine == P.REFINE_BALL_CENTRE:
        cx, cy, cz, r = desc.spheres[0]
        dx, dy, dz = x - cx, y - cy, z - cz
        return (dx * dx + dy * dy + dz * dz) < r * r
    if desc.refine == P.REFINE_SDF_BAND and t > 0:
        # a tile (the box [i, i+1] / nd per axis) meets the band of a sphere when the
        # sphere's signed distance, which runs over [dmin - r, dmax - r] on the box (nearest
        # and farthest distance from the centre), takes a value in (-band, band); boxes use
        # the centre test with the tile's half-diagonal
        ii, jj, kk = (np.asarray(v, np.float64) for v in (i, j, k))
        lo = [ii / nd, jj / nd, kk / nd]
        hi = [(ii + 1.0) / nd, (jj + 1.0) / nd, (kk + 1.0) / nd]
        out = np.zeros(x.shape, bool)
        for (cx, cy, cz, r) in desc.spheres:
            n2 = np.zeros(x.shape)
            f2 = np.zeros(x.shape)
            for a, c in enumerate((cx, cy, cz)):
                nearest = np.where(c < lo[a], lo[a], np.where(c > hi[a], hi[a], c))
                dn = nearest - c
                df = np.maximum(np.abs(lo[a] - c), np.abs(hi[a] - c))
                n2 = n2 + dn * dn
                f2 = f2 + df * df
            out |= (np.sqrt(n2) - r < desc.band) & (np.sqrt(f2) - r > -desc.band)
        if desc.boxes:
            phi = np.full(x.shape, np.inf)
            for box in desc.boxes:
                phi = np.minimum(phi, _box_sdf(box, x, y, z))
            out |= np.abs(phi) < desc.band + (0.5 * math.sqrt(3.0)) * (1.0 / nd)
        return out
    if desc.refine == P.REFINE_SDF_BAND:
        phi = np.full(x.shape, np.inf)
        for (cx, cy, cz, r) in desc.spheres:
            dx, dy, dz = x - cx, y - cy, z - cz
            phi = np.minimum(phi, np.sqrt(dx * dx + dy * dy + dz * dz) - r)
        for box in desc.boxes:
            phi = np.minimum(phi, _box_sdf(box, x, y, z))
        slack = desc.band + (0.5 * math.sqrt(3.0)) * (1.0 / nd)
        return np.abs(phi) < slack
    if desc.refine == P.REFINE_SINE_BAND:
        from . import trig
        s = np.zeros(x.shape)
        gx, gy, gz = np.zeros(x.shape), np.zeros(x.shape), np.zeros(x.shape)
        for (kap, dx, dy, dz, th) in desc.sines:
            w = trig.TWO_PI * kap
            a = w * (dx * x + dy * y + dz * z) + th
            s = s + trig.det_sin(a)
            g = w * trig.det_cos(a)
            gx, gy, gz = gx + g * dx, gy + g * dy, gz + g * dz
        n = float(len(desc.sines))
        phi = s / n
        grad = np.sqrt(gx * gx + gy * gy + gz * gz) / n
        slack = desc.band + (grad * (0.5 * math.sqrt(3.0))) * (1.0 / nd)
        return np.abs(phi) < slack
    if desc.refine == P.REFINE_STAR_BAND:
        if t > 0:
            # a tile meets the band when the star function takes a value below band and one
            # above -band among its 27 lattice points (i + q/2) / nd, q = 0, 1, 2 per axis
            ii, jj, kk = (np.asarray(v, np.float64) for v in (i, j, k))
            lo = np.full(x.shape, np.inf)
            hi = np.full(x.shape, -np.inf)
            for qz in range(3):
                for qy in range(3):
                    for qx in range(3):
                        f = _star_phi(desc, (ii + 0.5 * qx) / nd, (jj + 0.5 * qy) / nd, (kk + 0.5 * qz) / nd)
                        lo = np.minimum(lo, f)
                        hi = np.maximum(hi, f)
            return (lo < desc.band) & (hi > -desc.band)
        lip = desc.spheres[1][2]
        phi = _star_phi(desc, x, y, z)
        slack = desc.band + (lip * (0.5 * math.sqrt(3.0))) * (1.0 / nd)
        return np.abs(phi) < slack
    raise NotImplementedError("refine kind %d" % desc.refine)


class Octree:
    """Adaptive octree with face 2:1 balance.  Attributes:

    n0, D            root cells per axis, maximum depth
    exist[d]         sorted keys of every cell at depth d (leaf or inner)
    refined[d]       sorted keys of inner cells at depth d
    pred_refined[d]  cells refined by the predicate alone (before balancing)
    """

    def __init__(self, desc):
        self.desc = desc
        self.n0 = int(desc.n0)
        self.D = int(desc.max_depth)
        D = self.D
        self.exist = [None] * (D + 1)
        self.refined = [np.zeros(0, np.int64) for _ in range(D + 1)]
        n = self.n0
        ii, jj, kk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        self.exist[0] = np.unique(_key(ii.ravel(), jj.ravel(), kk.ravel(), n))
        for d in range(D):
            nd = self.nd(d)
            i, j, k = _unkey(self.exist[d], nd)
            sel = refine_predicate(desc, d, i, j, k)
            self.refined[d] = self.exist[d][sel]
            self.exist[d + 1] = self._children(d, self.refined[d])
        self.pred_refined = [r.copy() for r in self.refined]
        # face 2:1 balance, deepest inner cells first
        for e in range(D - 1, 0, -1):
            ne = self.nd(e)
            i, j, k = _unkey(self.refined[e], ne)
            add = [self.refined[e - 1]]
            for (a, s) in DIRS:
                c = [i.copy(), j.copy(), k.copy()]
                c[a] = c[a] + s
                ok = (c[a] >= 0) & (c[a] < ne)
                add.append(self._tile_cells(e - 1, c[0][ok] // 2, c[1][ok] // 2, c[2][ok] // 2))
            self.refined[e - 1] = np.unique(np.concatenate(add))
        for d in range(D):
            self.exist[d + 1] = self._children(d, self.refined[d])
        self._build_leaves()

    # --------------------------------------------------------------------------
    def _tile_cells(self, d, i, j, k):
        """Keys of the depth-d cells (i, j, k), each widened to its whole tile of
        2^tile_log2 cells per axis when the description refines by tiles (a tile is
        refined as a unit, by the predicate and by the 2:1 balance)."""
        t = int(getattr(self.desc, "tile_log2", 0))
        nd = self.nd(d)
        if t == 0 or len(i) == 0:
            return _key(i, j, k, nd)
        tk = np.unique(_key(i >> t, j >> t, k >> t, nd >> t))
        ti, tj, tk_ = _unkey(tk, nd >> t)
        w = 1 << t
        o = np.arange(w)
        oi, oj, ok = (a.ravel() for a in np.meshgrid(o, o, o, indexing="ij"))
        return _key((ti[:, None] * w + oi[None]).ravel(), (tj[:, None] * w + oj[None]).ravel(),
                    (tk_[:, None] * w + ok[None]).ravel(), nd)

    def nd(self, d):
        return self.n0 * 2 ** d

    def h(self, d):
        return 1.0 / self.nd(d)

    def _children(self, d, keys):
        nd = self.nd(d)
        i, j, k = _unkey(keys, nd)
        out = []
        for s in range(8):
            dx, dy, dz = s & 1, (s >> 1) & 1, (s >> 2) & 1
            out.append(_key(2 * i + dx, 2 * j + dy, 2 * k + dz, 2 * nd))
        if not out:
            return np.zeros(0, np.int64)
        return np.unique(np.concatenate(out))

    def is_refined(self, d, keys):
        if d > self.D:
            return np.zeros(np.shape(keys), bool)
        r = self.refined[d]
        if len(r) == 0:
            return np.zeros(np.shape(keys), bool)
        pos = np.minimum(np.searchsorted(r, keys), len(r) - 1)
        return r[pos] == keys

    def exists(self, d, keys):
        if d < 0 or d > self.D:
            return np.zeros(np.shape(keys), bool)
        e = self.exist[d]
        if len(e) == 0:
            return np.zeros(np.shape(keys), bool)
        pos = np.minimum(np.searchsorted(e, keys), len(e) - 1)
        return e[pos] == keys

    def _build_leaves(self):
        """Canonical leaf order: by (depth, Morton key)."""
        dep, I, J, K = [], [], [], []
        for d in range(self.D + 1):
            leaf = self.exist[d][~self.is_refined(d, self.exist[d])]
            i, j, k = _unkey(leaf, self.nd(d))
            order = np.argsort(morton(i, j, k), kind="stable")
            dep.append(np.full(len(leaf), d, np.int64))
            I.append(i[order]); J.append(j[order]); K.append(k[order])
        self.leaves = {"depth": np.concatenate(dep), "i": np.concatenate(I),
                       "j": np.concatenate(J), "k": np.concatenate(K)}
        self.n_leaves = len(self.leaves["depth"])
        # rank lookup per depth: sorted keys -> canonical rank
        self._rank_keys, self._rank_vals = [], []
        for d in range(self.D + 1):
            sel = self.leaves["depth"] == d
            ranks = np.nonzero(sel)[0]
            keys = _key(self.leaves["i"][sel], self.leaves["j"][sel], self.leaves["k"][sel], self.nd(d))
            o = np.argsort(keys)
            self._rank_keys.append(keys[o])
            self._rank_vals.append(ranks[o])

    def leaf_rank(self, d, i, j, k):
        """Canonical rank of the depth-d leaf at (i,j,k); -1 if it is not a leaf."""
        keys = _key(i, j, k, self.nd(d))
        rk, rv = self._rank_keys[d], self._rank_vals[d]
        if len(rk) == 0:
            return np.full(np.shape(keys), -1, np.int64)
        pos = np.minimum(np.searchsorted(rk, keys), len(rk) - 1)
        return np.where(rk[pos] == keys, rv[pos], -1)

    # --------------------------------------------------------------------------
    def neighbour_table(self):
        """Per leaf and direction (x-,x+,y-,y+,z-,z+): (kind, leaf rank).
        kind WALL / SAME (same-depth leaf) / COARSER (region covered by a leaf one depth
        coarser: the leaf is the fine side of a T-junction) / FINER (neighbour refined:
        the leaf is the coarse side).  Rank is -1 for WALL and FINER."""
        L = self.leaves
        n = self.n_leaves
        kind = np.zeros((n, 6), np.int8)
        rank = np.full((n, 6), -1, np.int64)
        for d in range(self.D + 1):
            sel = np.nonzero(L["depth"] == d)[0]
            if len(sel) == 0:
                continue
            nd = self.nd(d)
            for q, (a, s) in enumerate(DIRS):
                c = [L["i"][sel].copy(), L["j"][sel].copy(), L["k"][sel].copy()]
                c[a] = c[a] + s
                inside = (c[a] >= 0) & (c[a] < nd)
                cc = [np.clip(v, 0, nd - 1) for v in c]
                keys = _key(cc[0], cc[1], cc[2], nd)
                ex = inside & self.exists(d, keys)
                ref = ex & self.is_refined(d, keys)
                same = ex & ~ref
                coarse = inside & ~ex
                kk = np.full(len(sel), WALL, np.int8)
                rr = np.full(len(sel), -1, np.int64)
                kk[same] = SAME
                rr[same] = self.leaf_rank(d, cc[0][same], cc[1][same], cc[2][same])
                kk[ref] = FINER
                kk[coarse] = COARSER
                if np.any(coarse):
                    rr[coarse] = self.leaf_rank(d - 1, cc[0][coarse] // 2, cc[1][coarse] // 2,
                                                cc[2][coarse] // 2)
                kind[sel, q] = kk
                rank[sel, q] = rr
        return kind, rank

    def faces(self):
        """Interior faces in canonical order (axis, depth, Morton key of the +-side cell at
        that depth).  A face between same-depth leaves is the - face of its + leaf; a
        T-junction sub-face is named at the fine depth (its + cell is virtual when the
        fine leaf is on the - side).  Fields: axis, depth, i, j, k, minus, plus (leaf
        ranks of the two sides; the coarse leaf for the coarse side)."""
        kind, rank = self.neighbour_table()
        L = self.leaves
        ax, dp, fi, fj, fk, mi, pl = [], [], [], [], [], [], []
        idx = np.arange(self.n_leaves)
        for a in range(3):
            # - faces of leaves whose - neighbour is a same-depth leaf or a coarser leaf
            q = 2 * a
            sel = (kind[:, q] == SAME) | (kind[:, q] == COARSER)
            ax.append(np.full(sel.sum(), a)); dp.append(L["depth"][sel])
            fi.append(L["i"][sel]); fj.append(L["j"][sel]); fk.append(L["k"][sel])
            mi.append(rank[sel, q]); pl.append(idx[sel])
            # + faces of leaves whose + neighbour is coarser (virtual + cell)
            q = 2 * a + 1
            sel = kind[:, q] == COARSER
            c = [L["i"][sel].copy(), L["j"][sel].copy(), L["k"][sel].copy()]
            c[a] = c[a] + 1
            ax.append(np.full(sel.sum(), a)); dp.append(L["depth"][sel])
            fi.append(c[0]); fj.append(c[1]); fk.append(c[2])
            mi.append(idx[sel]); pl.append(rank[sel, q])
        f = {"axis": np.concatenate(ax).astype(np.int64), "depth": np.concatenate(dp),
             "i": np.concatenate(fi), "j": np.concatenate(fj), "k": np.concatenate(fk),
             "minus": np.concatenate(mi), "plus": np.concatenate(pl)}
        order = np.lexsort((morton(f["i"], f["j"], f["k"]), f["depth"], f["axis"]))
        return {k: v[order] for k, v in f.items()}

    def coarsest_n(self):
        """Multigrid levels below the root halve the root grid while its size is even
        and larger than 4 (the coarsest-level rule; the paper's tiles imply 8^3 but do
        not fix it)."""
        n = self.n0
        levels = 0
        while n % 2 == 0 and n > 4:
            n //= 2
            levels += 1
        return n, levels

    def level_cells(self, m):
        """Cells of multigrid level m (sorted by Morton key): depth-m cells (leaves and
        inner) for m >= 0, the uniform root coarsening of size n0/2^-m for m < 0.
        Returns (i, j, k, is_leaf)."""
        if m >= 0:
            nd = self.nd(m)
            i, j, k = _unkey(self.exist[m], nd)
            leaf = ~self.is_refined(m, self.exist[m])
        else:
            n = self.n0 >> (-m)
            ii, jj, kk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
            i, j, k = ii.ravel(), jj.ravel(), kk.ravel()
            leaf = np.zeros(len(i), bool)
        o = np.argsort(morton(i, j, k), kind="stable")
        return i[o], j[o], k[o], leaf[o]

    def min_level(self):
        return -self.coarsest_n()[1]
