"""Python face of libocg: Octree / Hierarchy handles and the solve calls.

Marshalling only: every arithmetic step runs inside libocg.so (host octree build, CUDA
kernels for set-up, operator, cycle and Krylov loop).  Device vectors are torch CUDA
tensors; the library fails loudly (ImportError / OcgError) when it is missing or a call
fails — there is no CPU path here.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import _lib as L
from . import problems as P


def _desc(d: P.OctreeDesc) -> L.OctreeDesc:
    out = L.OctreeDesc()
    out.n0 = d.n0
    out.max_depth = d.max_depth
    out.refine = d.refine
    out.band = d.band
    out.tile_log2 = d.tile_log2
    if len(d.spheres) > 4 or len(d.boxes) > 4 or len(d.sines) > 8:
        raise ValueError("at most 4 spheres, 4 boxes and 8 sine waves")
    out.n_sines = len(d.sines)
    for q, w in enumerate(d.sines):
        for c in range(5):
            out.sines[q][c] = float(w[c])
    out.n_spheres = len(d.spheres)
    out.n_boxes = len(d.boxes)
    for q, s in enumerate(d.spheres):
        for c in range(4):
            out.spheres[q][c] = float(s[c])
    for q, b in enumerate(d.boxes):
        for c in range(6):
            out.boxes[q][c] = float(b[c])
    return out


def sphere_change_box(old, new, band: float, n0: int):
    """The box for Octree.rebuild after one sphere of an SDF_BAND or BALL_CENTRE description
    moved or changed its radius from old = (cx, cy, cz, r) to new: the two spheres' bounding
    boxes grown by band + sqrt(3)/2 / n0, the farthest a cell centre can be from the sphere's
    surface and still have the sphere decide its refinement (outside it the signed distance
    to that sphere exceeds every depth's slack, so the minimum over the primitives, and with
    it the predicate, is unchanged)."""
    g = float(band) + 0.5 * math.sqrt(3.0) / n0
    lo = [min(old[a] - old[3], new[a] - new[3]) - g for a in range(3)]
    hi = [max(old[a] + old[3], new[a] + new[3]) + g for a in range(3)]
    return tuple(lo + hi)


class Octree:
    """Host-built octree (libocg ocg_octree_build) with its canonical exports."""

    def __init__(self, desc: P.OctreeDesc, _prev=None, _box=None):
        lib = L.lib()
        self._h = C.c_void_p()
        self.desc = desc
        if _prev is None:
            L.check(lib.ocg_octree_build(C.byref(_desc(desc)), C.byref(self._h)))
        else:
            bx = (C.c_double * 6)(*[float(v) for v in _box])
            L.check(lib.ocg_octree_rebuild(_prev._h, C.byref(_desc(desc)), bx, C.byref(self._h)))
        c = (C.c_int64 * 8)()
        L.check(lib.ocg_octree_counts(self._h, c))
        (self.n_leaves, self.n_faces, self.D, self.mc, self.n_cells, self.n_trec, self.n_tree,
         self.n_oct) = [int(v) for v in c]

    def rebuild(self, desc: P.OctreeDesc, box):
        """The octree of desc, built from this one after a change of the geometry confined
        to box = (lox, loy, loz, hix, hiy, hiz) (ocg_octree_rebuild: the refinement
        predicate is evaluated again only there)."""
        return Octree(desc, _prev=self, _box=box)

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            L.lib().ocg_octree_destroy(self._h)
            self._h = C.c_void_p()

    @property
    def handle(self):
        return self._h

    def leaves(self):
        n = self.n_leaves
        a = {k: np.empty(n, np.int32) for k in ("depth", "i", "j", "k")}
        L.check(L.lib().ocg_octree_export_leaves(self._h, L.ptr(a["depth"]), L.ptr(a["i"]),
                                                 L.ptr(a["j"]), L.ptr(a["k"])))
        return {k: v.astype(np.int64) for k, v in a.items()}

    def leaf_depths(self):
        """Depth of every leaf in canonical order (int32), without the coordinates."""
        d = np.empty(self.n_leaves, np.int32)
        L.check(L.lib().ocg_octree_export_leaves(self._h, L.ptr(d), None, None, None))
        return d

    def neighbours(self):
        kind = np.empty((self.n_leaves, 6), np.int8)
        rank = np.empty((self.n_leaves, 6), np.int64)
        L.check(L.lib().ocg_octree_export_neighbours(self._h, L.ptr(kind), L.ptr(rank)))
        return kind, rank

    def faces(self):
        n = self.n_faces
        a = {k: np.empty(n, np.int32) for k in ("axis", "depth", "i", "j", "k")}
        mi = np.empty(n, np.int64)
        pl = np.empty(n, np.int64)
        L.check(L.lib().ocg_octree_export_faces(self._h, L.ptr(a["axis"]), L.ptr(a["depth"]),
                                                L.ptr(a["i"]), L.ptr(a["j"]), L.ptr(a["k"]),
                                                L.ptr(mi), L.ptr(pl)))
        out = {k: v.astype(np.int64) for k, v in a.items()}
        out["minus"] = mi
        out["plus"] = pl
        return out

    def faces_range(self, first, count):
        """Canonical faces first .. first+count-1 as int32 / int64 numpy arrays."""
        a = {k: np.empty(count, np.int32) for k in ("axis", "depth", "i", "j", "k")}
        mi = np.empty(count, np.int64)
        pl = np.empty(count, np.int64)
        L.check(L.lib().ocg_octree_export_faces_range(self._h, first, count, L.ptr(a["axis"]),
                                                      L.ptr(a["depth"]), L.ptr(a["i"]), L.ptr(a["j"]),
                                                      L.ptr(a["k"]), L.ptr(mi), L.ptr(pl)))
        a["minus"] = mi
        a["plus"] = pl
        return a

    def level_size(self, m):
        """Number of cells of multigrid level m."""
        n = C.c_int64()
        L.check(L.lib().ocg_octree_export_level(self._h, m, C.byref(n), None, None, None, None))
        return int(n.value)

    def level(self, m):
        n = C.c_int64()
        L.check(L.lib().ocg_octree_export_level(self._h, m, C.byref(n), None, None, None, None))
        n = n.value
        i, j, k = (np.empty(n, np.int32) for _ in range(3))
        leaf = np.empty(n, np.int8)
        L.check(L.lib().ocg_octree_export_level(self._h, m, C.byref(C.c_int64(n)), L.ptr(i), L.ptr(j),
                                                L.ptr(k), L.ptr(leaf)))
        return i.astype(np.int64), j.astype(np.int64), k.astype(np.int64), leaf.astype(bool)


SWEEP_FORMS = {"auto": L.OCG_SWEEP_AUTO, "octet": L.OCG_SWEEP_OCTET, "cell": L.OCG_SWEEP_CELL,
               "quad": L.OCG_SWEEP_QUAD, "tile": L.OCG_SWEEP_TILE}
SWEEP_FORM_NAMES = {L.OCG_SWEEP_OCTET: "octet", L.OCG_SWEEP_CELL: "cell", L.OCG_SWEEP_QUAD: "quad",
                    L.OCG_SWEEP_TILE: "tile"}


_HOOKS = []   # callbacks stay alive: blocks made through them are released through them


def use_torch_allocator(enable=True):
    """Route the library's device allocations through torch's caching allocator
    (ocg_set_allocator), or back to cudaMalloc with enable=False."""
    import torch
    if not enable:
        L.check(L.lib().ocg_set_allocator(L.ALLOC_FN(), L.FREE_FN(), None))
        return

    def alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes))
        except RuntimeError:
            return None

    def free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    hooks = (L.ALLOC_FN(alloc), L.FREE_FN(free))
    _HOOKS.append(hooks)
    L.check(L.lib().ocg_set_allocator(hooks[0], hooks[1], None))


def mg_params(mu=1, nu_pre=2, nu_post=2, nu_coarsest=10, beta=2.0, alpha=2.0, coef="f32",
              bf16_coarse=False, sweep="auto", mu_min_cells=0, coarsening="algebraic") -> L.MGParams:
    """coarsening: "algebraic" (Alg. 3, the paper's method) or "geometric" (the geometric
    multigrid of Sec. 3.3, an ablation: cells with children rediscretised from the
    description's solids at their own resolution)."""
    p = L.MGParams()
    p.mu, p.nu_pre, p.nu_post, p.nu_coarsest = mu, nu_pre, nu_post, nu_coarsest
    p.mu_min_cells = mu_min_cells
    p.coarsening = {"algebraic": L.OCG_COARSEN_ALGEBRAIC, "geometric": L.OCG_COARSEN_GEOMETRIC}[coarsening]
    p.beta_restrict, p.alpha = beta, alpha
    p.coef_dtype = L.OCG_F64 if coef == "f64" else L.OCG_F32
    p.bf16_coarse = 1 if bf16_coarse else 0
    p.sweep_form = SWEEP_FORMS[sweep]
    return p


PRECISIONS = {"fp64": L.OCG_PREC_FP64, "fp32": L.OCG_PREC_FP32, "mixed": L.OCG_PREC_MIXED}


class Hierarchy:
    """Multigrid hierarchy on the current CUDA device (ocg_setup_hierarchy)."""

    def __init__(self, tree: Octree, beta, bc, prm: L.MGParams = None, stream=None):
        import torch
        lib = L.lib()
        self.tree = tree
        self.prm = prm or mg_params()
        if isinstance(beta, np.ndarray):
            beta = torch.from_numpy(np.ascontiguousarray(beta, np.float32)).cuda()
        assert beta.dtype == torch.float32 and beta.is_cuda and beta.numel() == tree.n_faces
        self._beta = beta
        self._bc = tuple(int(v) for v in bc)
        bcv = (C.c_int32 * 6)(*self._bc)
        self._h = C.c_void_p()
        st = C.c_void_p(stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream)
        L.check(lib.ocg_setup_hierarchy(tree.handle, L.ptr(beta), bcv, C.byref(self.prm), st,
                                        C.byref(self._h)))

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            L.lib().ocg_hier_destroy(self._h)
            self._h = C.c_void_p()

    @property
    def handle(self):
        return self._h

    def coefs(self, m):
        i, _, _, _ = self.tree.level(m)
        n = len(i)
        out = [np.empty(n) for _ in range(4)]
        L.check(L.lib().ocg_hier_export_coefs(self._h, m, *[L.ptr(a) for a in out]))
        return out

    def update_beta(self, beta, stream=None):
        """Recompute the coefficients in place for new face fractions beta on the same tree
        (ocg_hier_update_beta); captured graphs and batches stay valid."""
        import torch
        if isinstance(beta, np.ndarray):
            beta = torch.from_numpy(np.ascontiguousarray(beta, np.float32)).cuda()
        assert beta.dtype == torch.float32 and beta.is_cuda and beta.numel() == self.tree.n_faces
        beta = beta.contiguous()
        L.check(L.lib().ocg_hier_update_beta(self._h, L.ptr(beta), self._stream(stream)))

    def tuning(self):
        """{level: (form, us_octet, us_cell, us_quad, us_tile)} as chosen / measured at set-up."""
        out = {}
        for m in range(self.tree.mc, self.tree.D + 1):
            f = C.c_int32()
            us = [C.c_double() for _ in range(4)]
            L.check(L.lib().ocg_hier_tuning(self._h, m, C.byref(f), *[C.byref(v) for v in us]))
            out[m] = (f.value,) + tuple(v.value for v in us)
        return out

    @staticmethod
    def _stream(stream):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        return C.c_void_p(s.cuda_stream)

    def apply_A(self, x, stream=None, transpose=False):
        """y = A x (or A^T x) of the composite leaf operator."""
        import torch
        y = torch.empty_like(x)
        dt = L.OCG_F64 if x.dtype == torch.float64 else L.OCG_F32
        L.check(L.lib().ocg_apply_A(self._h, dt, L.ptr(x), L.ptr(y), 1 if transpose else 0,
                                    self._stream(stream)))
        return y

    @property
    def nullspace(self):
        """True when every wall is Neumann (constant null space, zero-mean solutions)."""
        return all(int(v) == 0 for v in self._bc)

    def face_grad(self, p, lam, stream=None):
        """dL/dbeta per canonical face from the solution p and the adjoint solution lam."""
        import torch
        assert p.dtype == torch.float64 and lam.dtype == torch.float64
        out = torch.empty(self.tree.n_faces, dtype=torch.float64, device=p.device)
        L.check(L.lib().ocg_face_grad(self._h, L.ptr(p), L.ptr(lam), L.ptr(out), self._stream(stream)))
        return out

    def vcycle(self, r, stream=None):
        import torch
        z = torch.empty_like(r)
        dt = L.OCG_F64 if r.dtype == torch.float64 else L.OCG_F32
        L.check(L.lib().ocg_vcycle(self._h, dt, L.ptr(r), L.ptr(z), self._stream(stream)))
        return z

    def vcycle_transpose(self, z, stream=None):
        """r = M^T z, the transpose of vcycle (preconditioner of the adjoint solve)."""
        import torch
        r = torch.empty_like(z)
        dt = L.OCG_F64 if z.dtype == torch.float64 else L.OCG_F32
        L.check(L.lib().ocg_vcycle_transpose(self._h, dt, L.ptr(z), L.ptr(r), self._stream(stream)))
        return r

    def solve(self, b, x=None, tol=1e-6, max_iter=100, precision="mixed", nullspace=-1,
              stream=None, raise_on_notconv=True, eager=False, transpose=False, unrolled=False,
              method="pcg", warm=False):
        """x with A x = b (PCG, Alg. 1), or A^T x = b with transpose=True (the adjoint
        system, preconditioned by the transposed cycle M^T: Alg. 1 with method="pcg",
        BiCGStab with method="bicgstab").  warm=True starts from the content of x (which
        must be given) instead of 0.  Returns (x, stats)."""
        import torch
        assert b.dtype == torch.float64 and b.is_cuda
        if x is None:
            if warm:
                raise ValueError("warm=True needs the initial guess in x")
            x = torch.empty_like(b)
        sp = L.SolveParams()
        sp.tol, sp.max_iter, sp.precision, sp.nullspace = tol, max_iter, PRECISIONS[precision], nullspace
        if method not in ("pcg", "bicgstab"):
            raise ValueError("method must be 'pcg' or 'bicgstab'")
        sp.flags = ((L.OCG_SOLVE_EAGER if eager else 0) | (L.OCG_SOLVE_TRANSPOSE if transpose else 0) |
                    (L.OCG_SOLVE_UNROLLED if unrolled else 0) |
                    (L.OCG_SOLVE_BICGSTAB if transpose and method == "bicgstab" else 0) |
                    (L.OCG_SOLVE_WARM if warm else 0))
        st = L.SolveStats()
        code = L.lib().ocg_pcg_solve(self._h, L.ptr(b), L.ptr(x), C.byref(sp), C.byref(st),
                                     self._stream(stream))
        if code not in (L.OCG_OK, L.OCG_ENOTCONV) or (code == L.OCG_ENOTCONV and raise_on_notconv):
            L.check(code)
        return x, st


class Batch:
    """Many independent hierarchies solved together (ocg_batch_create /
    ocg_pcg_solve_batched): one launch per phase for all problems, per-problem scalars
    and stop tests, one CUDA graph for the whole loop."""

    def __init__(self, hiers, stream=None):
        import torch
        self.hiers = list(hiers)          # kept alive for the batch's lifetime
        n = len(self.hiers)
        arr = (C.c_void_p * n)(*[h.handle.value for h in self.hiers])
        self._h = C.c_void_p()
        st = C.c_void_p(stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream)
        L.check(L.lib().ocg_batch_create(C.cast(arr, C.c_void_p), n, st, C.byref(self._h)))

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            L.lib().ocg_batch_destroy(self._h)
            self._h = C.c_void_p()

    def info(self):
        """{height: (form, us_octet, us_cell)} of the batched sweeps."""
        hts, f, a, b = C.c_int32(), C.c_int32(), C.c_double(), C.c_double()
        L.check(L.lib().ocg_batch_info(self._h, 1, C.byref(hts), C.byref(f), C.byref(a), C.byref(b)))
        out = {}
        for h in range(1, hts.value + 1):
            L.check(L.lib().ocg_batch_info(self._h, h, C.byref(hts), C.byref(f), C.byref(a), C.byref(b)))
            out[h] = (f.value, a.value, b.value)
        return out

    def solve(self, bs, xs=None, tol=1e-6, max_iter=100, nullspace=-1, stream=None, raise_on_notconv=True):
        import torch
        n = len(self.hiers)
        assert len(bs) == n and all(b.dtype == torch.float64 and b.is_cuda for b in bs)
        if xs is None:
            xs = [torch.empty_like(b) for b in bs]
        bp = (C.c_void_p * n)(*[b.data_ptr() for b in bs])
        xp = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
        sp = L.SolveParams()
        sp.tol, sp.max_iter, sp.precision, sp.nullspace, sp.flags = tol, max_iter, L.OCG_PREC_MIXED, nullspace, 0
        stats = (L.SolveStats * n)()
        s = stream if stream is not None else torch.cuda.current_stream()
        code = L.lib().ocg_pcg_solve_batched(self._h, C.cast(bp, C.c_void_p), C.cast(xp, C.c_void_p), C.byref(sp),
                                             C.cast(stats, C.c_void_p), C.c_void_p(s.cuda_stream))
        if code not in (L.OCG_OK, L.OCG_ENOTCONV) or (code == L.OCG_ENOTCONV and raise_on_notconv):
            L.check(code)
        return xs, list(stats)
