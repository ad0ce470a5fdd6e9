"""Seeded synthetic problem generators for the octree Poisson solve.

This module produces INPUTS only: octree descriptions (root size, depth, refinement
predicate parameters), per-face beta (fluid area fractions of cut faces), and
right-hand sides (manufactured solutions, random divergence fields). It holds none
of the solver's arithmetic (no operator, no coarsening, no cycle, no Krylov step);
both the CUDA library and the CPU oracle consume its arrays unchanged.

Geometry conventions shared by every consumer:
  * Domain is the unit cube; the root grid has n0^3 cells; depth d has cell size
    h_d = 1/(n0*2^d) and integer coordinates 0 <= i,j,k < n0*2^d.
  * A face is named by (axis, depth, i, j, k): the depth of its finer side and the
    integer coordinates, at that depth, of the cell on its + side (for a T-face whose
    fine cell sits on the - side, that + cell is the virtual fine cell inside the
    coarse leaf).  The face lies in the plane x_axis = i_axis * h_depth.
  * Wall order for boundary conditions: x-, x+, y-, y+, z-, z+; 1 = Dirichlet (value
    prescribed at the wall face), 0 = Neumann.

The configurations mirror the paper's test grids (Sec. 4.1): a ball refined around the
centre, narrow-band refinement around solid surfaces, and a band around the zero set
of a random smooth field.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NEUMANN = 0
DIRICHLET = 1

REFINE_NONE = 0
REFINE_BALL_CENTRE = 1
REFINE_SDF_BAND = 2
REFINE_SINE_BAND = 3
REFINE_STAR_BAND = 4

MAX_SPHERES = 4
MAX_BOXES = 4
MAX_SINES = 8


@dataclass
class OctreeDesc:
    """Refinement description of an adaptive octree (Sec. 3, Sec. 4.1).

    refine == REFINE_BALL_CENTRE: a depth-d cell (d < max_depth) is refined iff its
        centre lies strictly inside the first sphere (squared distance < r^2).
    refine == REFINE_SDF_BAND: refined iff |phi(centre)| < band + (sqrt(3)/2) h_d, with
        phi the minimum of the sphere and box signed distances.
    refine == REFINE_SINE_BAND: refined iff |phi(centre)| < band + |grad phi(centre)|
        (sqrt(3)/2) h_d, phi = (1/n) sum_m sin(2 pi kappa_m (d_m . x) + theta_m).
    refine == REFINE_STAR_BAND: refined iff |phi(centre)| < band + L (sqrt(3)/2) h_d with
        phi = r - (r0 + a cos(k theta) cos(k phi)) about spheres[0] = (c, r0) and
        spheres[1] = (a, k, L, 0) (the star surface of Sec. 4.1).
    tile_log2 = t > 0: every aligned tile of 2^t cells per axis takes one decision, the
        predicate of the depth-(d - t) cell covering it (Sec. 4.1 refines 8^3 tiles, t = 3).
    """

    n0: int
    max_depth: int
    refine: int = REFINE_NONE
    band: float = 0.0
    spheres: list = field(default_factory=list)   # (cx, cy, cz, r)
    boxes: list = field(default_factory=list)     # (lox, loy, loz, hix, hiy, hiz)
    sines: list = field(default_factory=list)     # (kappa, dx, dy, dz, theta)
    tile_log2: int = 0    # the predicate decides per aligned tile of 2^tile_log2 cells per axis


@dataclass
class Problem:
    name: str
    desc: OctreeDesc
    bc: tuple                 # 6 wall codes
    beta: str = "one"         # "one", "cut" (clamped fluid fraction), "cut_exact" or "cut_centre"
    rhs: str = "zero"         # "sin_dirichlet", "exp_sin_cos", "sinusoidal", "divergence", "tank", "normal"
    seed: int = 0
    mode: str = "mixed"       # suggested precision mode
    tol: float = 1e-6
    mu: int = 1
    solid_spheres: list = field(default_factory=list)
    solid_boxes: list = field(default_factory=list)
    solid_sines: list = field(default_factory=list)
    sine_offset: float = 0.0
    solid_star: list = field(default_factory=list)   # [(cx, cy, cz, r0), (a, k, ...)]

    @property
    def neumann(self) -> bool:
        return all(c == NEUMANN for c in self.bc)


# ----------------------------------------------------------------------------------
# configurations

CUT_SPHERE = (0.5, 0.5, 0.5, 0.2)
CUT_BOX = (0.65, 0.2, 0.3, 0.85, 0.8, 0.7)


def uniform(n0: int = 32) -> Problem:
    """Uniform n0^3 grid, beta = 1, homogeneous Dirichlet walls, p = sin(pi x)sin(pi y)sin(pi z)."""
    return Problem("uniform%d" % n0, OctreeDesc(n0, 0), (DIRICHLET,) * 6,
                   beta="one", rhs="sin_dirichlet", mode="fp64", tol=1e-10)


def two_level_ball(n0: int = 64, radius: float = 0.25) -> Problem:
    """n0^3 base, cells with centre within `radius` of the cube centre refined once;
    beta = 1, Dirichlet walls with the manufactured p = exp(x) sin(2 pi y) cos(2 pi z)."""
    d = OctreeDesc(n0, 1, REFINE_BALL_CENTRE, spheres=[(0.5, 0.5, 0.5, radius)])
    return Problem("ball%d" % n0, d, (DIRICHLET,) * 6, beta="one", rhs="exp_sin_cos",
                   mode="mixed", tol=1e-6)


def cut_cell(n0: int = 64, depth: int = 2, band: float = 0.05, seed: int = 4) -> Problem:
    """Cut-cell projection: band refinement around a solid sphere and box; fluid-fraction
    beta clamped to [1e-3, 1]; Neumann everywhere; rhs = divergence of N(0,1) face
    velocities, mean removed."""
    d = OctreeDesc(n0, depth, REFINE_SDF_BAND, band=band, spheres=[CUT_SPHERE], boxes=[CUT_BOX])
    return Problem("cut%d_d%d" % (n0, depth), d, (NEUMANN,) * 6, beta="cut", rhs="divergence",
                   seed=seed, mode="mixed_bf16", tol=1e-6,
                   solid_spheres=[CUT_SPHERE], solid_boxes=[CUT_BOX])


def batch_tree(k: int) -> Problem:
    """Tree k of the batched set: effective resolution from {64, 96, 128}, 2-3 levels,
    band refinement within 0.05 of a random sphere; even k Dirichlet beta=1, odd k cut-cell
    Neumann."""
    rng = np.random.default_rng(5 + k)
    eff = int(rng.choice([64, 96, 128]))
    levels = int(rng.choice([2, 3]))
    depth = levels - 1
    n0 = eff // (2 ** depth)
    r = float(rng.uniform(0.1, 0.3))
    c = rng.uniform(0.3, 0.7, size=3)
    sph = (float(c[0]), float(c[1]), float(c[2]), r)
    d = OctreeDesc(n0, depth, REFINE_SDF_BAND, band=0.05, spheres=[sph])
    if k % 2 == 0:
        return Problem("batch_t%d" % k, d, (DIRICHLET,) * 6, beta="one", rhs="normal",
                       seed=100 + k, mode="mixed", tol=1e-6)
    return Problem("batch_t%d" % k, d, (NEUMANN,) * 6, beta="cut", rhs="normal", seed=100 + k,
                   mode="mixed", tol=1e-6, solid_spheres=[sph])


def sine_waves(seed: int = 6, n: int = 8):
    """Random smooth field (1/n) sum sin(2 pi kappa (d.x) + theta), kappa in {1..4}."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        kappa = float(rng.integers(1, 5))
        v = rng.normal(size=3)
        v = v / np.linalg.norm(v)
        theta = float(rng.uniform(0.0, 2.0 * math.pi))
        out.append((kappa, float(v[0]), float(v[1]), float(v[2]), theta))
    return out


def sine_band(n0: int = 128, depth: int = 3, band: float = 0.02, seed: int = 7) -> Problem:
    sines = sine_waves()
    d = OctreeDesc(n0, depth, REFINE_SINE_BAND, band=band, sines=sines)
    return Problem("sine%d_d%d" % (n0, depth), d, (NEUMANN,) * 6, beta="cut",
                   rhs="divergence", seed=seed, mode="mixed", tol=1e-6, solid_sines=sines)


def by_name(name: str) -> Problem:
    table = {"uniform": uniform, "two_level_ball": two_level_ball, "cut_cell": cut_cell, "sine_band": sine_band}
    return table[name]()


# ----------------------------------------------------------------------------------
# geometry helpers (vectorised numpy, float64)

def solid_sdf(p: Problem, x, y, z):
    """Signed distance of the fluid region (positive in fluid, negative in solids):
    min over sphere and box distances, or the sine field."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    z = np.asarray(z, np.float64)
    phi = np.full(np.broadcast(x, y, z).shape, np.inf)
    for (cx, cy, cz, r) in p.solid_spheres:
        phi = np.minimum(phi, np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) - r)
    for (lx, ly, lz, hx, hy, hz) in p.solid_boxes:
        qx = np.abs(x - 0.5 * (lx + hx)) - 0.5 * (hx - lx)
        qy = np.abs(y - 0.5 * (ly + hy)) - 0.5 * (hy - ly)
        qz = np.abs(z - 0.5 * (lz + hz)) - 0.5 * (hz - lz)
        out = np.sqrt(np.maximum(qx, 0) ** 2 + np.maximum(qy, 0) ** 2 + np.maximum(qz, 0) ** 2)
        ins = np.minimum(np.maximum(qx, np.maximum(qy, qz)), 0.0)
        phi = np.minimum(phi, out + ins)
    if p.solid_sines:
        s = np.zeros_like(phi)
        for (kap, dx, dy, dz, th) in p.solid_sines:
            s = s + np.sin(2 * math.pi * kap * (dx * x + dy * y + dz * z) + th)
        phi = np.minimum(phi, s / len(p.solid_sines) - p.sine_offset)
    if p.solid_star:
        phi = np.minimum(phi, star_field(p.solid_star, x, y, z))
    return phi


def star_field(star, x, y, z):
    """r - (r0 + a cos(k theta) cos(k phi)) about (cx, cy, cz) (the star surface of
    Sec. 4.1; theta polar from +z, phi azimuth from +x), positive outside the star."""
    (cx, cy, cz, r0), (a, k) = star[0], star[1][:2]
    dx, dy, dz = x - cx, y - cy, z - cz
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    rho = np.sqrt(dx * dx + dy * dy)
    with np.errstate(divide="ignore", invalid="ignore"):
        th = np.arccos(np.where(r > 0, dz / np.where(r > 0, r, 1.0), 1.0))
        ph = np.arctan2(dy, dx)
    return r - (r0 + a * np.cos(k * th) * np.cos(k * ph))


def _tri_positive_fraction(a, b, c):
    """Area fraction of {phi > 0} on a triangle where phi is linear with vertex values a,b,c."""
    v = np.stack([a, b, c], axis=-1)
    v = np.sort(v, axis=-1)
    lo, mid, hi = v[..., 0], v[..., 1], v[..., 2]
    out = np.zeros(lo.shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        # exactly one vertex positive: similar triangle at the positive corner
        one = (hi > 0) & (mid <= 0)
        f1 = hi * hi / ((hi - lo) * (hi - mid))
        # two vertices positive: complement of the negative corner triangle
        two = (mid > 0) & (lo <= 0)
        f2 = 1.0 - lo * lo / ((mid - lo) * (hi - lo))
    out = np.where(lo > 0, 1.0, out)
    out = np.where(one, f1, out)
    out = np.where(two, f2, out)
    return out


def face_fluid_fraction(p: Problem, faces) -> np.ndarray:
    """Fluid area fraction of each face from the SDF at its four corners, splitting the
    face into two triangles along its (0,0)-(1,1) diagonal (local axes = the two other
    axes in increasing order) and integrating the linear interpolant exactly."""
    axis = faces["axis"]
    h = 1.0 / (p.desc.n0 * (2.0 ** faces["depth"]))
    ijk = np.stack([faces["i"], faces["j"], faces["k"]], axis=1).astype(np.float64)
    base = ijk * h[:, None]
    frac = np.empty(len(axis))
    for a in range(3):
        sel = axis == a
        if not np.any(sel):
            continue
        u, v = [b for b in range(3) if b != a]
        b0 = base[sel]
        hh = h[sel]

        def corner(du, dv):
            q = b0.copy()
            q[:, u] += du * hh
            q[:, v] += dv * hh
            return solid_sdf(p, q[:, 0], q[:, 1], q[:, 2])

        p00, p10, p11, p01 = corner(0, 0), corner(1, 0), corner(1, 1), corner(0, 1)
        t1 = _tri_positive_fraction(p00, p10, p11)
        t2 = _tri_positive_fraction(p00, p11, p01)
        frac[sel] = 0.5 * (t1 + t2)
    return frac


def face_beta(p: Problem, faces, leaves=None) -> np.ndarray:
    """Per-face beta in canonical face order (float32): 1 for beta="one"; the clamped
    fluid fraction max(1e-3, min(1, f)) for beta="cut"; the fraction itself in [0, 1]
    for beta="cut_exact" (cells inside the solid become inactive); for beta="cut_centre"
    (needs the leaves) the ghost-fluid classification of Sec. 2.1: a leaf whose centre lies
    in the solid (signed distance < 0) is a Neumann cell, no unknown, and every face that
    touches it gets 0; the faces between two cells whose centres are in the fluid keep
    their fluid fraction (the cut-cell coefficients)."""
    n = len(faces["axis"])
    if p.beta == "one":
        return np.ones(n, np.float32)
    f = face_fluid_fraction(p, faces)
    if p.beta == "cut_centre":
        if leaves is None:
            raise ValueError("beta='cut_centre' needs the leaves")
        h, x, y, z = _leaf_geometry(p, leaves)
        solid = solid_sdf(p, x, y, z) < 0.0
        touch = solid[np.asarray(faces["minus"])] | solid[np.asarray(faces["plus"])]
        return np.where(touch, 0.0, np.clip(f, 0.0, 1.0)).astype(np.float32)
    if p.beta == "cut_exact":
        # the exact fraction: faces inside the solid get 0, so a cell inside the solid has
        # no coefficient and drops out of the system (an inactive cell)
        return np.clip(f, 0.0, 1.0).astype(np.float32)
    return np.clip(f, 1e-3, 1.0).astype(np.float32)


# ----------------------------------------------------------------------------------
# right-hand sides

def _leaf_geometry(p: Problem, leaves):
    d = leaves["depth"].astype(np.float64)
    h = 1.0 / (p.desc.n0 * 2.0 ** d)
    x = (leaves["i"] + 0.5) * h
    y = (leaves["j"] + 0.5) * h
    z = (leaves["k"] + 0.5) * h
    return h, x, y, z


def exact_solution(p: Problem, x, y, z):
    if p.rhs == "sin_dirichlet":
        return np.sin(math.pi * x) * np.sin(math.pi * y) * np.sin(math.pi * z)
    if p.rhs == "exp_sin_cos":
        return np.exp(x) * np.sin(2 * math.pi * y) * np.cos(2 * math.pi * z)
    if p.rhs == "sinusoidal":
        # lap p = 4 pi G A sin(2 pi x) sin(2 pi y) sin(2 pi z) on the unit cube, G A = 1
        return -np.sin(2 * math.pi * x) * np.sin(2 * math.pi * y) * np.sin(2 * math.pi * z) / (3 * math.pi)
    raise ValueError("no closed-form solution for rhs kind %r" % p.rhs)


def _source(p: Problem, x, y, z):
    """f = -lap(p_exact)."""
    if p.rhs == "sin_dirichlet":
        return 3 * math.pi ** 2 * exact_solution(p, x, y, z)
    if p.rhs == "exp_sin_cos":
        return (8 * math.pi ** 2 - 1.0) * exact_solution(p, x, y, z)
    if p.rhs == "sinusoidal":
        return 12 * math.pi ** 2 * exact_solution(p, x, y, z)
    raise ValueError(p.rhs)


# ----------------------------------------------------------------------------------
# accuracy studies (Sec. 4: Laplacian accuracy and sinusoidal Poisson tests)

ACCURACY_GRIDS = ("uniform", "ball", "band", "star")

# the star surface of Sec. 4.1: r = 0.237 + 0.079 cos(6 theta) cos(6 phi) about the centre;
# L = 1 + a k / r0 = 3 bounds the field's gradient away from the axis
STAR = [(0.5, 0.5, 0.5, 0.237), (0.079, 6.0, 3.0, 0.0)]


def paper_grid(kind: str, n0: int, depth: int = 2) -> OctreeDesc:
    """The sphere and star grids of Sec. 4.1 as the paper builds them: the base grid n0^3
    (n0 = 8 * 2^l0) cut into 8^3 tiles, a tile refined while it meets the surface, down
    to `depth` levels below the base, 2:1 balance kept per tile.  A tile meets the sphere
    when the sphere's signed distance changes sign on it (exact box test), the star when
    the star function does among the tile's 27 lattice points.  The sphere grids have
    exactly the leaf counts of Table 1 (1.64453 Mi at 64~256, 7.55078 Mi at 128~512)."""
    if kind == "sphere":
        return OctreeDesc(n0, depth, REFINE_SDF_BAND, band=0.0, spheres=[(0.5, 0.5, 0.5, 0.25)], tile_log2=3)
    if kind == "star":
        return OctreeDesc(n0, depth, REFINE_STAR_BAND, band=0.0, spheres=list(STAR), tile_log2=3)
    raise ValueError(kind)


def accuracy_desc(kind: str, n0: int) -> OctreeDesc:
    """Grids of the accuracy studies: uniform n0^3; n0^3 with cells whose centre lies
    within 0.25 of the cube centre refined once; n0^3 refined twice within 0.05 of the
    sphere of radius 0.25 about the centre; n0^3 refined twice where the cells meet the
    star surface (the paper's sphere and star grids: two levels finer near the surface)."""
    if kind == "uniform":
        return OctreeDesc(n0, 0)
    if kind == "ball":
        return OctreeDesc(n0, 1, REFINE_BALL_CENTRE, spheres=[(0.5, 0.5, 0.5, 0.25)])
    if kind == "band":
        return OctreeDesc(n0, 2, REFINE_SDF_BAND, band=0.05, spheres=[(0.5, 0.5, 0.5, 0.25)])
    if kind == "star":
        return OctreeDesc(n0, 2, REFINE_STAR_BAND, band=0.0, spheres=list(STAR))
    raise ValueError(kind)


def sinusoidal(kind: str, n0: int) -> Problem:
    """Sinusoidal Poisson test: lap p = 4 pi G A sin(2 pi x) sin(2 pi y) sin(2 pi z)
    (G A = 1) on an accuracy grid; p vanishes on the walls, which are Dirichlet."""
    return Problem("sin_%s%d" % (kind, n0), accuracy_desc(kind, n0), (DIRICHLET,) * 6, beta="one",
                   rhs="sinusoidal", mode="mixed", tol=1e-6)


def laplacian_problem(kind: str, n0: int) -> Problem:
    """Laplacian accuracy test grid: beta = 1, Neumann walls (the outermost cell layer
    is the boundary; errors are measured on the cells that do not touch a wall)."""
    return Problem("lap_%s%d" % (kind, n0), accuracy_desc(kind, n0), (NEUMANN,) * 6, beta="one")


TANK_BC = (NEUMANN, NEUMANN, NEUMANN, DIRICHLET, NEUMANN, NEUMANN)   # open to air at y = 1


def tank(obstacle: str, n0: int, solid: str = "centre", tiles: bool = False) -> Problem:
    """Static tank (Sec. 4.4): liquid filling [0,1]^3, solid bottom and sides (Neumann),
    a free surface at y = 1 (zero-pressure Dirichlet), a solid obstacle (sphere of
    radius 0.25 or the star of Sec. 4.1) at the centre with fluid-fraction beta; rhs = the
    integrated divergence of the uniform velocity (0, -1, 0) (no flux through the solid
    walls, inflow through the open top).  solid: "centre" (the paper's solver: cells whose
    centre is in the solid are Neumann cells without an unknown, faces touching them get
    0, the others their fluid fraction; face_beta then needs the leaves), "exact" (the
    exact fraction on every face: only cells with no fluid on any face drop out) or
    "clamped" (the fraction clamped at 1e-3: every cell an unknown).  The grid is refined
    two levels near the obstacle's surface: cell by cell where cells meet the surface, or
    with tiles=True by the paper's 8^3 tiles (paper_grid; roots of 32 and more)."""
    kind = {"centre": "cut_centre", "exact": "cut_exact", "clamped": "cut"}[solid]
    tag = {"centre": "", "exact": "_exact", "clamped": "_clamped"}[solid]
    if obstacle == "sphere":
        sph = (0.5, 0.5, 0.5, 0.25)
        d = paper_grid("sphere", n0) if tiles else OctreeDesc(n0, 2, REFINE_SDF_BAND, band=0.0, spheres=[sph])
        return Problem("tank_sphere%d%s%s" % (n0, tag, "_tiles" if tiles else ""), d, TANK_BC, beta=kind,
                       rhs="tank", mode="mixed", tol=1e-6, mu=2, solid_spheres=[sph])
    if obstacle == "star":
        d = paper_grid("star", n0) if tiles else accuracy_desc("star", n0)
        return Problem("tank_star%d%s%s" % (n0, tag, "_tiles" if tiles else ""), d, TANK_BC, beta=kind,
                       rhs="tank", mode="mixed", tol=1e-6, mu=2, solid_star=list(STAR))
    raise ValueError(obstacle)


def laplacian_test_function(x, y, z):
    """f = (x^2 + y^2 + z^2) exp(-xyz)."""
    return (x * x + y * y + z * z) * np.exp(-x * y * z)


def laplacian_test_exact(x, y, z):
    """lap f for laplacian_test_function, differentiated from its definition:
    exp(-xyz) (6 - 12 xyz + (x^2 + y^2 + z^2)(x^2 y^2 + y^2 z^2 + z^2 x^2))."""
    r2 = x * x + y * y + z * z
    return np.exp(-x * y * z) * (6.0 - 12.0 * x * y * z + r2 * (x * x * y * y + y * y * z * z + z * z * x * x))


def leaf_centres(n0: int, leaves):
    """(h, x, y, z) of the leaves (canonical order)."""
    d = np.asarray(leaves["depth"]).astype(np.float64)
    h = 1.0 / (n0 * 2.0 ** d)
    return h, (np.asarray(leaves["i"]) + 0.5) * h, (np.asarray(leaves["j"]) + 0.5) * h, \
        (np.asarray(leaves["k"]) + 0.5) * h


def interior_leaves(n0: int, leaves):
    """Mask of the leaves that touch no domain wall."""
    nd = n0 * 2 ** np.asarray(leaves["depth"]).astype(np.int64)
    i, j, k = (np.asarray(leaves[c]) for c in ("i", "j", "k"))
    return (i > 0) & (j > 0) & (k > 0) & (i < nd - 1) & (j < nd - 1) & (k < nd - 1)


def t_junction_leaves(n_leaves: int, leaves, faces):
    """Mask of the leaves on either side of a T-junction face (the two sides of the face
    at different depths)."""
    dm = np.asarray(leaves["depth"])[np.asarray(faces["minus"])]
    dp = np.asarray(leaves["depth"])[np.asarray(faces["plus"])]
    t = dm != dp
    mask = np.zeros(n_leaves, bool)
    mask[np.asarray(faces["minus"])[t]] = True
    mask[np.asarray(faces["plus"])[t]] = True
    return mask


def rms_v(h, e, mask=None):
    """Volume-weighted RMS of e over the masked leaves (cell volume h^3)."""
    V = h ** 3
    if mask is not None:
        V, e = V[mask], e[mask]
    return math.sqrt(float(np.sum(V * e * e) / np.sum(V)))


def rhs(p: Problem, leaves, faces=None, beta=None) -> np.ndarray:
    """Right-hand side in canonical leaf order (float64).

    Manufactured kinds: b_i = V_i f(x_i) plus, for each Dirichlet wall face of leaf i,
    the boundary lift 2 h_i g(face centre) (the wall value enters through a half-cell
    distance, so the face weight is 2 beta h with beta = 1 on walls).
    "divergence": b_i = sum over the faces of i of +-beta_f h_f^2 u_f with u_f ~ N(0,1)
    (+ on the cell's + side, - on its - side), then the mean is removed.
    "normal": N(0,1) per leaf, mean removed when every wall is Neumann.
    """
    n = len(leaves["depth"])
    if p.rhs in ("sin_dirichlet", "exp_sin_cos", "sinusoidal"):
        h, x, y, z = _leaf_geometry(p, leaves)
        b = h ** 3 * _source(p, x, y, z)
        nd = p.desc.n0 * 2 ** leaves["depth"].astype(np.int64)
        coords = (leaves["i"], leaves["j"], leaves["k"])
        centre = (x, y, z)
        for a in range(3):
            for side in (0, 1):
                if p.bc[2 * a + side] != DIRICHLET:
                    continue
                on = coords[a] == 0 if side == 0 else coords[a] == nd - 1
                if not np.any(on):
                    continue
                fc = [c[on].copy() for c in centre]
                fc[a] = np.zeros(on.sum()) if side == 0 else np.ones(on.sum())
                g = exact_solution(p, fc[0], fc[1], fc[2])
                b[on] += 2.0 * h[on] * g
        return b
    if p.rhs == "tank":
        assert faces is not None and beta is not None
        b = np.zeros(n)
        hf = 1.0 / (p.desc.n0 * 2.0 ** np.asarray(faces["depth"], np.float64))
        u = np.where(np.asarray(faces["axis"]) == 1, -1.0, 0.0)
        flux = np.asarray(beta, np.float64) * hf * hf * u
        b += np.bincount(faces["minus"], weights=flux, minlength=n)
        b -= np.bincount(faces["plus"], weights=flux, minlength=n)
        # the open top (y = 1): inflow -h^2 through the + y face of the top leaves
        hl = 1.0 / (p.desc.n0 * 2.0 ** leaves["depth"].astype(np.float64))
        top = leaves["j"] == p.desc.n0 * 2 ** leaves["depth"].astype(np.int64) - 1
        b[top] += -hl[top] ** 2
        return b
    rng = np.random.default_rng(p.seed)
    if p.rhs == "divergence":
        assert faces is not None and beta is not None
        b = np.zeros(n)
        nf = len(faces["axis"])
        for first in range(0, nf, FACE_CHUNK):
            sl = slice(first, min(nf, first + FACE_CHUNK))
            divergence_accumulate(p, b, rng, {k: v[sl] for k, v in faces.items()}, beta[sl])
        return b - b.mean()
    if p.rhs == "normal":
        b = rng.standard_normal(n)
        if p.neumann:
            b = b - b.mean()
        return b
    if p.rhs == "zero":
        return np.zeros(n)
    raise ValueError(p.rhs)


# faces per piece when face arrays are processed in pieces (the divergence right-hand side
# accumulates piece by piece in this order whatever the tree size)
FACE_CHUNK = 1 << 25


def divergence_accumulate(p: Problem, b, rng, faces, beta):
    """Adds one piece of faces (in canonical order, continuing the draws of rng) to the
    integrated divergence b: flux_f = beta_f h_f^2 u_f, u_f ~ N(0,1), added to the - leaf
    and subtracted from the + leaf."""
    n = len(b)
    hf = 1.0 / (p.desc.n0 * 2.0 ** np.asarray(faces["depth"], np.float64))
    u = rng.standard_normal(len(hf))
    flux = np.asarray(beta, np.float64) * hf * hf * u
    b += np.bincount(faces["minus"], weights=flux, minlength=n)
    b -= np.bincount(faces["plus"], weights=flux, minlength=n)


def _solid_sdf_torch(p: Problem, x, y, z):
    import torch
    phi = torch.full_like(x, float("inf"))
    for (cx, cy, cz, r) in p.solid_spheres:
        phi = torch.minimum(phi, torch.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) - r)
    for (lx, ly, lz, hx, hy, hz) in p.solid_boxes:
        qx = torch.abs(x - 0.5 * (lx + hx)) - 0.5 * (hx - lx)
        qy = torch.abs(y - 0.5 * (ly + hy)) - 0.5 * (hy - ly)
        qz = torch.abs(z - 0.5 * (lz + hz)) - 0.5 * (hz - lz)
        out = torch.sqrt(qx.clamp(min=0) ** 2 + qy.clamp(min=0) ** 2 + qz.clamp(min=0) ** 2)
        ins = torch.clamp(torch.maximum(qx, torch.maximum(qy, qz)), max=0.0)
        phi = torch.minimum(phi, out + ins)
    if p.solid_sines:
        sfield = torch.zeros_like(x)
        for (kap, dx, dy, dz, th) in p.solid_sines:
            sfield = sfield + torch.sin(2 * math.pi * kap * (dx * x + dy * y + dz * z) + th)
        phi = torch.minimum(phi, sfield / len(p.solid_sines) - p.sine_offset)
    return phi


def _tri_positive_fraction_torch(a, b, c):
    import torch
    v, _ = torch.sort(torch.stack([a, b, c], dim=-1), dim=-1)
    lo, mid, hi = v[..., 0], v[..., 1], v[..., 2]
    one = (hi > 0) & (mid <= 0)
    two = (mid > 0) & (lo <= 0)
    f1 = hi * hi / torch.where(one, (hi - lo) * (hi - mid), torch.ones_like(hi))
    f2 = 1.0 - lo * lo / torch.where(two, (mid - lo) * (hi - lo), torch.ones_like(hi))
    out = torch.where(lo > 0, torch.ones_like(lo), torch.zeros_like(lo))
    out = torch.where(one, f1, out)
    return torch.where(two, f2, out)


def face_beta_torch(p: Problem, axis, depth, i, j, k):
    """face_beta for one piece of faces given as device tensors (the same formula as the
    numpy version, evaluated in float64 with the device's sin): float32 tensor."""
    import torch
    if p.beta == "one":
        return torch.ones(axis.shape, dtype=torch.float32, device=axis.device)
    h = 1.0 / (p.desc.n0 * torch.pow(2.0, depth.double()))
    base = torch.stack([i, j, k], dim=1).double() * h[:, None]
    frac = torch.empty(axis.shape, dtype=torch.float64, device=axis.device)
    for a in range(3):
        sel = axis == a
        if not bool(sel.any()):
            continue
        u, v = [q for q in range(3) if q != a]
        b0, hh = base[sel], h[sel]

        def corner(du, dv):
            q = b0.clone()
            q[:, u] += du * hh
            q[:, v] += dv * hh
            return _solid_sdf_torch(p, q[:, 0], q[:, 1], q[:, 2])

        p00, p10, p11, p01 = corner(0, 0), corner(1, 0), corner(1, 1), corner(0, 1)
        frac[sel] = 0.5 * (_tri_positive_fraction_torch(p00, p10, p11) + _tri_positive_fraction_torch(p00, p11, p01))
    return torch.clamp(frac, 1e-3, 1.0).float()


def large_inputs(p: Problem, n_leaves: int, n_faces: int, read_faces, device):
    """Face beta (float32, on `device`) and right-hand side (float64 numpy, canonical leaf
    order) of a problem too large to hold its face tables at once.  read_faces(first,
    count) returns one piece of the canonical faces as numpy arrays (axis, depth, i, j, k,
    minus, plus).  beta is evaluated on the device; the right-hand side follows rhs()."""
    import torch
    beta = torch.empty(n_faces, dtype=torch.float32, device=device)
    rng = np.random.default_rng(p.seed)
    b = np.zeros(n_leaves)
    for first in range(0, n_faces, FACE_CHUNK):
        cnt = min(FACE_CHUNK, n_faces - first)
        f = read_faces(first, cnt)
        t = {q: torch.from_numpy(f[q]).to(device) for q in ("axis", "depth", "i", "j", "k")}
        bt = face_beta_torch(p, t["axis"], t["depth"], t["i"], t["j"], t["k"])
        beta[first:first + cnt] = bt
        if p.rhs == "divergence":
            divergence_accumulate(p, b, rng, f, bt.cpu().numpy())
    if p.rhs == "divergence":
        b = b - b.mean()
    elif p.rhs == "normal":
        b = rng.standard_normal(n_leaves)
        if p.neumann:
            b = b - b.mean()
    else:
        raise ValueError("large_inputs supports the random right-hand sides only")
    return beta, b


def random_vector(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(n)
