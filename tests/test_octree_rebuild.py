"""Rebuild of an octree after a local change of the geometry (ocg_octree_rebuild: the
topology refresh between time steps, Sec. 3.4).  The minimal 2:1-balanced refinement of a
predicate is unique, so a rebuild that re-evaluates the predicate wherever it can have
changed must give exactly the octree a fresh build gives: every exported table is compared
bit for bit.  A box that misses the change must give back the previous octree."""
import math

import numpy as np
import pytest

from paper_2604_18886_b300 import _lib
from paper_2604_18886_b300 import problems as P
from paper_2604_18886_b300 import solver as S


def _tables(g):
    out = {"counts": (g.n_leaves, g.n_faces, g.D, g.mc, g.n_cells, g.n_trec, g.n_tree, g.n_oct)}
    out.update({"leaf_" + k: v for k, v in g.leaves().items()})
    kind, rank = g.neighbours()
    out["nb_kind"], out["nb_rank"] = kind, rank
    out.update({"face_" + k: v for k, v in g.faces().items()})
    for m in range(g.mc, g.D + 1):
        for q, v in enumerate(g.level(m)):
            out["level%d_%d" % (m, q)] = v
    return out


def _assert_same(a, b):
    ta, tb = _tables(a), _tables(b)
    assert ta["counts"] == tb["counts"]
    assert ta.keys() == tb.keys()
    for k in ta:
        if k != "counts":
            assert np.array_equal(ta[k], tb[k]), k


def _band(n0, depth, sphere, band=0.03, boxes=()):
    return P.OctreeDesc(n0, depth, P.REFINE_SDF_BAND, band=band, spheres=[sphere], boxes=list(boxes))


BOX = (0.62, 0.2, 0.3, 0.85, 0.8, 0.7)


@pytest.mark.parametrize("n0, depth", [(12, 2), (8, 3), (16, 2)])
def test_rebuild_after_a_moved_sphere_equals_a_fresh_build(n0, depth):
    s0 = (0.4, 0.5, 0.5, 0.18)
    s1 = (0.43, 0.48, 0.53, 0.18)
    d0, d1 = _band(n0, depth, s0, boxes=[BOX]), _band(n0, depth, s1, boxes=[BOX])
    g0 = S.Octree(d0)
    g1 = g0.rebuild(d1, S.sphere_change_box(s0, s1, 0.03, n0))
    _assert_same(g1, S.Octree(d1))
    # and back again, from the rebuilt octree
    _assert_same(g1.rebuild(d0, S.sphere_change_box(s1, s0, 0.03, n0)), g0)


def test_rebuild_after_a_radius_change_of_the_ball():
    s0, s1 = (0.5, 0.5, 0.5, 0.25), (0.5, 0.5, 0.5, 0.3)
    d0, d1 = P.two_level_ball(16, radius=0.25).desc, P.two_level_ball(16, radius=0.3).desc
    g1 = S.Octree(d0).rebuild(d1, S.sphere_change_box(s0, s1, 0.0, 16))
    _assert_same(g1, S.Octree(d1))


def test_a_sequence_of_moves_stays_equal_to_fresh_builds():
    n0, depth = 12, 2
    c = np.array([0.3, 0.45, 0.5])
    step = np.array([0.035, 0.01, -0.015])
    g = S.Octree(_band(n0, depth, tuple(c) + (0.15,)))
    for _ in range(5):
        s0, s1 = tuple(c) + (0.15,), tuple(c + step) + (0.15,)
        c = c + step
        d1 = _band(n0, depth, s1)
        g = g.rebuild(d1, S.sphere_change_box(s0, s1, 0.03, n0))
        _assert_same(g, S.Octree(d1))


def test_the_whole_cube_as_box_rebuilds_any_change():
    # no locality at all (star and sine fields change everywhere): the whole cube
    d0 = P.OctreeDesc(8, 2, P.REFINE_STAR_BAND, band=0.01, spheres=[(0.5, 0.5, 0.5, 0.2), (0.05, 4.0, 2.0, 0.0)])
    d1 = P.OctreeDesc(8, 2, P.REFINE_STAR_BAND, band=0.01, spheres=[(0.47, 0.52, 0.5, 0.21), (0.06, 6.0, 2.0, 0.0)])
    _assert_same(S.Octree(d0).rebuild(d1, (0.0, 0.0, 0.0, 1.0, 1.0, 1.0)), S.Octree(d1))
    s0, s1 = P.sine_band(8, 2, band=0.02).desc, P.sine_band(8, 2, band=0.03).desc
    _assert_same(S.Octree(s0).rebuild(s1, (-1.0, -1.0, -1.0, 2.0, 2.0, 2.0)), S.Octree(s1))


def test_a_box_that_misses_the_change_returns_the_previous_octree():
    s0, s1 = (0.3, 0.5, 0.5, 0.15), (0.34, 0.5, 0.5, 0.15)
    d0, d1 = _band(12, 2, s0), _band(12, 2, s1)
    g0 = S.Octree(d0)
    far = (0.8, 0.8, 0.8, 0.95, 0.95, 0.95)
    g1 = g0.rebuild(d1, far)
    _assert_same(g1, g0)
    fresh = S.Octree(d1).leaves()                 # the change itself is real
    assert any(not np.array_equal(fresh[k], g0.leaves()[k]) for k in ("i", "j", "k"))


def test_rebuild_rejects_incompatible_input():
    d0 = _band(12, 2, (0.4, 0.5, 0.5, 0.18))
    g0 = S.Octree(d0)
    with pytest.raises(_lib.OcgError):
        g0.rebuild(_band(16, 2, (0.4, 0.5, 0.5, 0.18)), (0, 0, 0, 1, 1, 1))
    with pytest.raises(_lib.OcgError):
        g0.rebuild(_band(12, 3, (0.4, 0.5, 0.5, 0.18)), (0, 0, 0, 1, 1, 1))
    with pytest.raises(_lib.OcgError):
        g0.rebuild(P.two_level_ball(12).desc, (0, 0, 0, 1, 1, 1))
    with pytest.raises(_lib.OcgError):
        g0.rebuild(d0, (0.5, 0, 0, 0.4, 1, 1))
    with pytest.raises(_lib.OcgError):
        g0.rebuild(d0, (math.nan, 0, 0, 1, 1, 1))
    # the previous octree is untouched by the failed calls
    _assert_same(g0, S.Octree(d0))


def test_uniform_octree_rebuild():
    d = P.uniform(8).desc
    _assert_same(S.Octree(d).rebuild(d, (0, 0, 0, 1, 1, 1)), S.Octree(d))


def test_grandchildren_of_a_newly_refined_cell_outside_the_box_are_evaluated():
    # Ball-centre rule on an 8^3 root with depths 0..2 refinable.  The radius grows by 2e-7
    # across the centre distance of one root cell T, so only T's predicate changes (checked
    # below over every cell centre): T becomes refined.  The box is a speck in T's far
    # corner: T meets it, so the contract holds, but the depth-2 cells under T's children on
    # the near side lie outside every index window and were never evaluated before (T was
    # not refined): they must be evaluated because their parents' flags changed.
    c = np.array([0.5113, 0.4871, 0.5037])
    tc = np.array([5.5, 4.5, 4.5]) / 8.0
    dist = float(np.sqrt(np.sum((tc - c) ** 2)))
    r0, r1 = dist - 1e-7, dist + 1e-7
    in_shell = 0
    for d in range(3):
        nd = 8 << d
        g = (np.arange(nd) + 0.5) / nd
        x, y, z = np.meshgrid(g, g, g, indexing="ij")
        s = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
        in_shell += int(np.sum((s >= r0 * r0) & (s < r1 * r1)))
    assert in_shell == 1
    d0 = P.OctreeDesc(8, 3, P.REFINE_BALL_CENTRE, spheres=[tuple(c) + (r0,)])
    d1 = P.OctreeDesc(8, 3, P.REFINE_BALL_CENTRE, spheres=[tuple(c) + (r1,)])
    speck = (0.7490, 0.6240, 0.6240, 0.7495, 0.6245, 0.6245)
    g1 = S.Octree(d0).rebuild(d1, speck)
    _assert_same(g1, S.Octree(d1))
    assert S.Octree(d1).n_leaves != S.Octree(d0).n_leaves


def test_one_of_several_primitives_changes():
    # the signed distance is the minimum over two spheres and a box; moving one sphere and
    # shrinking the other, each with its own box, rebuilt one after the other
    a0, a1 = (0.3, 0.35, 0.5, 0.12), (0.33, 0.37, 0.48, 0.12)
    b0, b1 = (0.55, 0.7, 0.45, 0.1), (0.55, 0.7, 0.45, 0.07)
    box = (0.7, 0.15, 0.2, 0.9, 0.5, 0.8)
    def desc(sa, sb):
        return P.OctreeDesc(12, 2, P.REFINE_SDF_BAND, band=0.02, spheres=[sa, sb], boxes=[box])
    g = S.Octree(desc(a0, b0))
    g = g.rebuild(desc(a1, b0), S.sphere_change_box(a0, a1, 0.02, 12))
    _assert_same(g, S.Octree(desc(a1, b0)))
    g = g.rebuild(desc(a1, b1), S.sphere_change_box(b0, b1, 0.02, 12))
    _assert_same(g, S.Octree(desc(a1, b1)))
