"""CPU tests of libocg: the library loads and exports every declared symbol, and its host
octree build reproduces the oracle's canonical tables bit for bit (leaves, neighbour
codes, faces, multigrid level cell sets)."""
import os
import re

import numpy as np
import pytest

from oracle import octree as O
from paper_2604_18886_b300 import _lib
from paper_2604_18886_b300 import problems as P
from paper_2604_18886_b300 import solver as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "ocg.h")).read()
    declared = set(re.findall(r"^\s*(?:int|void|const char\*)\s+(ocg_\w+)\s*\(", hdr, re.M))
    assert declared == set(_lib.EXPORTED)
    L = _lib.lib()
    for name in declared:
        assert hasattr(L, name), name


def _descs():
    yield P.uniform(8).desc
    yield P.two_level_ball(8).desc
    yield P.two_level_ball(16, radius=0.3).desc
    yield P.cut_cell(8, 2).desc
    yield P.OctreeDesc(4, 3, P.REFINE_SDF_BAND, band=0.02, spheres=[(0.3, 0.4, 0.55, 0.17)])
    yield P.OctreeDesc(6, 3, P.REFINE_SDF_BAND, band=0.01, spheres=[(0.21, 0.8, 0.5, 0.11)],
                       boxes=[(0.5, 0.1, 0.2, 0.9, 0.35, 0.6)])
    yield P.OctreeDesc(12, 2, P.REFINE_SDF_BAND, band=0.05, spheres=[(0.45, 0.55, 0.5, 0.23)])
    yield P.batch_tree(1).desc
    yield P.sine_band(8, 2).desc           # sine band: deterministic sin/cos in both builders
    yield P.sine_band(6, 3, band=0.01).desc
    yield P.sine_band(16, 2).desc
    yield P.accuracy_desc("star", 8)   # star surface: Chebyshev cosines in both builders
    yield P.accuracy_desc("star", 16)
    yield P.OctreeDesc(6, 3, P.REFINE_STAR_BAND, band=0.01,
                       spheres=[(0.47, 0.52, 0.5, 0.2), (0.05, 4.0, 2.0, 0.0)])
    # tiles (Sec. 4.1 refines the tiles that meet the surface): one decision per block
    yield P.OctreeDesc(16, 2, P.REFINE_SDF_BAND, band=0.0, spheres=[(0.5, 0.5, 0.5, 0.25)], tile_log2=2)
    yield P.OctreeDesc(8, 3, P.REFINE_STAR_BAND, band=0.0, spheres=list(P.STAR), tile_log2=1)
    yield P.OctreeDesc(8, 2, P.REFINE_SINE_BAND, band=0.02, sines=P.sine_waves(), tile_log2=2)
    yield P.paper_grid("sphere", 32)      # exact box test of the sphere, 2:1 balance per tile
    yield P.paper_grid("star", 32)        # 27-point star test
    yield P.OctreeDesc(16, 2, P.REFINE_SDF_BAND, band=0.01, spheres=[(0.3, 0.4, 0.55, 0.17)],
                       boxes=[(0.6, 0.1, 0.2, 0.9, 0.35, 0.6)], tile_log2=1)


@pytest.mark.parametrize("desc", list(_descs()))
def test_octree_tables_bit_exact(desc):
    t = O.Octree(desc)
    g = S.Octree(desc)
    assert g.n_leaves == t.n_leaves
    lo, lg = t.leaves, g.leaves()
    for k in ("depth", "i", "j", "k"):
        assert np.array_equal(lo[k], lg[k]), k
    ko, ro = t.neighbour_table()
    kg, rg = g.neighbours()
    assert np.array_equal(ko, kg)
    assert np.array_equal(ro, rg)
    fo, fg = t.faces(), g.faces()
    assert g.n_faces == len(fo["axis"])
    for k in ("axis", "depth", "i", "j", "k", "minus", "plus"):
        assert np.array_equal(fo[k], fg[k]), k
    assert g.mc == t.min_level() and g.D == t.D
    for m in range(g.mc, g.D + 1):
        io, jo, ko_, leafo = t.level_cells(m)
        ig, jg, kg_, leafg = g.level(m)
        assert np.array_equal(io, ig) and np.array_equal(jo, jg) and np.array_equal(ko_, kg_)
        assert np.array_equal(leafo, leafg)


def test_faces_bit_exact_when_a_group_is_merged_in_several_chunks():
    # the host build merges each (axis, depth) group of faces in chunks of about 2^20 of
    # its - faces; the cut-cell 64^3 tree has a group large enough for two chunks, with T
    # faces on both sides of the split
    desc = P.cut_cell(64, 2).desc
    g = S.Octree(desc)
    fg = g.faces()
    big = max(int(np.sum((fg["axis"] == a) & (fg["depth"] == d))) for a in range(3) for d in range(g.D + 1))
    assert big >= 2 ** 21
    fo = O.Octree(desc).faces()
    for k in ("axis", "depth", "i", "j", "k", "minus", "plus"):
        assert np.array_equal(fo[k], fg[k]), k


def test_paper_grids_at_128_have_the_leaf_counts_of_table1():
    # Table 1 (Sec. 4.5), 128~512 grids, in units of 2^20 leaves: sphere exactly, star
    # within 2 % (the bit-exact tables against the oracle are checked at a 32^3 root)
    import json
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_worked_values.json")))["table1_leaf_counts"]
    assert round(S.Octree(P.paper_grid("sphere", 128)).n_leaves / 2 ** 20, 5) == gold["sphere_128_512"]
    assert abs(S.Octree(P.paper_grid("star", 128)).n_leaves / 2 ** 20 / gold["star_128_512"] - 1.0) < 0.02


def test_config_leaf_counts():
    # two-level ball: 64^3 base with the central ball refined once
    g = S.Octree(P.two_level_ball(64).desc)
    assert g.n_leaves == 382936
    assert g.mc == -4 and g.D == 1


def test_invalid_descriptions_are_rejected():
    with pytest.raises(_lib.OcgError) as e:
        S.Octree(P.OctreeDesc(7, 1))
    assert e.value.code == _lib.OCG_EINVAL
    with pytest.raises(_lib.OcgError):
        S.Octree(P.OctreeDesc(8, 1, P.REFINE_BALL_CENTRE))   # no sphere given
    with pytest.raises(_lib.OcgError):                         # n0 not a multiple of the tile
        S.Octree(P.OctreeDesc(12, 1, P.REFINE_BALL_CENTRE, spheres=[(0.5, 0.5, 0.5, 0.25)], tile_log2=3))
