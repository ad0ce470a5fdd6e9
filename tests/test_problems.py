"""Pins for the seeded input generators (cut-face fractions, rhs invariants)."""
import numpy as np

from oracle import octree as O
from paper_2604_18886_b300 import problems as P


def test_triangle_fraction_linear_field():
    # phi linear on the triangle: the positive-area fraction has closed forms
    f = P._tri_positive_fraction
    assert np.allclose(f(np.array([1.0]), np.array([2.0]), np.array([3.0])), 1.0)
    assert np.allclose(f(np.array([-1.0]), np.array([-2.0]), np.array([0.0])), 0.0)
    # one positive vertex a=1 with b=c=-1: cut at the midpoints of both edges -> 1/4
    assert np.allclose(f(np.array([1.0]), np.array([-1.0]), np.array([-1.0])), 0.25)
    # two positive vertices: complement -> 3/4
    assert np.allclose(f(np.array([1.0]), np.array([1.0]), np.array([-1.0])), 0.75)


def test_face_fraction_of_a_plane():
    # solid half-space x < 0.3 (phi = x - 0.3, a box far larger than the domain): a face
    # normal to y spanning x in [0.25, 0.375] has fluid fraction (0.375-0.3)/0.125 = 0.6
    p = P.Problem("t", P.OctreeDesc(8, 0), (0,) * 6, beta="cut",
                  solid_boxes=[(-10.0, -10.0, -10.0, 0.3, 10.0, 10.0)])
    faces = {"axis": np.array([1, 0]), "depth": np.array([0, 0]),
             "i": np.array([2, 2]), "j": np.array([3, 3]), "k": np.array([1, 1])}
    fr = P.face_fluid_fraction(p, faces)
    assert abs(fr[0] - 0.6) < 1e-12
    assert abs(fr[1] - 0.0) < 1e-12       # x-face at x = 0.25 lies inside the solid
    assert P.face_beta(p, faces)[1] == np.float32(1e-3)


def test_divergence_rhs_sums_to_zero():
    p = P.cut_cell(8, 2)
    t = O.Octree(p.desc)
    f = t.faces()
    beta = P.face_beta(p, f)
    b = P.rhs(p, t.leaves, f, beta)
    assert abs(b.sum()) < 1e-12 and np.abs(b).max() > 0
    assert beta.min() >= np.float32(1e-3) and beta.max() <= 1.0 and (beta < 1).any()
