"""Static tank (Sec. 4.4) on the oracle: liquid in [0,1]^3, solid bottom and sides, open to
air at y = 1, a cut-cell sphere or star obstacle at the centre, the integrated divergence
of the uniform velocity (0, -1, 0) as rhs.

Pins: the velocity is minus the gradient of the linear field y, which the discretisation
reproduces exactly (regular faces, cut-cell faces with any beta, the T-junction ghost
value, the Dirichlet face at the open top), so the discrete pressure is p = y - 1 to
rounding (the field that cancels the motion: the paper's "nearly uniform gradient along
y"), whatever the obstacle and grid; and Alg. 1 with W-cycles (mu = 2, the paper's choice
for this test) reduces the residual by more than 5 per iteration on these small roots.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as sla

from oracle import mg
from oracle import octree as O
from oracle import operator as OP
from oracle import pcg
from paper_2604_18886_b300 import problems as P


def _setup(obstacle, n0):
    p = P.tank(obstacle, n0)
    t = O.Octree(p.desc)
    f = t.faces()
    beta = P.face_beta(p, f)
    H = OP.Hierarchy(t, beta, p.bc)
    return p, t, H, P.rhs(p, t.leaves, f, beta)


@pytest.mark.parametrize("obstacle", ["sphere", "star"])
def test_tank_pressure_is_the_hydrostatic_field(obstacle):
    for n0 in (8, 16):
        p, t, H, b = _setup(obstacle, n0)
        assert P.face_beta(p, t.faces()).min() < 0.01          # cut cells present
        x = sla.spsolve(H.A.tocsc(), b)
        h, xc, yc, zc = P.leaf_centres(n0, t.leaves)
        assert np.abs(x - (yc - 1.0)).max() <= 1e-11, n0


@pytest.mark.parametrize("obstacle", ["sphere", "star"])
def test_tank_w_cycle_reduces_the_residual_by_more_than_five(obstacle):
    for n0 in (8, 16):
        p, t, H, b = _setup(obstacle, n0)
        x, k, hist = pcg.pcg(H, b, tol=1e-6, prm=mg.CycleParams(mu=2), max_iter=100)
        red = math.exp(-math.log(hist[k]) / k)
        assert red > 5.0 and k <= 10, (n0, k, red)
