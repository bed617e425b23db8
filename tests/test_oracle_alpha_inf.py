"""alpha = infinity: the alpha complex is the whole weighted Delaunay (regular) triangulation.

Pins that do not go through the oracle's own predicates:
* the tetrahedra equal the lower facets of the convex hull of the lifted points
  (p, |p|^2 - r^2) in R^4 (the lifting-map view of the weighted Delaunay
  triangulation, Section 1.1), computed by Qhull through scipy;
* with equal radii they equal scipy's (unweighted) Delaunay tetrahedra;
* the complex triangulates the convex hull: Euler characteristic 1 and
  tetrahedron volumes summing to the hull volume.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle

scipy_spatial = pytest.importorskip("scipy.spatial")


def _points(seed, n, equal_radii=False):
    rng = np.random.default_rng(seed)
    c = np.round(rng.uniform(-6.0, 6.0, (n, 3)) * 1024) / 1024
    if equal_radii:
        r = np.full(n, 1.5)
    else:
        r = np.round(rng.uniform(0.8, 2.2, n) * 1024) / 1024
    return c, r


def _lower_hull_tets(c, r):
    lifted = np.column_stack([c, (c ** 2).sum(1) - r ** 2])
    hull = scipy_spatial.ConvexHull(lifted)
    tets = set()
    for simplex, eq in zip(hull.simplices, hull.equations):
        if eq[3] < -1e-12:  # outward normal points down in the lifted coordinate
            tets.add(tuple(sorted(int(v) for v in simplex)))
    return tets


@pytest.mark.parametrize("seed", range(6))
def test_tetrahedra_are_lower_hull_of_lifted_points(seed):
    c, r = _points(seed, 30)
    ac = oracle.alpha_complex(c, r, alpha_inf=True)
    got = {tuple(int(v) for v in t) for t in ac.simplices[3]}
    assert got == _lower_hull_tets(c, r)


@pytest.mark.parametrize("seed", range(4))
def test_equal_radii_reduce_to_delaunay(seed):
    c, r = _points(100 + seed, 30, equal_radii=True)
    ac = oracle.alpha_complex(c, r, alpha_inf=True)
    got = {tuple(int(v) for v in t) for t in ac.simplices[3]}
    dt = scipy_spatial.Delaunay(c)
    want = {tuple(sorted(int(v) for v in s)) for s in dt.simplices}
    assert got == want


def _tet_volume6(c, t):
    """Six times the volume of a tetrahedron, exactly (coordinates are dyadic)."""
    p = [[Fraction(float(x)) for x in c[v]] for v in t]
    a = [p[1][i] - p[0][i] for i in range(3)]
    b = [p[2][i] - p[0][i] for i in range(3)]
    d = [p[3][i] - p[0][i] for i in range(3)]
    det = a[0] * (b[1] * d[2] - b[2] * d[1]) - a[1] * (b[0] * d[2] - b[2] * d[0]) + a[2] * (b[0] * d[1] - b[1] * d[0])
    return abs(det)


@pytest.mark.parametrize("seed", range(6))
def test_triangulates_convex_hull(seed):
    c, r = _points(200 + seed, 25)
    ac = oracle.alpha_complex(c, r, alpha_inf=True)
    V, E, F, T = ac.counts()
    assert V - E + F - T == 1
    vol = sum(_tet_volume6(c, t) for t in ac.simplices[3]) / 6
    hull = scipy_spatial.ConvexHull(c)
    assert float(vol) == pytest.approx(hull.volume, rel=1e-12)
    # every hull vertex is a vertex of the triangulation (its power cell is unbounded)
    assert set(int(v) for v in hull.vertices) <= set(int(v) for v in ac.simplices[0][:, 0])
