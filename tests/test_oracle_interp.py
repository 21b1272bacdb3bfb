"""Pins of the oracle's leaf interpolant v~ (Section 3.1) against mathematics it does not use.

* Interpolation: v~ at every node of every leaf returns the value stored there.
* Exactness: leaf values of a polynomial of degree < k in each variable (in global coordinates)
  give that polynomial back at arbitrary points (a swapped x/y index, a transposed coefficient
  matrix or a wrong leaf centre breaks this).
* Location: the leaf found contains the point (closed box bounds from integer geometry), a
  point on an edge shared by two leaves goes to the upper or right one, points outside the root
  box get -1 and NaN.
"""
import numpy as np
import pytest

from oracle import interp
from oracle import tree as T

CAP = (0.13, -0.07, 0.31)


class _Cap:
    """A source for the oracle's tree builder: the paraboloid cap max(0, r^2 - |x - c|^2)."""
    kind = "cap"


def _cap_tree(monkeypatch, k, depth, cx=0.0, cy=0.0, width=1.0):
    from oracle import source as srcmod

    def ev(s, x, y):
        dx = x - (cx + CAP[0] * width)
        dy = y - (cy + CAP[1] * width)
        return np.maximum((CAP[2] * width) ** 2 - (dx * dx + dy * dy), 0.0)
    monkeypatch.setattr(srcmod, "evaluate_source", ev)
    return T.build_adaptive(cx, cy, width, k, _Cap(), 1e-6, depth)


@pytest.mark.parametrize("k", [4, 8, 16])
def test_interpolant_returns_the_values_at_the_nodes(monkeypatch, k):
    t = _cap_tree(monkeypatch, k, 4)
    X, Y = t.leaf_nodes()
    rng = np.random.default_rng(1)
    vals = rng.standard_normal((t.n_leaves, k * k))
    got = interp.interpolate(t, vals, X.reshape(-1), Y.reshape(-1))
    assert np.max(np.abs(got - vals.reshape(-1))) < 1e-12 * np.max(np.abs(vals))


@pytest.mark.parametrize("k,cx,cy,width", [(4, 0.0, 0.0, 1.0), (8, 0.3, -0.2, 2.0), (16, 0.0, 0.0, 1.0)])
def test_polynomials_of_degree_below_k_are_reproduced(monkeypatch, k, cx, cy, width):
    t = _cap_tree(monkeypatch, k, 4, cx, cy, width)
    rng = np.random.default_rng(k)
    a = rng.standard_normal((k, k)) / np.add.outer(np.arange(k), np.arange(k)).clip(1)

    def poly(x, y):
        u = (x - cx) / width
        v = (y - cy) / width
        return np.polynomial.polynomial.polyval2d(v, u, a)  # sum a[i, j] v^i u^j, degree < k in each

    X, Y = t.leaf_nodes()
    vals = poly(X, Y)
    lo = np.array([cx, cy]) - width / 2
    pts = lo + width * rng.random((500, 2))
    got = interp.interpolate(t, vals, pts[:, 0], pts[:, 1])
    ref = poly(pts[:, 0], pts[:, 1])
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


def test_location_contains_the_point_and_edges_go_up_and_right(monkeypatch):
    t = _cap_tree(monkeypatch, 8, 6)
    assert t.depth == 6 and t.n_leaves > 100
    rng = np.random.default_rng(7)
    pts = -0.5 + rng.random((2000, 2))
    leaf = interp.locate(t, pts[:, 0], pts[:, 1])
    assert np.all(leaf >= 0)
    b = t.leaves[leaf]
    h = t.h(b)
    x0 = -0.5 + t.ix[b] * h
    y0 = -0.5 + t.iy[b] * h
    assert np.all((pts[:, 0] >= x0) & (pts[:, 0] <= x0 + h) & (pts[:, 1] >= y0) & (pts[:, 1] <= y0 + h))
    # a point on the right edge of a leaf (not on the root's edge) belongs to the leaf to its right
    lf = int(leaf[0])
    bb = t.leaves[lf]
    hh = float(t.h(bb))
    ex = -0.5 + (t.ix[bb] + 1) * hh
    if ex < 0.5:
        ey = -0.5 + (t.iy[bb] + 0.5) * hh
        other = t.leaves[interp.locate(t, [ex], [ey])[0]]
        assert -0.5 + t.ix[other] * float(t.h(other)) == ex
    # root corners and outside points
    corners = interp.locate(t, [-0.5, 0.5, -0.5, 0.5], [-0.5, -0.5, 0.5, 0.5])
    assert np.all(corners >= 0)
    out = interp.locate(t, [0.5000001, -0.6, 0.0, np.nan], [0.0, 0.0, 0.51, 0.0])
    assert np.all(out == -1)
    vals = np.ones((t.n_leaves, 64))
    assert np.all(np.isnan(interp.interpolate(t, vals, [0.7], [0.0])))
