"""The oracle's evaluation at arbitrary points from stored expansions (Section 5.3: keep the FMM's
multipole and local expansions and evaluate new targets in O(p) for the far field; the near field
by box integrals at the point), pinned against quantities computed another way.

* At the leaf nodes it reproduces the box code's values (table apply + L2T + M2T), i.e. the same
  decomposition evaluated through per-point quadrature instead of the precomputed tables.
* At seeded random points it matches direct quadrature of V[f~] over every leaf (no FMM, no
  expansions, absolute coordinates) on uniform and adaptive trees that carry W and X lists, to the
  FMM's accuracy at p = 40.
* For f = 1 on a one-leaf tree it is the textbook antiderivative of the box integral at any point.
"""
import numpy as np
import pytest

import workloads as W
from oracle import brute, fmm, offnode
from oracle import tree as T

from test_oracle_cheb_quad import uniform_density_closed_form
from test_oracle_fmm import _mk

P = 40


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _tree(shape, k):
    if shape == "16leaf":
        return T.build_uniform(0.05, -0.02, 1.3, k, 2)
    if shape == "adaptive10":
        return _mk([(0, 0, 0), (1, 1, 1), (2, 3, 3)], k)
    return _mk([(0, 0, 0), (1, 0, 0), (2, 1, 1)], k, balance=True)


@pytest.mark.parametrize("shape", ["16leaf", "adaptive10", "adaptive19"])
def test_offnode_reproduces_the_box_code_at_nodes(shape, oracle_ops):
    k = 8
    t = _tree(shape, k)
    src = W.narrow_gaussians(9, n=3, sigma=0.15, spread=0.4)
    F = t.sample(src)
    L = T.build_lists(t)
    ref = fmm.solve(t, L, oracle_ops(k, P), F)
    X, Y = t.leaf_nodes()
    sel = np.arange(0, X.size, 7)
    got = offnode.evaluate(t, L, oracle_ops(k, P), F, X.reshape(-1)[sel], Y.reshape(-1)[sel])
    for q in range(3):
        assert _rel(got[q], ref[q].reshape(-1)[sel]) < 1e-14, (shape, q)


@pytest.mark.slow
@pytest.mark.parametrize("shape", ["16leaf", "adaptive10", "adaptive19"])
def test_offnode_matches_direct_quadrature_at_random_points(shape, oracle_ops):
    k = 8
    t = _tree(shape, k)
    L = T.build_lists(t)
    assert shape == "16leaf" or len(L["W"][1]) > 0  # the adaptive trees exercise M2T and S2L
    src = W.narrow_gaussians(9, n=3, sigma=0.15, spread=0.4)
    F = t.sample(src)
    rng = np.random.default_rng(11)
    lo_x, lo_y = t.cx - t.width / 2, t.cy - t.width / 2
    pts = np.column_stack([lo_x + t.width * rng.uniform(0.001, 0.999, 40),
                           lo_y + t.width * rng.uniform(0.001, 0.999, 40)])
    got = offnode.evaluate(t, L, oracle_ops(k, P), F, pts[:, 0], pts[:, 1])
    ref = brute.brute_potential(t, F, pts)
    for q in range(3):
        assert _rel(got[q], ref[q]) < 1e-13, (shape, q, _rel(got[q], ref[q]))


def test_offnode_constant_density_single_leaf(oracle_ops):
    """f = 1 on one leaf: the box integral's closed form at points inside and on the way out."""
    k = 4
    t = _mk([], k)  # the 1.3-wide root box at (0.05, -0.02)
    L = T.build_lists(t)
    F = np.ones((1, k * k))
    rng = np.random.default_rng(2)
    pts = np.column_stack([t.cx + t.width * rng.uniform(-0.499, 0.499, 25),
                           t.cy + t.width * rng.uniform(-0.499, 0.499, 25)])
    got = offnode.evaluate(t, L, oracle_ops(k, P), F, pts[:, 0], pts[:, 1])
    ref = np.column_stack([uniform_density_closed_form(x, np.array([t.cx, t.cy]), t.width) for x in pts])
    for q in range(3):
        assert _rel(got[q], ref[q]) < 1e-13, q


def test_offnode_outside_the_root_is_nan(oracle_ops):
    t = _mk([], 4)
    got = offnode.evaluate(t, T.build_lists(t), oracle_ops(4, P), np.ones((1, 16)), [5.0], [0.0])
    assert np.all(np.isnan(got))
