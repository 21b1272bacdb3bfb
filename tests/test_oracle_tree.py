"""Pins of the oracle's quadtree and interaction lists (Section 3.1, Fig. 1).

Invariants fixed by the definitions: leaves tile the root box, every split box
has four children, adjacent leaves differ by at most one level (the level
restriction of Section 3.1), the balance step adds only forced boxes, the
hashed list builder equals a pairwise test of the list definitions, and the
lists are symmetric (U, V) or mutually inverse (W, X).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import source, tables
from oracle import tree as T


def small_trees():
    out = []
    for seed, tol, depth, sig in ((3, 1e-3, 4, 0.05), (4, 1e-4, 5, 0.03), (7, 1e-2, 5, 0.01),
                                  (11, 1e-6, 4, 0.08)):
        src = W.narrow_gaussians(seed, n=2, sigma=sig, spread=0.35)
        out.append(T.build_adaptive(0.1, -0.2, 1.5, 6, src, tol, depth, return_info=True))
    return out


@pytest.mark.parametrize("depth", [0, 1, 2, 3])
def test_uniform_counts(depth):
    t = T.build_uniform(0, 0, 1, 4, depth)
    assert t.n_boxes == (4 ** (depth + 1) - 1) // 3
    assert t.n_leaves == 4 ** depth


def test_adaptive_trees_tile_and_balance():
    for t, info in small_trees():
        area = float(np.sum(t.h(t.leaves) ** 2))
        assert abs(area - t.width ** 2) < 1e-12 * t.width ** 2
        assert T.is_balanced(t)
        # every box the balance step added is forced: un-splitting it breaks the restriction
        refined = info["refined"]
        for b in range(t.n_boxes):
            ch = t.child[b]
            if ch[0] < 0 or not np.all(t.is_leaf[ch]):
                continue
            key = (int(t.level[ch[0]]), int(t.ix[ch[0]]), int(t.iy[ch[0]]))
            if key in refined:
                continue
            boxes = set(t.index.keys()) - {(int(t.level[c]), int(t.ix[c]), int(t.iy[c])) for c in ch}
            assert not T.is_balanced(T.Tree(t.cx, t.cy, t.width, t.k, boxes))


def test_lists_match_definitions_and_symmetry():
    for t, _ in small_trees() + [(T.build_uniform(0, 0, 1, 4, 3), None)]:
        L = T.build_lists(t)
        B = T.build_lists_bruteforce(t)
        for name in "UVWX":
            assert np.array_equal(L[name][0], B[name][0]), name
            assert np.array_equal(L[name][1], B[name][1]), name

        def pairs(name):
            p, i = L[name][0], L[name][1]
            return {(b, int(c)) for b in range(t.n_boxes) for c in i[p[b]:p[b + 1]]}
        U, V, Wl, X = pairs("U"), pairs("V"), pairs("W"), pairs("X")
        assert U == {(c, b) for (b, c) in U}
        assert V == {(c, b) for (b, c) in V}
        assert Wl == {(c, b) for (b, c) in X}
        sizes = {n: np.diff(L[n][0]).max(initial=0) for n in "UVWX"}
        assert sizes["U"] <= 13 and sizes["V"] <= 27 and sizes["W"] <= 20 and sizes["X"] <= 5


def test_list_configs_match_geometry():
    cfg = tables.near_configs()
    for t, _ in small_trees():
        L = T.build_lists(t)
        p, idx, cf = L["U"]
        for b in range(t.n_boxes):
            for e in range(p[b], p[b + 1]):
                s = idx[e]
                rho, dx, dy = cfg[cf[e]]
                hb = float(t.h(b))
                cb, cs = t.centre(b), t.centre(s)
                assert abs(float(t.h(s)) / hb - rho) < 1e-15
                assert abs((cs[0] - cb[0]) / hb - dx) < 1e-12 and abs((cs[1] - cb[1]) / hb - dy) < 1e-12
        for name, geo, scale in (("W", tables.w_configs(), 0.5), ("X", tables.x_configs(), 2.0)):
            p, idx, cf = L[name]
            for b in range(t.n_boxes):
                for e in range(p[b], p[b + 1]):
                    s = idx[e]
                    hb = float(t.h(b))
                    cb, cs = t.centre(b), t.centre(s)
                    dx, dy = geo[cf[e]]
                    assert abs(float(t.h(s)) / hb - scale) < 1e-15
                    assert abs((cs[0] - cb[0]) / hb - dx) < 1e-12 and abs((cs[1] - cb[1]) / hb - dy) < 1e-12


def test_refinement_decisions_follow_tail_test():
    """Every leaf below max_depth passes the tail test; every refined box failed it."""
    src = W.narrow_gaussians(5, n=3, sigma=0.04)
    tol, depth, k = 1e-5, 6, 8
    t, info = T.build_adaptive(0, 0, 1, k, src, tol, depth, return_info=True)
    X, Y = t.leaf_nodes()
    vals = source.evaluate_source(src, X, Y).reshape(-1, k, k)
    tl = T.cheb.tail(vals, k)
    lv = t.level[t.leaves]
    refined_leaf = np.array([(int(t.level[b]), int(t.ix[b]), int(t.iy[b])) in info["refined"] for b in t.leaves])
    assert np.all(tl[(lv < depth) & refined_leaf] <= tol * info["F"])
    assert info["min_margin"] > 1e-9


def _tail_by_vandermonde(vals, k):
    """Trailing-coefficient indicator by an independent route: the 2-D Chebyshev coefficients as the
    solution of the interpolation (Vandermonde) system on the nodes, numpy's chebvander, instead of
    the discrete orthogonality of the oracle's transform."""
    t = np.sin(0.5 * np.pi / k * np.arange(-k + 1, k + 1, 2))  # first-kind points, ascending
    Vinv = np.linalg.inv(np.polynomial.chebyshev.chebvander(t, k - 1))  # coefficients = Vinv @ values
    coef = np.einsum("mj,bji,ni->bmn", Vinv, vals, Vinv)
    mask = np.zeros((k, k), dtype=bool)
    mask[k - 2:, :] = True
    mask[:, k - 2:] = True
    return np.max(np.abs(coef[:, mask]), axis=-1)


@pytest.mark.parametrize("k,tol,depth,min_depth", [(8, 1e-5, 6, 0), (6, 1e-4, 7, 2)])
def test_refinement_decisions_against_an_independent_tail(k, tol, depth, min_depth):
    """Every box of the refinement (before balancing) below max_depth was split exactly when its tail,
    computed by the Vandermonde route and compared with tol times max |f| over the uniform level-5
    nodes (the F of the tolerance rule, Section 6.1), exceeds the threshold."""
    src = W.narrow_gaussians(5, n=3, sigma=0.04)
    t, info = T.build_adaptive(0, 0, 1, k, src, tol, depth, min_depth, return_info=True)
    assert info["min_margin"] > 1e-9
    m = min(5, depth)
    xs = np.sin(0.5 * np.pi / k * np.arange(-k + 1, k + 1, 2)) / 2  # nodes on [-1/2, 1/2]
    g = ((np.arange(1 << m)[:, None] + 0.5 + xs[None, :]) / (1 << m) - 0.5).reshape(-1)
    F = np.max(np.abs(source.evaluate_source(src, *np.meshgrid(g, g, indexing="xy"))))
    assert abs(F - info["F"]) <= 1e-15 * F
    boxes = sorted(b for b in info["refined"] if min_depth <= b[0] < depth)
    lv = np.array([b[0] for b in boxes])
    ix = np.array([b[1] for b in boxes])
    iy = np.array([b[2] for b in boxes])
    h = 1.0 / (1 << lv)
    X = (-0.5 + (ix + 0.5)[:, None, None] * h[:, None, None] + xs[None, None, :] * h[:, None, None])
    Y = (-0.5 + (iy + 0.5)[:, None, None] * h[:, None, None] + xs[None, :, None] * h[:, None, None])
    X, Y = np.broadcast_to(X, (len(boxes), k, k)), np.broadcast_to(Y, (len(boxes), k, k))
    tl = _tail_by_vandermonde(source.evaluate_source(src, X, Y), k)
    split = np.array([(b[0] + 1, 2 * b[1], 2 * b[2]) in info["refined"] for b in boxes])
    assert split.any() and (~split).any()
    assert np.array_equal(split, tl > tol * F)


def test_kinked_source_zero_set_is_the_curve():
    wl = W.kinked()
    prm = wl.sources[0].params
    a, c = prm[0:7], prm[7:14]
    th = np.linspace(0, 2 * math.pi, 97)
    r = 0.6 + sum(a[i] * np.cos((i + 2) * th + c[i]) for i in range(7))
    phi = source.kinked_phi(prm, r * np.cos(th), r * np.sin(th))
    assert np.max(np.abs(phi)) < 1e-14
    assert np.all(source.kinked_phi(prm, 0.5 * r * np.cos(th), 0.5 * r * np.sin(th)) > 0)
    assert np.all(source.kinked_phi(prm, 1.1 * r * np.cos(th), 1.1 * r * np.sin(th)) < 0)


# ----------------------------------------------------------------------------- leaf-count target
def _refined_leaves(refined):
    """Leaves of a refinement given as a set of boxes (before balancing)."""
    return [b for b in refined if (b[0] + 1, 2 * b[1], 2 * b[2]) not in refined]


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_greedy_constant_source_is_uniform(depth):
    """f = 1 has zero tails everywhere: every priority ties, so coarser-first order builds
    exactly the uniform tree when the target is 4^depth."""
    src = W.constant_source(1.0)
    ot = T.build_greedy(0.0, 0.0, 1.0, 8, src, 4 ** depth, 16)
    ref = T.build_uniform(0.0, 0.0, 1.0, 8, depth)
    assert ot.n_leaves == 4 ** depth
    assert sorted(zip(ot.level, ot.ix, ot.iy)) == sorted(zip(ref.level, ref.ix, ref.iy))


def test_greedy_counts_prefix_and_focus():
    """One split adds 3 leaves, so the refinement stops at the first count >= target; the split
    sequence is a prefix of the one for a larger target; a narrow Gaussian draws the deepest
    leaves to its centre; the result is level-restricted."""
    src = W.gauss_source([[0.31, -0.27]], 0.01, [1.0])
    prev = None
    for n in (10, 40, 100, 250):
        ot, info = T.build_greedy(0.0, 0.0, 1.0, 8, src, n, 16, return_info=True)
        leaves = _refined_leaves(info["refined"])
        assert n <= len(leaves) < n + 3 and (len(leaves) - 1) % 3 == 0
        if prev is not None:
            assert prev <= info["refined"]
        prev = info["refined"]
        assert T.is_balanced(ot)
    deepest = max(leaves, key=lambda b: b[0])
    h = 2.0 ** -deepest[0]
    cx, cy = -0.5 + (deepest[1] + 0.5) * h, -0.5 + (deepest[2] + 0.5) * h
    assert abs(cx - 0.31) <= 1.5 * h and abs(cy + 0.27) <= 1.5 * h


def test_greedy_max_depth_stops_refinement():
    src = W.gauss_source([[0.0, 0.0]], 0.001, [1.0])
    ot = T.build_greedy(0.0, 0.0, 1.0, 8, src, 10 ** 6, 2)
    assert ot.depth == 2 and ot.n_leaves == 16


# ----------------------------------------------------------------------------- Section 6.1 rules
class _Fn:
    """A source for the oracle's builders defined by a plain function (kind is not a built-in)."""
    kind = "fn"

    def __init__(self, fn):
        self.fn = fn


def _with_fn(monkeypatch, fn):
    from oracle import source as srcmod
    orig = srcmod.evaluate_source
    monkeypatch.setattr(srcmod, "evaluate_source",
                        lambda s, x, y: s.fn(np.asarray(x), np.asarray(y)) if isinstance(s, _Fn) else orig(s, x, y))
    return _Fn(fn)


@pytest.mark.parametrize("rule", ["interp", "interp_area", "interp_mixed"])
def test_interp_rules_do_not_refine_polynomials(monkeypatch, rule):
    k = 8
    rng = np.random.default_rng(3)
    a = rng.standard_normal((k, k)) / 10.0
    src = _with_fn(monkeypatch, lambda x, y: np.polynomial.polynomial.polyval2d(y, x, a))
    t = T.build_adaptive(0.0, 0.0, 1.0, k, src, 1e-10, 6, 2, rule=rule)
    assert t.n_leaves == 16 and t.depth == 2


def test_interp_error_of_chebyshev_polynomial_at_its_roots(monkeypatch):
    # p interpolates T_k at the k roots of T_k, so p = 0 and e = max |T_k| on the children's nodes
    from oracle import cheb
    for k in (4, 8, 16):
        src = _with_fn(monkeypatch, lambda x, y, k=k: np.cos(k * np.arccos(np.clip(2.0 * x, -1.0, 1.0))))
        e, meets = T.interp_error(0.0, 0.0, 1.0, k, src, [0], [0], [0])
        u = np.concatenate([-0.25 + cheb.nodes(k) / 2.0, 0.25 + cheb.nodes(k) / 2.0])
        exact = np.max(np.abs(np.cos(k * np.arccos(2.0 * u))))
        assert abs(e[0] - exact) < 1e-13 and not meets[0]


def test_rule_weights_area_and_side_length(monkeypatch):
    src = _with_fn(monkeypatch, lambda x, y: np.exp(3.0 * x) * np.sin(5.0 * y))
    lev, ix, iy = [2, 2], [1, 3], [0, 2]
    e = T.rule_indicator("interp", 0.0, 0.0, 1.0, 8, src, lev, ix, iy)
    assert np.all(e > 0)
    assert np.allclose(T.rule_indicator("interp_area", 0.0, 0.0, 1.0, 8, src, lev, ix, iy), e / 16.0, rtol=0, atol=0)
    assert np.allclose(T.rule_indicator("interp_mixed", 0.0, 0.0, 1.0, 8, src, lev, ix, iy), e / 4.0, rtol=0, atol=0)


def test_boundary_boxes_of_the_kinked_source():
    wl = W.kinked()
    src = wl.sources[0]
    a, c = np.asarray(src.params)[0:7], np.asarray(src.params)[7:14]
    r0 = 0.6 + np.sum(a * np.cos(c))  # the curve crosses the positive x axis at r0
    lev = 6
    h = 2.0 / (1 << lev)
    on = (int((r0 + 1.0) // h), int(1.0 // h))  # the box holding (r0, 0) (lower left of the axis)
    inside = (int((0.3 + 1.0) // h), int((0.1 + 1.0) // h))
    outside = (int((0.95 + 1.0) // h), int((0.1 + 1.0) // h))
    ixs = [on[0], inside[0], outside[0]]
    iys = [on[1], inside[1], outside[1]]
    _, meets = T.interp_error(0.0, 0.0, 2.0, wl.k, src, [lev] * 3, ixs, iys)
    assert meets.tolist() == [True, False, False]


@pytest.mark.parametrize("rule", ["tail", "interp"])
def test_depth_cap_count_with_zero_tolerance(rule):
    # tol = 0: every box with a nonzero test quantity splits, so the tree is uniform to max_depth and
    # every leaf there is capped
    src = W.narrow_gaussians(5, n=3, sigma=0.04)
    t, info = T.build_adaptive(0.0, 0.0, 1.0, 8, src, 0.0, 3, return_info=True, rule=rule)
    assert t.n_leaves == 64 and info["n_capped"] == 64
    t, info = T.build_adaptive(0.0, 0.0, 1.0, 8, src, 1e-6, 7, return_info=True, rule=rule)
    assert t.depth < 7 and info["n_capped"] == 0


def test_interp_rules_against_closed_form_potential():
    """Section 6.1: refining until the interpolation error is within tol gives an overall error
    well below tol; weighting it by the box area gets close to tol. Checked on Gaussians well
    inside the box (closed-form potential), k = 8, p = 20, tol = 1e-6."""
    pytest.importorskip("scipy.special")
    from oracle import fmm
    from test_oracle_fmm import _gauss_closed_form
    ops = tables.Ops(8, 20)
    src = W.narrow_gaussians(31, n=3, sigma=0.03, spread=0.2)
    errs = {}
    for rule in ("interp", "interp_area"):
        t = T.build_adaptive(0, 0, 1, 8, src, 1e-6, 12, rule=rule)
        u = fmm.solve(t, T.build_lists(t), ops, t.sample(src))
        X, Y = t.leaf_nodes()
        ref = _gauss_closed_form(src.params, X, Y)
        errs[rule] = float(np.max(np.abs(u[0] - ref[0])) / np.max(np.abs(ref[0])))
    assert errs["interp"] < 1e-7
    assert 1e-7 < errs["interp_area"] < 1e-5
