"""Convergence orders of the oracle's box code against what the paper's error analysis predicts.

* Spectral convergence in the node count k (Section 3.3): for smooth f on a fixed uniform tree the
  interpolation error, and with it the error of the computed potential and of its gradient, falls
  geometrically in k (order m = min(k, p) of the interpolant), at the same rate for u and grad u
  (the "super-convergence" remark at the end of Section 3.3). Checked against the closed-form
  potential of radially symmetric Gaussians (exponential integral).
* Orders for a continuous, piecewise smooth f (Section 4.1, Eqs. potBound and gradBound): nearly
  third order for u (h^3 |log h|) and second order for grad u on uniform trees. Checked against the
  closed-form potential of a paraboloid cap max(0, R^2 - |x - c|^2), whose gradient jumps across
  a circle, and by self-convergence on the kinked synthetic source (its C^0 curve is a perturbed
  circle), where the reference is the oracle on a deeper tree evaluated through the leaf
  interpolant v~.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import fmm, interp
from oracle import tree as T

from test_oracle_fmm import _gauss_closed_form

P = 40


def _errors(u, ref):
    """Relative L-infinity error of u, u_x, u_y (Section 6 error metric)."""
    return [float(np.max(np.abs(np.asarray(u[q]).reshape(-1) - np.asarray(ref[q]).reshape(-1))) /
                  np.max(np.abs(np.asarray(ref[q])))) for q in range(3)]


def _slope(xs, errs):
    """Least-squares slope of log2(err) against xs."""
    return float(np.polyfit(np.asarray(xs, dtype=np.float64), np.log2(np.asarray(errs)), 1)[0])


@pytest.mark.slow
def test_spectral_convergence_in_k(oracle_ops):
    pytest.importorskip("scipy.special")
    src = W.narrow_gaussians(31, n=3, sigma=0.03, spread=0.2)  # mass outside the box < 1e-16
    ks = (4, 6, 8, 10, 12, 14, 16)
    E = []
    for k in ks:
        t = T.build_uniform(0.0, 0.0, 1.0, k, 3)
        u = fmm.solve(t, T.build_lists(t), oracle_ops(k, P), t.sample(src))
        X, Y = t.leaf_nodes()
        E.append(_errors(u, _gauss_closed_form(src.params, X, Y)))
    E = np.array(E)  # [k, q]
    for q in range(3):
        # every step of 2 in k gains at least a factor 5 (measured: 10 to 20) ...
        assert np.all(E[1:, q] < E[:-1, q] / 5.0), (q, E[:, q])
        # ... and log E falls at least linearly in k, about 1.5 to 2 bits per node
        assert _slope(ks, E[:, q]) < -1.5, (q, _slope(ks, E[:, q]))
    # the gradient converges at the rate of the potential
    su = _slope(ks, E[:, 0])
    for q in (1, 2):
        assert abs(_slope(ks, E[:, q]) - su) < 0.25 * abs(su), (q, _slope(ks, E[:, q]), su)
    assert E[-1, 0] < 1e-8 and E[-1, 1] < 1e-7 and E[-1, 2] < 1e-7


CAP_C = (0.05, -0.03)
CAP_R = 0.3


def _cap_f(X, Y):
    """Paraboloid cap max(0, R^2 - |x - c|^2): continuous, its gradient jumps on |x - c| = R."""
    dx, dy = X - CAP_C[0], Y - CAP_C[1]
    return np.maximum(0.0, CAP_R * CAP_R - (dx * dx + dy * dy))


def _cap_potential(X, Y):
    """-(1/2pi) int log|x - y| f(y) dy for the cap, and its gradient (closed form).

    For a radial f the angular mean of log|x - y| over |y - c| = s is log max(r, s), so
    V(r) = -[log(r) m(r) + int_r^R f(s) s log(s) ds] with m(r) = int_0^r f(s) s ds, and
    grad V = -(x - c) m(r) / r^2 (Gauss's law).
    """
    R = CAP_R
    dx, dy = X - CAP_C[0], Y - CAP_C[1]
    r2 = dx * dx + dy * dy
    r = np.sqrt(r2)
    inside = r < R
    m = np.where(inside, R * R * r2 / 2.0 - r2 * r2 / 4.0, R ** 4 / 4.0)

    def antider(s):  # of (R^2 - s^2) s log s
        return R * R * (s * s / 2.0 * np.log(s) - s * s / 4.0) - (s ** 4 / 4.0 * np.log(s) - s ** 4 / 16.0)

    tail = np.where(inside, antider(R) - antider(np.minimum(r, R)), 0.0)
    g = -m / r2
    return -(np.log(r) * m + tail), g * dx, g * dy


def test_cap_potential_closed_form_is_the_potential():
    """The closed form itself: -Laplacian = f away from the kink (finite differences), continuity of
    the gradient across the circle, and the far field -(M/2pi) log r of the total mass."""
    h = 1e-4
    for (x, y) in ((0.1, 0.05), (0.3, -0.2), (-0.2, 0.1)):
        u0 = _cap_potential(np.array(x), np.array(y))[0]
        lap = sum(_cap_potential(np.array(x + a), np.array(y + b))[0] for a, b in
                  ((h, 0), (-h, 0), (0, h), (0, -h))) - 4 * u0
        assert abs(-lap / h ** 2 - _cap_f(np.array(x), np.array(y))) < 1e-5
    eps = 1e-9
    for sgn in (-1, 1):
        x = CAP_C[0] + CAP_R + sgn * eps
        assert abs(_cap_potential(np.array(x), np.array(CAP_C[1]))[1] + CAP_R ** 3 / 4.0) < 1e-7
    mass = 2 * math.pi * CAP_R ** 4 / 4.0
    xf = CAP_C[0] + 0.45
    assert abs(_cap_potential(np.array(xf), np.array(CAP_C[1]))[0] + mass / (2 * math.pi) * math.log(0.45)) < 1e-15


@pytest.mark.parametrize("k,depths", [(4, (2, 3, 4, 5, 6)), (8, (2, 3, 4, 5))])
def test_continuous_kink_orders_against_closed_form(k, depths, oracle_ops):
    E, hs = [], []
    for d in depths:
        t = T.build_uniform(0.0, 0.0, 1.0, k, d)
        X, Y = t.leaf_nodes()
        u = fmm.solve(t, T.build_lists(t), oracle_ops(k, P), _cap_f(X, Y).reshape(t.n_leaves, -1))
        E.append(_errors(u, _cap_potential(X, Y)))
        hs.append(2.0 ** -d)
    E = np.array(E)
    # slopes of log2 E against the depth are the observed orders
    su = _slope(depths, E[:, 0])
    assert su < -2.2, ("potential order", -su, E[:, 0])  # nearly third order (h^3 |log h|)
    for q in (1, 2):
        sg = _slope(depths, E[:, q])
        assert -2.4 < sg < -1.7, ("gradient order", q, -sg, E[:, q])  # second order
    if k == 4:
        # Eq. gradBound: E_grad / h^2 stays within a factor 2 of its first value; Eq. potBound:
        # E_u / (h^3 |log h|) does not grow beyond twice its first value
        for q in (1, 2):
            ratio = E[:, q] / np.square(hs)
            assert np.all(ratio < 2.0 * ratio[0]) and np.all(ratio > 0.5 * ratio[0]), (q, ratio)
        ratio_u = E[:, 0] / (np.power(hs, 3) * np.abs(np.log(hs)))
        assert np.all(ratio_u < 2.0 * ratio_u[0]), ratio_u


@pytest.mark.slow
def test_kinked_source_orders_by_self_convergence(oracle_ops):
    """The kinked synthetic source (C^0 on its polar curve), k = 4, root [-1, 1]^2: errors on
    uniform depths 3..5 against the depth-7 solution evaluated at the same nodes through v~."""
    k = 4
    src = W.kinked(k=k).sources[0]
    ops = oracle_ops(k, P)
    tr = T.build_uniform(0.0, 0.0, 2.0, k, 7)
    ur = fmm.solve(tr, T.build_lists(tr), ops, tr.sample(src))
    depths = (3, 4, 5)
    E = []
    for d in depths:
        t = T.build_uniform(0.0, 0.0, 2.0, k, d)
        X, Y = t.leaf_nodes()
        u = fmm.solve(t, T.build_lists(t), ops, t.sample(src))
        ref = [interp.interpolate(tr, ur[q], X.reshape(-1), Y.reshape(-1)) for q in range(3)]
        E.append(_errors(u, ref))
    E = np.array(E)
    assert _slope(depths, E[:, 0]) < -2.2, E[:, 0]
    for q in (1, 2):
        assert -2.6 < _slope(depths, E[:, q]) < -1.6, (q, E[:, q])
