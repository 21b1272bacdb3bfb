"""Pins of the oracle's collocation and quadrature against mathematics it does not use.

Section 3.1 (collocation on scaled nodes, precomputed near-field tables "up to
scale"), Section 3.2 (gradient kernels). Each test would fail on a plausible
slip: a wrong node sign or order, a dropped weight factor, a wrong sign in the
log-product weights, a transposed basis index, a wrong triangle orientation.
"""
import math

import numpy as np
import pytest

from oracle import cheb, quad


@pytest.mark.parametrize("k", [4, 8, 16])
def test_fejer_weights_integrate_monomials(k):
    w = cheb.fejer_weights(k)
    x = cheb.nodes(k)
    for m in range(k):
        exact = 0.0 if m % 2 else 2.0 * 0.5 ** (m + 1) / (m + 1)
        assert abs(np.dot(w, x ** m) - exact) < 1e-15


@pytest.mark.parametrize("k", [5, 8, 16])
def test_nodes_are_chebyshev_roots(k):
    x = cheb.nodes(k)
    assert np.all(np.diff(x) > 0)
    # T_k(2x) vanishes on first-kind nodes
    assert np.max(np.abs(np.cos(k * np.arccos(2 * x)))) < 1e-13


@pytest.mark.parametrize("k", [6, 16])
def test_lagrange_cardinal_and_reproduces_polynomials(k):
    x = cheb.nodes(k)
    assert np.max(np.abs(cheb.lagrange(k, x) - np.eye(k))) < 1e-15
    rng = np.random.default_rng(0)
    c = rng.normal(size=k)
    poly = np.polynomial.Polynomial(c)
    t = np.linspace(-0.5, 0.5, 41)
    assert np.max(np.abs(cheb.lagrange(k, t) @ poly(x) - poly(t))) < 1e-12


@pytest.mark.parametrize("k", [8, 16])
def test_values_to_coeffs_recovers_chebyshev_series(k):
    C = cheb.values_to_coeffs_matrix(k)
    t = 2 * cheb.nodes(k)
    for m in (0, 3, k - 1):
        v = np.cos(m * np.arccos(t))
        c = C @ v
        e = np.zeros(k)
        e[m] = 1.0
        assert np.max(np.abs(c - e)) < 1e-14
    # tail of a product T_a(x) T_b(y) is its coefficient when max(a, b) >= k - 2
    X, Y = np.meshgrid(t, t)  # [j, i]
    V = np.cos((k - 2) * np.arccos(X)) * np.cos(1 * np.arccos(Y))
    assert abs(cheb.tail(V, k) - 1.0) < 1e-13
    V = np.cos((k - 3) * np.arccos(X)) * np.cos((k - 3) * np.arccos(Y))
    assert cheb.tail(V, k) < 1e-14


@pytest.mark.parametrize("n", [8, 16, 32])
def test_log_product_weights_exact_moments(n):
    s, beta = quad.log_product_weights(n)
    for j in range(n):
        exact = -1.0 / (j + 2) ** 2  # int_0^1 s^(j+1) log s ds
        assert abs(np.dot(beta, s ** j) - exact) < 1e-15


def _F(u, v):
    # antiderivative with d2F/dudv = log(u^2 + v^2)
    return u * v * (np.log(u * u + v * v) - 3) + u * u * np.arctan(v / u) + v * v * np.arctan(u / v)


def _Fu(u, v):
    return v * np.log(u * u + v * v) - 2 * v + 2 * u * np.arctan(v / u)


def _Fv(u, v):
    return u * np.log(u * u + v * v) - 2 * u + 2 * v * np.arctan(u / v)


def _corners(fn, x, c, w):
    a1, a2 = c[0] - w / 2 - x[0], c[0] + w / 2 - x[0]
    b1, b2 = c[1] - w / 2 - x[1], c[1] + w / 2 - x[1]
    return fn(a2, b2) - fn(a1, b2) - fn(a2, b1) + fn(a1, b1)


def uniform_density_closed_form(x, c, w):
    """-(1/2pi) int_S log|x-y| dy and its gradient, from a textbook antiderivative."""
    g = -0.5 * _corners(_F, x, c, w) / (2 * math.pi)
    gx = 0.5 * _corners(_Fu, x, c, w) / (2 * math.pi)
    gy = 0.5 * _corners(_Fv, x, c, w) / (2 * math.pi)
    return np.array([g, gx, gy])


@pytest.mark.parametrize("k", [8, 16])
def test_box_integrals_uniform_density(k):
    """Sum over the basis = integral of f = 1 (Section 3.3: exact at nodes for f = 1)."""
    xs = cheb.nodes(k)
    c = np.array([0.0, 0.0])
    pts = np.array([[xs[0], xs[0]], [xs[2], xs[k - 1]], [0.0, 0.0],       # inside (self)
                    [0.5 + (0.5 + xs[0]) * 0.5, xs[3]],                   # fine neighbour node
                    [1.0 + xs[0], xs[2]], [1.0 + xs[0], 1.0 + xs[0]],     # colleague nodes
                    [0.5 + 1.0 + 2 * xs[0], 0.3], [3.1, -2.2]])           # coarse node, far
    G = quad.box_integrals(pts, c, 1.0, k).sum(axis=2)  # [3, m]
    for t, x in enumerate(pts):
        ref = uniform_density_closed_form(x, c, 1.0)
        assert np.max(np.abs(G[:, t] - ref)) < 2e-15 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.slow
def test_box_integrals_single_basis_vs_adaptive_quadpack():
    """Individual basis functions against scipy's adaptive quadrature (an independent rule)."""
    integrate = pytest.importorskip("scipy.integrate")
    k = 6
    xs = cheb.nodes(k)
    c = np.array([0.0, 0.0])
    cases = [(np.array([xs[1], xs[4]]), 7), (np.array([0.5 + 0.02, xs[2]]), 20), (np.array([1.3, 0.9]), 35)]
    for x, s in cases:
        G = quad.box_integrals(x[None, :], c, 1.0, k)[:, 0, s]
        i, j = s % k, s // k

        def f(y2, y1, q):
            l = cheb.lagrange(k, np.array([y1, y2]))
            r1, r2 = x[0] - y1, x[1] - y2
            rr = r1 * r1 + r2 * r2
            ker = (-0.5 * math.log(rr), -r1 / rr, -r2 / rr)[q] / (2 * math.pi)
            return ker * l[0, i] * l[1, j]
        for q in range(3):
            # split at the target so any singularity sits on a corner of each piece
            ref = 0.0
            xs1 = sorted({-0.5, 0.5, min(max(x[0], -0.5), 0.5)})
            xs2 = sorted({-0.5, 0.5, min(max(x[1], -0.5), 0.5)})
            for a, b in zip(xs1[:-1], xs1[1:]):
                for cc, d in zip(xs2[:-1], xs2[1:]):
                    v, _ = integrate.dblquad(f, a, b, cc, d, args=(q,), epsabs=1e-13, epsrel=1e-12)
                    ref += v
            assert abs(G[q] - ref) < 1e-10, (x, s, q, G[q], ref)


def test_box_integrals_on_the_boundary_of_the_source_box():
    """Targets on an edge or a corner of the source box (a point on an edge shared by two leaves):
    the potential and its gradient are continuous there; f = 1 against the antiderivative (at the
    corner, where the antiderivative's 0 log 0 terms need the limit, against a point 1e-12 inside)."""
    k = 8
    c = np.array([0.05, -0.02])
    w = 1.3
    hw = w / 2
    for x in ([c[0] + hw, c[1] + 0.1], [c[0] - hw, c[1] - 0.4], [c[0] + 0.2, c[1] - hw], [c[0] - 0.3, c[1] + hw]):
        x = np.array(x)
        G = quad.box_integrals(x[None, :], c, w, k).sum(axis=2)[:, 0]
        ref = uniform_density_closed_form(x, c, w)
        assert np.max(np.abs(G - ref)) < 2e-15, (x, G, ref)
    corner = c + np.array([hw, hw])
    G = quad.box_integrals(corner[None, :], c, w, k).sum(axis=2)[:, 0]
    ref = uniform_density_closed_form(corner - 1e-12, c, w)
    assert np.max(np.abs(G - ref)) < 1e-10, (G, ref)
