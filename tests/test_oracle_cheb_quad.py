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


# ---- Green's second identity: an independent route to single-basis box integrals
def _pmul(a, b):
    out = {}
    for (i, j), c in a.items():
        for (k, l), d in b.items():
            out[(i + k, j + l)] = out.get((i + k, j + l), 0) + c * d
    return out


def _lagrange_poly(mp, k, i, axis):
    """Monomial coefficients {(a, b): c} of the 1-D Lagrange basis l_i on first-kind nodes, in y1 or y2."""
    nodes = [-mp.cos(mp.pi * (2 * m + 1) / (2 * k)) / 2 for m in range(k)]
    p = {(0, 0): mp.mpf(1)}
    for m in range(k):
        if m != i:
            den = nodes[i] - nodes[m]
            p = _pmul(p, {((1, 0) if axis == 0 else (0, 1)): 1 / den, (0, 0): -nodes[m] / den})
    return p


def _pdiff(p, axis):
    out = {}
    for (a, b), c in p.items():
        e = a if axis == 0 else b
        if e > 0:
            key = (a - 1, b) if axis == 0 else (a, b - 1)
            out[key] = out.get(key, 0) + e * c
    return out


def _inverse_laplacian(mp, p):
    """A polynomial q with q_11 + q_22 = p: q = sum_m (-1)^m (d1^-2)^(m+1) d2^(2m) p (the series stops)."""
    out = {}
    for (a, b), c in p.items():
        m = 0
        while 2 * m <= b:
            f = mp.factorial(a) / mp.factorial(a + 2 * m + 2) * mp.factorial(b) / mp.factorial(b - 2 * m)
            key = (a + 2 * m + 2, b - 2 * m)
            out[key] = out.get(key, 0) + (-1) ** m * f * c
            m += 1
    return out


def _green_box(mp, p, x):
    """int_B -(1/2 pi) log|x - y| p(y) dy on B = [-1/2, 1/2]^2 (x off the boundary) by Green's second
    identity: -q(x) [x in B] + sum over the edges of int (G dq/dn - q dG/dn) ds, Laplacian q = p; the
    edge integrals by tanh-sinh, split where x projects onto the edge."""
    q = _inverse_laplacian(mp, p)
    dq = (_pdiff(q, 0), _pdiff(q, 1))
    ev = lambda poly, y1, y2: mp.fsum(c * y1 ** a * y2 ** b for (a, b), c in poly.items())  # noqa: E731
    x1, x2 = mp.mpf(x[0]), mp.mpf(x[1])
    total = -ev(q, x1, x2) if (abs(x1) < 0.5 and abs(x2) < 0.5) else mp.mpf(0)
    for ax in (0, 1):
        for val, sgn in ((mp.mpf(0.5), 1), (mp.mpf(-0.5), -1)):
            def f(s):
                y1, y2 = (val, s) if ax == 0 else (s, val)
                r1, r2 = x1 - y1, x2 - y2
                rr = r1 * r1 + r2 * r2
                return (-mp.log(rr) / (4 * mp.pi) * sgn * ev(dq[ax], y1, y2)
                        - ev(q, y1, y2) * sgn * (r1 if ax == 0 else r2) / (2 * mp.pi * rr))
            proj = x2 if ax == 0 else x1
            total += mp.quad(f, [mp.mpf(-0.5)] + ([proj] if abs(proj) < 0.5 else []) + [mp.mpf(0.5)])
    return total


def _green_box_gradient(mp, p, x, axis):
    """d/dx_axis of the same integral: V[dp/dy_axis](x) - int_dB G p n_axis ds (integration by parts)."""
    g = _green_box(mp, _pdiff(p, axis), x)
    ev = lambda poly, y1, y2: mp.fsum(c * y1 ** a * y2 ** b for (a, b), c in poly.items())  # noqa: E731
    x1, x2 = mp.mpf(x[0]), mp.mpf(x[1])
    for val, sgn in ((mp.mpf(0.5), 1), (mp.mpf(-0.5), -1)):
        def f(s):
            y1, y2 = (val, s) if axis == 0 else (s, val)
            return -mp.log((x1 - y1) ** 2 + (x2 - y2) ** 2) / (4 * mp.pi) * ev(p, y1, y2) * sgn
        proj = x2 if axis == 0 else x1
        g -= mp.quad(f, [mp.mpf(-0.5)] + ([proj] if abs(proj) < 0.5 else []) + [mp.mpf(0.5)])
    return g


def test_box_integrals_single_basis_vs_greens_identity():
    """Single tensor Lagrange basis functions (k = 6) against Green's second identity in 30-digit
    arithmetic: the area integral of the log kernel becomes a polynomial value plus edge integrals,
    an independent route (no area quadrature, no product weights). Targets inside the box (nodes
    and a non-node point), 0.02 outside an edge, and far; potential and both gradient components."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    k = 6
    xs = cheb.nodes(k)
    cases = [(np.array([xs[1], xs[4]]), 7), (np.array([xs[0], xs[0]]), 0), (np.array([0.0, 0.25]), 14),
             (np.array([0.5 + 0.02, xs[2]]), 20), (np.array([1.3, 0.9]), 35)]
    for x, s in cases:
        G = quad.box_integrals(x[None, :], np.array([0.0, 0.0]), 1.0, k)[:, 0, s]
        p = _pmul(_lagrange_poly(mp, k, s % k, 0), _lagrange_poly(mp, k, s // k, 1))
        ref = [_green_box(mp, p, x), _green_box_gradient(mp, p, x, 0), _green_box_gradient(mp, p, x, 1)]
        for q in range(3):
            assert abs(G[q] - float(ref[q])) < 1e-15, (x, s, q, G[q], float(ref[q]))


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
