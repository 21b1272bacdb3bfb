"""Integrals of the kernel against the leaf basis over one box (Section 3.1, 3.2).

For a target point x and a source box S (centre c, width w) this module returns,
for every basis function l_s of S (the tensor Lagrange basis on the nodes of
``cheb``, in S's normalised coordinates (y - c)/w),

    G_s(x)  = -(1/2pi) int_S log|x - y|        l_s(y) dy        (Eq. volumeint3)
    G1_s(x) = -(1/2pi) int_S (x1 - y1)/|x-y|^2 l_s(y) dy        (Eq. volumeint3x)
    G2_s(x) = -(1/2pi) int_S (x2 - y2)/|x-y|^2 l_s(y) dy

The paper computes these once for a unit box, to be scaled at every level, by an adaptive
brute-force quadrature (Section 1; Section 3.1 on precomputed tables). This oracle uses two
plain rules:

* x inside S: S is cut into four triangles with apex x. On the triangle (x, P0,
  P1) the map y = x + s (P0 + t (P1 - P0) - x), (s, t) in [0, 1]^2, has Jacobian
  s D with D = cross(P0 - x, P1 - P0), and log|x - y| = log s + log r(t) with
  r(t) = |P0 + t (P1 - P0) - x|. In s the integrand is s log s (or s) times a
  polynomial of degree 2k - 2, integrated exactly by Gauss-Legendre nodes with
  product weights for s log s. In t the integrand is a polynomial times log r(t)
  or (e(t) - x)/r(t)^2, smooth but nearly singular at the foot of the
  perpendicular from x; a composite Gauss-Legendre rule graded geometrically
  toward that foot resolves it.
* x outside S: S is split recursively into quarters until each piece lies at a
  distance of at least its own width from x; each piece gets a tensor
  Gauss-Legendre rule.
"""
from __future__ import annotations

import functools
import math

import numpy as np

from . import cheb

INV2PI = 1.0 / (2.0 * math.pi)


@functools.lru_cache(maxsize=None)
def _gl01(n: int):
    x, w = np.polynomial.legendre.leggauss(n)
    return (x + 1.0) / 2.0, w / 2.0


def gl01(n: int):
    """Gauss-Legendre nodes and weights on [0, 1]."""
    x, w = _gl01(n)
    return x.copy(), w.copy()


def log_product_weights(n: int):
    """Weights beta_a with sum_a beta_a q(s_a) = int_0^1 s log(s) q(s) ds for deg q < n.

    q is expanded in shifted Legendre polynomials P*_m through the discrete
    orthogonality of the n-point rule; the moments of s log s against P*_m follow
    from int_0^1 log(s) P*_m(s) ds = -1 (m = 0), (-1)^(m+1)/(m(m+1)) (m >= 1) and
    the recurrence s P*_m = ((m+1) P*_{m+1} + m P*_{m-1}) / (2(2m+1)) + P*_m / 2.
    """
    s, w = gl01(n)
    lam = np.zeros(n + 1)
    lam[0] = -1.0
    for m in range(1, n + 1):
        lam[m] = (-1.0) ** (m + 1) / (m * (m + 1.0))
    nu = np.zeros(n)
    for m in range(n):
        v = (m + 1) * lam[m + 1]
        if m >= 1:
            v += m * lam[m - 1]
        nu[m] = v / (2.0 * (2 * m + 1)) + lam[m] / 2.0
    # P*_m at the nodes
    P = np.polynomial.legendre.legvander(2.0 * s - 1.0, n - 1)  # [a, m]
    coef = (2.0 * np.arange(n) + 1.0)[None, :] * w[:, None] * P  # c_{a m}
    return s, coef @ nu


def graded_rule(t0: float, eta: float, n: int):
    """Composite Gauss-Legendre on [0, 1] with pieces doubling away from t0.

    The innermost pieces have length eta (the scale of a singularity at
    distance eta from the real axis above t0).
    """
    br = {0.0, 1.0, t0}
    if eta < 1.0:
        step = eta
        while step < 1.0:
            for v in (t0 - step, t0 + step):
                if 0.0 < v < 1.0:
                    br.add(v)
            step *= 2.0
    br = sorted(br)
    x, w = gl01(n)
    ts, ws = [], []
    for a, b in zip(br[:-1], br[1:]):
        if b - a <= 0.0:
            continue
        ts.append(a + (b - a) * x)
        ws.append((b - a) * w)
    return np.concatenate(ts), np.concatenate(ws)


def _accumulate(Wq, l1, l2):
    """sum_q W_q l1[q, i] l2[q, j] -> flat [j*k + i]."""
    return ((l2 * Wq[:, None]).T @ l1).reshape(-1)


def self_integrals(x, c, w, k):
    """(G, G1, G2) for one target x in the closed box S (triangles with apex x). On the boundary
    of S (a point of an edge shared with a neighbour leaf) the triangle over its own edge has no
    area and is dropped: the potential and its gradient are continuous there and the other
    triangles give their value at the point."""
    x = np.asarray(x, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    hw = w / 2.0
    corners = [c + np.array([-hw, -hw]), c + np.array([hw, -hw]),
               c + np.array([hw, hw]), c + np.array([-hw, hw])]
    ns = 2 * k
    s, beta = log_product_weights(ns)
    _, wgl = gl01(ns)
    alpha = wgl * s
    nt = 2 * k + 8
    out = np.zeros((3, k * k))
    for e in range(4):
        P0, P1 = corners[e], corners[(e + 1) % 4]
        E = P1 - P0
        L = math.hypot(E[0], E[1])
        D = (P0[0] - x[0]) * E[1] - (P0[1] - x[1]) * E[0]
        if D < 0.0:
            raise ValueError("target outside the source box")
        if D == 0.0:
            continue  # x on this edge's line: a triangle of zero area
        d = D / L
        t0 = min(max(float(np.dot(x - P0, E)) / (L * L), 0.0), 1.0)
        t, wt = graded_rule(t0, d / L, nt)
        et = P0[None, :] + t[:, None] * E[None, :]          # [nt, 2]
        rt = np.hypot(et[:, 0] - x[0], et[:, 1] - x[1])
        Y = x[None, None, :] + s[:, None, None] * (et[None, :, :] - x[None, None, :])  # [ns, nt, 2]
        l1 = cheb.lagrange(k, (Y[..., 0] - c[0]) / w).reshape(-1, k)
        l2 = cheb.lagrange(k, (Y[..., 1] - c[1]) / w).reshape(-1, k)
        # potential: -(1/2pi) D sum_b wt_b sum_a (beta_a + alpha_a log r_b) l(y_ab)
        Wp = -INV2PI * D * (beta[:, None] + alpha[:, None] * np.log(rt)[None, :]) * wt[None, :]
        # gradient: (D/2pi) wt_b (e_b - x)/r_b^2 * wgl_a
        g1 = INV2PI * D * ((et[:, 0] - x[0]) / (rt * rt)) * wt
        g2 = INV2PI * D * ((et[:, 1] - x[1]) / (rt * rt)) * wt
        W1 = wgl[:, None] * g1[None, :]
        W2 = wgl[:, None] * g2[None, :]
        out[0] += _accumulate(Wp.reshape(-1), l1, l2)
        out[1] += _accumulate(W1.reshape(-1), l1, l2)
        out[2] += _accumulate(W2.reshape(-1), l1, l2)
    return out


def _box_dist(X, cs, ws):
    dx = np.maximum(np.abs(X[:, 0] - cs[0]) - ws / 2.0, 0.0)
    dy = np.maximum(np.abs(X[:, 1] - cs[1]) - ws / 2.0, 0.0)
    return np.hypot(dx, dy)


def outside_integrals(X, c, w, k, cs=None, ws=None, ng=None):
    """(G, G1, G2) for targets X [m, 2] outside S: array [3, m, k*k]."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, 2)
    c = np.asarray(c, dtype=np.float64)
    if cs is None:
        cs, ws = c, w
    if ng is None:
        ng = k + 10
    m = X.shape[0]
    out = np.zeros((3, m, k * k))
    if m == 0:
        return out
    dist = _box_dist(X, cs, ws)
    if np.any(dist <= 0.0):
        raise ValueError("target inside a source piece")
    far = dist >= ws
    if np.any(far):
        xg, wg = gl01(ng)
        y1 = cs[0] - ws / 2.0 + ws * xg
        y2 = cs[1] - ws / 2.0 + ws * xg
        wq = ws * wg
        l1 = cheb.lagrange(k, (y1 - c[0]) / w)  # [a, i]
        l2 = cheb.lagrange(k, (y2 - c[1]) / w)  # [b, j]
        Xf = X[far]
        r1 = Xf[:, 0][:, None, None] - y1[None, :, None]   # [t, a, b]
        r2 = Xf[:, 1][:, None, None] - y2[None, None, :]
        rr = r1 * r1 + r2 * r2
        ww = wq[:, None] * wq[None, :]
        K0 = -INV2PI * 0.5 * np.log(rr) * ww
        K1 = -INV2PI * r1 / rr * ww
        K2 = -INV2PI * r2 / rr * ww
        for q, K in enumerate((K0, K1, K2)):
            tmp = K @ l2                                   # [t, a, j]
            out[q, far] = (np.swapaxes(tmp, 1, 2) @ l1).reshape(-1, k * k)  # [t, j, i]
    near = ~far
    if np.any(near):
        Xn = X[near]
        acc = np.zeros((3, Xn.shape[0], k * k))
        for qy in (-1, 1):
            for qx in (-1, 1):
                cc = cs + np.array([qx, qy]) * (ws / 4.0)
                acc += outside_integrals(Xn, c, w, k, cc, ws / 2.0, ng)
        out[:, near] = acc
    return out


def box_integrals(X, c, w, k):
    """(G, G1, G2) for any targets X [m, 2] (the closed box S included): [3, m, k*k]."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, 2)
    c = np.asarray(c, dtype=np.float64)
    inside = (np.abs(X[:, 0] - c[0]) <= w / 2.0) & (np.abs(X[:, 1] - c[1]) <= w / 2.0)
    out = np.zeros((3, X.shape[0], k * k))
    if np.any(~inside):
        out[:, ~inside] = outside_integrals(X[~inside], c, w, k)
    for t in np.nonzero(inside)[0]:
        out[:, t] = self_integrals(X[t], c, w, k)
    return out
