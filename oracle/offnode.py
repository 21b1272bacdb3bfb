"""The computed potential at arbitrary points from the stored expansions (Sections 3.1 and 5.3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 5.3 keeps the multipole and local expansions of every box of the hierarchy after the FMM
call, so that the potential at a new target needs O(p) work for its far field instead of a new
FMM. Here that is done for the volume potential V f~ at a point t of leaf b (the leaf holding t,
located as interp.locate does):

    V f~(t) = far(t) + near(t),
    far(t)  = -(1/2 pi) Re [ sum_l b_l ((t - z_b)/h)^l                       (b's local expansion)
                             + sum over W(b) of the box's multipole at t ],
    near(t) = sum over U(b) of -(1/2 pi) int_{B_s} log|t - y| f~_s(y) dy,

with the gradient from the differentiated expansions and kernels (Section 3.2). The near
integrals are the box integrals of quad.box_integrals at the point itself (absolute
coordinates): an on-the-fly quadrature per (point, neighbour leaf), which at a leaf node gives
what the precomputed tables give there. Points outside the closed root box get NaN.
"""
from __future__ import annotations

import math

import numpy as np

from . import fmm, interp, quad

INV2PI = 1.0 / (2.0 * math.pi)


def evaluate(tree, lists, ops, F, x, y):
    """u, u_x, u_y [3, n] at the points (x[i], y[i]) from the FMM of f~ with leaf values F."""
    F = np.asarray(F, dtype=np.float64).reshape(tree.n_leaves, ops.k ** 2)
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    M = fmm.upward(tree, ops, F)
    cache = {}
    leaf = interp.locate(tree, x, y)
    out = np.full((3, x.shape[0]), np.nan)
    up, ui, _ = lists["U"]
    wp, wi, wc = lists["W"]
    for i in np.nonzero(leaf >= 0)[0]:
        b = int(tree.leaves[leaf[i]])
        h = float(tree.h(b))
        cx, cy = tree.centre(b)
        zeta = complex((x[i] - cx) / h, (y[i] - cy) / h)
        # local expansion of b: Phi = sum_l b~_l zeta^l, Phi' = sum_l l b~_l zeta^(l-1) / h
        loc = fmm.local_of(tree, lists, ops, M, F, b, cache)
        phi, dphi = 0j, 0j
        zp = 1.0 + 0j
        for l in range(ops.p + 1):
            phi += loc[l] * zp
            if l + 1 <= ops.p:
                dphi += (l + 1) * loc[l + 1] * zp
            zp *= zeta
        dphi /= h
        # W list: multipoles of boxes of width h/2 at offset (dx, dy) / 4 in units of h
        for e in range(wp[b], wp[b + 1]):
            c = wi[e]
            dx, dy = ops.wcfg[wc[e]]
            hw = h / 2.0
            zw = 2.0 * (zeta - complex(dx, dy))
            a = M[c]
            p_w = a[0] * (math.log(hw) + np.log(zw))
            d_w = a[0] / zw
            zi = 1.0 / zw
            zq = 1.0 + 0j
            for n in range(1, ops.p + 1):
                d_w -= n * a[n] * zq * zi * zi
                zq *= zi
                p_w += a[n] * zq
            phi += p_w
            dphi += d_w / hw
        u = -INV2PI * phi.real
        ux = -INV2PI * dphi.real
        uy = INV2PI * dphi.imag
        # near field: box integrals at the point over every leaf of U(b)
        pt = np.array([[x[i], y[i]]])
        for e in range(up[b], up[b + 1]):
            s = ui[e]
            sx, sy = tree.centre(s)
            G = quad.box_integrals(pt, np.array([sx, sy]), float(tree.h(s)), ops.k)[:, 0, :]
            g = G @ F[tree.leaf_index[s]]
            u += g[0]
            ux += g[1]
            uy += g[2]
        out[:, i] = (u, ux, uy)
    return out
