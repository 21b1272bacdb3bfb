"""Values of the computed potential away from the collocation nodes: the leaf interpolant (Section 3.1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The box code computes the potential only at the collocation nodes of the leaves. At any other
point of the root box the paper takes the polynomial that interpolates the computed values on
the leaf holding the point; it calls this piecewise polynomial v~ (Section 3.1, right after f~ is
defined; Section 3.3 returns to values at points other than the nodes and to their error). Here the leaf is found from
integer coordinates and the interpolant is evaluated as a Chebyshev series: coefficients
c = C V C^T of the leaf's k x k values (cheb.values_to_coeffs_matrix; V indexed [y node, x node]),
then v~ = sum_mn c_mn T_m(y^) T_n(x^) in the leaf's coordinates x^ = 2 (x - centre_x) / h in
[-1, 1], with T_m from the three-term recurrence.

Reading taken here (the paper does not say which leaf owns a point on an edge shared by two
leaves): the point's integer coordinates at the finest level D are floor(2^D (x - lo) / W),
clamped to 2^D - 1 on the root's upper edges, so a point on a shared edge belongs to the leaf
above it or to its right. Points outside the closed root box, or with a NaN coordinate, belong
to no leaf: index -1 and value NaN.
"""
from __future__ import annotations

import numpy as np

from . import cheb


def locate(tree, x, y) -> np.ndarray:
    """Canonical leaf index of each point (-1 outside the closed root box)."""
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    D = tree.depth
    lox = tree.cx - tree.width / 2.0
    loy = tree.cy - tree.width / 2.0
    X = (x - lox) / tree.width
    Y = (y - loy) / tree.width
    out = np.full(x.shape, -1, dtype=np.int32)
    side = float(1 << D)
    for p in range(x.shape[0]):
        if not (0.0 <= X[p] <= 1.0 and 0.0 <= Y[p] <= 1.0):
            continue
        ixd = int(min(np.floor(X[p] * side), side - 1.0))
        iyd = int(min(np.floor(Y[p] * side), side - 1.0))
        # exactly one box on the path from the root down to level D is a leaf
        for level in range(D + 1):
            b = tree.index.get((level, ixd >> (D - level), iyd >> (D - level)))
            if b is not None and tree.is_leaf[b]:
                out[p] = tree.leaf_index[b]
                break
    return out


def _chebyshev_t(k: int, t: float) -> np.ndarray:
    """T_0(t) .. T_{k-1}(t) by T_{m+1} = 2 t T_m - T_{m-1} (valid for any real t)."""
    T = np.empty(k)
    T[0] = 1.0
    if k > 1:
        T[1] = t
    for m in range(1, k - 1):
        T[m + 1] = 2.0 * t * T[m] - T[m - 1]
    return T


def interpolate(tree, values, x, y) -> np.ndarray:
    """v~ at the points: values [n_leaves, k*k] (canonical leaf order, x-fastest nodes)."""
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    k = tree.k
    V = np.asarray(values, dtype=np.float64).reshape(tree.n_leaves, k, k)
    C = cheb.values_to_coeffs_matrix(k)
    leaf = locate(tree, x, y)
    out = np.full(x.shape, np.nan)
    coef = {}
    for p in np.nonzero(leaf >= 0)[0]:
        lf = int(leaf[p])
        if lf not in coef:
            coef[lf] = C @ V[lf] @ C.T  # [m (y), n (x)]
        b = tree.leaves[lf]
        cx, cy = tree.centre(b)
        h = float(tree.h(b))
        xh = (x[p] - cx) * (2.0 / h)
        yh = (y[p] - cy) * (2.0 / h)
        out[p] = _chebyshev_t(k, yh) @ coef[lf] @ _chebyshev_t(k, xh)
    return out
