"""The FMM passes of the box code (Section 3.1, with Section 3.2 for the gradient).

For every leaf node x_t the box code returns
    V~f~(x_t) = Phi_j(x_t) + sum over near leaves of int_{B_i} G(x_t, y) f~(y) dy,
where Phi_j collects the far field by expansions (Section 3.1) and the near sum
is a table apply per neighbour configuration (Section 3.1, tables computed once
for a unit box), with the gradient from the differentiated kernels and the
differentiated expansions (Section 3.2).

Steps, in the order the FMM takes them:
  1. S2M: leaf multipoles a~ = h^2 Q f.
  2. M2M: parents from children, finest level first.
  3. Downward, level 2 to the deepest level: b~ = L2L(parent) + sum_V M2L a~_c
     (+ a~_0 log h) + sum_X [(2h)^2 R f_c (+ (2h)^2 log(h) W.f_c)].
  4. Leaves: u = near + L2T + sum_W M2T.
"""
from __future__ import annotations

import math

import numpy as np

INV2PI = 1.0 / (2.0 * math.pi)


def upward(tree, ops, F):
    """Multipole coefficients of every box. F: [n_leaves, k*k] leaf values."""
    n = tree.n_boxes
    p = ops.p
    M = np.zeros((n, p + 1), dtype=np.complex128)
    hl = tree.h(tree.leaves)
    M[tree.leaves] = (hl * hl)[:, None] * (F @ ops.Q.T)
    for l in range(tree.depth - 1, -1, -1):
        a, b = tree.level_start[l], tree.level_start[l + 1]
        bx = np.arange(a, b)
        bx = bx[~tree.is_leaf[bx]]
        for pos in range(4):
            ch = tree.child[bx, pos]
            M[bx] += M[ch] @ ops.M2M[pos].T
    return M


def _pos(tree, b):
    return ((int(tree.iy[b]) & 1) << 1) | (int(tree.ix[b]) & 1)


def local_of(tree, lists, ops, M, F, box, cache):
    """Local expansion of one box (recursively through its ancestors)."""
    if box in cache:
        return cache[box]
    p = ops.p
    l = int(tree.level[box])
    acc = np.zeros(p + 1, dtype=np.complex128)
    if l < 2:
        cache[box] = acc
        return acc
    h = float(tree.h(box))
    if l >= 3:
        par = int(tree.parent[box])
        acc = acc + ops.L2L[_pos(tree, box)] @ local_of(tree, lists, ops, M, F, par, cache)
    vp, vi, vc = lists["V"]
    for e in range(vp[box], vp[box + 1]):
        c = vi[e]
        acc = acc + ops.M2L[vc[e]] @ M[c]
        acc[0] += M[c, 0].real * math.log(h)
    xp, xi, xc = lists["X"]
    for e in range(xp[box], xp[box + 1]):
        c = xi[e]
        fc = F[tree.leaf_index[c]]
        hc2 = (2.0 * h) ** 2
        acc = acc + hc2 * (ops.R[xc[e]] @ fc)
        acc[0] += hc2 * math.log(h) * float(ops.W @ fc)
    cache[box] = acc
    return acc


def leaf_potential(tree, lists, ops, M, F, b, cache):
    """u, u_x, u_y at the k*k nodes of leaf box b."""
    h = float(tree.h(b))
    T = ops.T
    u = np.zeros(ops.k ** 2)
    ux = np.zeros(ops.k ** 2)
    uy = np.zeros(ops.k ** 2)
    # near field (U list): tables scale by h^2 (potential) and h (gradient)
    up, ui, uc = lists["U"]
    for e in range(up[b], up[b + 1]):
        s = ui[e]
        cfg = uc[e]
        fs = F[tree.leaf_index[s]]
        u += h * h * (T[cfg, 0] @ fs) - INV2PI * h * h * math.log(h) * ops.rho[cfg] ** 2 * float(ops.W @ fs)
        ux += h * (T[cfg, 1] @ fs)
        uy += h * (T[cfg, 2] @ fs)
    # far field: local expansion
    loc = local_of(tree, lists, ops, M, F, b, cache)
    phi = ops.E @ loc
    dphi = (ops.dE @ loc) / h
    u += -INV2PI * phi.real
    ux += -INV2PI * dphi.real
    uy += INV2PI * dphi.imag
    # W list: multipoles of finer boxes evaluated directly
    wp, wi, wc = lists["W"]
    z = ops.Xt[:, 0] + 1j * ops.Xt[:, 1]
    for e in range(wp[b], wp[b + 1]):
        c = wi[e]
        dx, dy = ops.wcfg[wc[e]]
        hw = h / 2.0
        zeta = 2.0 * (z - complex(dx, dy))
        a = M[c]
        phi = a[0] * (math.log(hw) + np.log(zeta))
        dphi = a[0] / zeta
        zi = 1.0 / zeta
        zp = np.ones_like(zeta)
        for n in range(1, ops.p + 1):
            dphi = dphi - n * a[n] * zp * zi * zi
            zp = zp * zi
            phi = phi + a[n] * zp
        dphi = dphi / hw
        u += -INV2PI * phi.real
        ux += -INV2PI * dphi.real
        uy += INV2PI * dphi.imag
    return u, ux, uy


def solve(tree, lists, ops, F, leaves=None):
    """u, u_x, u_y [n_sel, k*k] for the selected leaf ranks (default: all leaves)."""
    F = np.asarray(F, dtype=np.float64).reshape(tree.n_leaves, ops.k ** 2)
    M = upward(tree, ops, F)
    cache = {}
    sel = np.arange(tree.n_leaves) if leaves is None else np.asarray(leaves)
    out = np.zeros((3, sel.shape[0], ops.k ** 2))
    for r, li in enumerate(sel):
        b = int(tree.leaves[li])
        out[:, r] = leaf_potential(tree, lists, ops, M, F, b, cache)
    return out
