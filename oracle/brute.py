"""Direct quadrature of V[f~] at leaf nodes: no FMM, no tables, no scaling.

Vf~(x_t) = sum over leaves c of sum_s f_{c,s} int_{B_c} G(x_t, y) l_s(y) dy in
absolute coordinates (Section 3.1: the quantity the box code approximates within
eps_V ||f~||_1). Cost is O(N^2): meant for trees of at most a few dozen leaves.
"""
from __future__ import annotations

import numpy as np

from . import quad


def brute_potential(tree, F, targets=None):
    """[3, n_targets] at the given points (default: all leaf nodes, leaf-major)."""
    k = tree.k
    F = np.asarray(F, dtype=np.float64).reshape(tree.n_leaves, k * k)
    if targets is None:
        X, Y = tree.leaf_nodes()
        targets = np.column_stack([X.reshape(-1), Y.reshape(-1)])
    out = np.zeros((3, targets.shape[0]))
    for li, b in enumerate(tree.leaves):
        cx, cy = tree.centre(b)
        G = quad.box_integrals(targets, np.array([cx, cy]), float(tree.h(b)), k)
        out += G @ F[li]
    return out
