"""Leaf collocation on tensor first-kind Chebyshev nodes (Section 3.1).

The paper collocates f on the same nodes, scaled, on every leaf and judges a
leaf by how well the interpolant represents f. It does not fix the node family;
this oracle reads it as first-kind Chebyshev nodes (interior points, so no
target ever sits on a box edge).

Unit box convention: nodes live on [-1/2, 1/2]; the node of index i is
x_i = -cos(pi (2i + 1) / (2k)) / 2, ascending. A leaf value array is stored
x-fastest: entry j*k + i is the node (x_i, x_j).
"""
from __future__ import annotations

import math

import numpy as np


def nodes(k: int) -> np.ndarray:
    """Ascending first-kind Chebyshev nodes on [-1/2, 1/2]."""
    j = np.arange(k, dtype=np.float64)
    return -np.cos(math.pi * (2.0 * j + 1.0) / (2.0 * k)) / 2.0


def fejer_weights(k: int) -> np.ndarray:
    """Fejer's first rule on [-1/2, 1/2] (interpolatory on the nodes above).

    On [-1, 1]: w_j = (2/k) (1 - 2 sum_{m=1}^{floor(k/2)} cos(2 m theta_j) / (4 m^2 - 1)),
    theta_j = pi (2j + 1) / (2k). Halved for the unit interval, so sum(w) = 1.
    """
    j = np.arange(k, dtype=np.float64)
    theta = math.pi * (2.0 * j + 1.0) / (2.0 * k)
    acc = np.zeros(k)
    for m in range(1, k // 2 + 1):
        acc += np.cos(2.0 * m * theta) / (4.0 * m * m - 1.0)
    return (2.0 / k) * (1.0 - 2.0 * acc) / 2.0


def fejer_weights_2d(k: int) -> np.ndarray:
    """Tensor weights on the unit box, flat x-fastest (sum 1)."""
    w = fejer_weights(k)
    return np.outer(w, w).reshape(-1)  # [j, i] -> j*k + i


def lagrange(k: int, x) -> np.ndarray:
    """Lagrange basis on the k nodes at points x (unit-box coordinates): [..., k].

    The product formula l_i(x) = prod_{m != i} (x - x_m)/(x_i - x_m), with the
    numerator formed from prefix and suffix products of the factors (x - x_m).
    """
    xs = nodes(k)
    x = np.asarray(x, dtype=np.float64)
    D = x[..., None] - xs  # [..., m]
    ones = np.ones(x.shape + (1,))
    pre = np.cumprod(np.concatenate([ones, D[..., :-1]], axis=-1), axis=-1)
    suf = np.cumprod(np.concatenate([ones, D[..., :0:-1]], axis=-1), axis=-1)[..., ::-1]
    denom = np.array([np.prod([xs[i] - xs[m] for m in range(k) if m != i]) for i in range(k)])
    return pre * suf / denom


def values_to_coeffs_matrix(k: int) -> np.ndarray:
    """C[m, i] = (2 - delta_m0)/k * T_m(t_i), t_i = 2 x_i in [-1, 1].

    For samples v_i = p(t_i) of a polynomial p = sum_m c_m T_m of degree < k,
    c = C v (discrete orthogonality of the cosines on first-kind nodes).
    """
    t = 2.0 * nodes(k)
    m = np.arange(k)
    T = np.cos(np.outer(m, np.arccos(np.clip(t, -1.0, 1.0))))
    C = (2.0 / k) * T
    C[0, :] *= 0.5
    return C


def tail(values_jk: np.ndarray, k: int, C: np.ndarray | None = None) -> np.ndarray:
    """Refinement indicator: max |c_mn| over coefficients with max(m, n) >= k - 2.

    values_jk: [..., k, k] samples indexed [y-node j, x-node i]. The two-dimensional
    coefficients are c = C V C^T. The last two rows and columns are used (a single
    trailing row misses functions that are even about the box centre).
    """
    if C is None:
        C = values_to_coeffs_matrix(k)
    coef = np.einsum("mj,...ji,ni->...mn", C, values_jk, C)
    mask = np.zeros((k, k), dtype=bool)
    mask[k - 2:, :] = True
    mask[:, k - 2:] = True
    return np.max(np.abs(coef[..., mask]), axis=-1)
