"""Evaluation of the synthetic right-hand sides f (plain numpy, libm functions).

The parameter layouts are the ones the seeded generators in ``workloads`` emit:
constant, sum of isotropic Gaussians A exp(-|x-c|^2 / (2 sigma^2)), and the kinked
source g max(0, phi) + h whose kink follows a closed polar curve (a synthetic
stand-in for the C^0 extension of Section 4.2).
"""
from __future__ import annotations

import math

import numpy as np

SRC_CONSTANT = 0
SRC_GAUSS_SUM = 1
SRC_KINKED = 2


def _gauss_sum(rows: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    out = np.zeros(np.broadcast(x, y).shape)
    for cx, cy, sig, amp in rows.reshape(-1, 4):
        dx = x - cx
        dy = y - cy
        out = out + amp * np.exp(-(dx * dx + dy * dy) / (2.0 * sig * sig))
    return out


def smooth_step(t: np.ndarray) -> np.ndarray:
    """psi(t) = e^{-1/t} / (e^{-1/t} + e^{-1/(1-t)}) on (0, 1); 0 below, 1 above."""
    t = np.asarray(t, dtype=np.float64)
    out = np.where(t >= 1.0, 1.0, 0.0)
    inside = (t > 0.0) & (t < 1.0)
    ti = np.where(inside, t, 0.5)
    a = np.exp(-1.0 / ti)
    b = np.exp(-1.0 / (1.0 - ti))
    return np.where(inside, a / (a + b), out)


def kinked_phi(params: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """phi(x) = r_chi(x)^2 - |x|^2 with r_chi = 0.6 + chi(|x|) sum_m a_m cos(m theta + c_m)."""
    a = params[0:7]
    c = params[7:14]
    rho = np.hypot(x, y)
    theta = np.arctan2(y, x)
    s = np.zeros(np.broadcast(x, y).shape)
    for idx in range(7):
        m = idx + 2
        s = s + a[idx] * np.cos(m * theta + c[idx])
    chi = smooth_step((rho - 0.1) / 0.2)
    r = 0.6 + chi * s
    return r * r - rho * rho


def evaluate(kind: int, params, x, y) -> np.ndarray:
    params = np.asarray(params, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if kind == SRC_CONSTANT:
        return np.full(np.broadcast(x, y).shape, params[0])
    if kind == SRC_GAUSS_SUM:
        return _gauss_sum(params, x, y)
    if kind == SRC_KINKED:
        g = _gauss_sum(params[14:34], x, y)
        h = _gauss_sum(params[34:54], x, y)
        return g * np.maximum(0.0, kinked_phi(params, x, y)) + h
    raise ValueError("unknown source kind %r" % kind)


def evaluate_source(src, x, y) -> np.ndarray:
    """Evaluate a ``workloads.Source``-like object (attributes kind, params)."""
    return evaluate(src.kind, src.params, x, y)


def gaussian_mass_in_box(rows, lo: float, hi: float) -> float:
    """int over [lo, hi]^2 of a Gaussian sum (closed form with erf)."""
    total = 0.0
    for cx, cy, sig, amp in np.asarray(rows, dtype=np.float64).reshape(-1, 4):
        s = sig * math.sqrt(2.0)
        fx = 0.5 * s * math.sqrt(math.pi) * (math.erf((hi - cx) / s) - math.erf((lo - cx) / s))
        fy = 0.5 * s * math.sqrt(math.pi) * (math.erf((hi - cy) / s) - math.erf((lo - cy) / s))
        total += amp * fx * fy
    return total
