"""Unit-scale operators of the box code (Section 3.1: the same operators at every level after scaling).

Scaling convention. A box of width h and centre z_b carries a multipole
expansion Phi(z) = a_0 log(z - z_b) + sum_{n>=1} a_n (z - z_b)^-n stored as
a~_n = a_n / h^n, and a local expansion Phi(z) = sum_l b_l (z - z_b)^l stored as
b~_l = b_l h^l. With these scalings every operator below is the same at every
level; the only level dependence left is an area factor h^2 and additive
log(h) terms, which the FMM applies itself. Phi represents
int log(z - w) f(w) dA(w), so u = -(1/2pi) Re Phi and u_x - i u_y = -(1/2pi) Phi'
(the complex form of Section 5.3/5.4).

Translation formulas (the paper defers to the FMM literature, Section 3.1; these
are the series of log(z - w) and (z - w)^-n written out):
  M2M, child c -> parent P, tau = (z_c - z_P)/h_P:
      A~_0 = a~_0,  A~_l = -a~_0 tau^l / l + sum_{n=1}^{l} a~_n 2^-n C(l-1, n-1) tau^(l-n)
  M2L, source c -> target b (same level h), D = (z_c - z_b)/h:
      b~_0 = a~_0 log|D| + sum_n a~_n (-D)^-n      (+ a~_0 log h, applied by the FMM)
      b~_l = -a~_0 / (l D^l) + D^-l sum_n a~_n (-D)^-n C(n+l-1, l)
  L2L, parent P -> child c, sigma = (z_c - z_P)/h_P:
      c~_m = 2^-m sum_{l>=m} b~_l C(l, m) sigma^(l-m)
The imaginary part of log(-D) in b~_0 is dropped: it changes Im Phi by a
constant and so affects neither u nor its gradient.
"""
from __future__ import annotations

import math

import numpy as np

from . import cheb, quad
from .tree import NEAR_PATTERN, FAR_PATTERN, V_OFFSETS


def near_configs():
    """(rho, Dx, Dy): source width / target width and source-centre offset in target widths."""
    out = []
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            out.append((1.0, float(dx), float(dy)))
    for (px, py) in NEAR_PATTERN:
        out.append((2.0, px / 2.0, py / 2.0))
    for (px, py) in NEAR_PATTERN:
        out.append((0.5, px / 4.0, py / 4.0))
    return out


def target_nodes(k):
    xh = cheb.nodes(k)
    gi = np.tile(np.arange(k), k)
    gj = np.repeat(np.arange(k), k)
    return np.column_stack([xh[gi], xh[gj]])  # [k*k, 2], flat j*k + i


def near_tables(k):
    """T[cfg, q, t, s]: q = 0 potential, 1, 2 gradient; unit target box [-1/2, 1/2]^2."""
    Xt = target_nodes(k)
    cfgs = near_configs()
    T = np.zeros((len(cfgs), 3, k * k, k * k))
    for ci, (rho, dx, dy) in enumerate(cfgs):
        T[ci] = quad.box_integrals(Xt, np.array([dx, dy]), rho, k)
    return T


def _contract(Wab, l1, l2):
    """sum_{a,b} W[a, b] l1[a, i] l2[b, j] -> [j, i]."""
    return l2.T @ Wab.T @ l1


def _gl_box(n, lo=-0.5, hi=0.5, splits=1):
    x, w = quad.gl01(n)
    edges = np.linspace(lo, hi, splits + 1)
    xs = np.concatenate([a + (b - a) * x for a, b in zip(edges[:-1], edges[1:])])
    ws = np.concatenate([(b - a) * w for a, b in zip(edges[:-1], edges[1:])])
    return xs, ws


def s2m_table(k, p):
    """Q[n, s] with a~_n = h^2 sum_s Q[n, s] f_s: Q_0s = int l_s, Q_ns = -(1/n) int l_s w^n."""
    ng = (p + k) // 2 + 4
    x, w = _gl_box(ng)
    l = cheb.lagrange(k, x)  # [a, i]
    Z = x[:, None] + 1j * x[None, :]  # [a (x), b (y)]
    Q = np.zeros((p + 1, k * k), dtype=np.complex128)
    ww = w[:, None] * w[None, :]
    Zn = np.ones_like(Z)
    for n in range(p + 1):
        if n == 0:
            val = _contract(ww, l, l)
        else:
            Zn = Zn * Z
            val = -(1.0 / n) * _contract(ww * Zn, l, l)
        Q[n] = val.reshape(-1)
    return Q


def l2t_tables(k, p):
    """E[t, l] = zeta_t^l and dE[t, l] = l zeta_t^(l-1), zeta_t the target node (unit box)."""
    X = target_nodes(k)
    z = X[:, 0] + 1j * X[:, 1]
    E = np.zeros((k * k, p + 1), dtype=np.complex128)
    dE = np.zeros((k * k, p + 1), dtype=np.complex128)
    for l in range(p + 1):
        E[:, l] = z ** l
        if l >= 1:
            dE[:, l] = l * z ** (l - 1)
    return E, dE


def w_configs():
    return [(px / 4.0, py / 4.0) for (px, py) in FAR_PATTERN]


def x_configs():
    return [(px / 2.0, py / 2.0) for (px, py) in FAR_PATTERN]


def s2l_tables(k, p):
    """R[cfg, l, s] for the X list: source leaf twice the target's width at D (target widths).

    b~_l += (2h)^2 sum_s R[l, s] f_s with R_ls = -(1/l) int l_s(w) (D + 2w)^-l dw (l >= 1)
    and R_0s = int l_s(w) log|D + 2w| dw, w over the unit box; the FMM adds
    (2h)^2 log(h) sum_s W_s f_s to b~_0.
    """
    ng = 24
    x, w = _gl_box(ng, splits=4)
    l = cheb.lagrange(k, x)
    ww = w[:, None] * w[None, :]
    out = np.zeros((20, p + 1, k * k), dtype=np.complex128)
    for ci, (dx, dy) in enumerate(x_configs()):
        Z = (dx + 2.0 * x[:, None]) + 1j * (dy + 2.0 * x[None, :])
        out[ci, 0] = _contract(ww * np.log(np.abs(Z)), l, l).reshape(-1)
        Zi = 1.0 / Z
        Zp = np.ones_like(Z)
        for n in range(1, p + 1):
            Zp = Zp * Zi
            out[ci, n] = (-(1.0 / n) * _contract(ww * Zp, l, l)).reshape(-1)
    return out


def binom(n, r):
    return float(math.comb(n, r)) if 0 <= r <= n else 0.0


def m2m_matrices(p):
    out = np.zeros((4, p + 1, p + 1), dtype=np.complex128)
    for pos in range(4):
        tau = ((2 * (pos & 1) - 1) + 1j * (2 * (pos >> 1) - 1)) / 4.0
        M = out[pos]
        M[0, 0] = 1.0
        for l in range(1, p + 1):
            M[l, 0] = -tau ** l / l
            for n in range(1, l + 1):
                M[l, n] = 2.0 ** (-n) * binom(l - 1, n - 1) * tau ** (l - n)
    return out


def l2l_matrices(p):
    out = np.zeros((4, p + 1, p + 1), dtype=np.complex128)
    for pos in range(4):
        sig = ((2 * (pos & 1) - 1) + 1j * (2 * (pos >> 1) - 1)) / 4.0
        M = out[pos]
        for m in range(p + 1):
            for l in range(m, p + 1):
                M[m, l] = 2.0 ** (-m) * binom(l, m) * sig ** (l - m)
    return out


def m2l_matrices(p):
    """One matrix per V offset (dx, dy) in V_OFFSETS; D = dx + i dy."""
    out = np.zeros((len(V_OFFSETS), p + 1, p + 1), dtype=np.complex128)
    for oi, (dx, dy) in enumerate(V_OFFSETS):
        D = complex(dx, dy)
        M = out[oi]
        M[0, 0] = math.log(abs(D))
        for n in range(1, p + 1):
            M[0, n] = (-D) ** (-n)
        for l in range(1, p + 1):
            M[l, 0] = -1.0 / (l * D ** l)
            for n in range(1, p + 1):
                M[l, n] = D ** (-l) * (-D) ** (-n) * binom(n + l - 1, l)
    return out


class Ops:
    """All unit-scale operators for one (k, p)."""

    def __init__(self, k, p, near=True):
        self.k, self.p = k, p
        self.W = cheb.fejer_weights_2d(k)
        self.near_cfgs = near_configs()
        self.rho = np.array([c[0] for c in self.near_cfgs])
        self.T = near_tables(k) if near else None
        self.Q = s2m_table(k, p)
        self.E, self.dE = l2t_tables(k, p)
        self.R = s2l_tables(k, p)
        self.M2M = m2m_matrices(p)
        self.L2L = l2l_matrices(p)
        self.M2L = m2l_matrices(p)
        self.wcfg = w_configs()
        self.xcfg = x_configs()
        self.Xt = target_nodes(k)
