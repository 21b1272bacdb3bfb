"""The plane-wave M2L's quadrature rules and factorisation, checked on the CPU against closed forms.

Section 3.1 attributes the box code's far-field speed to plane-wave (diagonalised) translations.
The library's rules (csrc/planewave_rule.h) discretise 1/u^n = 1/(n-1)! int lambda^(n-1)
e^(-lambda u) d lambda. Pins, independent of how the rules were built:
* every moment sum_j omega_j lambda_j^m e^(-lambda_j U0) against m! / U0^(m+1) (the Laplace
  transform of lambda^m) at the 14 rotated V offsets, weighted as the translation uses it;
* the outgoing / diagonal / incoming factorisation the kernels apply, composed here with the four
  side rotations and the exact log terms, against the oracle's dense M2L matrices for all 40 V
  offsets, including the point-source check the oracle's matrices are pinned by;
* the rule is not tuned to the 14 offsets alone: it holds on the segments between them.
"""
import math

import numpy as np
import pytest

from oracle import tables
from oracle.tree import V_OFFSETS
from paper_1610_00823_gb300 import planewave_rule as R

RULES = R.read_header()


def _side(dx, dy):
    if dy >= 2:
        return 3
    if dy <= -2:
        return 1
    return 2 if dx >= 2 else 0


def planewave_m2l(p, lam, om, dx, dy):
    """The (p+1) x (p+1) operator b~ = M a~ that the outgoing, diagonal and incoming steps compose to
    (M[l, n]: input coefficient n to output coefficient l), with the log column n = 0 exact."""
    q = _side(dx, dy)
    d = 1j ** q
    D = complex(dx, dy)
    U0 = -D / d
    M = np.zeros((p + 1, p + 1), dtype=complex)
    diag = om * np.exp(-lam * U0)
    for n in range(1, p + 1):
        out = d ** (-n) * lam ** (n - 1) / math.factorial(n - 1)  # X_q[j] per unit a~_n
        for l in range(p + 1):
            inc = (-lam) ** l / math.factorial(l) * d ** (-l)
            M[l, n] = np.sum(inc * diag * out)
    M[0, 0] = math.log(abs(D))
    for l in range(1, p + 1):
        M[l, 0] = -1.0 / (l * D ** l)
    return M


def test_header_holds_every_bucket_sorted_and_short():
    assert sorted(RULES) == [10, 20, 30, 40, 60]
    for pm, (lam, om) in RULES.items():
        assert len(lam) == len(om) <= 96  # three nodes per lane in the kernels
        assert np.all(np.diff(lam) > 0) and lam[0] > 0


def test_header_is_what_the_generator_writes():
    """The committed rules come from the committed script: regenerating the two smaller buckets gives
    the same nodes, and weights equal to rounding (a differently pivoted QR would change the node
    set, which the moment pins below would still have to accept)."""
    pytest.importorskip("scipy")
    for pm in (10, 20):
        lam, om = R.make_rule(pm)
        hl, ho = RULES[pm]
        assert len(lam) == len(hl)
        assert np.allclose(lam, hl, rtol=1e-13, atol=0.0)
        assert np.allclose(om, ho, rtol=1e-9, atol=1e-300)


@pytest.mark.parametrize("pmax", [10, 20, 30, 40, 60])
def test_moments_match_the_laplace_transform(pmax):
    lam, om = RULES[pmax]
    worst = 0.0
    for m in range(2 * pmax):
        c = 2.0 ** (m / 2) / math.factorial(m)
        for u0 in R.offsets_u0():
            got = np.sum(om * lam ** m * np.exp(-lam * u0))
            exact = math.factorial(m) / u0 ** (m + 1)
            worst = max(worst, abs(got - exact) * c)
    assert worst < 2e-14, worst


@pytest.mark.parametrize("p,pmax", [(8, 10), (20, 20), (30, 30), (40, 40), (60, 60)])
def test_factorisation_equals_the_dense_m2l(p, pmax):
    lam, om = RULES[pmax]
    dense = tables.m2l_matrices(p)  # [offset][l][n]
    w = 2.0 ** (-np.arange(p + 1) / 2.0)  # |a~_n| <= mass 2^(-n/2), |zeta| <= 2^(-1/2)
    worst = 0.0
    for oi, (dx, dy) in enumerate(V_OFFSETS):
        E = np.abs(planewave_m2l(p, lam, om, dx, dy) - dense[oi]) * w[:, None] * w[None, :]
        worst = max(worst, E.sum(axis=1).max())
    assert worst < 1e-14, worst


def test_point_sources_through_the_factorisation():
    """Unit charges in a source box of the V list: the local expansion built by the plane-wave
    steps reproduces sum log(z - w) at points of the target box (the field the oracle's M2L is
    pinned against), for every side."""
    p = 40
    lam, om = RULES[40]
    rng = np.random.default_rng(3)
    for (dx, dy) in [(-3, 0), (2, 1), (0, 3), (-1, -2), (3, 3), (-3, -3), (2, -3)]:
        D = complex(dx, dy)
        ws = D + (rng.random(5) - 0.5) + 1j * (rng.random(5) - 0.5)  # unit box around D
        a = np.zeros(p + 1, dtype=complex)  # scaled multipole about D
        a[0] = len(ws)
        for n in range(1, p + 1):
            a[n] = -np.sum((ws - D) ** n) / n
        b = planewave_m2l(p, lam, om, dx, dy) @ a
        z = (rng.random(6) - 0.5) + 1j * (rng.random(6) - 0.5)
        got = np.array([np.sum(b * zz ** np.arange(p + 1)) for zz in z])
        exact = np.array([np.sum(np.log(zz - ws)) for zz in z])
        # real parts (Im log carries a branch constant the expansions drop)
        assert np.max(np.abs(got.real - exact.real)) < 1e-12 * len(ws)


def test_rule_between_the_offsets():
    """Off the 14 design points (Re U0 in [2, 3], |Im U0| <= 3), the low moments stay accurate: the
    rule represents e^(-lambda U0) on the whole rectangle, not only at its integer points."""
    lam, om = RULES[40]
    worst = 0.0
    for a in np.linspace(2.0, 3.0, 5):
        for bb in np.linspace(-3.0, 3.0, 13):
            u0 = complex(a, bb)
            for m in range(0, 20):
                c = 2.0 ** (m / 2) / math.factorial(m)
                got = np.sum(om * lam ** m * np.exp(-lam * u0))
                worst = max(worst, abs(got - math.factorial(m) / u0 ** (m + 1)) * c)
    assert worst < 1e-9, worst
