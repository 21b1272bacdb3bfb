#!/usr/bin/env python3
"""Writes csrc/planewave_rule.h: the quadrature rules of the plane-wave (exponential) M2L.

The far-field translation of Section 3.1 can be diagonalised with plane waves, as the box code
the paper builds on does. In 2-D this rests on the Laplace transform

    1 / u^n = 1/(n-1)! * integral_0^inf lambda^(n-1) exp(-lambda u) d lambda,   Re u > 0,

applied to the multipole terms (z - z_c)^-n after a rotation d in {1, i, -1, -i} that puts the
source box on the negative real side of the target box: u = (z - z_c) / d = U0 + zeta / d, with
U0 = -D / d, D the source-centre offset in box widths and zeta the target point's offset from its
box centre. For the 40 offsets of the V list, Re U0 is 2 or 3 and |Im U0| <= 3.

The Taylor coefficient of zeta^l of (U0 + zeta/d)^-n needs the moments

    mu_m(U0) = integral_0^inf lambda^m exp(-lambda U0) d lambda = m! / U0^(m+1),  m = n + l - 1,

for 0 <= m <= 2p - 1 at the 14 points U0 = a + i b, a in {2, 3}, b in {-3..3}. A rule
(lambda_j, omega_j) with sum_j omega_j lambda_j^m exp(-lambda_j U0) = mu_m(U0) turns the dense
(p+1) x (p+1) translation into: multipole -> s exponential coefficients (per direction), one
complex multiplication per coefficient and V entry, exponential -> local.

Construction (discretise, then compress): a composite Gauss-Legendre rule on [0, 90] integrates
every moment to rounding; its columns lambda^m exp(-lambda U0) c_m sqrt(w) (real and imaginary
parts as rows, c_m = 2^(m/2) / m!: a scaled multipole coefficient of order n is at most
mass 2^(-n/2) and the local expansion is used at |zeta| <= 2^(-1/2), so c_m bounds how an error in
mu_m reaches the potential) are reduced by column-pivoted QR to the s columns whose R diagonal
exceeds eps of the first; the kept nodes' weights come from the interpolative decomposition of
the dropped columns, so the reduced rule reproduces the fine rule's sums.

Run: python paper_1610_00823_gb300/planewave_rule.py   (numpy + scipy; rewrites the header)
"""
from __future__ import annotations

import math
import os

import numpy as np

# largest p each rule serves; a solve takes the first rule whose bound is >= its p
P_BUCKETS = (10, 20, 30, 40, 60)
EPS = 1e-14
LAMBDA_MAX, PANELS, PANEL_NODES = 90.0, 90, 24


def offsets_u0():
    """The 14 rotated centre offsets U0 = -D/d of the V list (Re U0 in {2, 3}, Im U0 in -3..3)."""
    return [complex(a, b) for a in (2, 3) for b in range(-3, 4)]


def fine_rule():
    x, w = np.polynomial.legendre.leggauss(PANEL_NODES)
    edges = np.linspace(0.0, LAMBDA_MAX, PANELS + 1)
    lam = np.concatenate([(a + b) / 2 + (b - a) / 2 * x for a, b in zip(edges[:-1], edges[1:])])
    wt = np.concatenate([(b - a) / 2 * w for a, b in zip(edges[:-1], edges[1:])])
    return lam, wt


def moment_rows(lam, pmax):
    rows = []
    for m in range(2 * pmax):
        c = 2.0 ** (m / 2) / math.factorial(m)
        for u0 in offsets_u0():
            f = lam ** m * np.exp(-lam * u0) * c
            rows.append(f.real)
            rows.append(f.imag)
    return np.array(rows)


def make_rule(pmax, eps=EPS):
    """(lambda, omega) sorted by lambda, for every p <= pmax."""
    import scipy.linalg as sla

    lam, wt = fine_rule()
    sw = np.sqrt(wt)
    A = moment_rows(lam, pmax) * sw[None, :]
    _, R, piv = sla.qr(A, mode="economic", pivoting=True)
    d = np.abs(np.diag(R))
    s = int(np.sum(d > eps * d[0]))
    T = sla.solve_triangular(R[:s, :s], R[:s, s:])
    omega = sw[piv[:s]] * (sw[piv[:s]] + T @ sw[piv[s:]])
    lam_s = lam[piv[:s]]
    order = np.argsort(lam_s)
    return lam_s[order], omega[order]


def write_header(path):
    lines = [
        "// Generated by paper_1610_00823_gb300/planewave_rule.py: quadrature rules (lambda_j, omega_j)",
        "// of the plane-wave M2L, sum_j omega_j lambda_j^m exp(-lambda_j U0) = m! / U0^(m+1) for",
        "// 0 <= m < 2 pmax at the 14 rotated V-list offsets U0 (weighted by 2^(m/2) / m!, to %.0e)." % EPS,
        "#pragma once",
        "",
        "namespace vfmm {",
        "",
        "struct PlaneWaveRule {",
        "    int pmax;",
        "    int s;",
        "    const double* lambda;",
        "    const double* omega;",
        "};",
        "",
    ]
    names = []
    for pm in P_BUCKETS:
        lam, om = make_rule(pm)
        tag = "pw_p%d" % pm
        names.append((pm, len(lam), tag))
        lines.append("static const double %s_lambda[%d] = {" % (tag, len(lam)))
        lines += ["    %s," % float(v).hex() for v in lam]
        lines.append("};")
        lines.append("static const double %s_omega[%d] = {" % (tag, len(om)))
        lines += ["    %s," % float(v).hex() for v in om]
        lines.append("};")
        lines.append("")
    lines.append("static const PlaneWaveRule kPlaneWaveRules[%d] = {" % len(names))
    for pm, s, tag in names:
        lines.append("    {%d, %d, %s_lambda, %s_omega}," % (pm, s, tag, tag))
    lines.append("};")
    lines.append("")
    lines.append("}  // namespace vfmm")
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    return names


def read_header(path=None):
    """The rules stored in the header: {pmax: (lambda, omega)}."""
    import re

    path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "planewave_rule.h")
    text = open(path).read()
    out = {}
    for m in re.finditer(r"static const double pw_p(\d+)_(lambda|omega)\[(\d+)\] = \{(.*?)\};", text, re.S):
        vals = np.array([float.fromhex(v.strip()) for v in m.group(4).split(",") if v.strip()])
        out.setdefault(int(m.group(1)), {})[m.group(2)] = vals
    return {pm: (d["lambda"], d["omega"]) for pm, d in out.items()}


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    for pm, s, _ in write_header(os.path.join(here, "csrc", "planewave_rule.h")):
        print("p <= %d: %d nodes" % (pm, s))
