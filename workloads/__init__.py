"""Seeded synthetic inputs for the volume-potential box FMM.

This module only draws parameters. It holds none of the method's arithmetic
(no node placement, no kernel, no quadrature, no tree logic): both the oracle
under ``oracle/`` and the CUDA path read the parameter arrays it returns and
evaluate the source function f themselves, each with its own code.

The paper's own experiments use closed-form right-hand sides on a box
(Section 6, Examples 1 and 2); the workloads below are synthetic stand-ins with
the same structure: smooth sums of Gaussians of mixed widths (smooth f, as in
Section 3.3) and a continuous source with a kink along a closed polar curve
(the C^0 extended right-hand side of Section 4.2).

Flat parameter layouts (shared convention, also stated in include/vfmm.h):

* ``SRC_CONSTANT`` (kind 0): ``[A]``                      f = A
* ``SRC_GAUSS_SUM`` (kind 1): ``n`` rows of ``[cx, cy, sigma, A]``
  f(x) = sum A exp(-|x - c|^2 / (2 sigma^2))
* ``SRC_KINKED`` (kind 2): ``[a_2..a_8, c_2..c_8, g rows (5 x 4), h rows (5 x 4)]``
  f = g max(0, phi) + h with phi(x) = r_chi(x)^2 - |x|^2,
  r_chi = 0.6 + chi(|x|) sum_m a_m cos(m theta + c_m), chi the smooth step from
  0 (|x| <= 0.1) to 1 (|x| >= 0.3), and g, h Gaussian sums of the layout above.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List

import numpy as np

SRC_CONSTANT = 0
SRC_GAUSS_SUM = 1
SRC_KINKED = 2

SEED_BASE = 20161003


@dataclass
class Source:
    kind: int
    n: int
    params: np.ndarray  # float64, flat

    def as_list(self) -> List[float]:
        return [float(v) for v in self.params]


@dataclass
class Workload:
    name: str
    cx: float
    cy: float
    width: float
    k: int
    p: int
    tol: float
    max_depth: int
    min_depth: int
    uniform_depth: int  # >= 0: uniform tree of this depth; -1: adaptive
    sources: List[Source] = field(default_factory=list)


def constant_source(a: float = 1.0) -> Source:
    return Source(SRC_CONSTANT, 1, np.array([a], dtype=np.float64))


def gauss_source(centres, sigmas, amps) -> Source:
    centres = np.asarray(centres, dtype=np.float64).reshape(-1, 2)
    sigmas = np.broadcast_to(np.asarray(sigmas, dtype=np.float64), (centres.shape[0],))
    amps = np.asarray(amps, dtype=np.float64).reshape(-1)
    rows = np.column_stack([centres[:, 0], centres[:, 1], sigmas, amps])
    return Source(SRC_GAUSS_SUM, rows.shape[0], rows.reshape(-1).copy())


def _three_gaussians(rng: np.random.Generator) -> Source:
    centres = rng.uniform(-0.3, 0.3, size=(3, 2))
    amps = rng.uniform(-1.0, 1.0, size=3)
    return gauss_source(centres, 0.1, amps)


def uniform_gauss3(seed: int = SEED_BASE + 1, depth: int = 3, k: int = 8, p: int = 20) -> Workload:
    """Uniform tree, 3 Gaussians of width 0.1 on the unit box (the small case)."""
    rng = np.random.default_rng(seed)
    return Workload("uniform_d%d_k%d_p%d_gauss3" % (depth, k, p), 0.0, 0.0, 1.0, k, p,
                    0.0, depth, depth, depth, [_three_gaussians(rng)])


def adaptive_gauss20(seed: int = SEED_BASE + 2, k: int = 16, p: int = 40, tol: float = 1e-10,
                     max_depth: int = 16) -> Workload:
    """Adaptive tree, 20 Gaussians with log-uniform widths in [1e-3, 1e-1]."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-0.45, 0.45, size=(20, 2))
    sigmas = np.exp(rng.uniform(math.log(1e-3), math.log(1e-1), size=20))
    amps = rng.normal(0.0, 1.0, size=20)
    return Workload("adaptive_gauss20_k%d_p%d" % (k, p), 0.0, 0.0, 1.0, k, p, tol,
                    max_depth, 0, -1, [gauss_source(centres, sigmas, amps)])


def kinked(seed: int = SEED_BASE + 3, k: int = 16, p: int = 40, tol: float = 1e-10,
           max_depth: int = 14) -> Workload:
    """Continuous source with a kink on a closed polar curve, root box [-1, 1]^2."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, 0.03, size=7)
    c = rng.uniform(0.0, 2.0 * math.pi, size=7)
    rows = []
    for _ in range(2):
        centres = rng.uniform(-0.6, 0.6, size=(5, 2))
        amps = rng.normal(0.0, 1.0, size=5)
        rows.append(np.column_stack([centres[:, 0], centres[:, 1], np.full(5, 0.2), amps]))
    params = np.concatenate([a, c, rows[0].reshape(-1), rows[1].reshape(-1)])
    return Workload("kinked_k%d_p%d" % (k, p), 0.0, 0.0, 2.0, k, p, tol, max_depth, 0, -1,
                    [Source(SRC_KINKED, 5, params)])


def batch_members(n: int = 256, seed_base: int = SEED_BASE * 1000):
    """Independent uneven problems: leaf target log-uniform in [100, 5e4], k in {8, 16}."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed_base + i)
        src = _three_gaussians(rng)
        n_target = int(round(math.exp(rng.uniform(math.log(100.0), math.log(5e4)))))
        k = 8 if rng.uniform() < 0.5 else 16
        out.append({"source": src, "n_leaves_target": n_target, "k": k, "p": 20 if k == 8 else 40})
    return out


def shared_tree_rhs(n_rhs: int = 64, seed: int = SEED_BASE + 5):
    """Many right-hand sides (3 Gaussians each) for one uniform depth-3 tree."""
    rng = np.random.default_rng(seed)
    return [_three_gaussians(rng) for _ in range(n_rhs)]


def narrow_gaussians(seed: int, n: int = 3, sigma: float = 0.02, spread: float = 0.3) -> Source:
    """Gaussians whose mass outside the unit box is below 1e-16 (closed-form tests)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-spread, spread, size=(n, 2))
    amps = rng.uniform(-1.0, 1.0, size=n)
    return gauss_source(centres, sigma, amps)
