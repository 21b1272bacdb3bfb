"""vfmm_evaluate_points (V f~ at arbitrary points from the stored expansions, Section 5.3) against
the oracle's offnode.evaluate, element by element, through the C ABI.

Cases: a uniform tree and adaptive trees with W and X lists (k = 8 and 16), seeded random points,
points at leaf nodes (where it must give the solve's own values), points on shared leaf edges and
corners (the leaf convention), points 1e-3, 1e-6 and 1e-9 of a leaf width from a leaf edge (the
kernel's finer quadrature rules) and points outside the root (NaN). Bar: 1e-12 relative to the largest
|value| over the points (FP64 throughout; the near field by on-the-fly quadrature on both sides,
with different rules: tanh-sinh on the GPU, Gauss-Legendre with log-product weights in the oracle).
"""
import numpy as np
import pytest

import workloads as W
from oracle import offnode
from oracle import tree as T

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1610_00823_gb300 as v  # noqa: E402

TOL = 1e-12


def _rel(a, b):
    b = np.asarray(b)
    return float(np.max(np.abs(np.asarray(a) - b)) / np.max(np.abs(b)))


CASES = [
    ("uniform_k8", 8, 20, None, 0.0, 3),
    ("adaptive_k8", 8, 20, lambda: W.narrow_gaussians(5, n=3, sigma=0.04), 1e-6, 7),
    ("adaptive_k16", 16, 40, lambda: W.narrow_gaussians(8, n=2, sigma=0.02, spread=0.35), 1e-9, 8),
]


@pytest.mark.parametrize("name,k,p,mk,tol,depth", CASES)
def test_evaluate_points_matches_oracle(name, k, p, mk, tol, depth, oracle_ops):
    if mk is None:
        src = W.uniform_gauss3().sources[0]
        gt = v.tree_build_uniform(0.0, 0.0, 1.0, k, depth)
        ot = T.build_uniform(0.0, 0.0, 1.0, k, depth)
    else:
        src = mk()
        gt = v.tree_build(0.0, 0.0, 1.0, k, src, tol, depth)
        ot = T.build_adaptive(0.0, 0.0, 1.0, k, src, tol, depth)
    L = T.build_lists(ot)
    if mk is not None:
        assert len(L["W"][1]) > 0
    F = ot.sample(src)
    f = torch.from_numpy(F.reshape(-1)).cuda()
    ops = v.ops_create(k, p, v.FP64)
    ws = v.workspace(gt, ops, 1)
    sol = v.volume_potential(gt, ops, f, ws=ws)
    rng = np.random.default_rng(17)
    n_rand = 48 if k == 8 else 16
    pts = [rng.uniform(-0.5, 0.5, size=(n_rand, 2))]
    X, Y = ot.leaf_nodes()
    node_sel = rng.choice(X.size, size=8, replace=False)
    pts.append(np.column_stack([X.reshape(-1)[node_sel], Y.reshape(-1)[node_sel]]))
    # on shared edges and a corner of the level-2 grid, and outside the root box
    pts.append(np.array([[0.0, 0.1], [0.25, -0.3], [0.25, 0.25], [-0.5, 0.5], [0.7, 0.0]]))
    # 1e-3, 1e-6 and 1e-9 of a leaf width on either side of a leaf's right edge (the finer
    # quadrature rules of the kernel)
    for b in ot.leaves[len(ot.leaves) // 3:]:  # a leaf whose right edge is inside the root box
        hb = float(ot.h(int(b)))
        cx, cy = ot.centre(int(b))
        if cx + hb < 0.5:
            break
    for d in (1e-3, 1e-6, 1e-9):
        pts.append(np.array([[cx + hb / 2 - d * hb, cy + 0.1 * hb], [cx + hb / 2 + d * hb, cy - 0.2 * hb]]))
    pts = np.concatenate(pts)
    x = torch.from_numpy(pts[:, 0].copy()).cuda()
    y = torch.from_numpy(pts[:, 1].copy()).cuda()
    got = [o.cpu().numpy() for o in v.evaluate_points(gt, ops, f, ws, x, y)]
    ref = offnode.evaluate(ot, L, oracle_ops(k, p), F, pts[:, 0], pts[:, 1])
    inside = ~np.isnan(ref[0])
    assert np.array_equal(np.isnan(got[0]), ~inside)
    assert inside[-6:].all()
    for q in range(3):
        assert _rel(got[q][inside], ref[q][inside]) < TOL, (name, q, _rel(got[q][inside], ref[q][inside]))
    # at leaf nodes: the solve's own values
    for q in range(3):
        node_vals = sol[q].cpu().numpy()[node_sel]
        assert _rel(got[q][n_rand:n_rand + 8], node_vals) < TOL, (name, q)
