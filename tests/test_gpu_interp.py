"""Parity of v~ (vfmm_leaf_interpolate, Section 3.1) with the oracle's leaf interpolant.

The FP64 solve's u, u_x, u_y are interpolated at points of several kinds: uniform random
points, points clustered in the smallest leaves, exact leaf nodes, points on edges shared by
two leaves (which belong to the upper or right leaf), the root's corners, points outside the
root box and NaN. Leaf indices must match the oracle bit for bit; values within 1e-13 of the
largest |value| (the library evaluates the barycentric form, the oracle a Chebyshev series of
the same data, so only rounding separates them). Outside points give NaN and leaf -1.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import interp
from oracle import tree as T

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1610_00823_gb300 as v  # noqa: E402
from paper_1610_00823_gb300 import _lib  # noqa: E402

TOL = 1e-13


def _points(ot, rng):
    lo = np.array([ot.cx, ot.cy]) - ot.width / 2
    pts = [lo + ot.width * rng.random((4000, 2))]
    deep = ot.leaves[np.argsort(-ot.level[ot.leaves])[:8]]
    for b in deep:  # clustered in the smallest leaves
        h = float(ot.h(b))
        pts.append(lo + np.array([ot.ix[b], ot.iy[b]]) * h + h * rng.random((60, 2)))
    X, Y = ot.leaf_nodes()
    pick = rng.choice(ot.n_leaves, size=min(12, ot.n_leaves), replace=False)
    pts.append(np.stack([X[pick].reshape(-1), Y[pick].reshape(-1)], axis=1))  # exact nodes
    edges = []
    for b in ot.leaves[pick]:  # left and bottom edge midpoints, and the lower-left corner
        h = float(ot.h(b))
        x0 = lo[0] + ot.ix[b] * h
        y0 = lo[1] + ot.iy[b] * h
        edges += [(x0, y0 + 0.5 * h), (x0 + 0.5 * h, y0), (x0, y0)]
    pts.append(np.array(edges))
    hi = lo + ot.width
    pts.append(np.array([[lo[0], lo[1]], [hi[0], lo[1]], [lo[0], hi[1]], [hi[0], hi[1]]]))
    pts.append(np.array([[hi[0] + 1e-9, lo[1]], [lo[0] - 0.1, 0.0], [0.0, hi[1] * 1.5 + 1.0], [np.nan, 0.0]]))
    return np.concatenate(pts)


@pytest.mark.parametrize("k,p,depth", [(16, 40, 9), (8, 20, 7), (5, 0, 5)])
def test_leaf_interpolate_matches_oracle(k, p, depth):
    src = W.narrow_gaussians(8, n=2, sigma=0.01, spread=0.4) if k == 16 else W.narrow_gaussians(5, n=3, sigma=0.04)
    gt = v.tree_build(0.0, 0.0, 1.0, k, src, 1e-10 if k == 16 else 1e-6, depth)
    ot = T.build_adaptive(0.0, 0.0, 1.0, k, src, 1e-10 if k == 16 else 1e-6, depth)
    assert gt.n_leaves == ot.n_leaves
    f = v.source_sample(gt, src)
    if p:
        u = v.volume_potential(gt, v.ops_create(k, p), f)
    else:  # k without solve operators here: interpolate the source values and two random fields
        u = (f, torch.randn_like(f), torch.randn_like(f))
    pts = _points(ot, np.random.default_rng(k))
    x = torch.from_numpy(np.ascontiguousarray(pts[:, 0])).cuda()
    y = torch.from_numpy(np.ascontiguousarray(pts[:, 1])).cuda()
    got, leaf = v.leaf_interpolate(gt, list(u), x, y, with_leaf=True)
    torch.cuda.synchronize()
    leaf = leaf.cpu().numpy()
    assert np.array_equal(leaf, interp.locate(ot, pts[:, 0], pts[:, 1]))
    outside = leaf < 0
    assert outside.sum() == 4
    for q in range(3):
        vals = u[q].cpu().numpy().reshape(ot.n_leaves, k * k)
        ref = interp.interpolate(ot, vals, pts[:, 0], pts[:, 1])
        g = got[q].cpu().numpy()
        assert np.all(np.isnan(g[outside])) and np.all(np.isnan(ref[outside]))
        err = np.max(np.abs(g[~outside] - ref[~outside])) / np.max(np.abs(vals))
        assert err < TOL, (k, q, err)


def test_leaf_interpolate_reproduces_node_values_and_edge_cases():
    gt = v.tree_build_uniform(0.0, 0.0, 1.0, 8, 3)
    x, y = gt.leaf_nodes()
    vals = torch.randn(x.numel(), dtype=torch.float64, device="cuda")
    (got,) = v.leaf_interpolate(gt, [vals], x, y)
    assert torch.max(torch.abs(got - vals)).item() < 1e-13 * torch.max(torch.abs(vals)).item()
    empty = torch.empty(0, dtype=torch.float64, device="cuda")
    assert v.leaf_interpolate(gt, [vals], empty, empty)[0].numel() == 0
    lib = _lib.load()
    fp = (ctypes.c_void_p * 1)(vals.data_ptr())
    op = (ctypes.c_void_p * 1)(got.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    xp, yp = ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr())
    assert lib.vfmm_leaf_interpolate(gt.handle, 0, fp, x.numel(), xp, yp, op, None, stream) == -1
    assert lib.vfmm_leaf_interpolate(gt.handle, 9, fp, x.numel(), xp, yp, op, None, stream) == -1
    assert lib.vfmm_leaf_interpolate(gt.handle, 1, fp, -1, xp, yp, op, None, stream) == -1
