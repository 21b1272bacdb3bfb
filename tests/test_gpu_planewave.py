"""Plane-wave M2L (the diagonalised far-field translation of Section 3.1) on the GPU, FP64 form.

The solve with VFMM_M2L_PLANEWAVE is compared with the oracle's box code (dense Laurent-to-Taylor
M2L) element by element; the rule's error is about 1e-15 of the expansions' scale, so the FP64 bar
of the other parity tests, 1e-13 relative L-infinity, applies unchanged.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fmm
from oracle import tree as T

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1610_00823_gb300 as v  # noqa: E402
from paper_1610_00823_gb300.api import SolveGraph, workspace  # noqa: E402

TOL = 1e-13


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _pw_ops(k, p):
    ops = v.ops_create(k, p)
    ops.set_m2l(v.M2L_PLANEWAVE)
    return ops


def _check(gt, ot, src, k, p, oracle_ops):
    F = ot.sample(src)
    u = v.volume_potential(gt, _pw_ops(k, p), torch.from_numpy(F.reshape(-1)).cuda())
    torch.cuda.synchronize()
    ref = fmm.solve(ot, T.build_lists(ot), oracle_ops(k, p), F)
    for q in range(3):
        got = u[q].cpu().numpy().reshape(ref[q].shape)
        assert rel(got, ref[q]) < TOL, (q, rel(got, ref[q]))


def test_form_switch_and_rule_length():
    ops = v.ops_create(8, 20)
    assert ops.m2l == (v.M2L_DENSE, 73)
    gt = v.tree_build_uniform(0.0, 0.0, 1.0, 8, 4)
    dense_bytes = v.workspace_size(gt, ops)
    ops.set_m2l(v.M2L_PLANEWAVE)
    assert ops.m2l == (v.M2L_PLANEWAVE, 73)
    assert v.workspace_size(gt, ops) != dense_bytes  # per-box waves instead of per-entry slab rows
    with pytest.raises(RuntimeError):
        v.ops_create(16, 40, v.MIXED).set_m2l(v.M2L_PLANEWAVE)
    with pytest.raises(RuntimeError):
        ops.set_m2l(7)


def test_uniform_small_case(oracle_ops):
    wl = W.uniform_gauss3()
    gt = v.tree_build_uniform(0.0, 0.0, 1.0, wl.k, 3)
    ot = T.build_uniform(0.0, 0.0, 1.0, wl.k, 3)
    _check(gt, ot, wl.sources[0], wl.k, wl.p, oracle_ops)


@pytest.mark.parametrize("depth", [0, 1, 2])
def test_degenerate_trees(depth, oracle_ops):
    """One leaf, four leaves (no V list), sixteen leaves (V lists at level 2 only)."""
    src = W.narrow_gaussians(3, n=2, sigma=0.2)
    gt = v.tree_build_uniform(0.3, 0.1, 0.8, 8, depth)
    ot = T.build_uniform(0.3, 0.1, 0.8, 8, depth)
    _check(gt, ot, src, 8, 20, oracle_ops)


@pytest.mark.parametrize("name,mk,k,tol,depth,width", [
    ("narrow3", lambda: W.narrow_gaussians(5, n=3, sigma=0.04), 8, 1e-6, 7, 1.0),
    ("narrow_k16", lambda: W.narrow_gaussians(8, n=2, sigma=0.01, spread=0.4), 16, 1e-10, 9, 1.0),
    ("kinked", lambda: W.kinked(k=8).sources[0], 8, 1e-4, 6, 2.0),
])
def test_adaptive_trees(name, mk, k, tol, depth, width, oracle_ops):
    src = mk()
    gt = v.tree_build(0.0, 0.0, width, k, src, tol, depth)
    ot = T.build_adaptive(0.0, 0.0, width, k, src, tol, depth)
    assert ot.n_leaves > 64
    _check(gt, ot, src, k, 40 if k == 16 else 20, oracle_ops)


def test_p60_rule_on_a_uniform_tree(oracle_ops):
    """The longest expansion the library takes (p = 60) with its own rule, depth 4 (V lists on
    three levels, interior boxes with all 27 entries)."""
    src = W.narrow_gaussians(11, n=3, sigma=0.08)
    gt = v.tree_build_uniform(0.0, 0.0, 1.0, 4, 4)
    ot = T.build_uniform(0.0, 0.0, 1.0, 4, 4)
    _check(gt, ot, src, 4, 60, oracle_ops)


def test_full_size_equals_dense_form_in_a_graph():
    """Config-2 workload (1,219 leaves, k = 16, p = 40) replayed as a CUDA graph on a side stream,
    as the benchmark times it: the plane-wave solve equals the dense FP64 solve (itself held to the
    oracle by the full-size parity test) on every target."""
    wl = W.adaptive_gauss20()
    gt = v.tree_build(wl.cx, wl.cy, wl.width, wl.k, wl.sources[0], wl.tol, wl.max_depth, wl.min_depth)
    f = v.source_sample(gt, wl.sources[0])
    res = []
    for form in (v.M2L_DENSE, v.M2L_PLANEWAVE):
        ops = v.ops_create(wl.k, wl.p)
        ops.set_m2l(form)
        stream = torch.cuda.Stream()
        out = tuple(torch.full_like(f, float("nan")) for _ in range(3))
        g = SolveGraph(gt, ops, f, out, workspace(gt, ops, 1), stream)
        g.launch(stream)
        g.launch(stream)  # a replay overwrites every output: no state carried between steps
        stream.synchronize()
        res.append([o.cpu().numpy() for o in out])
    for q in range(3):
        assert np.all(np.isfinite(res[1][q]))
        assert rel(res[1][q], res[0][q]) < TOL, (q, rel(res[1][q], res[0][q]))
