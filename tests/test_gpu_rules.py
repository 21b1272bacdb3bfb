"""The a-priori refinement rules of Section 6.1 (vfmm_tree_build_rule) against the oracle.

Trees and lists must match the oracle's bit for bit for each rule (interpolation error on the
children's nodes; weighted by area; by area on boxes meeting the kinked source's curve and by
side length elsewhere), on Gaussians and on the kinked source. The decisions are checked to sit
well away from the threshold on both sides (margins), so rounding cannot decide them. The tail
rule through vfmm_tree_build_rule is vfmm_tree_build; an unknown rule is INVALID_ARG.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import tree as T

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1610_00823_gb300 as v  # noqa: E402
from paper_1610_00823_gb300 import _lib  # noqa: E402
from paper_1610_00823_gb300.api import _source  # noqa: E402

CASES = {"gauss": (lambda: W.narrow_gaussians(5, n=3, sigma=0.04), 8, 1e-6, 7, 1.0),
         "kinked": (lambda: W.kinked().sources[0], 8, 1e-5, 6, 2.0)}


def same_tree(gt, ot):
    lv, ix, iy = gt.export_boxes()
    assert gt.n_boxes == ot.n_boxes and gt.n_leaves == ot.n_leaves
    assert np.array_equal(lv, ot.level) and np.array_equal(ix, ot.ix) and np.array_equal(iy, ot.iy)
    L = T.build_lists(ot)
    for name in "UVWX":
        ptr, idx, cfg = gt.export_list(name)
        optr, oidx, ocfg = L[name]
        assert np.array_equal(ptr, optr) and np.array_equal(idx, oidx) and np.array_equal(cfg, ocfg), name


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("rule", ["interp", "interp_area", "interp_mixed"])
def test_rule_tree_bit_exact_with_oracle(case, rule):
    mk, k, tol, depth, width = CASES[case]
    src = mk()
    gt = v.tree_build(0.0, 0.0, width, k, src, tol, depth, rule=rule)
    ot, info = T.build_adaptive(0.0, 0.0, width, k, src, tol, depth, return_info=True, rule=rule)
    assert info["min_margin"] > 1e-3 and gt.min_margin > 1e-3
    same_tree(gt, ot)
    assert gt.n_leaves > 64


def test_tail_rule_is_tree_build_and_unknown_rule_is_rejected():
    src = W.narrow_gaussians(5, n=3, sigma=0.04)
    a = v.tree_build(0.0, 0.0, 1.0, 8, src, 1e-6, 7)
    prm = _lib.TreeParams(0.0, 0.0, 1.0, 8, 7, 0, 1e-6)
    s, keep = _source(src)
    h = ctypes.c_void_p()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    lib = _lib.load()
    assert lib.vfmm_tree_build_rule(ctypes.byref(prm), ctypes.byref(s), 0, stream, ctypes.byref(h)) == 0
    b = v.Tree(h, 8)
    for x, y in zip(a.export_boxes(), b.export_boxes()):
        assert np.array_equal(x, y)
    h2 = ctypes.c_void_p()
    assert lib.vfmm_tree_build_rule(ctypes.byref(prm), ctypes.byref(s), 4, stream, ctypes.byref(h2)) == -1
    del keep


@pytest.mark.parametrize("case,rule,depth", [("gauss", "tail", 4), ("kinked", "tail", 4), ("gauss", "interp", 3),
                                             ("kinked", "interp_mixed", 2), ("gauss", "tail", 7)])
def test_depth_capped_leaves_match_oracle(case, rule, depth):
    mk, k, tol, _, width = CASES[case]
    src = mk()
    gt = v.tree_build(0.0, 0.0, width, k, src, tol, depth, rule=rule)
    ot, info = T.build_adaptive(0.0, 0.0, width, k, src, tol, depth, return_info=True, rule=rule)
    same_tree(gt, ot)
    assert gt.n_depth_capped == info["n_capped"]
    if depth < 7:
        assert gt.n_depth_capped > 0


def test_depth_capped_conventions():
    assert v.tree_build_uniform(0.0, 0.0, 1.0, 8, 3).n_depth_capped == 0
    src = W.narrow_gaussians(5, n=3, sigma=0.04)
    assert v.tree_build_leaves(0.0, 0.0, 1.0, 8, src, 50).n_depth_capped == -1
    assert v.tree_build_pull(0.0, 0.0, 1.0, 8, lambda x, y: x * y, 1e-6, 2).n_depth_capped == -1
