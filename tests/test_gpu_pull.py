"""Adaptive trees for a caller-evaluated f (vfmm_tree_begin / pending / submit / finish).

* A paraboloid cap f = max(0, r^2 - |x - c|^2): continuous with a kink on a circle, so the tree
  refines along the circle. Every operation in it is exactly rounded, so the caller's values at
  the library's nodes equal the oracle's at its own, and the tree and lists must match the
  oracle's bit-exactly; the FP64 solve on that tree matches the oracle within 1e-13.
* f equal to a built-in Gaussian source, evaluated by the caller: the same tree as
  vfmm_tree_build with that source.
* Misuse of the protocol is rejected with INVALID_ARG and leaves the builder usable.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import fmm
from oracle import source as srcmod
from oracle import tree as T

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1610_00823_gb300 as v  # noqa: E402
from paper_1610_00823_gb300 import _lib  # noqa: E402

TOL = 1e-13
INVALID_ARG = -1
CAP = (0.13, -0.07, 0.31)  # centre x, centre y, radius


def cap_torch(x, y):
    dx = x - CAP[0]
    dy = y - CAP[1]
    return torch.clamp(CAP[2] * CAP[2] - (dx * dx + dy * dy), min=0.0)


def cap_numpy(x, y):
    dx = x - CAP[0]
    dy = y - CAP[1]
    return np.maximum(CAP[2] * CAP[2] - (dx * dx + dy * dy), 0.0)


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def same_tree(gt, ot):
    lv, ix, iy = gt.export_boxes()
    assert gt.n_boxes == ot.n_boxes and gt.n_leaves == ot.n_leaves
    assert np.array_equal(lv, ot.level) and np.array_equal(ix, ot.ix) and np.array_equal(iy, ot.iy)
    L = T.build_lists(ot)
    for name in "UVWX":
        ptr, idx, cfg = gt.export_list(name)
        optr, oidx, ocfg = L[name]
        assert np.array_equal(ptr, optr) and np.array_equal(idx, oidx) and np.array_equal(cfg, ocfg), name
    return L


@pytest.mark.parametrize("depth,min_depth", [(6, 0), (6, 3), (0, 0), (1, 1)])
def test_pull_tree_bit_exact_with_oracle(monkeypatch, depth, min_depth):
    monkeypatch.setattr(srcmod, "evaluate_source", lambda s, x, y: cap_numpy(x, y))
    gt = v.tree_build_pull(0.0, 0.0, 1.0, 8, cap_torch, 1e-6, depth, min_depth)
    ot, info = T.build_adaptive(0.0, 0.0, 1.0, 8, None, 1e-6, depth, min_depth, return_info=True)
    same_tree(gt, ot)
    assert gt.f_scale == info["F"]
    if depth == 6:
        assert gt.n_leaves > 300 and gt.depth == 6


def test_pull_tree_solve_matches_oracle(monkeypatch, oracle_ops):
    monkeypatch.setattr(srcmod, "evaluate_source", lambda s, x, y: cap_numpy(x, y))
    k, p = 8, 20
    gt = v.tree_build_pull(0.0, 0.0, 1.0, k, cap_torch, 1e-6, 5)
    ot = T.build_adaptive(0.0, 0.0, 1.0, k, None, 1e-6, 5)
    L = same_tree(gt, ot)
    x, y = gt.leaf_nodes()
    f = cap_torch(x, y)
    F = ot.sample(None)
    assert np.array_equal(f.cpu().numpy(), F.reshape(-1))
    u = v.volume_potential(gt, v.ops_create(k, p), f)
    torch.cuda.synchronize()
    ref = fmm.solve(ot, L, oracle_ops(k, p), F)
    for q in range(3):
        got = u[q].cpu().numpy().reshape(ref[q].shape)
        assert rel(got, ref[q]) < TOL, (q, rel(got, ref[q]))


def test_pull_with_builtin_source_values_equals_tree_build():
    src = W.narrow_gaussians(5, n=3, sigma=0.04)
    rows = np.asarray(src.params, dtype=np.float64).reshape(-1, 4)

    def gauss(x, y):
        acc = torch.zeros_like(x)
        for cx, cy, sig, amp in rows:
            dx = x - cx
            dy = y - cy
            acc = acc + amp * torch.exp(-(dx * dx + dy * dy) / (2.0 * sig * sig))
        return acc

    built = v.tree_build(0.0, 0.0, 1.0, 8, src, 1e-6, 7)
    pulled = v.tree_build_pull(0.0, 0.0, 1.0, 8, gauss, 1e-6, 7)
    # the two evaluations of exp may differ in the last bit; no decision is that close
    assert built.min_margin > 1e-9 and pulled.min_margin > 1e-9
    assert abs(pulled.f_scale - built.f_scale) <= 1e-14 * built.f_scale
    for a, b in zip(built.export_boxes(), pulled.export_boxes()):
        assert np.array_equal(a, b)
    for name in "UVWX":
        for a, b in zip(built.export_list(name), pulled.export_list(name)):
            assert np.array_equal(a, b), name


def test_pull_protocol_misuse_is_rejected():
    lib = _lib.load()
    prm = _lib.TreeParams(0.0, 0.0, 1.0, 8, 3, 0, 1e-6)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    b = ctypes.c_void_p()
    assert lib.vfmm_tree_begin(ctypes.byref(prm), stream, ctypes.byref(b)) == 0
    try:
        h = ctypes.c_void_p()
        assert lib.vfmm_tree_finish(b, ctypes.byref(h)) == INVALID_ARG  # f still pending
        n = ctypes.c_int64()
        assert lib.vfmm_tree_pending(b, ctypes.byref(n)) == 0
        assert n.value == 4 ** 3 * 64  # the f-scale grid: 4^min(5, 3) boxes, k^2 nodes each
        zeros = torch.zeros(n.value, dtype=torch.float64, device="cuda")
        assert lib.vfmm_tree_submit(b, ctypes.c_void_p(zeros.data_ptr())) == 0
        assert lib.vfmm_tree_pending(b, ctypes.byref(n)) == 0
        assert n.value == 64  # the root box
        assert lib.vfmm_tree_submit(b, ctypes.c_void_p(zeros.data_ptr())) == 0  # f = 0: nothing splits
        assert lib.vfmm_tree_pending(b, ctypes.byref(n)) == 0 and n.value == 0
        x = torch.empty(64, dtype=torch.float64, device="cuda")
        assert lib.vfmm_tree_pending_nodes(b, ctypes.c_void_p(x.data_ptr()),
                                           ctypes.c_void_p(x.data_ptr())) == INVALID_ARG
        assert lib.vfmm_tree_submit(b, ctypes.c_void_p(zeros.data_ptr())) == INVALID_ARG
        assert lib.vfmm_tree_finish(b, ctypes.byref(h)) == 0
        t = v.Tree(h, 8)
        assert t.n_leaves == 1 and t.n_boxes == 1
        h2 = ctypes.c_void_p()
        assert lib.vfmm_tree_finish(b, ctypes.byref(h2)) == INVALID_ARG  # once per builder
    finally:
        lib.vfmm_tree_builder_destroy(b)
    bad = _lib.TreeParams(0.0, 0.0, 1.0, 8, 3, 4, 1e-6)  # min_depth > max_depth
    b2 = ctypes.c_void_p()
    assert lib.vfmm_tree_begin(ctypes.byref(bad), stream, ctypes.byref(b2)) == INVALID_ARG
