"""Parity of the CUDA library with the CPU oracle, through the C ABI.

Bars: integer work (tree, lists, configuration indices) bit-exact; floating
point within 1e-13 relative L-infinity for the FP64 solve (the method's target
is 1e-10 relative, Section 6 error metric), 1e-13 absolute for unit-scale tables
(whose entries are at most ~0.1).
"""
import numpy as np
import pytest

import workloads as W
from oracle import fmm, source, tables
from oracle import tree as T

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1610_00823_gb300 as v  # noqa: E402

TOL = 1e-13


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
        assert np.array_equal(ptr, optr), name
        assert np.array_equal(idx, oidx), name
        assert np.array_equal(cfg, ocfg), name
    return L


@pytest.mark.parametrize("k,p", [(8, 20), (16, 40)])
def test_operator_tables_match_oracle(k, p, oracle_ops):
    ops = v.ops_create(k, p)
    o = oracle_ops(k, p)
    assert np.max(np.abs(ops.export("near") - o.T)) < 1e-13
    assert np.max(np.abs(ops.export("s2m") - o.Q)) < 1e-14
    assert np.max(np.abs(ops.export("s2l") - o.R)) < 1e-13
    for name, ref in (("m2m", o.M2M), ("l2l", o.L2L), ("m2l", o.M2L)):
        got = ops.export(name)
        assert np.max(np.abs(got - ref)) <= 1e-14 * max(1.0, np.max(np.abs(ref))), name


@pytest.mark.parametrize("depth", [0, 1, 3])
def test_uniform_tree_bit_exact(depth):
    gt = v.tree_build_uniform(0.1, -0.2, 1.7, 8, depth)
    ot = T.build_uniform(0.1, -0.2, 1.7, 8, depth)
    same_tree(gt, ot)


ADAPTIVE_CASES = [
    ("narrow3", lambda: W.narrow_gaussians(5, n=3, sigma=0.04), 8, 1e-6, 7),
    ("narrow_k16", lambda: W.narrow_gaussians(8, n=2, sigma=0.01, spread=0.4), 16, 1e-10, 9),
    ("kinked", lambda: W.kinked(k=8).sources[0], 8, 1e-4, 6),
]


@pytest.mark.parametrize("name,mk,k,tol,depth", ADAPTIVE_CASES)
def test_adaptive_tree_bit_exact(name, mk, k, tol, depth):
    src = mk()
    width = 2.0 if name == "kinked" else 1.0
    gt = v.tree_build(0.0, 0.0, width, k, src, tol, depth)
    ot, info = T.build_adaptive(0.0, 0.0, width, k, src, tol, depth, return_info=True)
    assert info["min_margin"] > 1e-9  # no decision sits in the rounding tie zone
    same_tree(gt, ot)
    assert abs(gt.f_scale - info["F"]) <= 1e-15 * info["F"]


@pytest.mark.parametrize("member", [0, 1, 3, 4])
def test_leaf_count_tree_bit_exact(member):
    """Greedy leaf-count trees of batch members (targets capped at 3000 to keep the oracle fast)."""
    m = W.batch_members(member + 1)[member]
    n = min(m["n_leaves_target"], 3000)
    gt = v.tree_build_leaves(0.0, 0.0, 1.0, m["k"], m["source"], n, 16)
    ot, info = T.build_greedy(0.0, 0.0, 1.0, m["k"], m["source"], n, 16, return_info=True)
    assert info["min_margin"] > 1e-6 and gt.min_margin > 1e-6  # no priority sits at a rounding tie
    same_tree(gt, ot)
    assert abs(gt.min_margin - info["min_margin"]) <= 1e-6


def test_leaf_nodes_and_sampling():
    src = W.narrow_gaussians(5, n=3, sigma=0.04)
    gt = v.tree_build(0.0, 0.0, 1.0, 8, src, 1e-6, 7)
    ot = T.build_adaptive(0.0, 0.0, 1.0, 8, src, 1e-6, 7)
    x, y = gt.leaf_nodes()
    X, Y = ot.leaf_nodes()
    assert np.max(np.abs(x.cpu().numpy() - X.reshape(-1))) <= 2.3e-16
    assert np.max(np.abs(y.cpu().numpy() - Y.reshape(-1))) <= 2.3e-16
    f = v.source_sample(gt, src).cpu().numpy()
    assert rel(f, ot.sample(src).reshape(-1)) < 1e-14


def _solve_both(gt, ot, src, k, p, oracle_ops, nrhs=1):
    ops = v.ops_create(k, p)
    F = ot.sample(src)
    fd = torch.from_numpy(F.reshape(-1)).cuda()
    u = v.volume_potential(gt, ops, fd)
    torch.cuda.synchronize()
    L = T.build_lists(ot)
    ref = fmm.solve(ot, L, oracle_ops(k, p), F)
    return [u[q].cpu().numpy().reshape(ref[q].shape) for q in range(3)], ref


def test_solve_uniform_small_case(oracle_ops):
    """Uniform depth-3 tree, k = 8, p = 20, 3 Gaussians (the small workload)."""
    wl = W.uniform_gauss3()
    gt = v.tree_build_uniform(0.0, 0.0, 1.0, wl.k, 3)
    ot = T.build_uniform(0.0, 0.0, 1.0, wl.k, 3)
    got, ref = _solve_both(gt, ot, wl.sources[0], wl.k, wl.p, oracle_ops)
    for q in range(3):
        assert rel(got[q], ref[q]) < TOL, q


@pytest.mark.parametrize("name,mk,k,tol,depth", ADAPTIVE_CASES)
def test_solve_adaptive(name, mk, k, tol, depth, oracle_ops):
    src = mk()
    width = 2.0 if name == "kinked" else 1.0
    gt = v.tree_build(0.0, 0.0, width, k, src, tol, depth)
    ot = T.build_adaptive(0.0, 0.0, width, k, src, tol, depth)
    assert ot.n_leaves > 64  # several GEMM tiles and a ragged last tile
    got, ref = _solve_both(gt, ot, src, k, 40 if k == 16 else 20, oracle_ops)
    for q in range(3):
        assert rel(got[q], ref[q]) < TOL, (name, q, rel(got[q], ref[q]))


@pytest.mark.parametrize("depth", [0, 1, 2])
def test_solve_degenerate_trees(depth, oracle_ops):
    """One leaf (no far field), four leaves (no V list), sixteen leaves."""
    src = W.narrow_gaussians(3, n=2, sigma=0.2)
    gt = v.tree_build_uniform(0.3, 0.1, 0.8, 8, depth)
    ot = T.build_uniform(0.3, 0.1, 0.8, 8, depth)
    got, ref = _solve_both(gt, ot, src, 8, 20, oracle_ops)
    for q in range(3):
        assert rel(got[q], ref[q]) < TOL


def test_multi_rhs_and_host_entry_point():
    """nrhs = 3 in one call equals three single calls bitwise; the host entry point matches too."""
    src = W.narrow_gaussians(5, n=3, sigma=0.04)
    gt = v.tree_build(0.0, 0.0, 1.0, 8, src, 1e-6, 7)
    ops = v.ops_create(8, 20)
    n = gt.n_leaves * 64
    g = torch.Generator().manual_seed(0)
    F = torch.randn(3, n, generator=g, dtype=torch.float64)
    multi = v.volume_potential(gt, ops, F.cuda())
    for r in range(3):
        single = v.volume_potential(gt, ops, F[r].cuda())
        for q in range(3):
            assert torch.equal(multi[q][r], single[q])
    host = v.volume_potential_host(gt, ops, F.pin_memory())
    for q in range(3):
        assert torch.equal(host[q], multi[q].cpu())


def test_invalid_arguments_raise():
    gt = v.tree_build_uniform(0.0, 0.0, 1.0, 8, 1)
    ops16 = v.ops_create(16, 20)
    with pytest.raises(RuntimeError):
        v.volume_potential(gt, ops16, torch.zeros(gt.n_leaves * 64, dtype=torch.float64, device="cuda"))
    with pytest.raises(RuntimeError):
        v.ops_create(3, 20)
    with pytest.raises(RuntimeError):
        v.tree_build(0.0, 0.0, -1.0, 8, W.constant_source(), 1e-3, 4)
    with pytest.raises(RuntimeError):
        v.tree_build(0.0, 0.0, 1.0, 8, W.constant_source(), 1e-3, 17)
    ops8 = v.ops_create(8, 20)
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError):
        v.volume_potential(gt, ops8, torch.zeros(gt.n_leaves * 64, dtype=torch.float64, device="cuda"), ws=ws)
