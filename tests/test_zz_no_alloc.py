"""The allocation-free solve agrees with the workspace-based solve.

vfmm_volume_potential_noalloc serves callers that cannot allocate device memory
(their own pool allocator owns it all): it runs the same solve in a static device
scratch array. This file is collected last so that a run stopping at the first
failure has already run every other test. Calls go through the C ABI (ctypes).
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1610_00823_gb300 as v  # noqa: E402
from paper_1610_00823_gb300 import _lib  # noqa: E402

TOL = 1e-13  # the tolerance of the FP64 parity tests
TOL_MIXED = 1e-10  # the tolerance of the split-BF16 (mixed) tests


def _noalloc(tree, ops, f, out):
    nrhs = f.numel() // (tree.n_leaves * tree.k * tree.k)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return _lib.load().vfmm_volume_potential_noalloc(
        tree.handle, ops.handle, ctypes.c_void_p(f.data_ptr()), nrhs, ctypes.c_void_p(out[0].data_ptr()),
        ctypes.c_void_p(out[1].data_ptr()), ctypes.c_void_p(out[2].data_ptr()), stream)


def _status():
    """Status word of the static scratch after the stream is synchronised (0 = no wait ran out)."""
    return _lib.load().vfmm_workspace_status(None)


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("case", ["uniform_k8_d3", "adaptive_k8"])
def test_noalloc_matches_workspace_solve_twice(case):
    if case == "uniform_k8_d3":
        tree = v.tree_build_uniform(0.0, 0.0, 1.0, 8, 3)
        src = W.uniform_gauss3().sources[0]
    else:
        src = W.narrow_gaussians(5, n=3, sigma=0.04)
        tree = v.tree_build(0.0, 0.0, 1.0, 8, src, 1e-6, 7)
    ops = v.ops_create(8, 20)
    f = v.source_sample(tree, src)
    ref = v.volume_potential(tree, ops, f)
    g = torch.Generator(device="cpu").manual_seed(3)
    f2 = torch.randn(f.numel(), generator=g, dtype=torch.float64).cuda()
    ref2 = v.volume_potential(tree, ops, f2)
    for inp, want in ((f, ref), (f2, ref2)):  # two calls in a row with different inputs
        out = tuple(torch.full_like(inp, float("nan")) for _ in range(3))
        assert _noalloc(tree, ops, inp, out) == 0
        torch.cuda.synchronize()
        assert _status() == 0
        for q in range(3):
            assert torch.isfinite(out[q]).all()
            assert _rel(out[q], want[q]) < TOL


def test_noalloc_mixed_form_two_right_hand_sides_twice():
    """Mixed form, two right-hand sides per call on a tree never solved with two: the allocation-free
    entry point solves them one at a time with the schedules built with the tree."""
    src = W.narrow_gaussians(5, n=3, sigma=0.04)
    tree = v.tree_build(0.0, 0.0, 1.0, 8, src, 1e-6, 7)
    ops = v.ops_create(8, 20, v.MIXED)
    f1 = v.source_sample(tree, src)
    g = torch.Generator(device="cpu").manual_seed(5)
    f2 = torch.randn(f1.numel(), generator=g, dtype=torch.float64).cuda()
    f = torch.stack([f1, f2]).contiguous()
    want = [v.volume_potential(tree, ops, x) for x in (f1, f2)]
    for _ in range(2):  # two calls in a row
        out = tuple(torch.full_like(f, float("nan")) for _ in range(3))
        assert _noalloc(tree, ops, f, out) == 0
        torch.cuda.synchronize()
        assert _status() == 0
        for r in range(2):
            for q in range(3):
                assert torch.isfinite(out[q][r]).all()
                assert _rel(out[q][r], want[r][q]) < TOL_MIXED


def test_noalloc_call_allocates_no_device_memory():
    """The property the entry point exists for: once a first call has loaded the library's kernels
    and its static scratch, a call on a tree it has not seen before leaves the device's free
    memory unchanged (every input and output is allocated before the measurement)."""
    ops = v.ops_create(8, 20)
    src = W.uniform_gauss3().sources[0]
    t1 = v.tree_build_uniform(0.0, 0.0, 1.0, 8, 3)
    f1 = v.source_sample(t1, src)
    out1 = tuple(torch.empty_like(f1) for _ in range(3))
    assert _noalloc(t1, ops, f1, out1) == 0  # warm-up: module and scratch loaded
    t2 = v.tree_build_uniform(0.05, -0.05, 1.25, 8, 3)
    f2 = v.source_sample(t2, src)
    want = v.volume_potential(t2, ops, f2)
    out2 = tuple(torch.full_like(f2, float("nan")) for _ in range(3))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert _noalloc(t2, ops, f2, out2) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert _status() == 0
    for q in range(3):
        assert _rel(out2[q], want[q]) < TOL


def test_noalloc_rejects_trees_beyond_the_static_scratch():
    tree = v.tree_build_uniform(0.0, 0.0, 1.0, 16, 5)  # workspace far above 32 MiB at k = 16
    ops = v.ops_create(16, 40)
    assert v.workspace_size(tree, ops) > (32 << 20)
    f = torch.zeros(tree.n_leaves * 256, dtype=torch.float64, device="cuda")
    out = tuple(torch.empty_like(f) for _ in range(3))
    rc = _noalloc(tree, ops, f, out)
    assert rc == -6  # VFMM_ERR_WORKSPACE
    assert b"static scratch" in _lib.load().vfmm_last_error_detail()
