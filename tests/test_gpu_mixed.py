"""Split-BF16 tensor-core near field (VFMM_MIXED) against the FP64 form and the oracle.

Bar: 1e-10 relative L-infinity for u, u_x, u_y (the method's accuracy target for the
mixed form); the slicing analysis predicts a few 1e-13.
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
from paper_1610_00823_gb300.api import volume_potential_profiled, workspace  # noqa: E402

TOL = 1e-10

CASES = [
    ("uniform_k8", None, 8, 20, 0.0, 3),
    ("narrow_k16", lambda: W.narrow_gaussians(8, n=2, sigma=0.01, spread=0.4), 16, 40, 1e-10, 9),
    ("kinked_k8", lambda: W.kinked(k=8).sources[0], 8, 20, 1e-4, 6),
]


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("name,mk,k,p,tol,depth", CASES)
def test_mixed_matches_fp64_and_oracle(name, mk, k, p, tol, depth, oracle_ops):
    width = 2.0 if name.startswith("kinked") else 1.0
    if mk is None:
        src = W.uniform_gauss3().sources[0]
        gt = v.tree_build_uniform(0.0, 0.0, width, k, depth)
        ot = T.build_uniform(0.0, 0.0, width, k, depth)
    else:
        src = mk()
        gt = v.tree_build(0.0, 0.0, width, k, src, tol, depth)
        ot = T.build_adaptive(0.0, 0.0, width, k, src, tol, depth)
    F = ot.sample(src)
    f = torch.from_numpy(F.reshape(-1)).cuda()
    ops64 = v.ops_create(k, p, v.FP64)
    opsmx = v.ops_create(k, p, v.MIXED)
    u64 = v.volume_potential(gt, ops64, f)
    out = tuple(torch.empty_like(f) for _ in range(3))
    ws = workspace(gt, opsmx, 1)
    stages, launches = volume_potential_profiled(gt, opsmx, f, out, ws)  # raises on a device timeout
    ref = fmm.solve(ot, T.build_lists(ot), oracle_ops(k, p), F)
    for q in range(3):
        got = out[q].cpu().numpy().reshape(ref[q].shape)
        assert rel(got, u64[q].cpu().numpy().reshape(ref[q].shape)) < TOL, (name, q)
        assert rel(got, ref[q]) < TOL, (name, q, rel(got, ref[q]))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_equals_direct_call(precision):
    from paper_1610_00823_gb300.api import SolveGraph
    src = W.narrow_gaussians(5, n=3, sigma=0.04)
    gt = v.tree_build(0.0, 0.0, 1.0, 8, src, 1e-6, 7)
    ops = v.ops_create(8, 20, v.MIXED if precision == "mixed" else v.FP64)
    f = v.source_sample(gt, src)
    ref = v.volume_potential(gt, ops, f)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    out = tuple(torch.full_like(f, float("nan")) for _ in range(3))
    ws = workspace(gt, ops, 1)
    g = SolveGraph(gt, ops, f, out, ws, stream)
    for _ in range(2):
        for q in range(3):
            out[q].fill_(float("nan"))
        torch.cuda.synchronize()
        g.launch(stream)
        stream.synchronize()
        for q in range(3):
            assert torch.equal(out[q], ref[q])


def _stack_sources(gt, sources):
    return torch.stack([v.source_sample(gt, s) for s in sources]).contiguous()


def test_folded_rhs_shared_tree(oracle_ops):
    """64 right-hand sides on the uniform depth-3, k = 8 tree (the shared-tree batch): the mixed form
    folds them into one solve; every right-hand side against the FP64 form (all targets) and four of
    them against the oracle."""
    srcs = W.shared_tree_rhs(64)
    gt = v.tree_build_uniform(0.0, 0.0, 1.0, 8, 3)
    ot = T.build_uniform(0.0, 0.0, 1.0, 8, 3)
    f = _stack_sources(gt, srcs)
    ops64 = v.ops_create(8, 20, v.FP64)
    opsmx = v.ops_create(8, 20, v.MIXED)
    u64 = [x.cpu().numpy() for x in v.volume_potential(gt, ops64, f)]
    umx = [x.cpu().numpy() for x in v.volume_potential(gt, opsmx, f)]
    for r in range(len(srcs)):
        for q in range(3):
            assert rel(umx[q][r], u64[q][r]) < TOL, (r, q)
    L = T.build_lists(ot)
    for r in (0, 17, 40, 63):
        ref = fmm.solve(ot, L, oracle_ops(8, 20), ot.sample(srcs[r]))
        for q in range(3):
            assert rel(umx[q][r].reshape(ref[q].shape), ref[q]) < TOL, (r, q)


def test_folded_rhs_adaptive_tree_and_graph():
    """Three right-hand sides on a deep adaptive k = 16 tree: folded mixed solve against the FP64
    form, a zero right-hand side stays exactly zero, and graph replay equals the direct call."""
    from paper_1610_00823_gb300.api import SolveGraph
    src = W.narrow_gaussians(8, n=2, sigma=0.01, spread=0.4)
    gt = v.tree_build(0.0, 0.0, 1.0, 16, src, 1e-10, 9)
    f1 = v.source_sample(gt, src)
    f2 = v.source_sample(gt, W.narrow_gaussians(9, n=3, sigma=0.03, spread=0.3))
    f = torch.stack([f1, 1e-6 * f2, torch.zeros_like(f1)]).contiguous()
    ops64 = v.ops_create(16, 40, v.FP64)
    opsmx = v.ops_create(16, 40, v.MIXED)
    u64 = v.volume_potential(gt, ops64, f)
    umx = v.volume_potential(gt, opsmx, f)
    for r in range(2):
        for q in range(3):
            assert rel(umx[q][r].cpu().numpy(), u64[q][r].cpu().numpy()) < TOL, (r, q)
    for q in range(3):
        assert torch.count_nonzero(umx[q][2]).item() == 0
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    out = tuple(torch.full_like(f, float("nan")) for _ in range(3))
    ws = workspace(gt, opsmx, 3)
    g = SolveGraph(gt, opsmx, f, out, ws, stream)
    for q in range(3):
        out[q].fill_(float("nan"))
    torch.cuda.synchronize()
    g.launch(stream)
    stream.synchronize()
    for q in range(3):
        assert torch.equal(out[q], umx[q])


@pytest.mark.parametrize("k,p,depth,tol", [(8, 20, 7, 1e-6), (16, 40, 9, 1e-10)])
def test_forked_solve_equals_single_stream_solve(k, p, depth, tol):
    """The mixed solve runs its near-field and S2L contractions on a second stream (joined back by
    events); the same kernels on one stream (the profiled call) give bit-identical results, also
    under graph capture and with two host threads solving at once (one second stream per thread)."""
    import threading
    from paper_1610_00823_gb300.api import SolveGraph
    src = W.narrow_gaussians(8, n=2, sigma=0.01, spread=0.4)
    gt = v.tree_build(0.0, 0.0, 1.0, k, src, tol, depth)
    f = v.source_sample(gt, src)
    ops = v.ops_create(k, p, v.MIXED)
    ws = workspace(gt, ops, 1)
    ref = tuple(torch.full_like(f, float("nan")) for _ in range(3))
    volume_potential_profiled(gt, ops, f, ref, ws)
    torch.cuda.synchronize()
    got = v.volume_potential(gt, ops, f)
    torch.cuda.synchronize()
    for q in range(3):
        assert torch.equal(got[q], ref[q]), q
    stream = torch.cuda.Stream()
    out = tuple(torch.full_like(f, float("nan")) for _ in range(3))
    g = SolveGraph(gt, ops, f, out, workspace(gt, ops, 1), stream)
    for q in range(3):
        out[q].fill_(float("nan"))
    torch.cuda.synchronize()
    g.launch(stream)
    stream.synchronize()
    for q in range(3):
        assert torch.equal(out[q], ref[q]), q
    results, errors = [None, None], []

    def worker(i):
        try:
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                o = tuple(torch.full_like(f, float("nan")) for _ in range(3))
                w = workspace(gt, ops, 1)
                st.synchronize()
                for _ in range(3):
                    v.volume_potential(gt, ops, f, o, w, stream=st)
                st.synchronize()
                results[i] = o
        except Exception as e:  # noqa: BLE001
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for o in results:
        for q in range(3):
            assert torch.equal(o[q], ref[q]), q


def test_autotuned_schedule_keeps_results():
    """vfmm_tune picks split-K factors by timing; the solution it leaves and later solves with the
    tuned schedule stay within the bar of the FP64 form."""
    from paper_1610_00823_gb300.api import tune
    src = W.narrow_gaussians(8, n=2, sigma=0.01, spread=0.4)
    gt = v.tree_build(0.0, 0.0, 1.0, 16, src, 1e-10, 9)
    f = v.source_sample(gt, src)
    u64 = v.volume_potential(gt, v.ops_create(16, 40, v.FP64), f)
    ops = v.ops_create(16, 40, v.MIXED)
    out = tuple(torch.empty_like(f) for _ in range(3))
    ws = workspace(gt, ops, 1)
    stream = torch.cuda.Stream()
    splits = tune(gt, ops, f, out, ws, stream)
    assert set(splits) == {"near", "m2l", "s2l", "far"} and all(s in (1, 2, 4, 8, 16) for s in splits.values())
    again = v.volume_potential(gt, ops, f, ws=ws, stream=stream)
    stream.synchronize()
    for q in range(3):
        assert rel(out[q].cpu().numpy(), u64[q].cpu().numpy()) < TOL
        assert rel(again[q].cpu().numpy(), u64[q].cpu().numpy()) < TOL


def test_co_schedule_caps_keep_results_bit_identical():
    """The near-field CTA cap and the tree-pass grid cap (vfmm_schedule_set, chosen by vfmm_tune's
    whole-step timing) only change which CTA takes which work item: forked solves under any caps,
    captured or not, equal the uncapped one-stream solve bit for bit."""
    from paper_1610_00823_gb300.api import SolveGraph, schedule, set_schedule
    src = W.narrow_gaussians(8, n=2, sigma=0.01, spread=0.4)
    gt = v.tree_build(0.0, 0.0, 1.0, 16, src, 1e-10, 9)
    f = v.source_sample(gt, src)
    ops = v.ops_create(16, 40, v.MIXED)
    ws = workspace(gt, ops, 1)
    set_schedule(gt, 0, 0)
    assert schedule(gt) == (0, 0)
    ref = tuple(torch.full_like(f, float("nan")) for _ in range(3))
    volume_potential_profiled(gt, ops, f, ref, ws)
    torch.cuda.synchronize()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for near, passes in [(sms, 0), (sms * 5 // 8, sms * 3 // 8), (sms // 2, 7), (1, 1)]:
        set_schedule(gt, near, passes)
        assert schedule(gt) == (near, passes)
        got = v.volume_potential(gt, ops, f)
        stream = torch.cuda.Stream()
        out = tuple(torch.full_like(f, float("nan")) for _ in range(3))
        g = SolveGraph(gt, ops, f, out, workspace(gt, ops, 1), stream)
        g.launch(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        for q in range(3):
            assert torch.equal(got[q], ref[q]), (near, passes, q)
            assert torch.equal(out[q], ref[q]), (near, passes, q)
    with pytest.raises(RuntimeError):
        set_schedule(gt, -1, 0)


def test_bounded_wait_reports_timeout_and_context_survives():
    """The failure path of the tensor-core kernels: a bounded wait that runs out (an mbarrier that
    nothing arrives on) is reported as VFMM_ERR_TIMEOUT, and the GPU context stays usable."""
    import ctypes
    import time
    from paper_1610_00823_gb300 import _lib
    lib = _lib.load()
    t0 = time.time()
    rc = lib.vfmm_selftest_wait_timeout(ctypes.c_int64(4096), ctypes.c_void_p(0))
    assert rc == -5  # VFMM_ERR_TIMEOUT
    assert b"bounded wait ran out" in lib.vfmm_last_error_detail()
    assert time.time() - t0 < 60.0
    # a solve afterwards still works and still matches the FP64 form
    src = W.narrow_gaussians(5, n=3, sigma=0.04)
    gt = v.tree_build(0.0, 0.0, 1.0, 8, src, 1e-6, 7)
    f = v.source_sample(gt, src)
    ref = v.volume_potential(gt, v.ops_create(8, 20, v.FP64), f)
    got = v.volume_potential(gt, v.ops_create(8, 20, v.MIXED), f)
    for q in range(3):
        assert rel(got[q].cpu().numpy(), ref[q].cpu().numpy()) < TOL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_workspace_status_reports_a_recorded_timeout(precision):
    """The asynchronous solve records a bounded wait that ran out in the status word at the start of
    its workspace; vfmm_workspace_status reads it after synchronisation. No wait is made to run out
    here: the word is written from the host side (as a kernel would), read back as TIMEOUT, and the
    next solve clears it again."""
    from paper_1610_00823_gb300._lib import VfmmError
    src = W.narrow_gaussians(5, n=3, sigma=0.04)
    gt = v.tree_build(0.0, 0.0, 1.0, 8, src, 1e-6, 7)
    f = v.source_sample(gt, src)
    ops = v.ops_create(8, 20, v.MIXED if precision == "mixed" else v.FP64)
    ws = workspace(gt, ops, 1)
    v.volume_potential(gt, ops, f, ws=ws)
    torch.cuda.synchronize()
    v.workspace_status(ws)  # a normal solve: no timeout recorded
    ws[:4].view(torch.int32).fill_(6)  # what a persistent tree pass records when a wait runs out
    torch.cuda.synchronize()
    with pytest.raises(VfmmError) as e:
        v.workspace_status(ws)
    assert e.value.code == -5 and "persistent tree pass" in str(e.value)
    v.volume_potential(gt, ops, f, ws=ws)  # every call clears the word
    torch.cuda.synchronize()
    v.workspace_status(ws)


def test_slice_counts_trade_accuracy_for_products():
    """vfmm_ops_set_slices: defaults, validation, and the error bound of each setting on a small
    adaptive k = 16 tree (fewer slices: the rounding at 2^(-7S - 1) of each operand's scale)."""
    from paper_1610_00823_gb300._lib import VfmmError
    from paper_1610_00823_gb300.api import solve_work
    src = W.narrow_gaussians(8, n=2, sigma=0.01, spread=0.4)
    gt = v.tree_build(0.0, 0.0, 1.0, 16, src, 1e-10, 9)
    f = v.source_sample(gt, src)
    u64 = v.volume_potential(gt, v.ops_create(16, 40, v.FP64), f)
    ops = v.ops_create(16, 40, v.MIXED)
    assert ops.slices == {"near": 6, "s2m": 6, "m2l": 6, "s2l": 6, "far": 6}
    for bad in (5, 9):
        with pytest.raises(VfmmError):
            ops.set_slices(near=bad)
    assert ops.slices["near"] == 6
    with pytest.raises(VfmmError):
        v.ops_create(16, 40, v.FP64).set_slices(near=7)
    base = solve_work(gt, ops)["near_tc_flops"]
    errs = {}
    for S in (8, 7, 6):
        ops.set_slices(**{c: S for c in ops.CONTRACTIONS})
        u = v.volume_potential(gt, ops, f)
        errs[S] = max(rel(u[q].cpu().numpy(), u64[q].cpu().numpy()) for q in range(3))
        assert solve_work(gt, ops)["near_tc_flops"] == base * (S * (S + 1) // 2) / 21
    # balanced base-128 digits: 6 (the default) hold the bar with a 5x margin; more digits, less error
    assert errs[6] < TOL / 5 and errs[7] < errs[6] and errs[8] < 1e-12, errs
