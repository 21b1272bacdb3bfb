"""Batch driver (many independent problems per call, one CUDA graph): every member's result
equals its own single call bit for bit (same kernels, same inputs, only the stream differs),
for both forms, mixed k, and a member with several right-hand sides."""
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1610_00823_gb300 as v  # noqa: E402
from paper_1610_00823_gb300.api import Batch, workspace  # noqa: E402


def _members(precision):
    mem = W.batch_members(10)
    ops = {k: v.ops_create(k, 20 if k == 8 else 40, precision) for k in (8, 16)}
    items, refs = [], []
    for i, m in enumerate(mem):
        k = m["k"]
        tol = (1e-6, 1e-9, 1e-12)[i % 3]
        tree = v.tree_build(0.0, 0.0, 1.0, k, m["source"], tol, 16)
        f = v.source_sample(tree, m["source"])
        if i == 3:  # two right-hand sides on one member
            f = torch.stack([f, 0.5 * f * f]).contiguous()
        ref = v.volume_potential(tree, ops[k], f)
        out = tuple(torch.full_like(f, float("nan")) for _ in range(3))
        items.append((tree, ops[k], f, out, workspace(tree, ops[k], f.numel() // (tree.n_leaves * k * k))))
        refs.append(ref)
    return items, refs


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_graph_equals_single_calls(precision):
    items, refs = _members(v.MIXED if precision == "mixed" else v.FP64)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    b = Batch(8)
    b.potential(items, stream)
    stream.synchronize()
    for (tree, ops, f, out, ws), ref in zip(items, refs):
        for q in range(3):
            assert torch.equal(out[q], ref[q])
    g = b.graph(items, stream)
    for _ in range(2):
        for it in items:
            for o in it[3]:
                o.fill_(float("nan"))
        torch.cuda.synchronize()
        g.launch(stream)
        stream.synchronize()
        for (tree, ops, f, out, ws), ref in zip(items, refs):
            for q in range(3):
                assert torch.equal(out[q], ref[q])


def test_batch_tune_picks_a_stream_count():
    items, refs = _members(v.MIXED)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    b = Batch(8)
    s, ms = b.tune(items, stream)
    assert s in (1, 2, 4, 8) and ms > 0.0 and b.streams == s
    for it in items:
        for o in it[3]:
            o.fill_(float("nan"))
    b.potential(items, stream)
    stream.synchronize()
    for (tree, ops, f, out, ws), ref in zip(items, refs):
        for q in range(3):
            assert torch.equal(out[q], ref[q])


def _rel(a, b):
    import numpy as np
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("mixed", 1e-10)])
def test_leaf_count_members_in_a_batch_match_the_oracle(precision, tol, oracle_ops):
    """Members of the uneven batch of leaf-count trees (member 224: k = 8, 103 leaves targeted;
    member 44: k = 16, 103 leaves targeted), solved together in one batch graph, against the
    oracle's solve on the oracle's own greedy tree, element by element."""
    from oracle import fmm
    from oracle import tree as T
    mem = W.batch_members(256)
    prec = v.MIXED if precision == "mixed" else v.FP64
    items, oracle_cases = [], []
    for i in (224, 44):
        m = mem[i]
        k, p, src = m["k"], m["p"], m["source"]
        tree = v.tree_build_leaves(0.0, 0.0, 1.0, k, src, m["n_leaves_target"], 16)
        ot = T.build_greedy(0.0, 0.0, 1.0, k, src, m["n_leaves_target"], 16)
        assert tree.n_leaves == ot.n_leaves
        F = ot.sample(src)
        f = torch.from_numpy(F.reshape(-1)).cuda()
        ops = v.ops_create(k, p, prec)
        out = tuple(torch.full_like(f, float("nan")) for _ in range(3))
        items.append((tree, ops, f, out, workspace(tree, ops, 1)))
        oracle_cases.append((ot, oracle_ops(k, p), F))
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    g = Batch(4).graph(items, stream)
    g.launch(stream)
    stream.synchronize()
    for (tree, ops, f, out, ws), (ot, oops, F) in zip(items, oracle_cases):
        ref = fmm.solve(ot, T.build_lists(ot), oops, F)
        for q in range(3):
            got = out[q].cpu().numpy().reshape(ref[q].shape)
            assert _rel(got, ref[q]) < tol, (precision, tree.k, q, _rel(got, ref[q]))


def test_tree_build_many_equals_single_builds():
    """vfmm_tree_build_many on 4 host threads: every tree (leaf-count and tolerance trees, k = 8 and
    16) has the boxes and the four lists of its own single build, entry for entry."""
    mem = W.batch_members(12)
    specs = []
    for i, m in enumerate(mem):
        sp = dict(cx=0.0, cy=0.0, width=1.0, k=m["k"], source=m["source"], max_depth=16)
        if i % 2:
            sp["n_leaves"] = 40 + 97 * i
        else:
            sp["tol"] = (1e-6, 1e-9, 1e-12)[i % 3]
        specs.append(sp)
    many = v.tree_build_many(specs, n_threads=4)
    for sp, t in zip(specs, many):
        if "n_leaves" in sp:
            ref = v.tree_build_leaves(sp["cx"], sp["cy"], sp["width"], sp["k"], sp["source"], sp["n_leaves"], 16)
        else:
            ref = v.tree_build(sp["cx"], sp["cy"], sp["width"], sp["k"], sp["source"], sp["tol"], 16)
        assert (t.n_boxes, t.n_leaves, t.depth, t.list_len) == (ref.n_boxes, ref.n_leaves, ref.depth, ref.list_len)
        for a, b in zip(t.export_boxes(), ref.export_boxes()):
            assert (a == b).all()
        for name in ("U", "V", "W", "X"):
            for a, b in zip(t.export_list(name), ref.export_list(name)):
                assert (a == b).all()
    assert v.tree_build_many([], n_threads=2) == []
