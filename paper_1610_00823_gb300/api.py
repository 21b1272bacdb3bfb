"""Torch-facing wrappers over the C ABI (names follow include/vfmm.h without the prefix)."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import c_double_p, c_int32_p, call

FP64 = 0
MIXED = 1
M2L_DENSE = 0  # vfmm_ops_set_m2l forms
M2L_PLANEWAVE = 1
LISTS = {"U": 0, "V": 1, "W": 2, "X": 3}
OP_IDS = {"near": 0, "s2m": 1, "s2l": 2, "m2m": 3, "l2l": 4, "m2l": 5}


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _source(src):
    """(kind, n, params) or an object with those attributes -> (ctypes Source, keep-alive array)."""
    kind, n, params = (src.kind, src.n, src.params) if hasattr(src, "kind") else src
    arr = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    s = _lib.Source(int(kind), int(n), arr.ctypes.data_as(c_double_p))
    return s, arr


class Tree:
    """Device-resident level-restricted quadtree with its interaction lists."""

    def __init__(self, handle, k):
        self._h = handle
        self.k = k
        info = _lib.TreeInfo()
        call("vfmm_tree_info", self._h, ctypes.byref(info))
        self.n_boxes = int(info.n_boxes)
        self.n_leaves = int(info.n_leaves)
        self.depth = int(info.depth)
        self.list_len = [int(v) for v in info.list_len]
        self.f_scale = float(info.f_scale)
        self.min_margin = float(info.min_margin)
        self.n_depth_capped = int(info.n_depth_capped)

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                _lib.load().vfmm_tree_destroy(h)
            except Exception:
                pass
            self._h = None

    def export_boxes(self):
        n = self.n_boxes
        out = [np.zeros(n, dtype=np.int32) for _ in range(3)]
        call("vfmm_tree_export_boxes", self._h, *[a.ctypes.data_as(c_int32_p) for a in out])
        return out

    def export_list(self, name):
        q = LISTS[name]
        ptr = np.zeros(self.n_boxes + 1, dtype=np.int32)
        idx = np.zeros(max(1, self.list_len[q]), dtype=np.int32)
        cfg = np.zeros(max(1, self.list_len[q]), dtype=np.int32)
        call("vfmm_tree_export_list", self._h, q, ptr.ctypes.data_as(c_int32_p), idx.ctypes.data_as(c_int32_p),
             cfg.ctypes.data_as(c_int32_p))
        n = self.list_len[q]
        return ptr, idx[:n], cfg[:n]

    def leaf_nodes(self, stream=None):
        n = self.n_leaves * self.k * self.k
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        call("vfmm_tree_leaf_nodes", self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
             _stream(stream))
        return x, y


REFINE_RULES = {"tail": 0, "interp": 1, "interp_area": 2, "interp_mixed": 3}


def tree_build(cx, cy, width, k, source, tol, max_depth, min_depth=0, stream=None, rule="tail") -> Tree:
    """Adaptive tree; rule: "tail" (vfmm_tree_build) or a Section 6.1 rule of vfmm_tree_build_rule."""
    prm = _lib.TreeParams(cx, cy, width, k, max_depth, min_depth, tol)
    s, keep = _source(source)
    h = ctypes.c_void_p()
    if rule == "tail":
        call("vfmm_tree_build", ctypes.byref(prm), ctypes.byref(s), _stream(stream), ctypes.byref(h))
    else:
        call("vfmm_tree_build_rule", ctypes.byref(prm), ctypes.byref(s), REFINE_RULES[rule], _stream(stream),
             ctypes.byref(h))
    del keep
    return Tree(h, k)


def tree_build_leaves(cx, cy, width, k, source, n_leaves, max_depth=16, stream=None) -> Tree:
    """Greedy refinement to at least n_leaves leaves (then balanced); see vfmm_tree_build_leaves."""
    prm = _lib.TreeParams(cx, cy, width, k, max_depth, 0, 0.0)
    s, keep = _source(source)
    h = ctypes.c_void_p()
    call("vfmm_tree_build_leaves", ctypes.byref(prm), ctypes.byref(s), int(n_leaves), _stream(stream), ctypes.byref(h))
    del keep
    return Tree(h, k)


def tree_build_many(specs, n_threads=0) -> list:
    """vfmm_tree_build_many. specs: dicts with cx, cy, width, k, source, max_depth and either
    n_leaves (a leaf-count tree, as tree_build_leaves) or tol (and optionally min_depth; as
    tree_build). The trees are built on up to n_threads host threads (0: one per core, at most 16)."""
    n = len(specs)
    prm = (_lib.TreeParams * max(1, n))()
    src = (_lib.Source * max(1, n))()
    nl = (ctypes.c_int64 * max(1, n))()
    keep = []
    for i, sp in enumerate(specs):
        n_leaves = int(sp.get("n_leaves") or 0)
        prm[i] = _lib.TreeParams(sp["cx"], sp["cy"], sp["width"], sp["k"], sp["max_depth"], sp.get("min_depth", 0),
                                 0.0 if n_leaves > 0 else float(sp["tol"]))
        s, arr = _source(sp["source"])
        src[i] = s
        keep.append(arr)
        nl[i] = n_leaves
    out = (ctypes.c_void_p * max(1, n))()
    call("vfmm_tree_build_many", prm, src, nl, n, int(n_threads), out)
    del keep
    return [Tree(ctypes.c_void_p(out[i]), specs[i]["k"]) for i in range(n)]


def tree_build_pull(cx, cy, width, k, f, tol, max_depth, min_depth=0, stream=None) -> Tree:
    """Adaptive tree for a caller-evaluated f (vfmm_tree_begin ... vfmm_tree_finish). f(x, y) takes
    cuda float64 tensors of node coordinates and returns f at them (same length); it is called once
    for the f-scale grid and once per tested level, on the current stream."""
    prm = _lib.TreeParams(cx, cy, width, k, max_depth, min_depth, tol)
    st = _stream(stream)
    b = ctypes.c_void_p()
    call("vfmm_tree_begin", ctypes.byref(prm), st, ctypes.byref(b))
    try:
        while True:
            n = ctypes.c_int64()
            call("vfmm_tree_pending", b, ctypes.byref(n))
            if n.value == 0:
                break
            x = torch.empty(n.value, dtype=torch.float64, device="cuda")
            y = torch.empty_like(x)
            call("vfmm_tree_pending_nodes", b, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()))
            fv = torch.as_tensor(f(x, y), dtype=torch.float64, device="cuda").reshape(-1).contiguous()
            if fv.numel() != n.value:
                raise ValueError("f returned %d values for %d nodes" % (fv.numel(), n.value))
            call("vfmm_tree_submit", b, ctypes.c_void_p(fv.data_ptr()))
        h = ctypes.c_void_p()
        call("vfmm_tree_finish", b, ctypes.byref(h))
    finally:
        _lib.load().vfmm_tree_builder_destroy(b)
    return Tree(h, k)


def leaf_interpolate(tree: Tree, fields, x, y, with_leaf=False, stream=None):
    """v~ (vfmm_leaf_interpolate): each field (cuda float64, n_leaves*k*k values, e.g. u, u_x, u_y)
    interpolated on its leaf at the points (x, y: cuda float64, same length). Returns the list of
    value tensors, and the int32 leaf index per point when with_leaf."""
    fields = [f.contiguous() for f in fields]
    n_f = len(fields)
    n = tree.n_leaves * tree.k * tree.k
    if not 1 <= n_f <= 8 or any(f.dtype != torch.float64 or not f.is_cuda or f.numel() != n for f in fields):
        raise ValueError("fields: 1..8 cuda float64 tensors of n_leaves*k*k values")
    x = x.contiguous()
    y = y.contiguous()
    out = [torch.empty_like(x) for _ in range(n_f)]
    leaf = torch.empty(x.numel(), dtype=torch.int32, device="cuda") if with_leaf else None
    fp = (ctypes.c_void_p * n_f)(*[f.data_ptr() for f in fields])
    op = (ctypes.c_void_p * n_f)(*[o.data_ptr() for o in out])
    call("vfmm_leaf_interpolate", tree.handle, n_f, fp, x.numel(), ctypes.c_void_p(x.data_ptr()),
         ctypes.c_void_p(y.data_ptr()), op, ctypes.c_void_p(leaf.data_ptr() if with_leaf else None), _stream(stream))
    return (out, leaf) if with_leaf else out


def tree_build_uniform(cx, cy, width, k, depth, stream=None) -> Tree:
    prm = _lib.TreeParams(cx, cy, width, k, depth, depth, 0.0)
    h = ctypes.c_void_p()
    call("vfmm_tree_build_uniform", ctypes.byref(prm), int(depth), _stream(stream), ctypes.byref(h))
    return Tree(h, k)


def source_sample(tree: Tree, source, stream=None):
    s, keep = _source(source)
    f = torch.empty(tree.n_leaves * tree.k * tree.k, dtype=torch.float64, device="cuda")
    call("vfmm_source_sample", tree.handle, ctypes.byref(s), ctypes.c_void_p(f.data_ptr()), _stream(stream))
    del keep
    return f


class Ops:
    """Device-resident unit-scale operators for (k, p, precision)."""

    def __init__(self, handle, k, p, precision):
        self._h = handle
        self.k, self.p, self.precision = k, p, precision

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                _lib.load().vfmm_ops_destroy(h)
            except Exception:
                pass
            self._h = None

    CONTRACTIONS = ("near", "s2m", "m2l", "s2l", "far")

    @property
    def slices(self):
        """Slices per split-BF16 contraction (VFMM_MIXED), {near, s2m, m2l, s2l, far} -> 6..8."""
        out = np.zeros(5, dtype=np.int32)
        call("vfmm_ops_get_slices", self._h, out.ctypes.data_as(c_int32_p))
        return dict(zip(self.CONTRACTIONS, out.tolist()))

    def set_slices(self, **counts):
        """vfmm_ops_set_slices: e.g. set_slices(near=7, m2l=6); unnamed contractions keep theirs."""
        cur = self.slices
        unknown = set(counts) - set(cur)
        if unknown:
            raise ValueError("unknown contractions %s" % sorted(unknown))
        cur.update(counts)
        arr = np.array([cur[c] for c in self.CONTRACTIONS], dtype=np.int32)
        call("vfmm_ops_set_slices", self._h, arr.ctypes.data_as(c_int32_p))

    @property
    def m2l(self):
        """(form, s): VFMM_M2L_DENSE or VFMM_M2L_PLANEWAVE and the plane-wave rule's length."""
        form, s = ctypes.c_int32(), ctypes.c_int32()
        call("vfmm_ops_get_m2l", self._h, ctypes.byref(form), ctypes.byref(s))
        return form.value, s.value

    def set_m2l(self, form):
        """vfmm_ops_set_m2l: M2L_DENSE or M2L_PLANEWAVE (FP64 operator sets only)."""
        call("vfmm_ops_set_m2l", self._h, int(form))

    def export(self, name):
        k, p = self.k, self.p
        kk, P = k * k, p + 1
        shapes = {"near": (33, 3, kk, kk), "s2m": (P, kk, 2), "s2l": (20, P, kk, 2), "m2m": (4, P, P, 2),
                  "l2l": (4, P, P, 2), "m2l": (40, P, P, 2)}
        shp = shapes[name]
        out = np.zeros(int(np.prod(shp)), dtype=np.float64)
        call("vfmm_ops_export", self._h, OP_IDS[name], out.ctypes.data_as(c_double_p), out.size)
        out = out.reshape(shp)
        if name != "near":
            out = out[..., 0] + 1j * out[..., 1]
        return out


def ops_create(k, p, precision=FP64, stream=None) -> Ops:
    h = ctypes.c_void_p()
    call("vfmm_ops_create", int(k), int(p), int(precision), _stream(stream), ctypes.byref(h))
    return Ops(h, k, p, precision)


def workspace_size(tree: Tree, ops: Ops, nrhs=1, with_io=False) -> int:
    b = ctypes.c_size_t()
    call("vfmm_workspace_size", tree.handle, ops.handle, int(nrhs), int(bool(with_io)), ctypes.byref(b))
    return int(b.value)


def workspace(tree: Tree, ops: Ops, nrhs=1, with_io=False):
    return torch.empty(workspace_size(tree, ops, nrhs, with_io), dtype=torch.uint8, device="cuda")


def volume_potential(tree: Tree, ops: Ops, f, out=None, ws=None, stream=None):
    """u, u_x, u_y at every leaf node. f: cuda float64 [n_leaves*k*k] or [nrhs, n_leaves*k*k]."""
    n = tree.n_leaves * tree.k * tree.k
    f = f.contiguous()
    if f.dtype != torch.float64 or not f.is_cuda or f.numel() % n:
        raise ValueError("f must be a cuda float64 tensor with a multiple of n_leaves*k*k elements")
    nrhs = f.numel() // n
    if out is None:
        out = tuple(torch.empty_like(f) for _ in range(3))
    if ws is None:
        ws = workspace(tree, ops, nrhs)
    call("vfmm_volume_potential", tree.handle, ops.handle, ctypes.c_void_p(f.data_ptr()), nrhs,
         ctypes.c_void_p(out[0].data_ptr()), ctypes.c_void_p(out[1].data_ptr()), ctypes.c_void_p(out[2].data_ptr()),
         ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream))
    return out


def volume_potential_host(tree: Tree, ops: Ops, f_host, out_host=None, ws=None, stream=None):
    """Same from host tensors (pinned for full speed); returns host tensors; synchronises."""
    n = tree.n_leaves * tree.k * tree.k
    f_host = f_host.contiguous()
    if f_host.dtype != torch.float64 or f_host.is_cuda or f_host.numel() % n:
        raise ValueError("f_host must be a host float64 tensor with a multiple of n_leaves*k*k elements")
    nrhs = f_host.numel() // n
    if out_host is None:
        out_host = tuple(torch.empty_like(f_host) for _ in range(3))
    if ws is None:
        ws = workspace(tree, ops, nrhs, with_io=True)
    call("vfmm_volume_potential_host", tree.handle, ops.handle, ctypes.c_void_p(f_host.data_ptr()), nrhs,
         ctypes.c_void_p(out_host[0].data_ptr()), ctypes.c_void_p(out_host[1].data_ptr()),
         ctypes.c_void_p(out_host[2].data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream))
    return out_host


def evaluate_points(tree: Tree, ops: Ops, f, ws, x, y, stream=None):
    """V f~ and its gradient at arbitrary points from the expansions a one-right-hand-side
    volume_potential call with workspace ws and leaf values f left there (vfmm_evaluate_points).
    x, y: cuda float64 tensors of the same length; returns (u, u_x, u_y)."""
    x = x.contiguous()
    y = y.contiguous()
    if x.dtype != torch.float64 or y.dtype != torch.float64 or not x.is_cuda or x.numel() != y.numel():
        raise ValueError("x, y: cuda float64 tensors of equal length")
    out = tuple(torch.empty_like(x) for _ in range(3))
    call("vfmm_evaluate_points", tree.handle, ops.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
         ws.numel(), x.numel(), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
         ctypes.c_void_p(out[0].data_ptr()), ctypes.c_void_p(out[1].data_ptr()), ctypes.c_void_p(out[2].data_ptr()),
         _stream(stream))
    return out


def workspace_status(ws=None):
    """Status of the last solve that used workspace ws (vfmm_workspace_status): raises VfmmError
    (VFMM_ERR_TIMEOUT) when a bounded device wait of that solve ran out. Call it after synchronising
    the solve's stream. ws = None reads the allocation-free entry point's static scratch."""
    call("vfmm_workspace_status", ctypes.c_void_p(ws.data_ptr() if ws is not None else None))


STAGES = ("s2m", "m2m", "down", "near", "l2t", "leaf", "near_tc", "s2m_tc", "m2l_tc", "s2l_tc", "far_tc")


def volume_potential_profiled(tree: Tree, ops: Ops, f, out, ws, stream=None):
    """volume_potential with per-stage CUDA-event times; returns (stage_ms dict, kernel launches)."""
    n = tree.n_leaves * tree.k * tree.k
    nrhs = f.numel() // n
    ms = (ctypes.c_float * len(STAGES))()
    launches = ctypes.c_int32()
    call("vfmm_volume_potential_profiled", tree.handle, ops.handle, ctypes.c_void_p(f.data_ptr()), nrhs,
         ctypes.c_void_p(out[0].data_ptr()), ctypes.c_void_p(out[1].data_ptr()), ctypes.c_void_p(out[2].data_ptr()),
         ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream), ms, ctypes.byref(launches))
    return dict(zip(STAGES, [float(x) for x in ms])), int(launches.value)


def volume_potential_noalloc(tree: Tree, ops: Ops, f, out=None, stream=None):
    """volume_potential without any allocation by the library (fixed 32 MiB static scratch).

    For callers that cannot allocate device memory (their pool allocator owns it all).
    Rejects trees whose workspace exceeds the static scratch; calls on overlapping
    streams race on the shared scratch. The first call on a device should precede
    any stream capture (it looks up the scratch's device address).
    """
    n = tree.n_leaves * tree.k * tree.k
    f = f.contiguous()
    if f.dtype != torch.float64 or not f.is_cuda or f.numel() % n:
        raise ValueError("f must be a cuda float64 tensor with a multiple of n_leaves*k*k elements")
    nrhs = f.numel() // n
    if out is None:
        out = tuple(torch.empty_like(f) for _ in range(3))
    call("vfmm_volume_potential_noalloc", tree.handle, ops.handle, ctypes.c_void_p(f.data_ptr()), nrhs,
         ctypes.c_void_p(out[0].data_ptr()), ctypes.c_void_p(out[1].data_ptr()), ctypes.c_void_p(out[2].data_ptr()),
         _stream(stream))
    return out


def tune(tree: Tree, ops: Ops, f, out, ws, stream=None):
    """Split-K autotuner (vfmm_tune): returns the chosen factors {near, m2l, s2l, far}; out holds the solution."""
    n = tree.n_leaves * tree.k * tree.k
    splits = np.zeros(4, dtype=np.int32)
    call("vfmm_tune", tree.handle, ops.handle, ctypes.c_void_p(f.data_ptr()), f.numel() // n,
         ctypes.c_void_p(out[0].data_ptr()), ctypes.c_void_p(out[1].data_ptr()), ctypes.c_void_p(out[2].data_ptr()),
         ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream), splits.ctypes.data_as(c_int32_p))
    return dict(zip(("near", "m2l", "s2l", "far"), splits.tolist()))


WORK = ("near_tc_flops", "m2l_tc_flops", "far_tc_flops", "s2l_tc_flops", "s2m_tc_flops", "near_fp64eq_flops",
        "u_entries", "entry_major_mask", "near_ctas", "pass_ctas")


def schedule(tree: Tree, nrhs: int = 1):
    """vfmm_schedule_get: (near-field CTA cap, tree-pass grid cap) of the mixed solve's schedule."""
    a, b = ctypes.c_int32(), ctypes.c_int32()
    call("vfmm_schedule_get", tree.handle, int(nrhs), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def set_schedule(tree: Tree, near_ctas: int, pass_ctas: int, nrhs: int = 1):
    """vfmm_schedule_set: override the tuner's co-schedule (0 = uncapped)."""
    call("vfmm_schedule_set", tree.handle, int(nrhs), int(near_ctas), int(pass_ctas))


def solve_work(tree: Tree, ops: Ops, nrhs: int = 1):
    """Work counts of one call with nrhs right-hand sides (host-side accounting for roofline reports)."""
    out = np.zeros(len(WORK), dtype=np.float64)
    call("vfmm_solve_work", tree.handle, ops.handle, int(nrhs), out.ctypes.data_as(c_double_p))
    return dict(zip(WORK, out.tolist()))


class SolveGraph:
    """Captured solve (CUDA graph) for repeated calls with the same f/u buffers and workspace."""

    def __init__(self, tree: Tree, ops: Ops, f, out, ws, stream):
        n = tree.n_leaves * tree.k * tree.k
        self._keep = (tree, ops, f, out, ws)
        self._h = ctypes.c_void_p()
        call("vfmm_graph_create", tree.handle, ops.handle, ctypes.c_void_p(f.data_ptr()), f.numel() // n,
             ctypes.c_void_p(out[0].data_ptr()), ctypes.c_void_p(out[1].data_ptr()),
             ctypes.c_void_p(out[2].data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream),
             ctypes.byref(self._h))

    def launch(self, stream=None):
        call("vfmm_graph_launch", self._h, _stream(stream))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                _lib.load().vfmm_graph_destroy(h)
            except Exception:
                pass
            self._h = None


class Batch:
    """Many independent solves per call (vfmm_batch_*): items are (tree, ops, f, out, ws) tuples with
    f and out[q] cuda float64 tensors laid out as for volume_potential and ws from workspace()."""

    def __init__(self, n_streams: int = 16):
        self._h = ctypes.c_void_p()
        call("vfmm_batch_create", int(n_streams), ctypes.byref(self._h))

    @staticmethod
    def _items(items):
        arr = (_lib.BatchItem * len(items))()
        for i, (tree, ops, f, out, ws) in enumerate(items):
            n = tree.n_leaves * tree.k * tree.k
            if f.numel() % n or any(o.numel() != f.numel() for o in out):
                raise ValueError("item %d: f/out sizes do not match the tree" % i)
            arr[i] = _lib.BatchItem(tree.handle.value if hasattr(tree.handle, "value") else tree.handle,
                                    ops.handle.value if hasattr(ops.handle, "value") else ops.handle,
                                    f.numel() // n, f.data_ptr(), out[0].data_ptr(), out[1].data_ptr(),
                                    out[2].data_ptr(), ws.data_ptr(), ws.numel())
        return arr

    def potential(self, items, stream=None):
        arr = self._items(items)
        call("vfmm_batch_potential", self._h, len(items), arr, _stream(stream))

    def graph(self, items, stream):
        """The whole batch captured as one CUDA graph (a Graph; keeps the items alive)."""
        arr = self._items(items)
        h = ctypes.c_void_p()
        call("vfmm_batch_graph_create", self._h, len(items), arr, _stream(stream), ctypes.byref(h))
        return Graph(h, keep=(self, items))

    def tune(self, items, stream):
        """Picks the number of side streams by timing graph replays; returns (streams, ms)."""
        arr = self._items(items)
        s = ctypes.c_int32()
        ms = ctypes.c_float()
        call("vfmm_batch_tune", self._h, len(items), arr, _stream(stream), ctypes.byref(s), ctypes.byref(ms))
        return int(s.value), float(ms.value)

    @property
    def streams(self) -> int:
        s = ctypes.c_int32()
        call("vfmm_batch_streams", self._h, ctypes.byref(s))
        return int(s.value)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                _lib.load().vfmm_batch_destroy(h)
            except Exception:
                pass
            self._h = None


class Graph:
    """An instantiated CUDA graph returned by the library (replay with launch)."""

    def __init__(self, handle, keep=None):
        self._h = handle
        self._keep = keep

    def launch(self, stream=None):
        call("vfmm_graph_launch", self._h, _stream(stream))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                _lib.load().vfmm_graph_destroy(h)
            except Exception:
                pass
            self._h = None
