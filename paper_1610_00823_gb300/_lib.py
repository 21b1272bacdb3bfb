"""ctypes declarations of the C ABI in include/vfmm.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvfmm.so")

c_double_p = ctypes.POINTER(ctypes.c_double)
c_int32_p = ctypes.POINTER(ctypes.c_int32)


class TreeParams(ctypes.Structure):
    _fields_ = [("cx", ctypes.c_double), ("cy", ctypes.c_double), ("width", ctypes.c_double),
                ("k", ctypes.c_int32), ("max_depth", ctypes.c_int32), ("min_depth", ctypes.c_int32),
                ("tol", ctypes.c_double)]


class Source(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n", ctypes.c_int32), ("params", c_double_p)]


class TreeInfo(ctypes.Structure):
    _fields_ = [("n_boxes", ctypes.c_int64), ("n_leaves", ctypes.c_int64), ("depth", ctypes.c_int32),
                ("k", ctypes.c_int32), ("list_len", ctypes.c_int64 * 4), ("f_scale", ctypes.c_double),
                ("min_margin", ctypes.c_double), ("n_depth_capped", ctypes.c_int64)]


class BatchItem(ctypes.Structure):
    _fields_ = [("tree", ctypes.c_void_p), ("ops", ctypes.c_void_p), ("nrhs", ctypes.c_int32),
                ("f", ctypes.c_void_p), ("u", ctypes.c_void_p), ("ux", ctypes.c_void_p), ("uy", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t)]


EXPORTS = {
    "vfmm_tree_build": [ctypes.POINTER(TreeParams), ctypes.POINTER(Source), ctypes.c_void_p,
                        ctypes.POINTER(ctypes.c_void_p)],
    "vfmm_tree_build_leaves": [ctypes.POINTER(TreeParams), ctypes.POINTER(Source), ctypes.c_int64, ctypes.c_void_p,
                               ctypes.POINTER(ctypes.c_void_p)],
    "vfmm_tree_build_uniform": [ctypes.POINTER(TreeParams), ctypes.c_int32, ctypes.c_void_p,
                                ctypes.POINTER(ctypes.c_void_p)],
    "vfmm_tree_build_many": [ctypes.POINTER(TreeParams), ctypes.POINTER(Source), ctypes.POINTER(ctypes.c_int64),
                             ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)],
    "vfmm_tree_build_rule": [ctypes.POINTER(TreeParams), ctypes.POINTER(Source), ctypes.c_int32, ctypes.c_void_p,
                             ctypes.POINTER(ctypes.c_void_p)],
    "vfmm_tree_begin": [ctypes.POINTER(TreeParams), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)],
    "vfmm_tree_pending": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)],
    "vfmm_tree_pending_nodes": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "vfmm_tree_submit": [ctypes.c_void_p, ctypes.c_void_p],
    "vfmm_tree_finish": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)],
    "vfmm_tree_builder_destroy": [ctypes.c_void_p],
    "vfmm_leaf_interpolate": [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p,
                              ctypes.c_void_p],
    "vfmm_tree_info": [ctypes.c_void_p, ctypes.POINTER(TreeInfo)],
    "vfmm_tree_export_boxes": [ctypes.c_void_p, c_int32_p, c_int32_p, c_int32_p],
    "vfmm_tree_export_list": [ctypes.c_void_p, ctypes.c_int32, c_int32_p, c_int32_p, c_int32_p],
    "vfmm_tree_leaf_nodes": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "vfmm_source_sample": [ctypes.c_void_p, ctypes.POINTER(Source), ctypes.c_void_p, ctypes.c_void_p],
    "vfmm_tree_destroy": [ctypes.c_void_p],
    "vfmm_ops_create": [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                        ctypes.POINTER(ctypes.c_void_p)],
    "vfmm_ops_export": [ctypes.c_void_p, ctypes.c_int32, c_double_p, ctypes.c_int64],
    "vfmm_ops_destroy": [ctypes.c_void_p],
    "vfmm_ops_set_slices": [ctypes.c_void_p, c_int32_p],
    "vfmm_ops_get_slices": [ctypes.c_void_p, c_int32_p],
    "vfmm_ops_set_m2l": [ctypes.c_void_p, ctypes.c_int32],
    "vfmm_schedule_get": [ctypes.c_void_p, ctypes.c_int32, c_int32_p, c_int32_p],
    "vfmm_schedule_set": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32],
    "vfmm_ops_get_m2l": [ctypes.c_void_p, c_int32_p, c_int32_p],
    "vfmm_workspace_size": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                            ctypes.POINTER(ctypes.c_size_t)],
    "vfmm_volume_potential": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_size_t, ctypes.c_void_p],
    "vfmm_volume_potential_host": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_size_t, ctypes.c_void_p],
    "vfmm_volume_potential_profiled": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_size_t, ctypes.c_void_p, ctypes.POINTER(ctypes.c_float),
                                       ctypes.POINTER(ctypes.c_int32)],
    "vfmm_workspace_status": [ctypes.c_void_p],
    "vfmm_evaluate_points": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                             ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_void_p, ctypes.c_void_p],
    "vfmm_volume_potential_noalloc": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "vfmm_solve_work": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, c_double_p],
    "vfmm_selftest_wait_timeout": [ctypes.c_int64, ctypes.c_void_p],
    "vfmm_tune": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, c_int32_p],
    "vfmm_graph_create": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                          ctypes.POINTER(ctypes.c_void_p)],
    "vfmm_graph_launch": [ctypes.c_void_p, ctypes.c_void_p],
    "vfmm_graph_destroy": [ctypes.c_void_p],
    "vfmm_batch_create": [ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)],
    "vfmm_batch_destroy": [ctypes.c_void_p],
    "vfmm_batch_potential": [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(BatchItem), ctypes.c_void_p],
    "vfmm_batch_graph_create": [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(BatchItem), ctypes.c_void_p,
                                ctypes.POINTER(ctypes.c_void_p)],
    "vfmm_batch_tune": [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(BatchItem), ctypes.c_void_p,
                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)],
    "vfmm_batch_streams": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)],
    "vfmm_strerror": [ctypes.c_int],
    "vfmm_last_error_detail": [],
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads the library; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libvfmm.so is missing at %s: build it with __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    for name, args in EXPORTS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name in ("vfmm_strerror", "vfmm_last_error_detail") else ctypes.c_int
    _lib = lib
    return lib


class VfmmError(RuntimeError):
    def __init__(self, fn: str, code: int):
        lib = load()
        detail = lib.vfmm_last_error_detail().decode(errors="replace")
        msg = lib.vfmm_strerror(code).decode()
        super().__init__("%s failed: %s (%d): %s" % (fn, msg, code, detail))
        self.code = code


def call(name: str, *args):
    lib = load()
    r = getattr(lib, name)(*args)
    if r != 0:
        raise VfmmError(name, r)
    return r
