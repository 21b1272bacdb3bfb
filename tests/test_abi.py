"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/vfmm.h declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vfmm.h")


def declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(vfmm_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1610_00823_gb300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared()
    for must in ("vfmm_tree_build", "vfmm_volume_potential", "vfmm_ops_create", "vfmm_workspace_size"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1610_00823_gb300 import _lib
    for name in declared():
        assert hasattr(lib, name), name
        assert name in _lib.EXPORTS, name


def test_error_strings_need_no_gpu(lib):
    assert lib.vfmm_strerror(0) == b"ok"
    assert lib.vfmm_strerror(-6) == b"workspace too small"
    assert lib.vfmm_strerror(12345) == b"unknown error code"


def _declared_arity():
    """Parameter count of every declared function, from the header text."""
    txt = open(HEADER).read()
    out = {}
    for m in re.finditer(r"^\s*(?:int|const char\*)\s+(vfmm_\w+)\s*\(([^;]*?)\)\s*;", txt, flags=re.M | re.S):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header():
    from paper_1610_00823_gb300 import _lib
    arity = _declared_arity()
    assert set(arity) == set(declared())
    for name, n in arity.items():
        assert len(_lib.EXPORTS[name]) == n, (name, len(_lib.EXPORTS[name]), n)
