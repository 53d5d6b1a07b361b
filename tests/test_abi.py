"""The C-ABI library loads and exports every entry point that include/bst.h declares
(no GPU needed: nothing here launches a kernel or creates a context)."""
import ctypes
import os
import re

from paper_1910_13555_gb300 import bst

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "bst.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bst_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1910_13555_gb300 import build as b
    b.build()
    lib = ctypes.CDLL(bst.LIB_PATH)
    names = declared()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(bst.exported_symbols()) == names


def test_status_names_and_version_without_gpu():
    lib = bst.load()
    assert lib.bst_status_name(0) == b"BST_OK"
    assert lib.bst_status_name(4) == b"BST_ERR_SHAPE_MISMATCH"
    assert bst.bst_version().startswith("bst")
