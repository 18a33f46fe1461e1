"""The C-ABI library builds, loads and exports every function that include/qhap.h declares.

No GPU needed: loading the shared library does not touch a device, and no compute
entry point is called here.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "qhap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qh_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2603_25762_gb300 import build
    return build.build()


def test_header_declares_the_path(libpath):
    names = _declared()
    for must in ("qh_build_graph", "qh_bsb_solve", "qh_phase", "qh_create", "qh_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(libpath):
    from paper_2603_25762_gb300 import qhap
    assert set(qhap._SIGS) == set(_declared())


def test_status_strings_without_device(libpath):
    lib = ctypes.CDLL(libpath)
    lib.qh_status_str.restype = ctypes.c_char_p
    assert lib.qh_status_str(0) == b"QH_OK"
    assert lib.qh_status_str(4) == b"QH_ETIMEOUT"


def test_struct_layouts_match_header():
    from paper_2603_25762_gb300 import qhap
    assert ctypes.sizeof(qhap.QhFragments) == 4 + 4 + 5 * 8 + 8
    assert ctypes.sizeof(qhap.QhGraphOpts) == 5 * 4 + 4 + 8
    assert ctypes.sizeof(qhap.QhBsbOpts) == 4 * 4 + 3 * 8 + 8 + 4 * 4 + 8 + 8 + 8
