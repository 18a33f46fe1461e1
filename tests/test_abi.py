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
    # replicas .. precision, dt a0 c0, seed, replica_base .. refine_max, step_kernel and
    # sb_variant, deform_h, deform_tries and check_mode, track_best (+ padding)
    assert ctypes.sizeof(qhap.QhBsbOpts) == 4 * 4 + 3 * 8 + 8 + 4 * 4 + 8 + 8 + 8 + 8
    # iterations_done (+ padding), six array pointers
    assert ctypes.sizeof(qhap.QhRefineState) == 8 + 6 * 8


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """Every field offset of the binding's structs equals the C compiler's for the
    header (gcc is the host compiler the library's host code is built with)."""
    import shutil
    import subprocess
    from paper_2603_25762_gb300 import qhap
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    lines = []
    for py, c in ((qhap.QhFragments, "qh_fragments"), (qhap.QhGraphOpts, "qh_graph_opts"),
                  (qhap.QhBsbOpts, "qh_bsb_opts"), (qhap.QhRefineState, "qh_refine_state")):
        lines.append(f'printf("{c} %zu\\n", sizeof({c}));')
        for name, _ in py._fields_:
            lines.append(f'printf("{c}.{name} %zu\\n", offsetof({c}, {name}));')
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "qhap.h"\n'
                   "int main(void) {\n" + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for py, c in ((qhap.QhFragments, "qh_fragments"), (qhap.QhGraphOpts, "qh_graph_opts"),
                  (qhap.QhBsbOpts, "qh_bsb_opts"), (qhap.QhRefineState, "qh_refine_state")):
        assert int(got[c]) == ctypes.sizeof(py), c
        for name, _ in py._fields_:
            assert int(got[f"{c}.{name}"]) == getattr(py, name).offset, (c, name)


def _header_enums():
    src = open(os.path.join(ROOT, "include", "qhap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return {k: int(v) for k, v in re.findall(r"\b(QH_[A-Z0-9_]+)\s*=\s*(\d+)", src)}


def test_binding_constants_match_header_enums():
    from paper_2603_25762_gb300 import qhap
    enums = _header_enums()
    assert len(enums) >= 20
    checked = 0
    for name, value in enums.items():
        short = name[len("QH_"):]
        if name.startswith("QH_SB_"):
            assert qhap.SB_VARIANTS[short[len("SB_"):].lower()] == value, name
            checked += 1
            continue
        for cand in (name, short):
            if hasattr(qhap, cand):
                assert getattr(qhap, cand) == value, name
                checked += 1
                break
        else:
            pytest.fail(f"{name} has no binding constant")
    assert checked == len(enums)


def test_every_status_has_its_string(libpath):
    from paper_2603_25762_gb300 import qhap
    lib = ctypes.CDLL(libpath)
    lib.qh_status_str.restype = ctypes.c_char_p
    for value, name in qhap._STATUS.items():
        assert lib.qh_status_str(value).decode() == name


def test_step_kernel_names_match_the_library_sources():
    """The binding's step-kernel list is the library's variant numbering: the tile
    variants in the order of their name table, then the CSR variants 10, 11, 12."""
    from paper_2603_25762_gb300 import qhap
    tc = open(os.path.join(ROOT, "paper_2603_25762_gb300", "csrc", "bsb_tc.cu")).read()
    table = re.search(r"static const char\* names\[\] = \{(.*?)\};", tc, flags=re.S).group(1)
    tile = re.findall(r'"([a-z0-9-]+)"', table)
    hdr = open(os.path.join(ROOT, "paper_2603_25762_gb300", "csrc", "qh_internal.cuh")).read()
    csr = {int(v): k for k, v in re.findall(r"constexpr int (CSR_[A-Z0-9]+) = (\d+);", hdr)}
    assert sorted(csr) == [len(tile), len(tile) + 1, len(tile) + 2]
    names = {"CSR_LANE4": "csr-lane4", "CSR_LANE8": "csr-lane8", "CSR_BAND8": "csr-band8"}
    assert qhap.STEP_KERNELS == tile + [names[csr[i]] for i in sorted(csr)]
