"""The C-ABI library: it builds for sm_103a, loads, and exports every symbol
that include/spc5.h declares.  Argument checks that happen before any CUDA
call are exercised here without a GPU."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

import paper_2307_14774_gb300 as spc5

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "spc5.h")


def declared_functions() -> list[str]:
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spc5_[a-z_0-9]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    lib = spc5.load()
    names = declared_functions()
    assert names, "no declarations found"
    for name in names:
        assert hasattr(lib, name), f"{name} declared in spc5.h but not exported"
    assert sorted(spc5.EXPORTS) == names


def test_library_is_built_for_sm103a():
    from paper_2307_14774_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_status_strings():
    for code, name in spc5.STATUS.items():
        assert spc5.spc5_status_str(code) == name


def test_rejects_unsupported_shape_before_touching_the_gpu():
    rowptr = np.array([0, 1], np.int32)
    col = np.array([0], np.int32)
    val = np.array([1.0])
    with pytest.raises(spc5.SPC5Error) as ei:
        spc5.spc5_convert_csr(1, 1, 1, rowptr, col, val, r=3, c=5, stream=0)
    assert ei.value.name == "SPC5_EUNSUPPORTED_RC"
    with pytest.raises(spc5.SPC5Error) as ei:
        spc5.spc5_convert_csr(-1, 1, 1, rowptr, col, val, r=4, c=8, stream=0)
    assert ei.value.name == "SPC5_EINVAL"
    with pytest.raises(spc5.SPC5Error) as ei:
        spc5.spc5_convert_csr(1, 1, 1, rowptr, col, val, r=4, c=8, vals_dtype=spc5.SPC5_F32,
                              stream=0)
    assert ei.value.name == "SPC5_EUNSUPPORTED"
    with pytest.raises(spc5.SPC5Error) as ei:
        spc5.spc5_convert_csr(3_000_000_000, 1, 1, rowptr, col, val, r=4, c=8, stream=0)
    assert ei.value.name == "SPC5_EOVERFLOW"
    lib = spc5.load()
    assert lib.spc5_spmv(None, None, None, 1.0, 0.0, None) == 1  # EINVAL on a NULL handle
    assert lib.spc5_matrix_info(None, None) == 1
    assert lib.spc5_destroy(None) == 0


@pytest.mark.parametrize("cname,pystruct", [("spc5_info", "Info"), ("spc5_cg_report", "CGReport")])
def test_struct_layout_matches_header(tmp_path, cname, pystruct):
    """The binding's ctypes mirrors of the header's structs have the C
    compiler's size and field offsets."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    cls = getattr(spc5.spc5, pystruct)
    lines = [f'printf("%zu\\n", sizeof({cname}));']
    lines += [f'printf("%zu\\n", offsetof({cname}, {f}));' for f, _ in cls._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "spc5.h"\n'
                   "int main(void) {\n" + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert got[0] == ctypes.sizeof(cls)
    assert got[1:] == [getattr(cls, f).offset for f, _ in cls._fields_]


def test_vector_placement_rule(tmp_path):
    """The rule by which spc5_spmv and spc5_spmv_noalloc classify a vector
    (spc5_pointer.h), compiled and checked on the host: host memory is
    staged, the matrix's own device memory and managed memory are read
    directly, another GPU's device memory is rejected."""
    import shutil
    import subprocess
    if shutil.which("g++") is None:
        pytest.skip("no C++ compiler")
    csrc = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_2307_14774_gb300",
                        "csrc")
    src = tmp_path / "placement.cpp"
    src.write_text('#include <cstdio>\n#include "spc5_pointer.h"\nusing namespace spc5;\n'
                   "int main() {\n"
                   "  int bad = 0;\n"
                   "  bad += placement_of(-1, -1, 0) != Placement::kHost;\n"
                   "  bad += placement_of(0, -2, 1) != Placement::kHost;\n"
                   "  bad += placement_of(1, 0, 1) != Placement::kHost;\n"
                   "  bad += placement_of(2, 1, 1) != Placement::kDevice;\n"
                   "  bad += placement_of(2, 0, 1) != Placement::kOtherDevice;\n"
                   "  bad += placement_of(2, 3, 0) != Placement::kOtherDevice;\n"
                   "  bad += placement_of(3, 0, 1) != Placement::kDevice;\n"
                   '  std::printf("%d\\n", bad);\n  return 0;\n}\n')
    exe = tmp_path / "placement"
    subprocess.run(["g++", "-std=c++17", "-I", csrc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    assert out.strip() == "0"
