"""CPU checks of the boundary: the shared library builds for sm_103a, loads
without a GPU, and exports every entry point include/blademaster.h declares
(no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared_symbols():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(bm_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2609_27342_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for core in ["bm_scene_create", "bm_add_blade", "bm_step", "bm_read_state", "bm_tool_wrench",
                 "bm_batch_create", "bm_batch_step", "bm_last_error"]:
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_2609_27342_gb300 import _abi
    assert set(declared_symbols()) <= set(_abi.SIGNATURES)


def test_version_string_without_gpu(lib):
    lib.bm_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.bm_version()


def test_library_built_for_sm103a():
    from paper_2609_27342_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_product_path_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_2609_27342_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.replace("the oracle", ""), f


def test_struct_layouts_match_header_sizes():
    """ctypes mirrors of the ABI structs have the sizes a C compiler gives."""
    import subprocess
    import tempfile
    from paper_2609_27342_gb300 import _abi as A
    src = ('#include <stdio.h>\n#include "blademaster.h"\nint main(){printf("%zu %zu %zu %zu %zu %zu\\n",'
           'sizeof(bm_scene_desc),sizeof(bm_blade_desc),sizeof(bm_segment),sizeof(bm_scene_info),'
           'sizeof(bm_batch_desc),sizeof(bm_alloc));return 0;}\n')
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        sizes = [int(t) for t in subprocess.check_output([exe]).split()]
    assert sizes == [ctypes.sizeof(A.SceneDesc), ctypes.sizeof(A.BladeDesc),
                     ctypes.sizeof(A.Segment), ctypes.sizeof(A.SceneInfo),
                     ctypes.sizeof(A.BatchDesc), ctypes.sizeof(A.Alloc)]
