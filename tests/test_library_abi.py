"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "st.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(st_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["st_scene_create", "st_scene_destroy", "st_refit", "st_render", "st_render_backward",
              "st_set_face_params", "st_get_stats", "st_last_error"]:
        assert n in names


def test_library_builds_loads_and_exports_all_symbols():
    from paper_2012_03939_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)            # loads on a machine without a GPU (static CUDA runtime)
    for n in _declared():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (st_[a-z0-9_]+)", out))
    assert set(_declared()) <= exported


def test_binding_names_match_header():
    from paper_2012_03939_gb300 import st
    assert sorted(st.EXPORTED) == _declared()


def test_last_error_is_callable_without_gpu():
    from paper_2012_03939_gb300 import st
    L = st.lib()
    assert isinstance(L.st_last_error(), bytes)
    # invalid arguments are rejected before any CUDA call
    assert L.st_scene_create(None, None, None) == 1
    h = ctypes.c_void_p()
    assert L.st_scene_create(None, None, ctypes.byref(h)) == 1
    assert b"mesh" in L.st_last_error()


def test_structure_sizes_match_c_layout():
    from paper_2012_03939_gb300 import st
    # st_view: 10 floats, 3 ints, 4 bytes padding, one long long
    assert ctypes.sizeof(st.View) == 10 * 4 + 3 * 4 + 4 + 8
    assert ctypes.sizeof(st.RenderOpts) == 9 * 4
    assert ctypes.sizeof(st.PointLight) == 24
