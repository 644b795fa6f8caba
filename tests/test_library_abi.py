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


def test_structure_sizes_match_c_layout(tmp_path):
    # every ctypes structure of the binding against the C compiler's layout of include/st.h
    import subprocess
    from paper_2012_03939_gb300 import st
    pairs = {"st_view": st.View, "st_scene_desc": st.SceneDesc, "st_render_opts": st.RenderOpts,
             "st_stats": st.Stats, "st_point_light": st.PointLight, "st_envmap": st.EnvMap}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "st.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for cname, py in pairs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got["%s.%s" % (cname, f)]) == getattr(py, f).offset, (cname, f)


def test_binding_constants_match_header():
    # every constant the binding restates has the header's value
    from paper_2012_03939_gb300 import st
    src = open(os.path.join(ROOT, "include", "st.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"#define ST_([A-Z0-9_]+)\s+(-?\d+)", src)}
    pairs = {"MODE_BATCHED": st.MODE_BATCHED, "MODE_PER_VIEW": st.MODE_PER_VIEW,
             "EDGE_SILHOUETTE": st.EDGE_SILHOUETTE, "EDGE_ALL": st.EDGE_ALL,
             "EDGE_TERM_PRIMARY": st.EDGE_TERM_PRIMARY, "EDGE_TERM_SECONDARY": st.EDGE_TERM_SECONDARY,
             "EDGE_TERM_SHADOW": st.EDGE_TERM_SHADOW, "BVH_PLOC": st.BVH_PLOC, "BVH_LBVH": st.BVH_LBVH,
             "MAX_VIEW_LIGHTS": st.MAX_VIEW_LIGHTS, "MAX_VIEWS": st.MAX_VIEWS,
             "SEC_PICK_TREE": st.SEC_PICK_TREE, "SEC_PICK_UNIFORM": st.SEC_PICK_UNIFORM,
             "FRESNEL_HELD": st.FRESNEL_HELD, "FRESNEL_SCHLICK": st.FRESNEL_SCHLICK}
    for k, v in pairs.items():
        assert defs[k] == v, k


def test_make_opts_maps_names_to_header_values():
    from paper_2012_03939_gb300 import st
    o = st.make_opts()
    assert (o.sec_pick, o.edge_mode, o.mode, o.use_graph, o.edge_term) == (st.SEC_PICK_TREE, st.EDGE_SILHOUETTE,
                                                                           st.MODE_BATCHED, 1, 0)
    o = st.make_opts(sec_pick="uniform", edge_mode="all", mode="per_view",
                     edge_term=st.EDGE_TERM_SECONDARY | st.EDGE_TERM_SHADOW)
    assert (o.sec_pick, o.edge_mode, o.mode, o.edge_term) == (st.SEC_PICK_UNIFORM, st.EDGE_ALL, st.MODE_PER_VIEW, 6)
    with pytest.raises(KeyError):
        st.make_opts(sec_pick="random")


def test_fault_injection_hook_validates_its_site_without_gpu():
    # arming and disarming the host-side fault hook makes no CUDA call
    from paper_2012_03939_gb300 import st
    L = st.lib()
    assert L.st_inject_fault(0, 0) == 1 and b"fault site" in L.st_last_error()
    assert L.st_inject_fault(3, 0) == 1
    for site in (st.FAULT_ALLOC, st.FAULT_COPY):
        assert L.st_inject_fault(site, 5) == 0
        assert L.st_inject_fault(site, -1) == 0
    src = open(os.path.join(ROOT, "include", "st.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"#define ST_([A-Z0-9_]+)\s+(-?\d+)", src)}
    assert (defs["FAULT_ALLOC"], defs["FAULT_COPY"]) == (st.FAULT_ALLOC, st.FAULT_COPY)
