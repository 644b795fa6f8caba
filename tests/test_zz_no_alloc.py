"""st_build_bvh_noalloc against the BVH that st_scene_create builds.

The allocation-free entry point serves callers that cannot allocate device
memory when they need a BVH; its scratch lives in one fixed device array that
every call shares. This checks, through the C ABI, that two calls in a row
(different meshes, so the second starts from the first one's leftovers) each
reproduce exactly the nodes, leaf order and leaf triangles of the allocating
path with the same builder (the radix tree), and that oversized or invalid
meshes are refused. This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2012_03939_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def st():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_03939_gb300 import build
    build.build()
    from paper_2012_03939_gb300 import st as _st
    _st.lib()
    return _st


def _noalloc(st, V, F):
    n = len(F)
    dV = torch.from_numpy(np.ascontiguousarray(V, np.float32)).cuda()
    dF = torch.from_numpy(np.ascontiguousarray(F, np.int32)).cuda()
    nodes = torch.full((max(n - 1, 1), 16), -7.0, dtype=torch.float32, device="cuda")
    tris = torch.full((n, 12), -7.0, dtype=torch.float32, device="cuda")
    leaf = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = st.lib().st_build_bvh_noalloc(dV.data_ptr(), dF.data_ptr(), len(V), n, nodes.data_ptr(),
                                           tris.data_ptr(), leaf.data_ptr(), stream)
    torch.cuda.synchronize()
    return status, nodes.cpu().numpy()[: n - 1], tris.cpu().numpy(), leaf.cpu().numpy()


def _reference(st, sc):
    scene = st.Scene.from_scene(sc, bvh_builder="lbvh")
    nodes, leaf = scene.debug_bvh()
    scene.close()
    return nodes, leaf


def test_noalloc_bvh_matches_allocating_build_twice_in_a_row(st):
    meshes = [S.edges(), S.tiny()]          # 5120 faces, then 320 faces reusing the scratch
    for sc in meshes:
        status, nodes, tris, leaf = _noalloc(st, sc.vertices, sc.faces)
        assert status == 0, st.lib().st_last_error()
        ref_nodes, ref_leaf = _reference(st, sc)
        np.testing.assert_array_equal(leaf, ref_leaf)
        np.testing.assert_array_equal(nodes, ref_nodes)
        # leaf records: v0 (w = face id bits), v1, v2 of each leaf's face
        exp = np.zeros_like(tris)
        P = sc.vertices[sc.faces[ref_leaf]]
        exp[:, 0:3], exp[:, 4:7], exp[:, 8:11] = P[:, 0], P[:, 1], P[:, 2]
        exp[:, 3] = ref_leaf.view(np.float32)
        np.testing.assert_array_equal(tris, exp)


def test_noalloc_leaves_free_device_memory_unchanged(st):
    # buffers made first, then two builds: the device's free memory does not move
    sc = S.edges()
    _noalloc(st, sc.vertices, sc.faces)            # the first call on the device looks up the scratch address
    n = len(sc.faces)
    dV = torch.from_numpy(sc.vertices).cuda()
    dF = torch.from_numpy(sc.faces).cuda()
    nodes = torch.empty((n - 1, 16), dtype=torch.float32, device="cuda")
    tris = torch.empty((n, 12), dtype=torch.float32, device="cuda")
    leaf = torch.empty((n,), dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        assert st.lib().st_build_bvh_noalloc(dV.data_ptr(), dF.data_ptr(), len(sc.vertices), n, nodes.data_ptr(),
                                             tris.data_ptr(), leaf.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_refuses_oversized_and_invalid_meshes(st):
    V, F = S.uv_sphere(300, 120)                 # 71,400 faces > 65,536
    status, *_ = _noalloc(st, V, F)
    assert status == 6 and b"65536" in st.lib().st_last_error()
    sc = S.tiny()
    bad = sc.faces.copy()
    bad[5, 1] = len(sc.vertices) + 3
    status, *_ = _noalloc(st, sc.vertices, bad)
    assert status == 1
    # and a valid call still works afterwards
    status, nodes, _, leaf = _noalloc(st, sc.vertices, sc.faces)
    ref_nodes, ref_leaf = _reference(st, sc)
    assert status == 0
    np.testing.assert_array_equal(leaf, ref_leaf)
    np.testing.assert_array_equal(nodes, ref_nodes)
