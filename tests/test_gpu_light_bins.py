"""Point-light shadow lists: shadow rays to the scene's lights test leaf lists binned from each light.

Calls with at least 2^20 primary rays bin the leaves, seen from each scene light
outside the mesh's bounding sphere, into a frustum of cells around the mesh; a
shadow ray to that light tests the leaves of its origin's cell with the
traversal's test and bound. For one closed, consistently wound surface the faces
wound away from the light are left out. The visibility must be exactly the
traversal's, so a view rendered in such a call must equal, bitwise, the same view
rendered alone (a small call, which traces every shadow ray through the BVH).
"""
import dataclasses

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


def _two_spheres():
    # two closed surfaces: two components, so no face is left out
    V, F = S.icosphere(3)
    V2 = np.concatenate([V * 0.5 + [-0.6, 0, 0], V * 0.5 + [0.6, 0, 0]]).astype(np.float32)
    F2 = np.concatenate([F, F + len(V)]).astype(np.int32)
    rng = np.random.default_rng(3)
    return S.Scene("two", V2, F2, S.random_face_params(rng, len(F2)),
                   light_pos=np.array([[0, 2.5, 2.5], [-2.0, 0.3, -2.2]], np.float32),
                   light_intensity=np.array([[9, 9, 9], [5, 4, 3]], np.float32))


def _scene(name):
    if name == "two_spheres":
        return _two_spheres()
    if name == "color_bleed_far_light":
        # an open mesh (no face left out) lit by its own light, inside the bounds (BVH), and a far one (lists)
        sc = S.make("color_bleed")
        sc.light_pos = np.array([[1.3, 1.6, 1.3], [5.0, 6.0, 4.0]], np.float32)
        sc.light_intensity = np.array([[4, 4, 4], [30, 30, 30]], np.float32)
        return sc
    if name == "scale":
        return S.make("scale")
    return S.make(name)


@pytest.mark.parametrize("name,B", [("edges", 3), ("two_spheres", 2), ("color_bleed_far_light", 3), ("scale", 2),
                                    ("edges_view_lights", 2)])
def test_listed_shadow_rays_equal_traversal(st, name, B):
    sc = _scene(name.replace("_view_lights", ""))
    vs = S.fibonacci_views(4, [448, 384, 512, 320], [448, 384, 256, 320], [2, 2, 3, 2])
    if name.endswith("_view_lights"):
        # each view's own two lights (camera and offset) trace the BVH beside the scene's listed lights
        vs = S.with_view_lights(vs, intensity=(2.0, 2.0, 2.0))
    if name == "color_bleed_far_light":
        vs = [dataclasses.replace(v, eye=tuple(np.array(v.eye) * 1.2 + [1.5, 1.0, 1.5]), target=(0.6, 0.5, 0.6))
              for v in vs]
    sc.views = vs
    assert sum(v.width * v.height * v.spp for v in vs) >= 1 << 20   # large enough to build the lists
    scene = st.Scene.from_scene(sc)
    opts = st.make_opts(count_visits=1, use_graph=0)
    full = scene.render(vs, B, 31, opts).cpu().numpy()
    big = scene.stats()
    visits, rays = 0, 0
    for v in vs:
        alone = scene.render([v], B, 31, opts).cpu().numpy()
        s = scene.stats()
        visits += s["shadow_node_visits"]
        rays += s["shadow_rays"]
        rows = slice(v.pixel_offset, v.pixel_offset + v.width * v.height)
        np.testing.assert_array_equal(full[rows], alone[rows])
    assert big["device_error"] == 0
    assert big["shadow_rays"] == rays
    # the listed rays fetch no node: the big call's any-hit node fetches fall well below the traversal's
    assert big["shadow_node_visits"] < 0.8 * visits, (big["shadow_node_visits"], visits)
    scene.close()


def test_light_lists_follow_the_vertices(st):
    # a refit moves the mesh: the next call bins again, and equals a scene created at the new vertices
    sc = S.make("edges")
    vs = S.fibonacci_views(3, [512, 512, 384], [512, 384, 384], [2, 2, 2])
    sc.views = vs
    scene = st.Scene.from_scene(sc)
    a = scene.render(vs, 2, 7).cpu().numpy()
    V2 = (sc.vertices * np.float32(1.1) + np.float32(0.05)).astype(np.float32)
    scene.refit(torch.from_numpy(V2).cuda())
    b = scene.render(vs, 2, 7).cpu().numpy()
    fresh = st.Scene.from_scene(sc, vertices=V2)
    c = fresh.render(vs, 2, 7).cpu().numpy()
    assert scene.stats()["device_error"] == 0 and fresh.stats()["device_error"] == 0
    np.testing.assert_array_equal(b, c)
    assert not np.array_equal(a, b)
    scene.close()
    fresh.close()
