"""Primary-visibility bins drop back faces of a closed, consistently wound surface.

Calls with at least 2^20 primary rays test the leaves binned to each pixel
instead of traversing the BVH; for a single closed surface seen from outside
its bounds, faces wound away from the eye are left out of the bins (they can
never be a primary ray's closest hit). A view rendered in such a call must
equal, bitwise, the same view rendered alone (a small call, which traverses the
BVH with every face): identical samples, identical hits.
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
    # two closed surfaces: two components, so nothing is culled
    V, F = S.icosphere(3)
    V2 = np.concatenate([V * 0.5 + [-0.6, 0, 0], V * 0.5 + [0.6, 0, 0]]).astype(np.float32)
    F2 = np.concatenate([F, F + len(V)]).astype(np.int32)
    rng = np.random.default_rng(3)
    return S.Scene("two", V2, F2, S.random_face_params(rng, len(F2)), light_pos=np.array([[0, 2.5, 2.5]], np.float32),
                   light_intensity=np.array([[9, 9, 9]], np.float32))


@pytest.mark.parametrize("name,B", [("batched", 3), ("env", 2), ("color_bleed", 2), ("two_spheres", 2)])
def test_binned_call_equals_views_rendered_alone(st, name, B):
    sc = _two_spheres() if name == "two_spheres" else S.make(name)
    vs = S.fibonacci_views(4, [448, 384, 512, 320], [448, 384, 256, 320], [2, 2, 3, 2])
    if name == "color_bleed":
        vs = [dataclasses.replace(v, eye=tuple(np.array(v.eye) * 1.2 + [1.5, 1.0, 1.5]), target=(0.6, 0.5, 0.6))
              for v in vs]
    sc.views = vs
    assert sum(v.width * v.height * v.spp for v in vs) >= 1 << 20
    scene = st.Scene.from_scene(sc)
    full = scene.render(vs, B, 31).cpu().numpy()
    for v in vs:
        alone = scene.render([v], B, 31).cpu().numpy()
        rows = slice(v.pixel_offset, v.pixel_offset + v.width * v.height)
        np.testing.assert_array_equal(full[rows], alone[rows])
    assert scene.stats()["device_error"] == 0
    scene.close()
