"""Mesh colors at resolution r > 0 (Sec. 3.3) on the GPU path, against the FP64 oracle.

Each face carries (r+1)(r+2)/2 parameter sets (texels); a hit uses the texel
its barycentric coordinates fall in. The texel choice draws no random numbers,
so with every texel of a face set to the face's parameters the image must be
bit-identical to the per-face (r = 0) render, and the per-texel gradients of a
face must sum to the per-face gradient.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2012_03939_gb300 import scenes as S
from tests.gpu_util import GRAD_REL, assert_image_parity, rel_l2

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


def _textured(sc, r, seed):
    n = (r + 1) * (r + 2) // 2
    rng = np.random.default_rng(seed)
    P = np.repeat(sc.face_params.astype(np.float64), n, axis=0)
    P[:, :3] = np.clip(P[:, :3] + rng.normal(0.0, 0.2, (len(P), 3)), 0.02, 0.98)
    P[:, 3] = np.clip(P[:, 3] + rng.normal(0.0, 0.1, len(P)), 0.0, 1.0)
    P[:, 4] = np.clip(P[:, 4] + rng.normal(0.0, 0.1, len(P)), 0.05, 1.0)
    sc.face_params = P.astype(np.float32)
    sc.color_res = r
    return sc


@pytest.mark.parametrize("r", [1, 3])
def test_mesh_colors_image_and_gradient_match_oracle(st, r):
    sc = _textured(S.tiny(res=32, spp=4), r, 40 + r)
    scene = st.Scene.from_scene(sc)
    img = scene.render(sc.views, 3, 11).cpu().numpy()
    w = np.random.default_rng(r).normal(size=img.shape)
    dV, dF = scene.backward(sc.views, 3, 11, torch.from_numpy(w.astype(np.float32)).cuda(), st.make_opts(edge_term=0))
    assert scene.stats()["device_error"] == 0
    scene.close()
    assert dF.shape == (len(sc.faces) * (r + 1) * (r + 2) // 2, 5)
    osc = O.OracleScene(sc)
    ref, _ = O.render_pixels(osc, O.params(3, 11), O.all_pixels(sc))
    assert_image_parity(img, ref, what=f"mesh colors r={r}")
    rv, rf, _ = O.grad_pixels(osc, O.params(3, 11), O.all_pixels(sc), w)
    assert rel_l2([dV.cpu().numpy(), dF.cpu().numpy()], [rv, rf]) <= GRAD_REL


def test_uniform_texels_reproduce_per_face_render(st):
    r = 2
    n = (r + 1) * (r + 2) // 2
    base = S.tiny(res=32, spp=4)
    tex = S.tiny(res=32, spp=4)
    tex.face_params = np.repeat(base.face_params, n, axis=0)
    tex.color_res = r
    out = []
    for sc in (base, tex):
        scene = st.Scene.from_scene(sc)
        img = scene.render(sc.views, 3, 5).clone()
        w = torch.ones_like(img)
        dV, dF = scene.backward(sc.views, 3, 5, w, st.make_opts(edge_term=0))
        scene.close()
        out.append((img.cpu().numpy(), dV.cpu().numpy(), dF.cpu().numpy()))
    np.testing.assert_array_equal(out[1][0], out[0][0])
    np.testing.assert_allclose(out[1][1], out[0][1], rtol=1e-4, atol=1e-6 * np.abs(out[0][1]).max())
    per_face = out[1][2].reshape(len(base.faces), n, 5).sum(1)
    np.testing.assert_allclose(per_face, out[0][2], rtol=1e-4, atol=1e-6 * np.abs(out[0][2]).max())


def test_color_res_out_of_range_is_rejected(st):
    sc = S.tiny(res=16, spp=1)
    sc.color_res = 65
    sc.face_params = np.repeat(sc.face_params, 66 * 67 // 2, axis=0)
    with pytest.raises(RuntimeError):
        st.Scene.from_scene(sc)
