"""RGB specular (7 parameters per texel: kd rgb, ks rgb, roughness) on the GPU path.

The paper gives each material a specular colour (Sec. 3.3); the library takes
either one specular value for all channels (5 parameters per texel) or one per
channel (7). Images and gradients are compared with the FP64 oracle, and equal
channels must reproduce the scalar form.
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


def _rgb(P5, ks):
    return np.c_[P5[:, :3], ks, P5[:, 4]].astype(np.float32)


def _run(st, sc, B, seed, w):
    scene = st.Scene.from_scene(sc)
    img = scene.render(sc.views, B, seed).cpu().numpy()
    dV, dF = scene.backward(sc.views, B, seed, torch.from_numpy(w.astype(np.float32)).cuda(),
                            st.make_opts(edge_term=0))
    assert scene.stats()["device_error"] == 0
    scene.close()
    return img, dV.cpu().numpy(), dF.cpu().numpy()


@pytest.mark.parametrize("workload,B,r", [("tiny", 2, 0), ("edges", 3, 0), ("tiny", 2, 2)])
def test_rgb_specular_matches_oracle(st, workload, B, r):
    sc = S.tiny(res=32, spp=4) if workload == "tiny" else S.small_variant(S.make(workload), 2, 32, 4)
    rng = np.random.default_rng(8)
    if r:
        n = (r + 1) * (r + 2) // 2
        sc.face_params = np.repeat(sc.face_params, n, axis=0)
        sc.color_res = r
    sc.face_params = _rgb(sc.face_params, rng.uniform(0.02, 0.5, (len(sc.face_params), 3)))
    w = rng.normal(size=(sc.n_pixels, 3))
    img, dV, dF = _run(st, sc, B, 23, w)
    assert dF.shape == (len(sc.face_params), 7)
    osc = O.OracleScene(sc)
    ref, _ = O.render_pixels(osc, O.params(B, 23), O.all_pixels(sc))
    assert_image_parity(img, ref, what="rgb specular")
    rv, rf, _ = O.grad_pixels(osc, O.params(B, 23), O.all_pixels(sc), w)
    assert rel_l2([dV, dF], [rv, rf]) <= GRAD_REL


def test_equal_channels_reproduce_scalar_specular(st):
    sc5 = S.tiny(res=32, spp=4)
    sc7 = S.tiny(res=32, spp=4)
    sc7.face_params = _rgb(sc5.face_params, np.repeat(sc5.face_params[:, 3:4], 3, axis=1))
    w = np.random.default_rng(9).normal(size=(sc5.n_pixels, 3))
    i5, v5, f5 = _run(st, sc5, 3, 4, w)
    i7, v7, f7 = _run(st, sc7, 3, 4, w)
    np.testing.assert_array_equal(i5, i7)
    np.testing.assert_allclose(v7, v5, rtol=1e-4, atol=1e-6 * np.abs(v5).max())
    np.testing.assert_allclose(f7[:, 3:6].sum(1), f5[:, 3], rtol=1e-4, atol=1e-6 * np.abs(f5).max())
    np.testing.assert_allclose(f7[:, [0, 1, 2, 6]], f5[:, [0, 1, 2, 4]], rtol=1e-4, atol=1e-6 * np.abs(f5).max())
