"""Schlick's Fresnel factor (scene option fresnel = 1) on the GPU path against the FP64 oracle.

The Torrance-Sparrow specular lobe (Sec. 3.3 "Representation") is scaled by
F = ks + (1 - ks)(1 - wi.h)^5 per channel. Images, path signatures and
gradients (where the factor moves with the point-light direction, hence with
the hit point and the vertices) are compared with the oracle on identical
samples; the held form stays the default and is unchanged.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2012_03939_gb300 import scenes as S
from tests.gpu_util import GRAD_REL, PIX_ABS, PIX_REL, assert_image_parity, rel_l2

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


def _glossy(sc):
    # a stronger, rougher specular so the factor carries weight in the image and the gradient
    P = sc.face_params.copy()
    P[:, 3 if P.shape[1] == 5 else slice(3, 6)] = 0.3
    P[:, -1] = np.clip(P[:, -1], 0.2, 0.5)
    return dataclasses.replace(sc, face_params=P, fresnel=1)


def _scene(name):
    if name == "tiny":
        return _glossy(S.tiny(res=32, spp=4))
    if name == "tiny_beckmann":
        sc = _glossy(S.tiny(res=32, spp=4))
        sc.brdf = "beckmann"
        return sc
    if name == "rgb":
        sc = S.tiny(res=32, spp=4)
        P = sc.face_params
        rng = np.random.default_rng(3)
        sc = dataclasses.replace(sc, face_params=np.c_[P[:, :3], rng.uniform(0.1, 0.5, (len(P), 3)),
                                                       P[:, 4]].astype(np.float32))
        return dataclasses.replace(sc, fresnel=1)
    if name == "smooth":
        return dataclasses.replace(_glossy(S.small_variant(S.make("edges"), n_views=2, max_res=24, spp=2)),
                                   smooth_normals=True)
    return _glossy(S.small_variant(S.make(name), n_views=2, max_res=24, spp=2))


def _B(name):
    return {"tiny": 2, "tiny_beckmann": 2, "rgb": 2, "edges": 3, "env": 4, "color_bleed": 3, "smooth": 3}[name]


@pytest.mark.parametrize("name", ["tiny", "tiny_beckmann", "rgb", "edges", "env", "color_bleed", "smooth"])
def test_schlick_image_signatures_and_interior_gradient_match_oracle(st, name):
    sc = _scene(name)
    B = _B(name)
    scene = st.Scene.from_scene(sc)
    sig = torch.zeros(sc.n_pixels, dtype=torch.int64, device="cuda")
    img = scene.render(sc.views, B, 51, signatures=sig).cpu().numpy()
    sig = sig.cpu().numpy().view(np.uint64)
    w = np.random.default_rng(5).normal(size=img.shape)
    dV, dF = scene.backward(sc.views, B, 51, torch.from_numpy(w.astype(np.float32)).cuda(), st.make_opts(edge_term=0))
    assert scene.stats()["device_error"] == 0
    scene.close()
    osc = O.OracleScene(sc)
    pix = O.all_pixels(sc)
    ref, _ = O.render_pixels(osc, O.params(B, 51), pix)
    assert_image_parity(img, ref, what=name)
    rsig = O.render_signatures(osc, O.params(B, 51), pix)
    same = sig == rsig
    assert same.mean() >= 0.999
    out = np.any(np.abs(img - ref) > PIX_REL * np.abs(ref) + PIX_ABS, axis=1)
    assert not np.any(out & same)
    rv, rf, _ = O.grad_pixels(osc, O.params(B, 51), pix, w)
    r = rel_l2([dV.cpu().numpy(), dF.cpu().numpy()], [rv, rf])
    assert r <= GRAD_REL, r


def test_schlick_edge_term_matches_oracle(st):
    sc = _scene("tiny")
    w = np.random.default_rng(8).normal(size=(sc.n_pixels, 3))
    scene = st.Scene.from_scene(sc)
    wt = torch.from_numpy(w.astype(np.float32)).cuda()
    dVe, _ = scene.backward(sc.views, 2, 19, wt, st.make_opts(edge_term=1, edge_mode=1))
    dVi, _ = scene.backward(sc.views, 2, 19, wt, st.make_opts(edge_term=0))
    scene.close()
    ev, _ = O.edge_grad(O.OracleScene(sc), O.params(2, 19, edge_mode=1), w)
    r = rel_l2([(dVe - dVi).cpu().numpy()], [ev])
    assert r <= 5e-3, r


def test_schlick_changes_the_specular_image_and_held_stays_default(st):
    sc = _scene("tiny")
    held = dataclasses.replace(sc, fresnel=0)
    a = st.Scene.from_scene(sc)
    b = st.Scene.from_scene(held)
    ia = a.render(sc.views, 2, 7).cpu().numpy()
    ib = b.render(sc.views, 2, 7).cpu().numpy()
    a.close()
    b.close()
    assert np.all(ia >= ib - 1e-6)               # F >= ks at every angle
    assert (ia > ib + 1e-6).mean() > 0.05        # and larger toward grazing
    # the default scene (no option given) renders as the held form
    c = st.Scene(torch.from_numpy(sc.vertices).cuda(), torch.from_numpy(sc.faces).cuda(),
                 torch.from_numpy(sc.face_params).cuda(), light_pos=sc.light_pos, light_intensity=sc.light_intensity)
    np.testing.assert_array_equal(c.render(sc.views, 2, 7).cpu().numpy(), ib)
    c.close()
    with pytest.raises(st.StError):
        st.Scene.from_scene(dataclasses.replace(sc, fresnel=2))
