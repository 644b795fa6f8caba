"""Interpolated shading normals (scene option smooth_normals) on the GPU path against the FP64 oracle.

Vertex normals are recomputed on the device after every vertex update; the
shading normal at a hit is their barycentric blend. Both sides take the same
samples, so images, path signatures and gradients (interior, then with the
primary, secondary and shadow edge terms) agree up to rounding. The gradient
through the vertex normals reaches every vertex around a hit face.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2012_03939_gb300 import scenes as S
from tests.gpu_util import GRAD_REL, assert_image_parity, rel_l2
from tests.test_gpu_shadow_edges import _sphere_on_floor

pytestmark = pytest.mark.gpu

EDGE_REL = 2e-3


@pytest.fixture(scope="module")
def st():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_03939_gb300 import build
    build.build()
    from paper_2012_03939_gb300 import st as _st
    _st.lib()
    return _st


def _smooth(name, **kw):
    sc = S.small_variant(S.make(name), **({"n_views": 2, "max_res": 32, "spp": 4} | kw))
    sc.smooth_normals = True
    return sc


def _backward(st, sc, B, seed, w, edge_term=0, **kw):
    scene = st.Scene.from_scene(sc)
    dV, dF = scene.backward(sc.views, B, seed, torch.from_numpy(w.astype(np.float32)).cuda(),
                            st.make_opts(edge_term=edge_term, **kw))
    assert scene.stats()["device_error"] == 0
    scene.close()
    return dV.cpu().numpy(), dF.cpu().numpy()


@pytest.mark.parametrize("name,B", [("tiny", 2), ("edges", 3), ("env", 3)])
def test_smooth_image_and_signatures_match_oracle(st, name, B):
    sc = _smooth(name)
    scene = st.Scene.from_scene(sc)
    sig = torch.zeros(sc.n_pixels, dtype=torch.int64, device="cuda")
    img = scene.render(sc.views, B, 21, signatures=sig).cpu().numpy()
    assert scene.stats()["device_error"] == 0
    scene.close()
    osc = O.OracleScene(sc)
    pix = O.all_pixels(sc)
    ref = O.render_pixels(osc, O.params(B, 21), pix)[0]
    assert_image_parity(img, ref, what=name)
    same = sig.cpu().numpy().view(np.uint64) == O.render_signatures(osc, O.params(B, 21), pix)
    assert same.mean() >= 0.999
    # the option changes the image: shading normals differ from the face normals
    flat = dataclasses.replace(sc, smooth_normals=False)
    assert np.abs(O.render_pixels(O.OracleScene(flat), O.params(B, 21), pix)[0] - ref).max() > 1e-3 * ref.max()


@pytest.mark.parametrize("name,B", [("tiny", 2), ("edges", 3), ("env", 2)])
def test_smooth_gradient_matches_oracle(st, name, B):
    sc = _smooth(name)
    w = np.random.default_rng(3).normal(size=(sc.n_pixels, 3))
    dV, dF = _backward(st, sc, B, 33, w)
    rv, rf, _ = O.grad_pixels(O.OracleScene(sc), O.params(B, 33), O.all_pixels(sc), w)
    assert rel_l2([dV], [rv]) <= GRAD_REL and rel_l2([dF], [rf]) <= GRAD_REL


def test_smooth_gradient_with_every_edge_term(st):
    sc = _sphere_on_floor()
    sc.smooth_normals = True
    w = np.random.default_rng(4).normal(size=(sc.n_pixels, 3))
    et = st.EDGE_TERM_PRIMARY | st.EDGE_TERM_SECONDARY | st.EDGE_TERM_SHADOW
    dV, dF = _backward(st, sc, 2, 12, w, et)
    osc = O.OracleScene(sc)
    prm = O.params(2, 12, secondary=2)
    rv, rf, _ = O.grad_pixels(osc, prm, O.all_pixels(sc), w)
    rv = rv + O.edge_grad(osc, prm, w)[0] + O.shadow_edge_grad(osc, prm, w)[0]
    assert rel_l2([dV, dF], [rv, rf]) <= EDGE_REL


def test_smooth_gradient_does_not_depend_on_the_launch_path(st):
    sc = _smooth("edges", spp=2)
    w = np.random.default_rng(6).normal(size=(sc.n_pixels, 3))
    et = st.EDGE_TERM_PRIMARY | st.EDGE_TERM_SECONDARY
    ref = _backward(st, sc, 3, 8, w, et)
    for kw in [dict(use_graph=0), dict(chunk_paths=1024), dict(mode="per_view")]:
        assert rel_l2(_backward(st, sc, 3, 8, w, et, **kw), ref) <= 1e-5, kw


def test_refit_recomputes_the_vertex_normals(st):
    sc = _smooth("tiny")
    V1 = sc.vertices + np.random.default_rng(7).normal(0, 0.03, sc.vertices.shape).astype(np.float32)
    moved = st.Scene.from_scene(sc)
    moved.refit(torch.from_numpy(V1).cuda())
    a = moved.render(sc.views, 2, 5).cpu().numpy()
    moved.close()
    fresh = st.Scene.from_scene(sc, vertices=V1)
    b = fresh.render(sc.views, 2, 5).cpu().numpy()
    fresh.close()
    np.testing.assert_array_equal(a, b)
    assert_image_parity(a, O.render_pixels(O.OracleScene(sc, vertices=V1), O.params(2, 5), O.all_pixels(sc))[0])


def test_smooth_normals_with_rgb_specular_and_mesh_colors(st):
    # the smooth adjoint with 7 parameters per texel at mesh-colors resolution 2
    sc = S.tiny(res=32, spp=4)
    sc.smooth_normals = True
    rng = np.random.default_rng(12)
    sc.face_params = np.repeat(sc.face_params, 6, axis=0)
    sc.color_res = 2
    P = sc.face_params
    sc.face_params = np.c_[P[:, :3], rng.uniform(0.02, 0.5, (len(P), 3)), P[:, 4]].astype(np.float32)
    w = rng.normal(size=(sc.n_pixels, 3))
    dV, dF = _backward(st, sc, 2, 17, w)
    assert dF.shape == (len(sc.face_params), 7)
    rv, rf, _ = O.grad_pixels(O.OracleScene(sc), O.params(2, 17), O.all_pixels(sc), w)
    assert rel_l2([dV], [rv]) <= GRAD_REL and rel_l2([dF], [rf]) <= GRAD_REL
