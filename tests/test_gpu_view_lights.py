"""Per-view point lights on the GPU path against the FP64 oracle.

Each view may carry up to two point lights of its own, seen only by its paths
(camera paths, edge side paths and secondary side paths), after the scene's
lights; the paper lights every capture from the camera and from a point offset
from it (Sec. 4).
"""
import dataclasses

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


def _colocated(workload, keep_scene_lights, n_views=3, res=24, spp=4):
    sc = S.small_variant(S.make(workload), n_views=n_views, max_res=res, spp=spp)
    sc.views = S.with_view_lights(sc.views, intensity=(3.0, 2.5, 2.0))
    # views differ: the last one gets a single light of its own
    sc.views[-1] = dataclasses.replace(sc.views[-1], lights=sc.views[-1].lights[:1])
    if not keep_scene_lights:
        sc.light_pos = np.zeros((0, 3), np.float32)
        sc.light_intensity = np.zeros((0, 3), np.float32)
    return sc


@pytest.mark.parametrize("workload,keep", [("edges", False), ("edges", True), ("env", False)])
def test_view_lights_image_and_gradient_match_oracle(st, workload, keep):
    sc = _colocated(workload, keep)
    B = 2
    scene = st.Scene.from_scene(sc)
    img = scene.render(sc.views, B, 17).cpu().numpy()
    w = np.random.default_rng(2).normal(size=img.shape)
    dV, dF = scene.backward(sc.views, B, 17, torch.from_numpy(w.astype(np.float32)).cuda(),
                            st.make_opts(edge_term=0))
    assert scene.stats()["device_error"] == 0
    scene.close()
    osc = O.OracleScene(sc)
    ref, _ = O.render_pixels(osc, O.params(B, 17), O.all_pixels(sc))
    assert_image_parity(img, ref, what="view lights %s" % workload)
    rv, rf, _ = O.grad_pixels(osc, O.params(B, 17), O.all_pixels(sc), w)
    assert rel_l2([dV.cpu().numpy(), dF.cpu().numpy()], [rv, rf]) <= GRAD_REL


def test_view_lights_with_both_edge_terms(st):
    sc = _colocated("color_bleed", False)
    w = np.random.default_rng(3).normal(size=(sc.n_pixels, 3))
    scene = st.Scene.from_scene(sc)
    dV, _ = scene.backward(sc.views, 3, 5, torch.from_numpy(w.astype(np.float32)).cuda(),
                           st.make_opts(edge_term=st.EDGE_TERM_PRIMARY | st.EDGE_TERM_SECONDARY, edge_spp=4))
    scene.close()
    osc = O.OracleScene(sc)
    rv, _, _ = O.grad_pixels(osc, O.params(3, 5, secondary=2), O.all_pixels(sc), w)
    ev, _ = O.edge_grad(osc, O.params(3, 5, edge_spp=4), w)
    assert rel_l2([dV.cpu().numpy()], [rv + ev]) <= 2e-3


def test_graph_replays_moved_view_lights(st):
    # the view lights live in the call's device view table, so a captured graph
    # replays with new lights exactly as a fresh, ungraphed call renders them
    sc = _colocated("edges", True)
    scene = st.Scene.from_scene(sc)
    a = scene.render(sc.views, 2, 9).clone()
    moved = S.with_view_lights(sc.views, intensity=(1.0, 2.0, 3.0), offset=0.8)
    b = scene.render(moved, 2, 9).clone()
    c = scene.render(moved, 2, 9, st.make_opts(use_graph=0)).clone()
    d = scene.render(moved, 2, 9, st.make_opts(mode="per_view")).clone()
    scene.close()
    assert not torch.equal(a, b)
    assert torch.equal(b, c) and torch.equal(b, d)


def test_view_light_limits_are_enforced(st):
    sc = _colocated("edges", True)
    scene = st.Scene.from_scene(sc)
    too_many = [dataclasses.replace(sc.views[0], lights=sc.views[0].lights * 2)]
    with pytest.raises(ValueError):
        scene.render(too_many, 2, 1)
    bad = [dataclasses.replace(sc.views[0], lights=(((0.0, 0.0, 0.0), (-1.0, 1.0, 1.0)),))]
    with pytest.raises(st.StError):
        scene.render(bad, 2, 1)
    scene.close()
