"""Point-light shadow-edge term on the GPU path against the FP64 oracle (same samples).

For every point light of every view the backward call samples the light's
shadow boundary on the surfaces the camera sees (ST_EDGE_TERM_SHADOW): an edge
that is a silhouette seen from the light, a point on it, the light ray through
it continued to the receiving surface, and camera paths on both sides of the
receiving point's image. Both sides pick the same edges and points by the same
integer map and counters.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2012_03939_gb300 import scenes as S
from tests.gpu_util import rel_l2
from tests.test_oracle_shadow_edges import _scene as _shadow_scene

pytestmark = pytest.mark.gpu

SH_REL = 2e-3


@pytest.fixture(scope="module")
def st():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_03939_gb300 import build
    build.build()
    from paper_2012_03939_gb300 import st as _st
    _st.lib()
    return _st


def _gpu(st, sc, B, seed, w, edge_term, **kw):
    scene = st.Scene.from_scene(sc)
    dV, dF = scene.backward(sc.views, B, seed, torch.from_numpy(w.astype(np.float32)).cuda(),
                            st.make_opts(edge_term=edge_term, **kw))
    assert scene.stats()["device_error"] == 0
    scene.close()
    return dV.cpu().numpy(), dF.cpu().numpy()


def _oracle(sc, B, seed, w, primary=False, edge_spp=0):
    osc = O.OracleScene(sc)
    prm = O.params(B, seed, edge_spp=edge_spp)
    dv, df, _ = O.grad_pixels(osc, prm, O.all_pixels(sc), w)
    sv, _ = O.shadow_edge_grad(osc, prm, w)
    if primary:
        dv = dv + O.edge_grad(osc, prm, w)[0]
    return dv + sv, df


def test_shadow_edges_match_oracle_on_the_pinned_scene(st):
    sc = _shadow_scene(spp=16)
    w = np.random.default_rng(4).normal(size=(sc.n_pixels, 3))
    dV, dF = _gpu(st, sc, 1, 12, w, st.EDGE_TERM_SHADOW)
    rv, rf = _oracle(sc, 1, 12, w)
    assert rel_l2([dV, dF], [rv, rf]) <= SH_REL
    dV0, _ = _gpu(st, sc, 1, 12, w, 0)
    # the term moves the occluder's gradient substantially (its shadow spans many pixels)
    assert np.abs(dV[4:] - dV0[4:]).max() > 0.1 * np.abs(dV[4:]).max()


def _sphere_on_floor(spp=4):
    """An icosphere floating over a floor under one light: its shadow falls on the floor and on itself."""
    V, F = S.icosphere(2)
    V = V * 0.45 + [0.0, 0.75, 0.0]
    floor = np.array([[-4, 0, -4], [4, 0, -4], [4, 0, 4], [-4, 0, 4]], np.float64)
    F2 = np.concatenate([F, np.array([[0, 2, 1], [0, 3, 2]]) + len(V)]).astype(np.int32)
    V2 = np.concatenate([V, floor]).astype(np.float32)
    rng = np.random.default_rng(11)
    vs = [S.View((2.4, 2.6, 2.2), (0.0, 0.3, 0.0), (0.0, 1.0, 0.0), 45.0, 32, 24, spp),
          S.View((-2.0, 2.8, 2.4), (0.0, 0.3, 0.0), (0.0, 1.0, 0.0), 45.0, 27, 32, spp)]
    sc = S.Scene("sphere_floor", V2, F2, S.random_face_params(rng, len(F2)), "ggx",
                 light_pos=np.array([[0.6, 2.6, 0.4]], np.float32), light_intensity=np.full((1, 3), 8.0, np.float32),
                 views=vs, max_bounces=2)
    return sc.subset_views(range(len(vs)))


@pytest.mark.parametrize("view_light", [False, True])
def test_shadow_edges_with_primary_edges_on_a_shadowing_mesh(st, view_light):
    sc = _sphere_on_floor()
    if view_light:
        sc.views = [dataclasses.replace(v, lights=(((-1.2, 2.0, 0.8), (4.0, 4.0, 4.0)),)) for v in sc.views]
    w = np.random.default_rng(5).normal(size=(sc.n_pixels, 3))
    dV, dF = _gpu(st, sc, 2, 31, w, st.EDGE_TERM_PRIMARY | st.EDGE_TERM_SHADOW)
    rv, rf = _oracle(sc, 2, 31, w, primary=True)
    assert rel_l2([dV, dF], [rv, rf]) <= SH_REL
    # the shadow term itself, on its own, against the oracle's
    d = dV - _gpu(st, sc, 2, 31, w, st.EDGE_TERM_PRIMARY)[0]
    sv, _ = O.shadow_edge_grad(O.OracleScene(sc), O.params(2, 31), w)
    assert np.abs(sv).max() > 0
    assert rel_l2([d], [sv]) <= 10 * SH_REL


def test_a_convex_mesh_casts_no_shadow_edge_on_itself(st):
    # the light grazes the sphere's light silhouette; the ray continued past it
    # leaves the sphere, and the edge's own faces are no receivers
    sc = S.small_variant(S.make("tiny"), n_views=2, max_res=32, spp=4)
    sc.light_pos = np.array([[0.3, 1.6, 0.9]], np.float32)
    w = np.random.default_rng(8).normal(size=(sc.n_pixels, 3))
    g0, _ = _gpu(st, sc, 2, 3, w, 0)
    g1, _ = _gpu(st, sc, 2, 3, w, st.EDGE_TERM_SHADOW)
    assert np.abs(g1 - g0).max() <= 1e-4 * np.abs(g0).max()


def test_shadow_edges_do_not_depend_on_the_launch_path(st):
    sc = S.small_variant(S.make("edges"), n_views=2, max_res=32, spp=2)
    w = np.random.default_rng(6).normal(size=(sc.n_pixels, 3))
    ref = _gpu(st, sc, 2, 8, w, st.EDGE_TERM_SHADOW)
    for kw in [dict(use_graph=0), dict(chunk_paths=1024), dict(mode="per_view")]:
        assert rel_l2(_gpu(st, sc, 2, 8, w, st.EDGE_TERM_SHADOW, **kw), ref) <= 1e-5, kw


def test_shadow_edges_in_a_binned_call_equal_the_views_traced_alone(st):
    # six views of a closed torus knot under a point light: together they pass
    # the 2^20 primary jobs that turn on the screen-space bins (back faces
    # culled), alone each stays below and traverses the BVH; the knot's loops
    # shadow one another, and every sample is the same in both
    sc = S.make("env")
    sc.light_pos = np.array([[0.4, 2.6, 1.2]], np.float32)
    sc.light_intensity = np.full((1, 3), 8.0, np.float32)
    sc.views = S.fibonacci_views(6, [160] * 6, [152] * 6, [4] * 6)
    w = np.random.default_rng(9).normal(size=(sc.n_pixels, 3)).astype(np.float32)
    scene = st.Scene.from_scene(sc)
    et = st.EDGE_TERM_PRIMARY | st.EDGE_TERM_SHADOW
    full = scene.backward(sc.views, 2, 17, torch.from_numpy(w).cuda(), st.make_opts(edge_term=et))
    sh_full = full[0] - scene.backward(sc.views, 2, 17, torch.from_numpy(w).cuda(),
                                       st.make_opts(edge_term=st.EDGE_TERM_PRIMARY))[0]
    dv = torch.zeros_like(full[0])
    df = torch.zeros_like(full[1])
    for v in sc.views:
        m = np.zeros_like(w)
        rows = slice(v.pixel_offset, v.pixel_offset + v.width * v.height)
        m[rows] = w[rows]
        a, b = scene.backward([v], 2, 17, torch.from_numpy(m).cuda(), st.make_opts(edge_term=et))
        dv += a
        df += b
    assert scene.stats()["device_error"] == 0
    scene.close()
    assert rel_l2([full[0].cpu().numpy(), full[1].cpu().numpy()], [dv.cpu().numpy(), df.cpu().numpy()]) <= 1e-5
    assert sh_full.abs().max() > 0.05 * full[0].abs().max()


def test_shadow_bit_adds_nothing_without_point_lights(st):
    # an environment-only scene has no point light to cast a shadow edge
    sc = S.small_variant(S.make("env"), n_views=1, max_res=24, spp=2)
    assert len(sc.light_pos) == 0
    w = np.random.default_rng(2).normal(size=(sc.n_pixels, 3))
    a = _gpu(st, sc, 2, 4, w, st.EDGE_TERM_PRIMARY | st.EDGE_TERM_SHADOW)
    b = _gpu(st, sc, 2, 4, w, st.EDGE_TERM_PRIMARY)
    assert rel_l2(a, b) <= 1e-6


def test_call_limits_on_views_and_shadow_pairs(st):
    # grids index views (and shadow (view, light) pairs) in their y dimension:
    # a call beyond the limit is refused before any launch
    sc = S.tiny(res=8, spp=1)
    scene = st.Scene.from_scene(sc)
    v = sc.views[0]
    many = [dataclasses.replace(v, width=1, height=1, pixel_offset=i) for i in range(65536)]
    w = torch.zeros((65536, 3), device="cuda")
    with pytest.raises(st.StError):
        scene.render(many, 1, 1)
    few = many[:40000]
    two = [dataclasses.replace(u, lights=(((0.0, 2.0, 0.0), (1.0, 1.0, 1.0)),)) for u in few]
    with pytest.raises(st.StError):     # 40000 views x (1 scene + 1 view light) pairs
        scene.backward(two, 1, 1, w, st.make_opts(edge_term=st.EDGE_TERM_SHADOW))
    scene.close()
