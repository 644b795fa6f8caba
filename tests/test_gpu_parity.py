"""GPU path (through the C ABI) against the FP64 oracle on identical seeded inputs."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2012_03939_gb300 import scenes as S
from tests.gpu_util import GRAD_REL, assert_image_parity, oracle_pixels, rel_l2, sample_pixels

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


def gpu_image(st, sc, B, seed, opts=None, vertices=None):
    scene = st.Scene.from_scene(sc, vertices=vertices)
    img = scene.render(sc.views, B, seed, opts).cpu().numpy()
    stats = scene.stats()
    scene.close()
    assert stats["device_error"] == 0
    return img, stats


def rows_of(sc, pix):
    return O.pixel_index(sc, pix)


# ---------------------------------------------------------------------------- BVH
def test_bvh_structure_is_valid(st):
    sc = S.edges()
    scene = st.Scene.from_scene(sc)
    nodes, leaf = scene.debug_bvh()
    F = len(sc.faces)
    assert sorted(leaf.tolist()) == list(range(F))
    V = sc.vertices
    tri = V[sc.faces[leaf]]                      # leaf order
    lo_t, hi_t = tri.min(1), tri.max(1)
    kids = nodes[:, 12:14].view(np.int32)
    seen_leaf = np.zeros(F, int)
    seen_node = np.zeros(F - 1, int)
    box = np.zeros((F - 1, 2, 2, 3), np.float32)   # node, child, lo/hi, xyz
    box[:, 0, 0] = nodes[:, [0, 2, 4]]
    box[:, 0, 1] = nodes[:, [1, 3, 5]]
    box[:, 1, 0] = nodes[:, [6, 8, 10]]
    box[:, 1, 1] = nodes[:, [7, 9, 11]]
    stack = [0]
    seen_node[0] = 1

    def subtree_box(c):
        if c < 0:
            return lo_t[~c], hi_t[~c]
        return np.minimum(box[c, 0, 0], box[c, 1, 0]), np.maximum(box[c, 0, 1], box[c, 1, 1])

    while stack:
        n = stack.pop()
        for k in range(2):
            c = kids[n, k]
            lo, hi = subtree_box(c)
            assert np.all(box[n, k, 0] <= lo) and np.all(box[n, k, 1] >= hi)
            if c < 0:
                seen_leaf[~c] += 1
            else:
                seen_node[c] += 1
                stack.append(c)
    assert np.all(seen_leaf == 1) and np.all(seen_node == 1)
    scene.close()


def test_refit_equals_rebuild_and_oracle(st):
    sc = S.tiny()
    rng = np.random.default_rng(3)
    V2 = (sc.vertices + rng.normal(0, 0.02, sc.vertices.shape)).astype(np.float32)
    scene = st.Scene.from_scene(sc)
    scene.refit(torch.from_numpy(V2).cuda())
    a = scene.render(sc.views, sc.max_bounces, 5).cpu().numpy()
    scene.rebuild(torch.from_numpy(V2).cuda())
    b = scene.render(sc.views, sc.max_bounces, 5).cpu().numpy()
    scene.close()
    np.testing.assert_array_equal(a, b)
    osc = O.OracleScene(sc, vertices=V2)
    ref, _ = O.render_pixels(osc, O.params(sc.max_bounces, 5), O.all_pixels(sc))
    assert_image_parity(a, ref, what="refit")


def test_closest_hit_matches_brute_force(st):
    for sc in (S.tiny(), S.edges()):
        rng = np.random.default_rng(11)
        n = 4000
        o = rng.normal(size=(n, 3))
        o = 3 * o / np.linalg.norm(o, axis=1, keepdims=True)
        d = rng.normal(size=(n, 3)) * 0.35 - o / 3
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        rays = np.zeros((n, 8), np.float32)
        rays[:, :3], rays[:, 4:7], rays[:, 7] = o, d, np.inf
        scene = st.Scene.from_scene(sc)
        tri, t = scene.trace_closest(torch.from_numpy(rays).cuda())
        tri, t = tri.cpu().numpy(), t.cpu().numpy()
        scene.close()
        r64 = np.c_[rays[:, :3], rays[:, 4:7], np.full(n, np.inf)].astype(np.float64)
        rt, tt = O.closest_hit(O.OracleScene(sc), r64)
        agree = tri == rt
        assert agree.mean() > 0.999, agree.mean()
        hit = agree & (rt >= 0)
        np.testing.assert_allclose(t[hit], tt[hit], rtol=2e-5, atol=1e-6)


# ---------------------------------------------------------------------------- forward
@pytest.mark.parametrize("brdf", ["ggx", "beckmann"])
def test_forward_tiny_full_image(st, brdf):
    sc = S.tiny()
    sc.brdf = brdf
    img, stats = gpu_image(st, sc, sc.max_bounces, 1234)
    ref, seg = O.render_pixels(O.OracleScene(sc), O.params(sc.max_bounces, 1234), O.all_pixels(sc))
    assert_image_parity(img, ref, what="tiny " + brdf)
    assert stats["extension_rays"] + stats["shadow_rays"] == seg   # identical ray-query count


@pytest.mark.parametrize("name,B", [("edges", 3), ("env", 4), ("batched", 3)])
def test_forward_small_variants_full_image(st, name, B):
    # oracle-sized: two views of ragged size (several 32-path warps and a ragged tail)
    sc = S.small_variant(S.make(name), n_views=2, max_res=26, spp=2)
    img, stats = gpu_image(st, sc, B, 77)
    ref, seg = O.render_pixels(O.OracleScene(sc), O.params(B, 77), O.all_pixels(sc))
    assert_image_parity(img, ref, what=name)
    assert abs(stats["extension_rays"] + stats["shadow_rays"] - seg) <= 2e-4 * seg


def test_batched_per_view_and_graph_agree_bitwise(st):
    sc = S.small_variant(S.batched(), n_views=5, max_res=40, spp=3)
    scene = st.Scene.from_scene(sc)
    imgs = []
    for opts in (st.make_opts(mode="batched", use_graph=1), st.make_opts(mode="batched", use_graph=0),
                 st.make_opts(mode="per_view"), st.make_opts(mode="batched", use_graph=1, chunk_paths=1000)):
        imgs.append(scene.render(sc.views, 3, 99, opts).cpu().numpy())
    # graph replay with a new seed equals an ungraphed call with that seed
    g2 = scene.render(sc.views, 3, 100, st.make_opts(use_graph=1)).cpu().numpy()
    u2 = scene.render(sc.views, 3, 100, st.make_opts(use_graph=0)).cpu().numpy()
    scene.close()
    for im in imgs[1:]:
        np.testing.assert_array_equal(imgs[0], im)
    np.testing.assert_array_equal(g2, u2)
    assert not np.array_equal(g2, imgs[0])


def test_graph_replay_writes_each_calls_output_and_rejects_overlaps(st):
    # one captured graph serves calls with different output tensors (the image
    # pointer is a per-call argument, not part of the graph)
    sc = S.small_variant(S.batched(), n_views=3, max_res=32, spp=2)
    scene = st.Scene.from_scene(sc)
    a = torch.full((sc.n_pixels, 3), 7.0, device="cuda")
    b = torch.full((sc.n_pixels, 3), -3.0, device="cuda")
    scene.render(sc.views, 3, 5, st.make_opts(use_graph=1), out=a)
    scene.render(sc.views, 3, 5, st.make_opts(use_graph=1), out=b)
    ref = scene.render(sc.views, 3, 5, st.make_opts(use_graph=0)).cpu().numpy()
    np.testing.assert_array_equal(a.cpu().numpy(), ref)
    np.testing.assert_array_equal(b.cpu().numpy(), ref)
    import dataclasses
    bad = [sc.views[0], dataclasses.replace(sc.views[1], pixel_offset=sc.views[0].width * sc.views[0].height - 5)]
    with pytest.raises(st.StError) as e:
        scene.render(bad, 3, 5)
    assert e.value.status == 1
    scene.close()


# ---------------------------------------------------------------------------- adjoint
def _grad_gpu(st, sc, B, seed, dLdI, opts):
    scene = st.Scene.from_scene(sc)
    dV, dF = scene.backward(sc.views, B, seed, torch.from_numpy(dLdI.astype(np.float32)).cuda(), opts)
    out = dV.cpu().numpy(), dF.cpu().numpy()
    assert scene.stats()["device_error"] == 0
    scene.close()
    return out


@pytest.mark.parametrize("brdf", ["ggx", "beckmann"])
def test_interior_gradient_tiny(st, brdf):
    sc = S.tiny()
    sc.brdf = brdf
    rng = np.random.default_rng(1)
    w = rng.normal(size=(sc.n_pixels, 3))
    dV, dF = _grad_gpu(st, sc, sc.max_bounces, 4321, w, st.make_opts(edge_term=0))
    rv, rf, _ = O.grad_pixels(O.OracleScene(sc), O.params(sc.max_bounces, 4321), O.all_pixels(sc), w)
    r = rel_l2([dV, dF], [rv, rf])
    assert r <= GRAD_REL, r


@pytest.mark.parametrize("name,B,npix", [("edges", 3, 0), ("env", 4, 0), ("scale", 5, 10)])
def test_interior_gradient_multibounce(st, name, B, npix):
    sc = S.small_variant(S.make(name), n_views=2, max_res=24, spp=2)
    rng = np.random.default_rng(2)
    pix = O.all_pixels(sc) if npix == 0 else sample_pixels(sc, npix, seed=1)
    w = np.zeros((sc.n_pixels, 3))
    w[rows_of(sc, pix)] = rng.normal(size=(len(pix), 3))
    dV, dF = _grad_gpu(st, sc, B, 55, w, st.make_opts(edge_term=0))
    rv, rf, _ = O.grad_pixels(O.OracleScene(sc), O.params(B, 55), pix, w[rows_of(sc, pix)])
    r = rel_l2([dV, dF], [rv, rf])
    assert r <= GRAD_REL, r


def test_interior_gradient_full_size_pixel_subset(st):
    # full-size displaced icosphere, 16 views: dL/dI nonzero on a sampled subset only
    sc = S.edges()
    pix = sample_pixels(sc, 64, seed=9)
    w = np.zeros((sc.n_pixels, 3))
    w[rows_of(sc, pix)] = np.random.default_rng(3).normal(size=(len(pix), 3))
    dV, dF = _grad_gpu(st, sc, sc.max_bounces, 8, w, st.make_opts(edge_term=0))
    rv, rf, _ = O.grad_pixels(O.OracleScene(sc), O.params(sc.max_bounces, 8), pix, w[rows_of(sc, pix)])
    r = rel_l2([dV, dF], [rv, rf])
    assert r <= GRAD_REL, r


@pytest.mark.parametrize("mode", [0, 1])
def test_edge_term_matches_oracle(st, mode):
    sc = S.tiny(res=48, spp=2)
    rng = np.random.default_rng(4)
    w = rng.normal(size=(sc.n_pixels, 3))
    opts_e = st.make_opts(edge_term=1, edge_mode=mode)
    opts_i = st.make_opts(edge_term=0)
    dVe, _ = _grad_gpu(st, sc, sc.max_bounces, 77, w, opts_e)
    dVi, _ = _grad_gpu(st, sc, sc.max_bounces, 77, w, opts_i)
    ev, _ = O.edge_grad(O.OracleScene(sc), O.params(sc.max_bounces, 77, edge_mode=mode), w)
    r = rel_l2([dVe - dVi], [ev])
    assert r <= 5e-3, r


def test_edge_plus_interior_matches_gpu_finite_differences(st):
    # every edge sampled, B = 1: mean over seeds of <grad, delta> vs central
    # differences of high-spp renders with common random numbers, within 3 sigma
    sc = S.tiny(res=32, spp=256)
    sc.max_bounces = 1
    rng = np.random.default_rng(6)
    delta = rng.normal(size=sc.vertices.shape)
    w = rng.normal(size=(sc.n_pixels, 3)).astype(np.float32)
    scene = st.Scene.from_scene(sc)
    V0 = torch.from_numpy(sc.vertices).cuda()
    D = torch.from_numpy(delta.astype(np.float32)).cuda()
    wt = torch.from_numpy(w).cuda()
    h = 1e-3
    g, f = [], []
    for seed in range(10):
        scene.refit(V0)
        dV, _ = scene.backward(sc.views, 1, seed, wt, st.make_opts(edge_term=1, edge_mode=1, edge_spp=64))
        g.append(float((dV * D).sum()))
        scene.refit(V0 + h * D)
        ip = scene.render(sc.views, 1, 1000 + seed)
        scene.refit(V0 - h * D)
        im = scene.render(sc.views, 1, 1000 + seed)
        f.append(float(((ip - im) * wt).sum()) / (2 * h))
    scene.close()
    g, f = np.array(g), np.array(f)
    se = math.sqrt(g.var(ddof=1) / len(g) + f.var(ddof=1) / len(f))
    assert abs(g.mean() - f.mean()) <= 3 * se + 1e-3 * abs(f.mean()), (g.mean(), f.mean(), se)


def test_autograd_function_matches_direct_calls(st):
    sc = S.tiny(res=20, spp=2)
    scene = st.Scene.from_scene(sc)
    V = torch.from_numpy(sc.vertices).cuda().requires_grad_(True)
    P = torch.from_numpy(sc.face_params).cuda().requires_grad_(True)
    target = torch.zeros((sc.n_pixels, 3), device="cuda")
    img = st.render(V, P, scene, sc.views, 2, 31, None, st.make_opts(edge_term=1))
    loss = ((img - target) ** 2).mean()
    loss.backward()
    gI = 2 * (img.detach() - target) / img.numel()
    dV, dF = scene.backward(sc.views, 2, 31, gI, st.make_opts(edge_term=1))
    torch.testing.assert_close(V.grad, dV, rtol=1e-4, atol=1e-6)
    torch.testing.assert_close(P.grad, dF, rtol=1e-4, atol=1e-6)
    scene.close()


# ---------------------------------------------------------------------------- errors
def test_invalid_inputs_are_rejected(st):
    sc = S.tiny()
    scene = st.Scene.from_scene(sc)
    bad = [S.View((0, 0, 3), (0, 0, 3), (0, 1, 0), 45.0, 8, 8, 1),      # eye == target
           S.View((0, 0, 3), (0, 0, 0), (0, 1, 0), 45.0, 0, 8, 1),      # empty view
           S.View((0, 0, 3), (0, 0, 0), (0, 1, 0), 45.0, 8, 8, -1)]     # negative spp
    for v in bad:
        with pytest.raises(st.StError) as e:
            scene.render([v], 2, 1)
        assert e.value.status == 1
    with pytest.raises(st.StError) as e:
        scene.render(sc.views, 9, 1)
    assert e.value.status == 6
    F = torch.from_numpy(sc.faces.copy()).cuda()
    F[0, 0] = 10 ** 6
    with pytest.raises(st.StError):
        st.Scene(torch.from_numpy(sc.vertices).cuda(), F, torch.from_numpy(sc.face_params).cuda(),
                 light_pos=sc.light_pos, light_intensity=sc.light_intensity)
    V = torch.from_numpy(sc.vertices.copy()).cuda()
    V[3, 1] = float("nan")
    with pytest.raises(st.StError):
        st.Scene(V, torch.from_numpy(sc.faces).cuda(), torch.from_numpy(sc.face_params).cuda(),
                 light_pos=sc.light_pos, light_intensity=sc.light_intensity)
    scene.close()


def test_empty_and_degenerate_views(st):
    sc = S.tiny()
    scene = st.Scene.from_scene(sc)
    # a view looking away from the mesh renders black; a 1x1 view works
    away = S.View((0, 0, 3), (0, 0, 6), (0, 1, 0), 45.0, 7, 5, 2, 0)
    one = S.View((0, 0, 3), (0, 0, 0), (0, 1, 0), 45.0, 1, 1, 3, 35)
    img = scene.render([away, one], 2, 3).cpu().numpy()
    assert np.all(img[:35] == 0)
    ref = oracle_pixels(S.Scene("t", sc.vertices, sc.faces, sc.face_params, light_pos=sc.light_pos,
                                light_intensity=sc.light_intensity, views=[away, one]), 2, 3,
                        np.array([[1, 0, 0]], np.int32))
    assert_image_parity(img[35:36], ref, what="1x1")
    scene.close()


def test_primary_bins_and_bvh_fallback_views(st):
    # one view outside the mesh (primary rays use the screen-space bins) and one
    # inside it, where triangles straddle the eye plane and the view's primary
    # rays fall back to the BVH; both match the oracle
    # over 2^20 primary rays, so the library builds the bins (at ordinary spp: the
    # per-pixel check assumes few samples per pixel, as in the workloads)
    sc = S.tiny()
    out = S.View((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 45.0, 384, 360, 4, 0)
    inside = S.View((0.1, 0.2, 0.3), (0.0, 0.0, -2.0), (0.0, 1.0, 0.0), 90.0, 370, 352, 4, 384 * 360)
    sc.views = [out, inside]
    sc.light_pos = np.array([[0.0, 0.0, 0.0], [0.0, 2.1, 2.1]], np.float32)
    sc.light_intensity = np.array([[0.5, 0.5, 0.5], [9.0, 9.0, 9.0]], np.float32)
    img, stats = gpu_image(st, sc, 2, 41)
    ref, seg = O.render_pixels(O.OracleScene(sc), O.params(2, 41), O.all_pixels(sc))
    assert_image_parity(img, ref, what="bins + fallback")
    assert stats["extension_rays"] + stats["shadow_rays"] == seg


@pytest.mark.parametrize("name,npix,views", [("batched", 256, None), ("scale", 64, 8)])
def test_full_size_gradient_in_bench_configuration(st, name, npix, views):
    # the benchmark's launch configuration (batched, CUDA graph, 16M-path chunks as the autotuner
    # picks for these workloads, silhouette edge term) at full size; dL/dI nonzero on a pixel
    # sample so the oracle can follow
    sc = S.make(name)
    if views:
        sc = sc.subset_views(range(views))
    pix = sample_pixels(sc, npix, seed=13)
    rows = rows_of(sc, pix)
    w = np.zeros((sc.n_pixels, 3))
    w[rows] = np.random.default_rng(14).normal(size=(len(pix), 3))
    opts = st.make_opts(mode="batched", use_graph=1, chunk_paths=1 << 24, edge_term=1, edge_mode=0)
    dV, dF = _grad_gpu(st, sc, sc.max_bounces, 2025, w, opts)
    osc = O.OracleScene(sc)
    prm = O.params(sc.max_bounces, 2025, edge_mode=0)
    rv, rf, _ = O.grad_pixels(osc, prm, pix, w[rows])
    ev, _ = O.edge_grad(osc, prm, w)
    r_int = rel_l2([dF], [rf])                      # parameters: interior term only
    r_tot = rel_l2([dV, dF], [rv + ev, rf])         # vertices: interior + edge term
    assert r_int <= GRAD_REL, r_int
    assert r_tot <= 5e-3, r_tot


@pytest.mark.parametrize("n_faces", [1, 2])
def test_one_and_two_triangle_scenes(st, n_faces):
    # the smallest meshes: a single face (no internal node: traversal tests the one
    # leaf, the 4-wide tree is empty) and two faces sharing an edge (one internal
    # node); every edge is a boundary edge except the shared one. Image, interior
    # gradient and edge term against the oracle; a refit equals a fresh scene.
    V = np.array([[-0.8, -0.6, 0.0], [0.7, -0.7, 0.1], [0.6, 0.8, 0.0], [-0.7, 0.7, -0.1]], np.float32)
    F = np.array([[0, 1, 2], [0, 2, 3]], np.int32)[:n_faces]
    P = np.array([[0.7, 0.5, 0.3, 0.04, 0.3], [0.2, 0.6, 0.8, 0.04, 0.5]], np.float32)[:n_faces]
    views = [S.View((0.2, -0.3, 3.0), (0.0, 0.0, 0.0), (0, 1, 0), 45.0, 24, 20, 4, 0),
             S.View((-1.5, 0.4, 2.2), (0.0, 0.1, 0.0), (0, 1, 0), 50.0, 16, 16, 3, 480)]
    sc = S.Scene("tri%d" % n_faces, V, F, P, light_pos=np.array([[0.3, 0.5, 2.0]], np.float32),
                 light_intensity=np.array([[6.0, 6.0, 6.0]], np.float32), views=views, max_bounces=2)
    img, stats = gpu_image(st, sc, 2, 19)
    ref, seg = O.render_pixels(O.OracleScene(sc), O.params(2, 19), O.all_pixels(sc))
    assert_image_parity(img, ref, what="%d face(s)" % n_faces)
    assert stats["extension_rays"] + stats["shadow_rays"] == seg
    assert img.max() > 0.0

    w = np.random.default_rng(20).normal(size=(sc.n_pixels, 3))
    dVi, dFi = _grad_gpu(st, sc, 2, 19, w, st.make_opts(edge_term=0))
    rv, rf, _ = O.grad_pixels(O.OracleScene(sc), O.params(2, 19), O.all_pixels(sc), w)
    r = rel_l2([dVi, dFi], [rv, rf])
    assert r <= GRAD_REL, r
    dVe, _ = _grad_gpu(st, sc, 2, 19, w, st.make_opts(edge_term=1, edge_mode=0))
    ev, _ = O.edge_grad(O.OracleScene(sc), O.params(2, 19, edge_mode=0), w)
    assert np.abs(ev).max() > 0.0
    r = rel_l2([dVe - dVi], [ev])
    assert r <= 5e-3, r

    V2 = V + np.float32(0.05) * np.random.default_rng(21).normal(size=V.shape).astype(np.float32)
    scene = st.Scene.from_scene(sc)
    scene.refit(torch.from_numpy(V2).cuda())
    refit = scene.render(views, 2, 19).cpu().numpy()
    scene.close()
    fresh, _ = gpu_image(st, sc, 2, 19, vertices=V2)
    np.testing.assert_array_equal(refit, fresh)


def test_maximum_bounces_and_lights(st):
    # ST_MAX_BOUNCES (8) vertices per path and ST_MAX_LIGHTS (8) point lights per path, six of the scene's
    # and two of each view's own, on the concave three-plane scene where paths keep bouncing between the
    # walls: image (with path signatures) and interior gradient against the oracle
    sc = S.small_variant(S.make("color_bleed"), n_views=2, max_res=20, spp=2)
    rng = np.random.default_rng(30)
    sc.light_pos = rng.uniform(0.3, 1.8, size=(6, 3)).astype(np.float32)   # inside the open corner
    sc.light_intensity = rng.uniform(0.5, 2.0, size=(6, 3)).astype(np.float32)
    sc.views = S.with_view_lights(sc.views, intensity=(1.5, 1.5, 1.5))
    B = 8
    scene = st.Scene.from_scene(sc)
    sig = torch.zeros(sc.n_pixels, dtype=torch.int64, device="cuda")
    img = scene.render(sc.views, B, 23, signatures=sig).cpu().numpy()
    stats = scene.stats()
    assert stats["device_error"] == 0
    scene.close()
    osc = O.OracleScene(sc)
    pix = O.all_pixels(sc)
    ref, seg = O.render_pixels(osc, O.params(B, 23), pix)
    assert_image_parity(img, ref, what="B = 8, 8 lights")
    assert stats["extension_rays"] + stats["shadow_rays"] == seg
    same = sig.cpu().numpy().view(np.uint64) == O.render_signatures(osc, O.params(B, 23), pix)
    assert same.mean() >= 0.999, same.mean()
    w = rng.normal(size=(sc.n_pixels, 3))
    dV, dF = _grad_gpu(st, sc, B, 23, w, st.make_opts(edge_term=0))
    rv, rf, _ = O.grad_pixels(osc, O.params(B, 23), pix, w)
    r = rel_l2([dV, dF], [rv, rf])
    assert r <= GRAD_REL, r


def test_many_small_views_in_one_call(st):
    # 5000 views of 2 x 3 pixels (uneven spp, some with their own lights, the widest view 1 x 1) in one
    # batched, graph-captured call: 5000+ job segments, each a few jobs, found by every job's segment
    # search; every pixel against the oracle, and the gradient on a pixel sample
    sc = S.tiny()
    n = 5000
    rng = np.random.default_rng(40)
    vs = S.fibonacci_views(n, np.full(n, 2), np.full(n, 3), rng.choice([1, 2, 3], size=n), fov=20.0)
    vs[7] = S.View(vs[7].eye, vs[7].target, vs[7].up, 20.0, 1, 1, 4)
    S._pack_offsets(vs)
    vs[::97] = S.with_view_lights(vs[::97], intensity=(2.0, 2.0, 2.0))
    sc.views = vs
    img, stats = gpu_image(st, sc, 2, 29)
    ref, seg = O.render_pixels(O.OracleScene(sc), O.params(2, 29), O.all_pixels(sc))
    assert_image_parity(img, ref, what="5000 views")
    assert stats["extension_rays"] + stats["shadow_rays"] == seg
    pix = sample_pixels(sc, 400, seed=41)
    w = np.zeros((sc.n_pixels, 3))
    w[rows_of(sc, pix)] = rng.normal(size=(len(pix), 3))
    dV, dF = _grad_gpu(st, sc, 2, 29, w, st.make_opts(edge_term=0))
    rv, rf, _ = O.grad_pixels(O.OracleScene(sc), O.params(2, 29), pix, w[rows_of(sc, pix)])
    r = rel_l2([dV, dF], [rv, rf])
    assert r <= GRAD_REL, r
