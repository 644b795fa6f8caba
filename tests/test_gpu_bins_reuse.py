"""Primary-visibility bins are built once per (vertices, views) and reused by later calls.

The leaf lists depend only on the vertices and on each view's camera frame, size
and bin-cell layout. A call whose views equal those of the last build, with no
vertex update since, tests the lists already on the device instead of building
them again (a forward render and the adjoint of the same views share one build).
Every such call must render bitwise what a scene building its lists afresh
renders, and a refit, a rebuild or a moved camera must build them again.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2012_03939_gb300 import scenes as S

pytestmark = pytest.mark.gpu

BIN_BUILD_LAUNCHES = 6   # fill, count, three scan stages, fill of the lists


@pytest.fixture(scope="module")
def st():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_03939_gb300 import build
    build.build()
    from paper_2012_03939_gb300 import st as _st
    _st.lib()
    return _st


def _render(scene, vs, B, seed):
    img = scene.render(vs, B, seed).cpu().numpy()
    s = scene.stats()
    assert s["device_error"] == 0
    return img, s["kernel_launches"]


def test_reused_bins_equal_fresh_builds(st):
    sc = S.make("batched")
    vs = S.fibonacci_views(3, [512, 384, 448], [512, 384, 320], [2, 2, 2])
    sc.views = vs
    assert sum(v.width * v.height * v.spp for v in vs) >= 1 << 20   # large enough to use the bins
    B, seed = 2, 17
    scene = st.Scene.from_scene(sc)
    a, la = _render(scene, vs, B, seed)
    b, lb = _render(scene, vs, B, seed)
    assert lb == la - BIN_BUILD_LAUNCHES          # the second call built nothing
    fresh = st.Scene.from_scene(sc)
    c, lc = _render(fresh, vs, B, seed)
    assert lc == la
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, c)
    # per-view calls (host-sized grids) and ungraphed calls reuse the same lists
    for opts in (st.make_opts(mode="per_view", use_graph=0), st.make_opts(use_graph=0)):
        pv = scene.render(vs, B, seed, opts).cpu().numpy()
        assert scene.stats()["device_error"] == 0
        np.testing.assert_array_equal(pv, a)

    # the adjoint of the same views reuses the forward's lists: same gradient as a scene that builds them
    g = torch.from_numpy(np.random.default_rng(5).normal(size=a.shape).astype(np.float32)).cuda()
    out = []
    for sc_ in (scene, fresh):
        dV = torch.zeros((sc_.nv, 3), device="cuda")
        sc_.backward(vs, B, seed, g, st.make_opts(edge_term=1), d_vertices=dV)
        out.append((dV.cpu().numpy(), sc_.stats()["kernel_launches"]))
    fresh.close()
    (dv_reused, l_reused), (dv_fresh, l_fresh) = out
    assert l_reused == l_fresh   # both scenes' lists match these views: neither builds
    np.testing.assert_allclose(dv_reused, dv_fresh, rtol=1e-4, atol=1e-5 * np.abs(dv_fresh).max())

    # a vertex update builds them again, and the image is that of a scene created with those vertices
    V2 = (sc.vertices * np.float32(1.03)).astype(np.float32)
    scene.refit(torch.from_numpy(V2).cuda())
    d, ld = _render(scene, vs, B, seed)
    assert ld == la
    moved = st.Scene.from_scene(sc, vertices=V2)
    e, _ = _render(moved, vs, B, seed)
    np.testing.assert_array_equal(d, e)
    assert not np.array_equal(a, d)

    # so does a moved camera
    vs2 = [dataclasses.replace(vs[0], eye=tuple(np.array(vs[0].eye, np.float64) * 1.01))] + vs[1:]
    f, lf = _render(scene, vs2, B, seed)
    assert lf == la
    h, _ = _render(moved, vs2, B, seed)
    np.testing.assert_array_equal(f, h)
    assert not np.array_equal(f[: vs[0].width * vs[0].height], d[: vs[0].width * vs[0].height])

    # and a rebuild of the tree (new leaf order) as well
    scene.rebuild(torch.from_numpy(V2).cuda())
    k, lk = _render(scene, vs2, B, seed)
    assert lk == la
    np.testing.assert_array_equal(k, h)
    moved.close()
    scene.close()
