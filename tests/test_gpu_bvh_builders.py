"""The two tree builders: PLOC clustering (default) and the Karras radix tree.

Both order the leaves by Morton code; PLOC merges mutual nearest neighbours by
merged-box surface area in a window of that order (Meister and Bittner 2018),
which gives trees of lower surface-area cost. The trees differ, the closest hits
do not: the traversal's result is the closest t with the lower face id on ties,
whatever the tree.
"""
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


def _tree(scene):
    nodes, leaf = scene.debug_bvh()
    kids = nodes[:, 12:14].copy().view(np.int32)
    lo = np.minimum(nodes[:, [0, 2, 4]], nodes[:, [6, 8, 10]])
    hi = np.maximum(nodes[:, [1, 3, 5]], nodes[:, [7, 9, 11]])
    return nodes, leaf, kids, lo, hi


def _check_tree(nodes, leaf, kids, lo, hi, V, Fc):
    F = len(Fc)
    assert sorted(leaf.tolist()) == list(range(F))
    tri = V[Fc[leaf]]
    tlo, thi = tri.min(1), tri.max(1)
    # every node but the root and every leaf has exactly one parent
    refs = kids.ravel()
    assert sorted(refs[refs >= 0].tolist()) == list(range(1, F - 1))
    assert sorted((~refs[refs < 0]).tolist()) == list(range(F))
    # child boxes contain their subtrees
    for k in range(2):
        c = kids[:, k]
        blo = nodes[:, [0, 2, 4]] if k == 0 else nodes[:, [6, 8, 10]]
        bhi = nodes[:, [1, 3, 5]] if k == 0 else nodes[:, [7, 9, 11]]
        leafc = (c < 0)[:, None]
        sub_lo = np.where(leafc, tlo[np.where(c < 0, ~c, 0)], lo[np.where(c >= 0, c, 0)])
        sub_hi = np.where(leafc, thi[np.where(c < 0, ~c, 0)], hi[np.where(c >= 0, c, 0)])
        assert np.all(blo <= sub_lo) and np.all(bhi >= sub_hi)


def _sah(lo, hi):
    d = np.maximum(hi - lo, 0).astype(np.float64)
    a = d[:, 0] * d[:, 1] + d[:, 1] * d[:, 2] + d[:, 2] * d[:, 0]
    return a.sum() / a[0]


@pytest.mark.parametrize("workload", ["edges", "env", "batched"])
def test_ploc_tree_is_valid_and_cheaper_than_the_radix_tree(st, workload):
    sc = S.make(workload)
    cost = {}
    for b in ("ploc", "lbvh"):
        scene = st.Scene.from_scene(sc, bvh_builder=b)
        nodes, leaf, kids, lo, hi = _tree(scene)
        _check_tree(nodes, leaf, kids, lo, hi, sc.vertices, sc.faces)
        cost[b] = _sah(lo, hi)
        assert scene.stats()["device_error"] == 0
        scene.close()
    assert cost["ploc"] < 0.97 * cost["lbvh"], cost


def test_builders_give_identical_hits_and_images(st):
    sc = S.small_variant(S.make("env"), n_views=2, max_res=64, spp=2)
    rng = np.random.default_rng(4)
    n = 1 << 16
    o = rng.uniform(-1.2, 1.2, (n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = torch.from_numpy(np.c_[o, np.zeros(n), d, np.full(n, 1e30)].astype(np.float32)).cuda()
    out = {}
    for b in ("ploc", "lbvh"):
        scene = st.Scene.from_scene(sc, bvh_builder=b)
        tri, t = scene.trace_closest(rays)
        img = scene.render(sc.views, 3, 12)
        out[b] = (tri.cpu().numpy(), t.cpu().numpy(), img.cpu().numpy())
        scene.close()
    assert (out["ploc"][0] >= 0).mean() > 0.1
    for k in range(3):
        np.testing.assert_array_equal(out["ploc"][k], out["lbvh"][k])


def test_ploc_rebuild_after_moving_vertices(st):
    sc = S.make("edges")
    rng = np.random.default_rng(5)
    V2 = (sc.vertices + rng.normal(0, 0.01, sc.vertices.shape)).astype(np.float32)
    scene = st.Scene.from_scene(sc)
    scene.rebuild(torch.from_numpy(V2).cuda())
    nodes, leaf, kids, lo, hi = _tree(scene)
    _check_tree(nodes, leaf, kids, lo, hi, V2, sc.faces)
    assert scene.stats()["device_error"] == 0
    scene.close()
