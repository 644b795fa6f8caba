"""Chunks of a batched call overlapped on two engines and two streams.

Consecutive chunks alternate between two sets of wavefront buffers on two
streams; forward chunks resolve in order, so each pixel still adds its samples
in sample order. The images must be bitwise those of a call run chunk after
chunk on one stream (calls that time their kernels, and per-view calls, do not
overlap), for any chunk size, graphed or not; the counters of both engines add
up to the same ray counts; gradients agree up to the order of FP32 atomics.
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


def _scene(name):
    if name == "shadow_edges":
        from tests.test_gpu_shadow_edges import _sphere_on_floor
        return _sphere_on_floor()
    return S.small_variant(S.make(name), n_views=4, max_res=48, spp=4)


@pytest.mark.parametrize("name,B", [("batched", 3), ("env", 4), ("edges", 3)])
def test_overlapped_chunks_give_the_single_stream_image(st, name, B):
    sc = _scene(name)
    scene = st.Scene.from_scene(sc)
    sig0 = torch.zeros(sc.n_pixels, dtype=torch.int64, device="cuda")
    # one stream, one chunk after the other: the timed-kernel path never overlaps
    ref = scene.render(sc.views, B, 17, st.make_opts(use_graph=0, time_kernels=1, chunk_paths=2048),
                       signatures=sig0).cpu().numpy()
    ref_stats = scene.stats()
    for chunk in (2048, 4096, 1 << 20):
        for graph in (0, 1):
            sig = torch.zeros(sc.n_pixels, dtype=torch.int64, device="cuda")
            img = scene.render(sc.views, B, 17, st.make_opts(use_graph=graph, chunk_paths=chunk),
                               signatures=sig).cpu().numpy()
            stats = scene.stats()
            np.testing.assert_array_equal(img, ref)
            np.testing.assert_array_equal(sig.cpu().numpy(), sig0.cpu().numpy())
            for k in ("paths", "extension_rays", "shadow_rays"):
                assert stats[k] == ref_stats[k], (k, chunk, graph)
            assert stats["device_error"] == 0
    scene.close()


@pytest.mark.parametrize("name,B,term", [("batched", 3, 1), ("env", 4, 0), ("shadow_edges", 2, 5)])
def test_overlapped_chunks_give_the_single_stream_gradient(st, name, B, term):
    sc = _scene(name)
    scene = st.Scene.from_scene(sc)
    w = torch.from_numpy(np.random.default_rng(2).normal(size=(sc.n_pixels, 3)).astype(np.float32)).cuda()
    r0 = scene.backward(sc.views, B, 9, w, st.make_opts(use_graph=0, time_kernels=1, chunk_paths=2048, edge_term=term))
    s0 = scene.stats()
    ref = np.concatenate([x.cpu().numpy().ravel() for x in r0]).astype(np.float64)
    for chunk in (2048, 1 << 20):
        r1 = scene.backward(sc.views, B, 9, w, st.make_opts(use_graph=1, chunk_paths=chunk, edge_term=term))
        s1 = scene.stats()
        got = np.concatenate([x.cpu().numpy().ravel() for x in r1]).astype(np.float64)
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref), chunk
        for k in ("paths", "extension_rays", "shadow_rays", "edge_samples"):
            assert s1[k] == s0[k], (k, chunk)
        assert s1["device_error"] == 0
    scene.close()
