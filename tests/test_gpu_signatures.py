"""Path signatures: the GPU path and the oracle take the same discrete decisions.

Each path hashes its decisions (faces hit, environment texels drawn, BSDF lobes,
shadow-ray visibility) and each pixel sums its paths' hashes. Where the two
implementations' signatures agree they took the same decisions, so their values
may differ only by rounding: every pixel outside the image tolerance must have a
different signature (a decision that FP32 and FP64 took differently).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2012_03939_gb300 import scenes as S
from tests.gpu_util import PIX_ABS, PIX_REL

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


def _gpu(st, sc, B, seed, opts=None):
    scene = st.Scene.from_scene(sc)
    sig = torch.zeros(sc.n_pixels, dtype=torch.int64, device="cuda")
    img = scene.render(sc.views, B, seed, opts, signatures=sig).cpu().numpy()
    assert scene.stats()["device_error"] == 0
    scene.close()
    return img, sig.cpu().numpy().view(np.uint64)


def _scene(name):
    if name == "tiny":
        return S.tiny(res=32, spp=4)
    if name == "mesh_colors":
        # mesh colors at r = 3: the texel a hit picks is one of the hashed decisions
        sc = S.tiny(res=32, spp=4)
        r, n = 3, 10
        rng = np.random.default_rng(8)
        P = np.repeat(sc.face_params.astype(np.float64), n, axis=0)
        P[:, :3] = np.clip(P[:, :3] + rng.normal(0.0, 0.2, (len(P), 3)), 0.02, 0.98)
        sc.face_params = P.astype(np.float32)
        sc.color_res = r
        return sc
    return S.small_variant(S.make(name), n_views=2, max_res=32, spp=4)


@pytest.mark.parametrize("name,B", [("tiny", 2), ("edges", 3), ("env", 4), ("color_bleed", 3), ("mesh_colors", 3)])
def test_signatures_match_oracle_and_explain_every_value_difference(st, name, B):
    sc = _scene(name)
    img, sig = _gpu(st, sc, B, 61)
    osc = O.OracleScene(sc)
    pix = O.all_pixels(sc)
    ref_sig = O.render_signatures(osc, O.params(B, 61), pix)
    ref, _ = O.render_pixels(osc, O.params(B, 61), pix)
    same = sig == ref_sig
    assert same.mean() >= 0.999, same.mean()
    out = np.any(np.abs(img - ref) > PIX_REL * np.abs(ref) + PIX_ABS, axis=1)
    assert not np.any(out & same), np.flatnonzero(out & same)[:10]


def test_signatures_do_not_depend_on_the_launch_path(st):
    sc = S.small_variant(S.make("edges"), n_views=3, max_res=40, spp=3)
    ref = _gpu(st, sc, 3, 5)[1]
    for kw in [dict(use_graph=0), dict(mode="per_view"), dict(chunk_paths=1000)]:
        np.testing.assert_array_equal(_gpu(st, sc, 3, 5, st.make_opts(**kw))[1], ref)
