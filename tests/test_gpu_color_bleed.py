"""The paper's colour-bleeding study (Sec. 3.3, "Effects of Global Illumination") on the GPU path.

Three intersecting planes with constant albedos (red wall, blue wall, white
floor) are rendered with global illumination as the target. Optimising one
albedo per plane from neutral gray through the path tracer recovers the white
floor with multi-bounce transport, while the one-bounce ("local + shadows")
renderer explains the red and blue light reflected onto the floor by baking a
purple tint into the floor's albedo -- the paper's qualitative finding.
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


def test_color_bleed_scene_matches_oracle(st):
    sc = S.color_bleed(res=24, spp=4)
    scene = st.Scene.from_scene(sc)
    img = scene.render(sc.views, 3, 8).cpu().numpy()
    w = np.random.default_rng(0).normal(size=img.shape)
    dV, dF = scene.backward(sc.views, 3, 8, torch.from_numpy(w.astype(np.float32)).cuda(), st.make_opts(edge_term=0))
    scene.close()
    osc = O.OracleScene(sc)
    ref, _ = O.render_pixels(osc, O.params(3, 8), O.all_pixels(sc))
    assert_image_parity(img, ref, what="color bleed")
    rv, rf, _ = O.grad_pixels(osc, O.params(3, 8), O.all_pixels(sc), w)
    assert rel_l2([dV.cpu().numpy(), dF.cpu().numpy()], [rv, rf]) <= GRAD_REL


def _recover_albedos(st, bounces, iters=70):
    sc = S.color_bleed(res=48, spp=16)
    plane = torch.from_numpy(sc.face_plane).cuda()
    scene = st.Scene.from_scene(sc)
    target = scene.render(sc.views, 3, 4242).clone()            # global illumination target
    V = torch.from_numpy(sc.vertices).cuda()
    rest = torch.tensor([0.0, 0.5], device="cuda").expand(len(sc.faces), 2)
    theta = torch.full((3, 3), 0.5, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([theta], lr=0.04)
    for it in range(iters):
        opt.zero_grad()
        P = torch.cat([theta[plane], rest], 1)
        img = st.render(V, P, scene, sc.views, bounces, 1000 + it, None, st.make_opts(edge_term=0))
        torch.mean((img - target) ** 2).backward()
        opt.step()
        with torch.no_grad():
            theta.clamp_(0.0, 1.0)
    scene.close()
    return theta.detach().cpu().numpy()


def test_global_illumination_disambiguates_color_bleeding(st):
    truth = np.array([[0.8, 0.1, 0.1], [0.1, 0.1, 0.8], [0.8, 0.8, 0.8]])
    gi = _recover_albedos(st, bounces=3)
    local = _recover_albedos(st, bounces=1)
    floor_gi, floor_local = gi[2], local[2]
    purple = lambda c: 0.5 * (c[0] + c[2]) - c[1]      # red + blue above green
    # multi-bounce recovers the white floor; one-bounce bakes the bleeding in
    assert np.abs(floor_gi - truth[2]).max() < 0.08, gi
    assert purple(floor_gi) < 0.04, gi
    assert purple(floor_local) > purple(floor_gi) + 0.04, (local, gi)
    assert np.abs(floor_local - truth[2]).max() > np.abs(floor_gi - truth[2]).max(), (local, gi)
