"""Autotuner and Adam driver on the GPU (through the C ABI)."""
import dataclasses
import os

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


def test_autotune_caches_and_keeps_the_image(st, tmp_path):
    from paper_2012_03939_gb300 import autotune
    sc = S.small_variant(S.batched(), n_views=4, max_res=48, spp=4)
    scene = st.Scene.from_scene(sc)
    cache = str(tmp_path / "tune.json")
    r1 = autotune.tune(scene, sc.views, 3, chunks=(4096, 1 << 16), persist=(0, 1), cache_path=cache, repeats=1)
    assert not r1["cached"] and len(r1["tried"]) == 4 and os.path.exists(cache)
    r2 = autotune.tune(scene, sc.views, 3, chunks=(4096, 1 << 16), persist=(0, 1), cache_path=cache)
    assert r2["cached"] and r2["chunk_paths"] == r1["chunk_paths"]
    tuned = scene.render(sc.views, 3, 5, st.make_opts(chunk_paths=r1["chunk_paths"],
                                                      persist_blocks=r1["persist_blocks"])).cpu().numpy()
    plain = scene.render(sc.views, 3, 5).cpu().numpy()
    scene.close()
    np.testing.assert_array_equal(tuned, plain)


def test_adam_recovers_material_and_resumes_from_checkpoint(st, tmp_path):
    from paper_2012_03939_gb300 import optimize as Opt
    sc = S.tiny(res=48, spp=8)
    sc.views = S.ring_views(4, 40, 8)
    true_P = sc.face_params.copy()
    targets = Opt.render_targets(sc, max_bounces=2)
    start_P = true_P.copy()
    start_P[:, :3] = np.clip(start_P[:, :3] + 0.25, 0, 1)
    scene = st.Scene.from_scene(sc)
    cfg = Opt.AdamConfig(max_bounces=2, minibatch=2, lr_vertices=0.0, lr_params=0.03, edge_term=1, seed=3)
    rec = Opt.Reconstruction(scene, sc.views, targets, torch.from_numpy(sc.vertices).cuda(),
                             torch.from_numpy(start_P).cuda(), cfg)

    def full_loss(P):
        scene.set_face_params(P)
        img = scene.render(sc.views, 2, 99)
        return float(torch.mean((img - targets) ** 2))

    l0 = full_loss(rec.P.detach())
    for _ in range(25):
        rec.step()
    l1 = full_loss(rec.P.detach())
    assert l1 < 0.5 * l0, (l0, l1)
    # checkpoint, take three steps, restore, take the same three steps
    ck = str(tmp_path / "ck.pt")
    rec.save(ck)
    for _ in range(3):
        rec.step()
    after = rec.P.detach().clone()
    rec.load(ck)
    for _ in range(3):
        rec.step()
    torch.testing.assert_close(rec.P.detach(), after, rtol=1e-5, atol=1e-6)
    scene.close()


def test_adam_with_rgb_specular_recovers_colour_and_keeps_roughness_in_range(st):
    # 7 parameters per texel (kd rgb, ks rgb, roughness): the step clamps by that layout
    from paper_2012_03939_gb300.optimize import clamp_params_
    from paper_2012_03939_gb300 import optimize as Opt
    sc = S.tiny(res=40, spp=8)
    sc.views = S.ring_views(4, 32, 8)
    P5 = sc.face_params
    rng = np.random.default_rng(21)
    true_P = np.c_[P5[:, :3], rng.uniform(0.02, 0.3, (len(P5), 3)), P5[:, 4]].astype(np.float32)
    sc.face_params = true_P
    targets = Opt.render_targets(sc, max_bounces=2)
    start = true_P.copy()
    start[:, :3] = np.clip(start[:, :3] + 0.25, 0, 1)
    start[:, 6] = 0.02                 # roughness near its lower bound: a 5-column clamp would leave it unclamped
    scene = st.Scene.from_scene(sc)
    assert scene.face_params.shape[1] == 7
    cfg = Opt.AdamConfig(max_bounces=2, minibatch=2, lr_vertices=0.0, lr_params=0.03, edge_term=1, seed=5)
    rec = Opt.Reconstruction(scene, sc.views, targets, torch.from_numpy(sc.vertices).cuda(),
                             torch.from_numpy(start).cuda(), cfg)

    def full_loss(P):
        scene.set_face_params(P)
        return float(torch.mean((scene.render(sc.views, 2, 99) - targets) ** 2))

    l0 = full_loss(rec.P.detach())
    for _ in range(25):
        rec.step()
        P = rec.P.detach()
        assert float(P[:, 6].min()) >= float(np.float32(0.01)) and float(P[:, 6].max()) <= 1.0
        assert float(P[:, :6].min()) >= 0.0 and float(P[:, :6].max()) <= 1.0
    l1 = full_loss(rec.P.detach())
    assert l1 < 0.5 * l0, (l0, l1)
    P = rec.P.detach().clone()
    assert torch.equal(clamp_params_(P.clone()), P)
    scene.close()


def test_refit_every_step_keeps_parity_with_a_fresh_scene(st):
    # vertex updates through the autograd wrapper refit the BVH; a scene built
    # from scratch on the same vertices renders the identical image
    sc = S.tiny(res=32, spp=2)
    scene = st.Scene.from_scene(sc)
    V = torch.from_numpy(sc.vertices).cuda()
    P = torch.from_numpy(sc.face_params).cuda()
    rng = np.random.default_rng(0)
    for k in range(3):
        V = V + torch.from_numpy(rng.normal(0, 0.01, sc.vertices.shape).astype(np.float32)).cuda()
        a = st.render(V, P, scene, sc.views, 2, 11 + k).cpu().numpy()
        fresh = st.Scene(V, torch.from_numpy(sc.faces).cuda(), P, light_pos=sc.light_pos,
                         light_intensity=sc.light_intensity)
        b = fresh.render(sc.views, 2, 11 + k).cpu().numpy()
        fresh.close()
        np.testing.assert_array_equal(a, b)
    scene.close()
