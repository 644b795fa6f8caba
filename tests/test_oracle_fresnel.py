"""Pins of the oracle's Fresnel option (Schlick's approximation with F0 = ks).

The paper's reflectance is a Torrance-Sparrow BRDF (Sec. 3.3 "Representation"),
whose specular lobe carries a Fresnel factor. The scene option fresnel = 1
takes Schlick's F = ks + (1 - ks)(1 - wi.h)^5; fresnel = 0 holds F at ks.
Each pin below holds for the definition whatever D and G are, so a mistake in
the factor (a wrong angle, a wrong power, F applied to the diffuse term, a
missing channel) fails one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2012_03939_gb300 import scenes as S
from tests.test_oracle_pins import _book_scene, _hemi_quad, _rand_dir


def _h(wi, wo):
    h = wi + wo
    return h / np.linalg.norm(h)


@pytest.mark.parametrize("brdf", [0, 1])
def test_schlick_brdf_is_reciprocal(brdf):
    rng = np.random.default_rng(40 + brdf)
    for _ in range(50):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        p5 = np.r_[rng.uniform(0.1, 0.9, 3), rng.uniform(0, 1), rng.uniform(0.05, 0.8)]
        a, b = _rand_dir(rng, n), _rand_dir(rng, n)
        np.testing.assert_allclose(O.brdf_eval(brdf, p5, n, a, b, fresnel=1),
                                   O.brdf_eval(brdf, p5, n, b, a, fresnel=1), rtol=1e-12)


@pytest.mark.parametrize("brdf", [0, 1])
def test_schlick_equals_held_form_at_normal_incidence(brdf):
    # wi = wo = n: h = n, wi.h = 1, F = ks: f = kd/pi + ks/(4 pi a^2) as without the option
    n = np.array([0.0, 0, 1])
    p5 = np.array([0.2, 0.4, 0.6, 0.3, 0.25])
    f = O.brdf_eval(brdf, p5, n, n, n, fresnel=1)
    np.testing.assert_allclose(f, p5[:3] / math.pi + p5[3] / (4 * math.pi * p5[4] ** 2), rtol=1e-12)


@pytest.mark.parametrize("brdf", [0, 1])
def test_schlick_factor_isolated_against_the_held_lobe(brdf):
    # kd = 0: with ks = 0 the lobe is (1 - wi.h)^5 D G / (4 ci co), with ks = 1 and F held it is
    # D G / (4 ci co); their ratio is (1 - wi.h)^5, wi.h computed here from the directions alone.
    # With ks = 1, F = 1 at every angle: Schlick equals the held lobe.
    rng = np.random.default_rng(7 + brdf)
    n = np.array([0.0, 0, 1])
    for _ in range(60):
        a, b = _rand_dir(rng, n), _rand_dir(rng, n)
        al = rng.uniform(0.05, 0.8)
        f0 = O.brdf_eval(brdf, np.array([0, 0, 0, 0.0, al]), n, a, b, fresnel=1)
        f1 = O.brdf_eval(brdf, np.array([0, 0, 0, 1.0, al]), n, a, b, fresnel=0)
        np.testing.assert_allclose(f0, f1 * (1.0 - a @ _h(a, b)) ** 5, rtol=1e-12, atol=1e-300)
        g = O.brdf_eval(brdf, np.array([0, 0, 0, 1.0, al]), n, a, b, fresnel=1)
        np.testing.assert_allclose(g, f1, rtol=1e-14)
        # per channel: F_c = ks_c + (1 - ks_c) x^5 with the diffuse term untouched
        p7 = np.array([0.3, 0.5, 0.7, 0.6, al])
        fs = O.brdf_eval(brdf, p7, n, a, b, fresnel=1)
        fh = O.brdf_eval(brdf, p7, n, a, b, fresnel=0)
        x5 = (1.0 - a @ _h(a, b)) ** 5
        lobe = f1                                   # D G / (4 ci co) in every channel
        np.testing.assert_allclose(fs - fh, (1 - 0.6) * x5 * lobe, rtol=1e-9, atol=1e-14)


def test_schlick_albedo_bounds():
    # F >= ks everywhere and F <= 1: the directional albedo lies between the held form's and 1,
    # and rises toward grazing view where (1 - wi.h) grows
    n = np.array([0.0, 0, 1])
    p5 = np.array([0.0, 0.0, 0.0, 0.5, 0.3])
    out = []
    for th in (0.2, 1.2, 1.45):
        wo = np.array([math.sin(th), 0.0, math.cos(th)])
        a_s = _hemi_quad(lambda wi: O.brdf_eval(0, p5, n, wi, wo, fresnel=1)[0] * wi[2], 96, 96)
        a_h = _hemi_quad(lambda wi: O.brdf_eval(0, p5, n, wi, wo, fresnel=0)[0] * wi[2], 96, 96)
        one = _hemi_quad(lambda wi: O.brdf_eval(0, np.array([0, 0, 0, 1.0, 0.3]), n, wi, wo)[0] * wi[2], 96, 96)
        assert a_h - 1e-12 <= a_s <= one + 1e-12 <= 1.0 + 1e-6
        out.append(a_s / a_h)
    assert out[0] < out[1] < out[2]


def _grazing_scene(ks, fresnel):
    # a triangle in z = 0 seen from a low camera on one side, lit by a low point light on the other:
    # wi and wo far apart, so 1 - wi.h is large
    V = np.array([[-0.8, -0.6, 0.0], [0.8, -0.6, 0.0], [0.0, 0.8, 0.0]], np.float32)
    F = np.array([[0, 1, 2]], np.int32)
    P = np.array([[0.0, 0.0, 0.0, ks, 0.35]], np.float32)
    vs = [S.View((0.0, -3.0, 0.8), (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), 30.0, 16, 16, 1)]
    sc = S.Scene("grazing", V, F, P, "ggx", light_pos=np.array([[0.0, 3.0, 0.6]], np.float32),
                 light_intensity=np.array([[1.0, 1.0, 1.0]], np.float32), views=vs, max_bounces=1)
    sc.fresnel = fresnel
    return sc


def test_schlick_factor_at_exact_screen_points():
    # direct light only (one vertex): L = F D G / (4 ci co) ci I / d^2 at every screen point the
    # triangle covers, so L(ks = 0, Schlick) / L(ks = 1, held) = (1 - wi.h)^5 with wi toward the
    # light and wo toward the eye from the hit point, both restated here from the camera model
    sc = _grazing_scene(0, 0)
    v = sc.views[0]
    # the scene's positions as the oracle receives them (float32 views and lights)
    e, t, up = (np.array(a, np.float32).astype(np.float64) for a in (v.eye, v.target, v.up))
    L = sc.light_pos[0].astype(np.float64)
    fwd = (t - e) / np.linalg.norm(t - e)
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    th = math.tan(math.radians(v.fov_y_deg) / 2)
    a = O.OracleScene(_grazing_scene(0.0, 1))
    b = O.OracleScene(_grazing_scene(1.0, 0))
    prm = O.params(1, 5)
    seen = 0
    for px in np.linspace(0.5, 15.5, 16):
        for py in np.linspace(0.5, 15.5, 31):
            d = fwd + right * (2 * px / v.width - 1) * th * v.width / v.height + upv * (1 - 2 * py / v.height) * th
            d /= np.linalg.norm(d)
            La = O.trace_screen(a, prm, 0, px, py)
            Lb = O.trace_screen(b, prm, 0, px, py)
            if Lb[0] <= 0:
                continue
            p = e + d * (-e[2] / d[2])
            wi = L - p
            wi /= np.linalg.norm(wi)
            x5 = (1.0 - wi @ _h(wi, -d)) ** 5
            np.testing.assert_allclose(La, Lb * x5, rtol=1e-10)
            seen += 1
    assert seen >= 40


@pytest.mark.parametrize("brdf,B", [("ggx", 1), ("ggx", 3), ("beckmann", 2)])
def test_schlick_gradient_matches_tape_replay_fd(brdf, B):
    # dual numbers through the Fresnel factor (it depends on the point-light direction, hence on the
    # hit point and the vertices, and on ks) against central differences of the taped estimator
    sc = _book_scene(brdf)
    sc.fresnel = 1
    V0 = sc.vertices.astype(np.float64)
    P0 = sc.face_params.astype(np.float64)
    prm = O.params(B, 4321)
    w = np.array([0.4, -0.6, 0.5])
    checked = 0
    for (px, py, c1) in [(5.3, 9.1, 0), (8.7, 11.2, 1), (10.1, 6.4, 2), (6.6, 12.8, 3)]:
        osc = O.OracleScene(sc, vertices=V0, face_params=P0)
        _, dv, df = O.trace_screen(osc, prm, 0, px, py, c0=13, c1=c1, grad_w=w)
        _, tape = O.trace_screen_taped(osc, prm, 0, px, py, c0=13, c1=c1)
        h = 1e-6
        for (vi, k) in [(i, k) for i in range(len(V0)) for k in range(3) if dv[i, k] != 0]:
            Vp, Vm = V0.copy(), V0.copy()
            Vp[vi, k] += h
            Vm[vi, k] -= h
            fp = O.trace_screen_taped(O.OracleScene(sc, vertices=Vp, face_params=P0), prm, 0, px, py, 13, c1, tape=tape)
            fm = O.trace_screen_taped(O.OracleScene(sc, vertices=Vm, face_params=P0), prm, 0, px, py, 13, c1, tape=tape)
            fd = (w @ fp - w @ fm) / (2 * h)
            assert abs(fd - dv[vi, k]) < 1e-5 * max(1.0, abs(fd)), (vi, k, fd, dv[vi, k])
            checked += 1
        for (fi, k) in [(i, k) for i in range(len(P0)) for k in range(5) if df[i, k] != 0]:
            Pp, Pm = P0.copy(), P0.copy()
            Pp[fi, k] += h
            Pm[fi, k] -= h
            fp = O.trace_screen_taped(O.OracleScene(sc, vertices=V0, face_params=Pp), prm, 0, px, py, 13, c1, tape=tape)
            fm = O.trace_screen_taped(O.OracleScene(sc, vertices=V0, face_params=Pm), prm, 0, px, py, 13, c1, tape=tape)
            fd = (w @ fp - w @ fm) / (2 * h)
            assert abs(fd - df[fi, k]) < 1e-5 * max(1.0, abs(fd)), (fi, k, fd, df[fi, k])
            checked += 1
    assert checked > 20
