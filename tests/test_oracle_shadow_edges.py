"""Pin of the oracle's shadow-edge term (point-light shadows on surfaces the camera sees).

A point light's shadow on a visible floor ends where light rays graze the
occluder's silhouette edges; the image integral over a pixel is discontinuous
across the projected boundary, and moving the occluder or the floor moves it.
Closed form: a Lambertian floor plane lit by one point light, shadowed by a
floating triangle. The shadow is the triangle's projection from the light onto
the floor, whose image is a triangle T_S, so every pixel value is the integral
of the smooth lit radiance over (pixel minus T_S): polygon clipping and Gauss
quadrature evaluate it to high accuracy, and central differences give the
derivative with respect to each occluder vertex and to a translation of the
floor, against which the estimator (interior term + shadow-edge term) is tested.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2012_03939_gb300 import scenes as S
from tests import _geom as G

KD = np.array([0.7, 0.5, 0.3])
LIGHT = np.array([0.4, 2.0, 0.3])
INTENSITY = 5.0


def _scene(spp=1):
    V = np.array([[-10, 0, -10], [10, 0, -10], [10, 0, 10], [-10, 0, 10],
                  [-0.30, 0.50, -0.20], [0.35, 0.55, -0.10], [0.00, 0.52, 0.35]], np.float64)
    F = np.array([[0, 2, 1], [0, 3, 2], [4, 5, 6]], np.int32)
    P = np.array([np.r_[KD, 0.0, 0.5]] * 2 + [[0.5, 0.5, 0.5, 0.0, 0.5]], np.float32)
    vs = [S.View((1.6, 2.4, 2.2), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 40.0, 16, 16, spp)]
    return S.Scene("shadow", V.astype(np.float32), F, P, "ggx", light_pos=np.array([LIGHT], np.float32),
                   light_intensity=np.full((1, 3), INTENSITY, np.float32), views=vs, max_bounces=1)


def _rays(v, pts):
    """Eye and unit directions through screen points [n, 2] (the pinhole model of _geom, vectorised)."""
    eye, fwd, right, up, th = G.camera_frame(v)
    pts = np.asarray(pts, np.float64)
    sx = 2 * pts[:, 0] / v.width - 1
    sy = 1 - 2 * pts[:, 1] / v.height
    d = fwd[None, :] + right[None, :] * (sx * th * v.width / v.height)[:, None] + up[None, :] * (sy * th)[:, None]
    return eye, d / np.linalg.norm(d, axis=1, keepdims=True)


def _h(v, V, pts):
    """Lit radiance at screen points: camera ray onto the floor plane y = V[0,1], Lambertian under the light."""
    eye, d = _rays(v, pts)
    yf = V[0, 1]
    t = (yf - eye[1]) / d[:, 1]
    p = eye + d * t[:, None]
    wl = LIGHT - p
    dist = np.linalg.norm(wl, axis=1)
    cos = np.maximum(wl[:, 1] / dist, 0.0)
    return np.outer(cos / dist ** 2 * INTENSITY / math.pi, KD)


def _pixel_values(sc, V, pix):
    v = sc.views[0]
    yf = V[0, 1]
    # shadow of the occluder on the floor plane, then its image (a triangle)
    occ = V[4:7]
    s = (LIGHT[1] - yf) / (LIGHT[1] - occ[:, 1])
    shadow = LIGHT + (occ - LIGHT) * s[:, None]
    T = G.project(v, shadow)
    out = np.zeros((len(pix), 3))
    for i, (_, x, y) in enumerate(pix):
        sq = np.array([[x, y], [x + 1, y], [x + 1, y + 1], [x, y + 1]], np.float64)
        p_all, w_all = G.polygon_quadrature(sq, subdiv=2)
        full = w_all @ _h(v, V, p_all)
        C = G.clip_polygon(T, x, y, x + 1, y + 1)
        if len(C) >= 3:
            p_s, w_s = G.polygon_quadrature(np.array(C), subdiv=2)
            full = full - w_s @ _h(v, V, p_s)
        out[i] = full
    return out


def _pixels(sc):
    v = sc.views[0]
    V = sc.vertices.astype(np.float64)
    occ_img = G.project(v, V[4:7])
    out = []
    for y in range(v.height):
        for x in range(v.width):
            if len(G.clip_polygon(occ_img, x - 0.05, y - 0.05, x + 1.05, y + 1.05)) < 3:
                out.append((0, x, y))
    return np.array(out, np.int32)


def test_closed_form_shadowed_floor_value():
    spp = 4096
    sc = _scene(spp)
    pix = _pixels(sc)[::6]
    exp = _pixel_values(sc, sc.vertices.astype(np.float64), pix)
    got, _ = O.render_pixels(O.OracleScene(sc), O.params(1, 2), pix)
    # per-sample values are 0 or h (smooth): binomial spread within the pixel
    se = exp.max() / math.sqrt(spp)
    assert np.all(np.abs(got - exp) < 4 * se + 1e-6 * exp.max()), (got, exp)
    assert (exp[:, 0] < 0.5 * exp[:, 0].max()).any() and (exp[:, 0] > 0.9 * exp[:, 0].max()).any()


def test_shadow_edge_gradient_matches_closed_form():
    sc = _scene(spp=64)
    pix = _pixels(sc)
    rows = O.pixel_index(sc, pix)
    V0 = sc.vertices.astype(np.float64)
    rng = np.random.default_rng(41)
    w = rng.normal(size=(len(pix), 3))
    wfull = np.zeros((sc.n_pixels, 3))
    wfull[rows] = w
    h = 1e-5
    # directions: the nine occluder coordinates and a translation of the whole floor along y
    dirs = []
    for vi in range(4, 7):
        for k in range(3):
            D = np.zeros_like(V0)
            D[vi, k] = 1.0
            dirs.append(D)
    D = np.zeros_like(V0)
    D[0:4, 1] = 1.0
    dirs.append(D)
    exp = np.array([((_pixel_values(sc, V0 + h * D, pix) - _pixel_values(sc, V0 - h * D, pix)) * w).sum() / (2 * h)
                    for D in dirs])
    osc = O.OracleScene(sc)
    ests = []
    for seed in range(8):
        prm = O.params(1, 600 + seed, edge_spp=64)
        dv, _, _ = O.grad_pixels(osc, prm, pix, w)
        sv, _ = O.shadow_edge_grad(osc, prm, wfull)
        ests.append([((dv + sv) * D).sum() for D in dirs])
    ests = np.array(ests)
    mean, se = ests.mean(0), ests.std(0, ddof=1) / math.sqrt(len(ests))
    scale = np.abs(exp).max()
    assert np.all(np.abs(mean - exp) < 4 * se + 2e-3 * scale), (mean, exp, se)
    # without the shadow-edge term the occluder receives no gradient at all
    plain = np.array([(O.grad_pixels(osc, O.params(1, 600), pix, w)[0] * D).sum() for D in dirs[:9]])
    assert np.all(plain == 0) and np.abs(exp[:9]).max() > 0.2 * scale


def test_a_convex_mesh_receives_no_shadow_edge_from_itself():
    # a line through a point of a convex surface's light silhouette touches the
    # surface there only: no receiver, so the term is exactly zero, for lights
    # near and far (a near light makes the light rays graze the edge's faces)
    sc = S.small_variant(S.make("tiny"), n_views=1, max_res=24, spp=2)
    w = np.random.default_rng(2).normal(size=(sc.n_pixels, 3))
    for L in ([0.3, 1.6, 0.9], [0.0, 1.2, 0.0], [2.0, 0.0, -3.0]):
        sc.light_pos = np.array([L], np.float32)
        sv, _ = O.shadow_edge_grad(O.OracleScene(sc), O.params(1, 5), w)
        assert np.all(sv == 0)


# ---------------------------------------------------------------------------- tilted receiver
# The same construction on a floor tilted about two axes, so the receiver's
# normal has no zero component: the shadow is the occluder projected from the
# light onto the tilted plane, and the directions include a rigid rotation of
# the floor (its normal turns) as well as its translation along the normal.
def _rot(ax, ay, az):
    cx, sx, cy, sy, cz, sz = math.cos(ax), math.sin(ax), math.cos(ay), math.sin(ay), math.cos(az), math.sin(az)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def _tilted_scene(spp=1):
    sc = _scene(spp)
    V = sc.vertices.astype(np.float64)
    V[:4] = V[:4] @ _rot(0.25, 0.1, -0.18).T
    sc.vertices = V.astype(np.float32)
    return sc


def _plane(V):
    """Point and unit normal of the floor (faces (0, 2, 1) and (0, 3, 2) wind upward)."""
    n = np.cross(V[1] - V[0], V[2] - V[0])
    n = -n / np.linalg.norm(n)
    return V[0], n


def _h_tilted(v, V, pts):
    eye, d = _rays(v, pts)
    x0, n = _plane(V)
    t = ((x0 - eye) @ n) / (d @ n)
    p = eye + d * t[:, None]
    wl = LIGHT - p
    dist = np.linalg.norm(wl, axis=1)
    cos = np.maximum((wl @ n) / dist, 0.0)
    return np.outer(cos / dist ** 2 * INTENSITY / math.pi, KD)


def _pixel_values_tilted(sc, V, pix):
    v = sc.views[0]
    x0, n = _plane(V)
    occ = V[4:7]
    s = ((x0 - LIGHT) @ n) / ((occ - LIGHT) @ n)
    T = G.project(v, LIGHT + (occ - LIGHT) * s[:, None])
    out = np.zeros((len(pix), 3))
    for i, (_, x, y) in enumerate(pix):
        sq = np.array([[x, y], [x + 1, y], [x + 1, y + 1], [x, y + 1]], np.float64)
        p_all, w_all = G.polygon_quadrature(sq, subdiv=2)
        full = w_all @ _h_tilted(v, V, p_all)
        C = G.clip_polygon(T, x, y, x + 1, y + 1)
        if len(C) >= 3:
            p_s, w_s = G.polygon_quadrature(np.array(C), subdiv=2)
            full = full - w_s @ _h_tilted(v, V, p_s)
        out[i] = full
    return out


def test_shadow_edge_gradient_on_a_tilted_floor():
    sc = _tilted_scene(spp=64)
    pix = _pixels(sc)
    rows = O.pixel_index(sc, pix)
    V0 = sc.vertices.astype(np.float64)
    # the closed form holds for the tilted floor (value check, many samples)
    val = O.render_pixels(O.OracleScene(_tilted_scene(spp=2048)), O.params(1, 5), pix[::9])[0]
    exp_val = _pixel_values_tilted(sc, V0, pix[::9])
    assert np.all(np.abs(val - exp_val) < 4 * exp_val.max() / math.sqrt(2048) + 1e-6 * exp_val.max())
    rng = np.random.default_rng(43)
    w = rng.normal(size=(len(pix), 3))
    wfull = np.zeros((sc.n_pixels, 3))
    wfull[rows] = w
    h = 1e-5
    dirs = []
    for vi in range(4, 7):
        for k in range(3):
            D = np.zeros_like(V0)
            D[vi, k] = 1.0
            dirs.append(D)
    x0, n = _plane(V0)
    c = V0[:4].mean(0)
    D = np.zeros_like(V0)
    D[:4] = n
    dirs.append(D)                                  # the floor along its normal
    axis = np.cross(n, [1.0, 0.0, 0.0])
    axis /= np.linalg.norm(axis)
    D = np.zeros_like(V0)
    D[:4] = np.cross(axis, V0[:4] - c) * 0.1
    dirs.append(D)                                  # the floor turned about an axis in it
    exp = np.array([((_pixel_values_tilted(sc, V0 + h * D, pix) - _pixel_values_tilted(sc, V0 - h * D, pix)) * w).sum()
                    / (2 * h) for D in dirs])
    osc = O.OracleScene(sc)
    ests = []
    for seed in range(8):
        prm = O.params(1, 640 + seed, edge_spp=64)
        dv, _, _ = O.grad_pixels(osc, prm, pix, w)
        sv, _ = O.shadow_edge_grad(osc, prm, wfull)
        ests.append([((dv + sv) * D).sum() for D in dirs])
    ests = np.array(ests)
    mean, se = ests.mean(0), ests.std(0, ddof=1) / math.sqrt(len(ests))
    scale = np.abs(exp).max()
    assert np.all(np.abs(mean - exp) < 4 * se + 2e-3 * scale), (mean, exp, se)
    assert np.abs(exp[:9]).max() > 0.2 * scale and abs(exp[10]) > 0.02 * scale


def test_view_light_gives_the_scene_lights_shadow_edges():
    # the same light as the view's own instead of the scene's: same index (the
    # scene has no other), same counters, the same estimate bit for bit
    import dataclasses
    sc = _scene(spp=4)
    w = np.random.default_rng(5).normal(size=(sc.n_pixels, 3))
    a = O.shadow_edge_grad(O.OracleScene(sc), O.params(1, 9), w)[0]
    sv = dataclasses.replace(sc, light_pos=np.zeros((0, 3), np.float32), light_intensity=np.zeros((0, 3), np.float32))
    sv.views = [dataclasses.replace(v, lights=((tuple(LIGHT), (INTENSITY,) * 3),)) for v in sc.views]
    b = O.shadow_edge_grad(O.OracleScene(sv), O.params(1, 9), w)[0]
    assert np.abs(a).max() > 0
    np.testing.assert_array_equal(a, b)
