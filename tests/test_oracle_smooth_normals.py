"""Pins of the oracle's interpolated shading normals (scene option ``smooth_normals``).

The shading normal at a hit is the barycentric blend of vertex normals, each
the normalised sum of e1 x e2 over the faces around the vertex, turned with
the geometric normal toward the incoming ray; a direction counts only above
both the geometric and the shading plane. Pinned by: a planar mesh renders as
with flat normals; direct light at exact screen points equals a numpy
evaluation written from that definition (own ray casting, vertex normals,
blend, shadow test); the dual-number gradient (which now reaches every vertex
around the hit face) equals central differences of the taped estimator; the
secondary edge term is unchanged where vertex normals equal face normals; and
the gradient around a vertex of valence 200 matches the taped central differences.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2012_03939_gb300 import scenes as S
from tests import _geom as G
from tests.test_oracle_secondary_edges import _occluder_scene


def _sphere_scene(brdf="ggx", smooth=True, env=True, ks=None, seed=5):
    V, F = S.icosphere(1)
    V = V * 0.8
    rng = np.random.default_rng(seed)
    P = S.random_face_params(rng, len(F))
    if ks is not None:
        P[:, 3] = ks
    vs = [S.View((0.375, 0.875, 2.625), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 45.0, 16, 16, 1)]   # exact in float32
    return S.Scene("sphere", V.astype(np.float32), F, P, brdf, light_pos=np.array([[1.2, 1.6, 1.4]], np.float32),
                   light_intensity=np.array([[3.0, 2.5, 2.0]], np.float32),
                   env=S.lognormal_env(rng, 16, 8, sigma=0.5) if env else None, views=vs, max_bounces=2,
                   smooth_normals=smooth)


def test_planar_mesh_renders_as_with_flat_normals():
    P, F = S._grid_quad((-1, 0, -1), (0, 0, 2), (2, 0, 0), 4)
    rng = np.random.default_rng(2)
    vs = S.fibonacci_views(2, [12, 10], [10, 12], [2, 2])
    vs = [S.View(tuple(np.array(v.eye) * [1, 0, 1] * 0.6 + [0, 2.2, 0]), (0, 0, 0), (0, 0, 1), 50.0, v.width,
                 v.height, v.spp, v.pixel_offset) for v in vs]
    base = S.Scene("grid", P.astype(np.float32), F.astype(np.int32), S.random_face_params(rng, len(F)), "ggx",
                   light_pos=np.array([[0.3, 1.5, 0.2]], np.float32), light_intensity=np.full((1, 3), 3.0, np.float32),
                   env=S.lognormal_env(rng, 16, 8, sigma=0.5), views=vs, max_bounces=3)
    pix = O.all_pixels(base)
    prm = O.params(3, 44)
    flat = O.render_pixels(O.OracleScene(base), prm, pix)[0]
    smooth_sc = S.Scene(**{**base.__dict__, "smooth_normals": True})
    smooth = O.render_pixels(O.OracleScene(smooth_sc), prm, pix)[0]
    assert flat.max() > 0
    np.testing.assert_allclose(smooth, flat, rtol=1e-12, atol=1e-14)
    np.testing.assert_array_equal(O.render_signatures(O.OracleScene(smooth_sc), prm, pix),
                                  O.render_signatures(O.OracleScene(base), prm, pix))


def _vertex_normals(V, F):
    M = np.zeros_like(V)
    c = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    for k in range(3):
        np.add.at(M, F[:, k], c)
    return M / np.linalg.norm(M, axis=1, keepdims=True)


def _cast(V, F, o, d, exclude=-1, tmax=np.inf):
    """Moller-Trumbore over all faces: (face, t, b1, b2) of the nearest hit with t in (1e-5, tmax)."""
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    e1, e2 = b - a, c - a
    pv = np.cross(d, e2)
    det = np.einsum("ij,ij->i", e1, pv)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / det
        tv = o - a
        u = np.einsum("ij,ij->i", tv, pv) * inv
        qv = np.cross(tv, e1)
        v = (qv @ d) * inv
        t = np.einsum("ij,ij->i", e2, qv) * inv
    ok = (np.abs(det) > 0) & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 1e-5) & (t < tmax)
    ok[exclude] = ok[exclude] and exclude < 0
    if not ok.any():
        return -1, np.inf, 0.0, 0.0
    f = int(np.argmin(np.where(ok, t, np.inf)))
    return f, t[f], u[f], v[f]


@pytest.mark.parametrize("inward", [False, True])
def test_direct_light_equals_the_definition_at_screen_points(inward):
    # inward: faces wound the other way, so every hit turns both normals around
    sc = _sphere_scene(env=False, ks=0.0)
    sc.max_bounces = 1
    if inward:
        sc.faces = np.ascontiguousarray(sc.faces[:, [0, 2, 1]])
    V = sc.vertices.astype(np.float64)
    F = sc.faces
    N = _vertex_normals(V, F)
    L = sc.light_pos[0].astype(np.float64)
    I = sc.light_intensity[0].astype(np.float64)
    osc = O.OracleScene(sc)
    prm = O.params(1, 3)
    v = sc.views[0]
    rng = np.random.default_rng(8)
    n_hit = n_tilted = n_split = 0
    for px, py in rng.uniform([3, 3], [13, 13], size=(300, 2)):
        got = O.trace_screen(osc, prm, 0, px, py)
        o, d = G.pixel_ray(v, px, py)
        f, t, b1, b2 = _cast(V, F, o, d)
        exp = np.zeros(3)
        if f >= 0:
            n_hit += 1
            a, b, c = V[F[f]]
            ng = np.cross(b - a, c - a)
            ng /= np.linalg.norm(ng)
            s = (1 - b1 - b2) * N[F[f, 0]] + b1 * N[F[f, 1]] + b2 * N[F[f, 2]]
            ns = s / np.linalg.norm(s)
            if ng @ -d < 0:
                ng, ns = -ng, -ns
            n_tilted += math.acos(min(1.0, ns @ ng)) > 1e-2
            p = o + t * d
            wi = L - p
            dist = np.linalg.norm(wi)
            wi /= dist
            n_split += (ng @ wi > 0) != (ns @ wi > 0)
            if ng @ wi > 0 and ns @ wi > 0 and _cast(V, F, p, wi, exclude=f, tmax=dist - 1e-5)[0] < 0:
                exp = sc.face_params[f, :3].astype(np.float64) / math.pi * I * (ns @ wi) / dist ** 2
        np.testing.assert_allclose(got, exp, rtol=1e-9, atol=1e-12)
    assert n_hit > 150 and n_tilted > 100 and n_split > 0


@pytest.mark.parametrize("brdf,B", [("ggx", 1), ("ggx", 3), ("beckmann", 2)])
def test_smooth_gradient_matches_tape_replay_fd(brdf, B):
    sc = _sphere_scene(brdf)
    V0 = sc.vertices.astype(np.float64)
    P0 = sc.face_params.astype(np.float64)
    prm = O.params(B, 77)
    w = np.array([0.4, -0.6, 0.5])
    checked = ring = 0
    for (px, py, c1) in [(6.3, 7.1, 0), (9.7, 8.2, 1), (8.1, 10.4, 2), (7.6, 5.8, 3)]:
        osc = O.OracleScene(sc, vertices=V0, face_params=P0)
        rgb, dv, df = O.trace_screen(osc, prm, 0, px, py, c0=5, c1=c1, grad_w=w)
        _, tape = O.trace_screen_taped(osc, prm, 0, px, py, c0=5, c1=c1)
        np.testing.assert_array_equal(rgb, O.trace_screen_taped(osc, prm, 0, px, py, c0=5, c1=c1, tape=tape))
        o, d = G.pixel_ray(sc.views[0], px, py)
        f = _cast(V0, sc.faces, o, d)[0]
        ring += np.count_nonzero(np.delete(np.abs(dv).sum(1), sc.faces[f])) if f >= 0 else 0
        h = 1e-6
        for (vi, k) in [(i, k) for i in range(len(V0)) for k in range(3) if dv[i, k] != 0]:
            Vp, Vm = V0.copy(), V0.copy()
            Vp[vi, k] += h
            Vm[vi, k] -= h
            fp = O.trace_screen_taped(O.OracleScene(sc, vertices=Vp, face_params=P0), prm, 0, px, py, 5, c1, tape=tape)
            fm = O.trace_screen_taped(O.OracleScene(sc, vertices=Vm, face_params=P0), prm, 0, px, py, 5, c1, tape=tape)
            fd = (w @ fp - w @ fm) / (2 * h)
            assert abs(fd - dv[vi, k]) < 1e-5 * max(1.0, abs(fd)), (vi, k, fd, dv[vi, k])
            checked += 1
        for (fi, k) in [(i, k) for i in range(len(P0)) for k in range(5) if df[i, k] != 0]:
            Pp, Pm = P0.copy(), P0.copy()
            Pp[fi, k] += h
            Pm[fi, k] -= h
            fp = O.trace_screen_taped(O.OracleScene(sc, vertices=V0, face_params=Pp), prm, 0, px, py, 5, c1, tape=tape)
            fm = O.trace_screen_taped(O.OracleScene(sc, vertices=V0, face_params=Pm), prm, 0, px, py, 5, c1, tape=tape)
            fd = (w @ fp - w @ fm) / (2 * h)
            assert abs(fd - df[fi, k]) < 1e-5 * max(1.0, abs(fd)), (fi, k, fd, df[fi, k])
            checked += 1
    # the shading normals reach the vertices around the hit face, not just its own
    assert checked > 40 and ring > 0


def test_secondary_term_unchanged_where_vertex_normals_are_face_normals():
    # floor and floating triangle share no vertex: every vertex normal is its
    # face's normal, so the shading normal equals the geometric one and the
    # secondary edge samples (their planes, sides and weights) are the flat ones
    sc = _occluder_scene(spp=2)
    pix = O.all_pixels(sc)[::7]
    w = np.random.default_rng(3).normal(size=(len(pix), 3))
    out = []
    for smooth in (False, True):
        s = S.Scene(**{**sc.__dict__, "smooth_normals": smooth})
        osc = O.OracleScene(s)
        g1 = O.grad_pixels(osc, O.params(1, 9, secondary=1), pix, w)[0]
        g0 = O.grad_pixels(osc, O.params(1, 9), pix, w)[0]
        out.append(g1 - g0)
    assert np.abs(out[0]).max() > 0
    np.testing.assert_allclose(out[1], out[0], rtol=1e-9, atol=1e-9 * np.abs(out[0]).max())


def test_high_valence_vertex_gradient_matches_tape_replay_fd():
    # a fan of 200 triangles around a raised centre: the centre's normal depends
    # on all 201 vertices; each vertex normal is one variable of the path and
    # its derivative reaches every vertex around it
    n = 200
    ang = np.linspace(0, 2 * np.pi, n, endpoint=False)
    rng = np.random.default_rng(1)
    V = np.r_[[[0.0, 0.3, 0.0]], np.c_[np.cos(ang), rng.uniform(-0.05, 0.05, n), np.sin(ang)]].astype(np.float32)
    F = np.array([[0, 1 + (i + 1) % n, 1 + i] for i in range(n)], np.int32)
    vs = [S.View((0.125, 2.5, 0.5), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 40.0, 8, 8, 1)]
    P = S.random_face_params(rng, n)
    P[:, 3] = 0.0
    sc = S.Scene("fan", V, F, P, "ggx", light_pos=np.array([[0.5, 2.0, 0.25]], np.float32),
                 light_intensity=np.full((1, 3), 3.0, np.float32), views=vs, max_bounces=1, smooth_normals=True)
    V0 = V.astype(np.float64)
    prm = O.params(1, 1)
    w = np.array([0.3, 0.5, -0.2])
    checked = far = 0
    for px, py in [(3.6, 4.1), (4.4, 3.7), (4.05, 4.2)]:
        osc = O.OracleScene(sc, vertices=V0)
        _, dv, _ = O.trace_screen(osc, prm, 0, px, py, grad_w=w)
        _, tape = O.trace_screen_taped(osc, prm, 0, px, py)
        far += np.count_nonzero(np.abs(dv[1:]).sum(1)) > 10
        h = 1e-6
        for vi in [0] + list(rng.choice(np.arange(1, n + 1), 12, replace=False)):
            for k in range(3):
                Vp, Vm = V0.copy(), V0.copy()
                Vp[vi, k] += h
                Vm[vi, k] -= h
                fp = O.trace_screen_taped(O.OracleScene(sc, vertices=Vp), prm, 0, px, py, tape=tape)
                fm = O.trace_screen_taped(O.OracleScene(sc, vertices=Vm), prm, 0, px, py, tape=tape)
                fd = (w @ fp - w @ fm) / (2 * h)
                assert abs(fd - dv[vi, k]) < 1e-5 * max(1.0, abs(fd)), (vi, k, fd, dv[vi, k])
                checked += 1
    assert checked == 3 * 13 * 3 and far == 3


def _valley(spp):
    """Two faces meeting in a valley (concave, open below): the near face's vertex normals at the valley are the
    mean of both faces', so its shading normal stands up out of the face toward the far face. The far face hides
    part of the near face's sky; nothing lies below the near face."""
    V = np.array([[-1.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.6, 1.2], [0.0, 0.6, -1.2]], np.float32)
    F = np.array([[0, 2, 1], [0, 1, 3]], np.int32)
    P = np.array([[0.6, 0.5, 0.4, 0.0, 0.5], [0.6, 0.5, 0.4, 0.0, 0.5]], np.float32)
    vs = [S.View((0.25, 2.25, 2.5), (0.0, 0.25, 0.5), (0.0, 1.0, 0.0), 30.0, 16, 16, spp)]
    return S.Scene("valley", V, F, P, "ggx", env=np.full((16, 32, 3), 0.7, np.float32), views=vs, max_bounces=1,
                   smooth_normals=True)


def _hits_triangle(o, W, a, b, c):
    """Does the ray o + t w (t > 1e-5) meet triangle (a, b, c), for every direction w in W?"""
    e1, e2 = b - a, c - a
    pv = np.cross(W, e2)
    det = pv @ e1
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / det
        tv = o - a
        u = (pv @ tv) * inv
        qv = np.cross(tv, e1)
        v = (W @ qv) * inv
        t = (qv @ e2) * inv
    return (np.abs(det) > 0) & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 1e-5)


def test_uniform_sky_counts_directions_above_both_planes():
    # a Lambertian point under a uniform sky of radiance L0, one vertex (the
    # environment sample's MIS weight is 1): E[L] = kd/pi L0 I, I the integral of
    # (n_s.w)+ over the directions above the face's plane as well and not hidden
    # by the far face. Expected pixel values: I by quadrature over the sphere
    # with each direction cast against the far face, n_s from the definition
    # (vertex normals, barycentric blend), averaged over the pixel by Gauss points
    spp = 1 << 19
    sc = _valley(spp)
    V = sc.vertices.astype(np.float64)
    N = _vertex_normals(V, sc.faces)
    v = sc.views[0]
    ng = np.cross(V[2] - V[0], V[1] - V[0])
    ng /= np.linalg.norm(ng)
    nz, nph = 240, 480
    z = (np.arange(nz) + 0.5) / nz * 2 - 1
    ph = (np.arange(nph) + 0.5) / nph * 2 * np.pi
    zz, pp = np.meshgrid(z, ph, indexing="ij")
    rr = np.sqrt(1 - zz ** 2)
    W = np.stack([rr * np.cos(pp), rr * np.sin(pp), zz], -1).reshape(-1, 3)
    dw = 4 * np.pi / len(W)

    def expected(px, py):
        o, d = G.pixel_ray(v, px, py)
        f, t, b1, b2 = _cast(V, sc.faces, o, d)
        assert f == 0
        p = o + t * d
        s = (1 - b1 - b2) * N[0] + b2 * N[1] + b1 * N[2]    # face (0, 2, 1): b1 weighs vertex 2, b2 vertex 1
        ns = s / np.linalg.norm(s)
        keep = (W @ ng > 0) & ~_hits_triangle(p, W, V[0], V[1], V[3])
        return (np.maximum(W @ ns, 0) * keep).sum() * dw

    img = G.project(v, V[[0, 2, 1]])
    pix, exp = [], []
    for y in range(v.height):
        for x in range(v.width):
            C = G.clip_polygon(img, x, y, x + 1, y + 1)
            if len(C) >= 3 and G.polygon_area(np.array(C)) > 0.999:
                pix.append((0, x, y))
    pix = pix[::4]
    for _, x, y in pix:
        pts, wts = G.polygon_quadrature(np.array([[x, y], [x + 1, y], [x + 1, y + 1], [x, y + 1]], float), 1)
        exp.append(0.6 / math.pi * 0.7 * sum(w * expected(px, py) for (px, py), w in zip(pts, wts)))
    pix, exp = np.array(pix, np.int32), np.array(exp)
    assert len(pix) >= 6
    got = O.render_pixels(O.OracleScene(sc), O.params(1, 4), pix)[0][:, 0]
    # the sky sample is uniform over the sphere (pdf 1/(4 pi)), so a sample is at
    # most 4 kd L0 (n_s.w)+: E[X^2] <= 16 (kd L0)^2 / 6
    se = 4 * 0.6 * 0.7 / math.sqrt(6 * spp)
    assert np.all(np.abs(got - exp) < 4 * se), (got, exp, se)
    # the rule matters here: counting the open sky below the face (above the
    # shading plane) would raise some pixels by far more than the resolution
    def without_face_plane(px, py):
        o, d = G.pixel_ray(v, px, py)
        f, t, b1, b2 = _cast(V, sc.faces, o, d)
        p = o + t * d
        s_ = (1 - b1 - b2) * N[0] + b2 * N[1] + b1 * N[2]
        ns = s_ / np.linalg.norm(s_)
        keep = ~_hits_triangle(p, W, V[0], V[1], V[3])
        return (np.maximum(W @ ns, 0) * keep).sum() * dw

    alt = []
    for _, x, y in pix:
        pts, wts = G.polygon_quadrature(np.array([[x, y], [x + 1, y], [x + 1, y + 1], [x, y + 1]], float), 1)
        alt.append(0.6 / math.pi * 0.7 * sum(w * without_face_plane(px, py) for (px, py), w in zip(pts, wts)))
    assert (np.array(alt) - exp).max() > 12 * se


def test_point_light_below_the_face_is_not_seen():
    # the valley's near face under two lights: one above its plane, one low
    # beyond its outer edge -- below the face's plane everywhere, but above the
    # shading plane near the valley, with nothing in between (open below): by
    # the definition that light adds nothing. Exact screen points; expected
    # values restated in numpy (casts, vertex normals, blend, both plane tests,
    # the far face as the only occluder)
    import dataclasses
    LP = np.array([[0.0, 1.0, 6.0], [0.3, 2.5, 0.5]])
    I0 = np.array([[30.0, 20.0, 10.0], [3.0, 2.5, 2.0]])
    sc = dataclasses.replace(_valley(1), env=None, light_pos=LP.astype(np.float32),
                             light_intensity=I0.astype(np.float32))
    LP = sc.light_pos.astype(np.float64)    # the values the scene holds (float32)
    V = sc.vertices.astype(np.float64)
    N = _vertex_normals(V, sc.faces)
    ng = np.cross(V[2] - V[0], V[1] - V[0])
    ng /= np.linalg.norm(ng)
    v = sc.views[0]
    osc = O.OracleScene(sc)
    prm = O.params(1, 2)
    img = G.project(v, V[[0, 2, 1]])
    lo, hi = img.min(0), img.max(0)
    rng = np.random.default_rng(3)
    n_pts = n_below = n_lit = 0
    for px, py in rng.uniform(lo, hi, size=(600, 2)):
        o, d = G.pixel_ray(v, px, py)
        f, t, b1, b2 = _cast(V, sc.faces, o, d)
        if f != 0:
            continue
        n_pts += 1
        p = o + t * d
        s = (1 - b1 - b2) * N[0] + b2 * N[1] + b1 * N[2]
        ns = s / np.linalg.norm(s)
        exp = np.zeros(3)
        for L, I in zip(LP, I0):
            wl = L - p
            dist = np.linalg.norm(wl)
            wl /= dist
            n_below += ns @ wl > 0 and not ng @ wl > 0
            if ng @ wl > 0 and ns @ wl > 0 and not _hits_triangle(p, wl[None], V[0], V[1], V[3])[0]:
                exp += sc.face_params[0, :3].astype(np.float64) / math.pi * I * (ns @ wl) / dist ** 2
                n_lit += 1
        got = O.trace_screen(osc, prm, 0, px, py)
        np.testing.assert_allclose(got, exp, rtol=1e-9, atol=1e-12)
    assert n_pts > 200 and n_below > 20 and n_lit > 100


def _fnv(words):
    h = 0xcbf29ce484222325
    for x in words:
        h = ((h ^ (int(x) & 0xffffffff)) * 0x100000001b3) & 0xffffffffffffffff
    return h


def test_path_decisions_over_the_valley_match_a_restatement():
    # two-vertex paths over the valley under a point light, one sample per
    # pixel: every decision the path signature hashes -- the faces hit, the
    # shadow rays traced and their visibility, the BSDF lobe and whether its
    # direction is valid (above the shading plane by the sampler, above the
    # face's plane by the rule) -- restated in numpy from the counters
    import dataclasses
    seed = 77
    LP = np.array([[0.3, 2.5, 0.5]])
    sc = dataclasses.replace(_valley(1), env=None, light_pos=LP.astype(np.float32),
                             light_intensity=np.full((1, 3), 3.0, np.float32))
    sc.views = [dataclasses.replace(sc.views[0], width=32, height=32)]
    sc.max_bounces = 2
    L = sc.light_pos.astype(np.float64)[0]
    V = sc.vertices.astype(np.float64)
    F = sc.faces
    N = _vertex_normals(V, F)
    v = sc.views[0]
    key = np.array([seed & 0xffffffff, seed >> 32], np.uint32)
    unif = lambda w: (int(w) >> 8) * 2.0 ** -24
    P5 = sc.face_params.astype(np.float64)

    def normals(f, p, wo):
        a, b, c = V[F[f]]
        m = np.cross(b - a, c - a)
        ng = m / np.linalg.norm(m)
        q = p - a
        b1 = np.cross(q, c - a) @ m / (m @ m)
        b2 = np.cross(b - a, q) @ m / (m @ m)
        s = (1 - b1 - b2) * N[F[f, 0]] + b1 * N[F[f, 1]] + b2 * N[F[f, 2]]
        ns = s / np.linalg.norm(s)
        sg = -1.0 if ng @ wo < 0 else 1.0
        return ng * sg, ns * sg

    def nee(f, p, ng, ns):
        wl = L - p
        dist = np.linalg.norm(wl)
        wl /= dist
        if not (ng @ wl > 0 and ns @ wl > 0 and dist > 2e-5):
            return False, 0
        seen = _cast(V, F, p, wl, exclude=f, tmax=dist - 1e-5)[0] < 0
        return True, (1 if seen else 0)

    pix = O.all_pixels(sc)
    expect = []
    n_invalid = n_bounce = 0
    for _, x, y in pix:
        c0 = v.pixel_offset + y * v.width + x
        u = O.philox([c0, 0, 0, 0], key)
        o, d = G.pixel_ray(v, x + unif(u[0]), y + unif(u[1]))
        words = []
        f, t, _, _ = _cast(V, F, o, d)
        if f < 0:
            expect.append(_fnv([0xffffffff]))
            continue
        words.append(f)
        p = o + t * d
        ng, ns = normals(f, p, -d)
        traced, vis = nee(f, p, ng, ns)
        ub = O.philox([c0, 0, (0 << 4) | 2, 0], key)
        m = P5[f]
        ps = min(max(m[3] / (m[3] + m[:3].mean()), 0.05), 0.95)
        lobe = 1 if unif(ub[0]) < ps else 0
        wi, pdf = O.brdf_sample(0, m, ns, -d, unif(ub[0]), unif(ub[1]), unif(ub[2]))
        valid = pdf > 0 and ng @ wi > 0
        n_invalid += pdf > 0 and not valid
        words.append(lobe | (2 if valid else 0))
        if traced:
            words.append(vis)
        if valid:
            n_bounce += 1
            f2, t2, _, _ = _cast(V, F, p, wi, exclude=f)
            if f2 < 0:
                words.append(0xffffffff)
            else:
                words.append(f2)
                p2 = p + t2 * wi
                ng2, ns2 = normals(f2, p2, -wi)
                traced2, vis2 = nee(f2, p2, ng2, ns2)
                if traced2:
                    words.append(vis2)
        expect.append(_fnv(words))
    got = O.render_signatures(O.OracleScene(sc), O.params(2, seed), pix).astype(np.uint64)
    same = got == np.array(expect, np.uint64)
    assert same.mean() >= 0.998, (same.mean(), np.nonzero(~same)[0][:5])
    assert n_invalid > 10 and n_bounce > 300
