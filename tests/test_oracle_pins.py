"""Pins of the FP64 oracle against facts the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, definitions written independently here, invariants, or finite
differences of its own forward pass. None needs a GPU.
"""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle as O
from paper_2012_03939_gb300 import scenes as S
from tests import _geom as G

MASK = 0xFFFFFFFF


# ---------------------------------------------------------------------------- Philox4x32-10
def _weyl():
    # Salmon et al. SC'11 key schedule: golden ratio and sqrt(3) - 1, as 32-bit fixed point.
    getcontext().prec = 60
    phi = (1 + Decimal(5).sqrt()) / 2
    return int((phi - 1) * (1 << 32)), int((Decimal(3).sqrt() - 1) * (1 << 32))


def _philox_inverse(out, key):
    M0, M1 = 0xD2511F53, 0xCD9E8D57      # multipliers given in Salmon et al. SC'11
    W0, W1 = _weyl()
    i0, i1 = pow(M0, -1, 1 << 32), pow(M1, -1, 1 << 32)
    y = [int(v) for v in out]
    for r in reversed(range(10)):
        k0 = (key[0] + r * W0) & MASK
        k1 = (key[1] + r * W1) & MASK
        x0 = (y[3] * i0) & MASK
        x2 = (y[1] * i1) & MASK
        hi0 = (M0 * x0) >> 32
        hi1 = (M1 * x2) >> 32
        y = [x0, y[0] ^ hi1 ^ k0, x2, y[2] ^ hi0 ^ k1]
    return y


def test_philox_inverts_to_counter():
    rng = np.random.default_rng(1)
    for _ in range(200):
        ctr = rng.integers(0, 1 << 32, size=4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 1 << 32, size=2, dtype=np.uint64).astype(np.uint32)
        out = O.philox(ctr, key)
        assert _philox_inverse(out, [int(k) for k in key]) == [int(c) for c in ctr]


def test_philox_uniformity_and_counter_sensitivity():
    key = np.array([0x1234, 0x5678], np.uint32)
    words = np.array([O.philox(np.array([i, 7, 2, 0], np.uint32), key) for i in range(8192)])
    u = (words >> 8).astype(np.float64) / 2 ** 24
    for k in range(4):
        hist = np.histogram(u[:, k], bins=32, range=(0, 1))[0]
        e = len(u) / 32
        chi2 = ((hist - e) ** 2 / e).sum()
        assert chi2 < 80, chi2          # 31 dof; p ~ 1e-6 at 80
    # neighbouring counters differ in about half of the output bits
    a = O.philox(np.array([5, 7, 2, 0], np.uint32), key)
    b = O.philox(np.array([5, 7, 3, 0], np.uint32), key)
    flips = sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b))
    assert 40 < flips < 88


# ---------------------------------------------------------------------------- alias table
def _env_weights(env):
    h = env.shape[0]
    e = env.astype(np.float64)
    lum = 0.2126 * e[..., 0] + 0.7152 * e[..., 1] + 0.0722 * e[..., 2]
    return (lum * np.sin(np.pi * (np.arange(h) + 0.5) / h)[:, None]).ravel()


def test_alias_table_distribution_exact():
    env = S.lognormal_env(np.random.default_rng(3), 32, 16)
    prob, alias, pmf = O.env_alias(env)
    w = _env_weights(env)
    np.testing.assert_allclose(pmf, w / w.sum(), rtol=1e-12, atol=0)
    N = len(prob)
    implied = prob / N
    np.add.at(implied, alias, (1 - prob) / N)
    np.testing.assert_allclose(implied, w / w.sum(), rtol=0, atol=1e-12)


def test_alias_sampling_chi2():
    env = S.lognormal_env(np.random.default_rng(4), 8, 4)
    prob, alias, pmf = O.env_alias(env)
    rng = np.random.default_rng(5)
    words = rng.integers(0, 1 << 32, size=(40000, 2), dtype=np.uint64)
    counts = np.bincount([O.alias_pick(prob, alias, int(a), int(b)) for a, b in words], minlength=len(pmf))
    e = pmf * len(words)
    chi2 = ((counts - e) ** 2 / e).sum()
    assert chi2 < len(pmf) + 6 * math.sqrt(2 * len(pmf))


# ---------------------------------------------------------------------------- BRDF
def _rand_dir(rng, n):
    while True:
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        if v @ n > 0.05:
            return v


@pytest.mark.parametrize("brdf", [0, 1])
def test_brdf_reciprocity(brdf):
    rng = np.random.default_rng(10 + brdf)
    for _ in range(50):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        p5 = np.r_[rng.uniform(0.1, 0.9, 3), rng.uniform(0, 1), rng.uniform(0.05, 0.8)]
        a, b = _rand_dir(rng, n), _rand_dir(rng, n)
        np.testing.assert_allclose(O.brdf_eval(brdf, p5, n, a, b), O.brdf_eval(brdf, p5, n, b, a), rtol=1e-12)


@pytest.mark.parametrize("brdf,alpha", [(0, 0.1), (0, 0.35), (0, 0.6), (1, 0.1), (1, 0.35), (1, 0.6)])
def test_microfacet_D_normalised(brdf, alpha):
    from scipy.integrate import quad
    f = lambda th: O.microfacet(brdf, alpha, math.cos(th))[0] * math.cos(th) * math.sin(th)
    val = 2 * math.pi * quad(f, 0, math.pi / 2, points=[alpha, 2 * alpha], limit=200, epsabs=1e-12)[0]
    assert abs(val - 1) < 1e-7


@pytest.mark.parametrize("brdf,alpha,theta_o", [(0, 0.3, 0.4), (0, 0.6, 1.1), (1, 0.3, 0.7), (1, 0.6, 1.2)])
def test_smith_G1_projected_area(brdf, alpha, theta_o):
    # Smith masking: G1(wo) * integral of max(0, wo.h) D(h) dh equals cos(theta_o).
    wo = np.array([math.sin(theta_o), 0, math.cos(theta_o)])
    xg, wg = np.polynomial.legendre.leggauss(400)
    th = (xg + 1) * math.pi / 4
    wth = wg * math.pi / 4
    ph = (np.arange(720) + 0.5) * 2 * math.pi / 720
    T, P = np.meshgrid(th, ph, indexing="ij")
    h = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1)
    D = np.vectorize(lambda c: O.microfacet(brdf, alpha, c)[0])(np.cos(th))
    integrand = np.maximum(0, h @ wo) * D[:, None] * np.sin(T)
    I = (integrand * wth[:, None]).sum() * (2 * math.pi / 720)
    G1 = O.microfacet(brdf, alpha, math.cos(theta_o))[1]
    assert abs(G1 * I - math.cos(theta_o)) < 2e-5


@pytest.mark.parametrize("brdf", [0, 1])
def test_brdf_peak_closed_form(brdf):
    # wi = wo = n: h = n, D(1) = 1/(pi a^2), G1(1) = 1 -> f = kd/pi + ks/(4 pi a^2)
    n = np.array([0.0, 0, 1])
    p5 = np.array([0.2, 0.4, 0.6, 0.3, 0.25])
    f = O.brdf_eval(brdf, p5, n, n, n)
    np.testing.assert_allclose(f, p5[:3] / math.pi + p5[3] / (4 * math.pi * p5[4] ** 2), rtol=1e-12)


def _hemi_quad(fn, nth=200, nph=400):
    xg, wg = np.polynomial.legendre.leggauss(nth)
    th = (xg + 1) * math.pi / 4
    wth = wg * math.pi / 4
    tot = 0.0
    for t, w in zip(th, wth):
        for p in (np.arange(nph) + 0.5) * 2 * math.pi / nph:
            wi = np.array([math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t)])
            tot += w * (2 * math.pi / nph) * fn(wi) * math.sin(t)
    return tot


def test_diffuse_albedo_equals_kd():
    n = np.array([0.0, 0, 1])
    wo = np.array([0.3, 0.1, 0.9])
    wo /= np.linalg.norm(wo)
    p5 = np.array([0.3, 0.5, 0.7, 0.0, 0.4])
    alb = np.array([_hemi_quad(lambda wi, c=c: O.brdf_eval(0, p5, n, wi, wo)[c] * wi[2], 64, 64) for c in range(3)])
    np.testing.assert_allclose(alb, p5[:3], rtol=1e-9)


@pytest.mark.parametrize("brdf,alpha", [(0, 0.2), (0, 0.5), (1, 0.2), (1, 0.5)])
def test_sampling_pdf_mass_closed_form(brdf, alpha):
    # kd = 0, ks = 1 -> p_spec = 0.95. At wo = n the reflected direction leaves the
    # hemisphere iff theta_h > 45 deg, whose probability is a^2/(1+a^2) (GGX) or
    # exp(-1/a^2) (Beckmann); the diffuse share integrates to 1.
    from scipy.integrate import quad
    n = np.array([0.0, 0, 1])
    p5 = np.array([0, 0, 0, 1.0, alpha])
    f = lambda th: O.brdf_pdf(brdf, p5, n, np.array([math.sin(th), 0, math.cos(th)]), n) * math.sin(th)
    mass = 2 * math.pi * quad(f, 0, math.pi / 2, points=[alpha, 2 * alpha], limit=400, epsabs=1e-12)[0]
    tail = alpha ** 2 / (1 + alpha ** 2) if brdf == 0 else math.exp(-1 / alpha ** 2)
    assert abs(mass - (0.05 + 0.95 * (1 - tail))) < 1e-7


@pytest.mark.parametrize("brdf", [0, 1])
def test_sampled_direction_is_continuous_across_coordinate_planes(brdf):
    # the tangent frame may rotate about n, but a normal on a coordinate plane
    # (every face of a mirror-symmetric mesh has some) must not switch frames
    # when rounding moves it off the plane by an ulp: the same numbers give the
    # same direction on both sides of the plane, and at a signed zero
    p5 = np.array([0.4, 0.3, 0.2, 0.5, 0.3])
    rng = np.random.default_rng(3)
    for base in ([0.983104336, -0.183046071, 0.0], [0.0, 1.0, 0.0], [0.6, 0.0, -0.8], [-1.0, 0.0, 0.0]):
        base = np.array(base) / np.linalg.norm(base)
        wo = base + np.array([0.31, -0.22, 0.17]) * 0.5
        wo /= np.linalg.norm(wo)
        for ul, u1, u2 in rng.random((40, 3)):
            ref, pref = O.brdf_sample(brdf, p5, base, wo, ul, u1, u2)
            for k in np.nonzero(base == 0)[0]:
                for eps in (-1e-9, 1e-9, -0.0):
                    n = base.copy()
                    n[k] = eps
                    n /= np.linalg.norm(n)
                    wi, pdf = O.brdf_sample(brdf, p5, n, wo, ul, u1, u2)
                    assert np.abs(wi - ref).max() < 1e-6 and abs(pdf - pref) <= 1e-6 * max(pref, 1.0)


@pytest.mark.parametrize("brdf", [0, 1])
def test_sampling_matches_pdf_histogram(brdf):
    rng = np.random.default_rng(20 + brdf)
    n = np.array([0.0, 0, 1])
    wo = np.array([math.sin(0.6), 0, math.cos(0.6)])
    p5 = np.array([0.2, 0.3, 0.1, 0.3, 0.3])
    N = 60000
    U = rng.random((N, 3))
    dirs = []
    fcos_over_pdf = []
    for ul, u1, u2 in U:
        wi, pdf = O.brdf_sample(brdf, p5, n, wo, ul, u1, u2)
        if pdf > 0:
            dirs.append(wi)
            fcos_over_pdf.append(O.brdf_eval(brdf, p5, n, wi, wo)[0] * wi[2] / pdf)
            assert abs(O.brdf_pdf(brdf, p5, n, wi, wo) - pdf) <= 1e-12 * pdf
    dirs = np.array(dirs)
    # histogram in (cos theta, phi) bins versus the pdf integrated over each bin
    nc, nphi = 8, 8
    cth = np.clip(dirs[:, 2], 0, 1 - 1e-12)
    phi = np.mod(np.arctan2(dirs[:, 1], dirs[:, 0]), 2 * np.pi)
    counts = np.histogram2d(cth, phi, bins=[nc, nphi], range=[[0, 1], [0, 2 * np.pi]])[0]
    exp = np.zeros((nc, nphi))
    sub = 12
    for i in range(nc):
        for j in range(nphi):
            cs = (i + (np.arange(sub) + 0.5) / sub) / nc
            ps = (j + (np.arange(sub) + 0.5) / sub) * 2 * np.pi / nphi
            acc = 0.0
            for c in cs:
                s = math.sqrt(1 - c * c)
                for p in ps:
                    acc += O.brdf_pdf(brdf, p5, n, np.array([s * math.cos(p), s * math.sin(p), c]), wo)
            exp[i, j] = acc / sub ** 2 * (1 / nc) * (2 * np.pi / nphi) * N
    m = exp > 20
    chi2 = ((counts[m] - exp[m]) ** 2 / exp[m]).sum()
    assert chi2 < m.sum() + 6 * math.sqrt(2 * m.sum()), chi2
    # E[f cos / pdf] = directional albedo by quadrature (red channel)
    alb = _hemi_quad(lambda wi: O.brdf_eval(brdf, p5, n, wi, wo)[0] * wi[2], 96, 96)
    mc = np.sum(fcos_over_pdf) / N
    se = np.std(np.r_[fcos_over_pdf, np.zeros(N - len(fcos_over_pdf))]) / math.sqrt(N)
    assert abs(mc - alb) < 4 * se + 1e-4


# ---------------------------------------------------------------------------- mesh colors
def test_mesh_color_index():
    # r = 0 is one texel per face (k = t), the per-face parameters used here.
    for t in (0, 1, 7, 319):
        assert O.mesh_color_index(0, t, 0.3, 0.2) == t
    # r > 0: the (r+1)(r+2)/2 texel positions of face t map one-to-one onto its block.
    for r in (1, 2, 3, 5):
        n = (r + 1) * (r + 2) // 2
        for t in (0, 3):
            ks = sorted(O.mesh_color_index(r, t, (i + 0.5) / r if i < r else 1.0, (j + 0.5) / r if j < r else 1.0)
                        for i in range(r + 1) for j in range(r + 1 - i))
            assert ks == list(range(t * n, (t + 1) * n))


# ---------------------------------------------------------------------------- intersection
def test_watertight_closed_mesh_never_misses():
    V, F = S.icosphere(2)
    sc = S.Scene("ico", V.astype(np.float32), F, S.random_face_params(np.random.default_rng(0), len(F)))
    osc = O.OracleScene(sc)
    rng = np.random.default_rng(6)
    Vf = V.astype(np.float32).astype(np.float64)
    targets = list(Vf)
    E = {(min(a, b), max(a, b)) for f in F for a, b in ((f[0], f[1]), (f[1], f[2]), (f[2], f[0]))}
    targets += [(Vf[a] + Vf[b]) / 2 for a, b in list(E)]
    rays = []
    for t in targets:
        # approach each vertex / edge midpoint from outside, roughly head-on
        o = 3 * t + 0.3 * rng.normal(size=3)
        d = t - o
        d /= np.linalg.norm(d)
        rays.append(np.r_[o, d, np.inf])
    tri, _ = O.closest_hit(osc, np.array(rays))
    assert (tri >= 0).all()


def test_closest_hit_matches_moller_trumbore():
    V, F = S.icosphere(1)
    V = V * np.array([1.0, 0.7, 1.3])
    sc = S.Scene("ico", V.astype(np.float32), F, S.random_face_params(np.random.default_rng(0), len(F)))
    osc = O.OracleScene(sc)
    Vd = V.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(7)
    o = rng.normal(size=(400, 3))
    o = 3 * o / np.linalg.norm(o, axis=1, keepdims=True)
    d = rng.normal(size=(400, 3)) * 0.3 - o / 3
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    tri, t = O.closest_hit(osc, np.c_[o, d, np.full(400, np.inf)])
    for i in range(400):
        best, bt, margin = -1, np.inf, np.inf
        for f, (a, b, c) in enumerate(F):
            e1, e2 = Vd[b] - Vd[a], Vd[c] - Vd[a]
            p = np.cross(d[i], e2)
            det = e1 @ p
            if abs(det) < 1e-14:
                continue
            s = o[i] - Vd[a]
            u = (s @ p) / det
            q = np.cross(s, e1)
            v = (d[i] @ q) / det
            tt = (e2 @ q) / det
            if u >= 0 and v >= 0 and u + v <= 1 and tt > 1e-5 and tt < bt:
                best, bt, margin = f, tt, min(u, v, 1 - u - v)
        if margin < 1e-9:
            continue
        assert tri[i] == best
        if best >= 0:
            assert abs(t[i] - bt) < 1e-12 * max(1, bt)


# ---------------------------------------------------------------------------- camera + coverage
def test_pixel_coverage_of_a_black_triangle_on_a_constant_sky():
    # A black triangle in front of a constant environment L0: each camera sample is
    # L0 on a miss and 0 on a hit, so the pixel mean is L0 * (1 - covered area).
    sc = S.single_triangle(12, 10)
    sc.face_params = np.array([[0, 0, 0, 0, 0.5]], np.float32)
    sc.light_pos = np.zeros((0, 3), np.float32)
    sc.light_intensity = np.zeros((0, 3), np.float32)
    sc.env = np.full((8, 16, 3), 0.7, np.float32)
    sc.views[0].spp = 1024
    osc = O.OracleScene(sc)
    img, _ = O.render_pixels(osc, O.params(1, 99), O.all_pixels(sc))
    v = sc.views[0]
    tri2d = G.project(v, sc.vertices.astype(np.float64))
    pix = O.all_pixels(sc)
    for k, (_, x, y) in enumerate(pix):
        A = G.polygon_area(G.clip_polygon(tri2d, x, y, x + 1, y + 1))
        exp = 0.7 * (1 - A)
        sd = 0.7 * math.sqrt(max(A * (1 - A), 1e-4) / v.spp)
        assert abs(img[k, 0] - exp) < 5 * sd + 1e-12, (x, y, img[k, 0], exp)


# ---------------------------------------------------------------------------- point light closed form
def test_point_light_lambertian_closed_form():
    # Radiance is linear in kd; the difference of two renders isolates
    # (kd_a - kd_b)/pi * I cos(theta) / d^2 at every covered screen point.
    sc = S.single_triangle(16, 16, light_dist=2.5)
    sc.light_pos = np.array([[0.7, 0.4, 2.2]], np.float32)
    sc.light_intensity = np.array([[3.0, 4.0, 5.0]], np.float32)
    pa = np.array([[0.8, 0.5, 0.3, 0.3, 0.4]], np.float32)
    pb = np.array([[0.2, 0.1, 0.6, 0.3, 0.4]], np.float32)
    oa, ob = O.OracleScene(sc, face_params=pa), O.OracleScene(sc, face_params=pb)
    prm = O.params(1, 5)
    V = sc.vertices.astype(np.float64)
    nrm = np.cross(V[1] - V[0], V[2] - V[0])
    nrm /= np.linalg.norm(nrm)
    hits = 0
    for px in np.linspace(0.5, 15.5, 13):
        for py in np.linspace(0.5, 15.5, 13):
            o, d = G.pixel_ray(sc.views[0], px, py)
            t = ((V[0] - o) @ nrm) / (d @ nrm)
            p = o + t * d
            lam = np.linalg.solve(np.c_[V[1] - V[0], V[2] - V[0], nrm], p - V[0])
            if min(lam[0], lam[1], 1 - lam[0] - lam[1]) < 1e-3:
                continue
            n = nrm if nrm @ -d > 0 else -nrm
            Lp = sc.light_pos[0].astype(np.float64)
            wl = Lp - p
            dist = np.linalg.norm(wl)
            cos = max(0.0, n @ wl / dist)
            dkd = pa[0, :3].astype(np.float64) - pb[0, :3].astype(np.float64)
            exp = dkd / math.pi * sc.light_intensity[0].astype(np.float64) * cos / dist ** 2
            got = O.trace_screen(oa, prm, 0, px, py) - O.trace_screen(ob, prm, 0, px, py)
            np.testing.assert_allclose(got, exp, rtol=1e-10, atol=1e-14)
            hits += 1
    assert hits > 40


@pytest.mark.parametrize("where", ["view", "scene+view", "two view lights"])
def test_view_lights_lambertian_closed_form(where):
    # the same closed form with lights that belong to the view (a light at the
    # camera and one offset from it, as in the paper's captures, Sec. 4): the
    # radiance is the sum over the scene's and the view's lights
    import dataclasses
    sc = S.single_triangle(16, 16, light_dist=2.5)
    eye = np.array(sc.views[0].eye, np.float64)
    A = ((0.7, 0.4, 2.2), (3.0, 4.0, 5.0))
    Bl = (tuple(eye + np.array([0.3, 0.0, 0.0])), (2.0, 1.0, 0.5))
    Cl = (tuple(eye), (1.5, 1.5, 1.5))
    scene_l, view_l = {"view": ([], [A]), "scene+view": ([A], [Bl]), "two view lights": ([], [Cl, Bl])}[where]
    sc.light_pos = np.array([l[0] for l in scene_l], np.float32).reshape(-1, 3)
    sc.light_intensity = np.array([l[1] for l in scene_l], np.float32).reshape(-1, 3)
    sc.views = [dataclasses.replace(sc.views[0], lights=tuple(view_l))]
    pa = np.array([[0.8, 0.5, 0.3, 0.3, 0.4]], np.float32)
    pb = np.array([[0.2, 0.1, 0.6, 0.3, 0.4]], np.float32)
    oa, ob = O.OracleScene(sc, face_params=pa), O.OracleScene(sc, face_params=pb)
    prm = O.params(1, 5)
    V = sc.vertices.astype(np.float64)
    nrm = np.cross(V[1] - V[0], V[2] - V[0])
    nrm /= np.linalg.norm(nrm)
    dkd = pa[0, :3].astype(np.float64) - pb[0, :3].astype(np.float64)
    hits = 0
    for px in np.linspace(0.5, 15.5, 9):
        for py in np.linspace(0.5, 15.5, 9):
            o, d = G.pixel_ray(sc.views[0], px, py)
            t = ((V[0] - o) @ nrm) / (d @ nrm)
            p = o + t * d
            lam = np.linalg.solve(np.c_[V[1] - V[0], V[2] - V[0], nrm], p - V[0])
            if min(lam[0], lam[1], 1 - lam[0] - lam[1]) < 1e-3:
                continue
            n = nrm if nrm @ -d > 0 else -nrm
            exp = np.zeros(3)
            for pos, inten in scene_l + view_l:
                wl = np.array(pos, np.float32).astype(np.float64) - p
                dist = np.linalg.norm(wl)
                exp += dkd / math.pi * np.array(inten, np.float32).astype(np.float64) * max(0.0, n @ wl / dist) / dist ** 2
            got = O.trace_screen(oa, prm, 0, px, py) - O.trace_screen(ob, prm, 0, px, py)
            np.testing.assert_allclose(got, exp, rtol=1e-10, atol=1e-14)
            hits += 1
    assert hits > 20


# ---------------------------------------------------------------------------- white furnace
@pytest.mark.parametrize("B", [1, 2, 3])
def test_white_furnace(B):
    V, F = S.icosphere(1)
    P = np.tile(np.array([[1.0, 1.0, 1.0, 0.0, 0.5]], np.float32), (len(F), 1))
    vs = S.ring_views(1, 20, 64)
    sc = S.Scene("furnace", V.astype(np.float32), F, P, env=np.full((16, 32, 3), 0.7, np.float32), views=vs)
    img, _ = O.render_pixels(O.OracleScene(sc), O.params(B, 17 + B), O.all_pixels(sc))
    x = img[:, 1]
    se = x.std() / math.sqrt(len(x))
    assert abs(x.mean() - 0.7) < 4 * se + 1e-12
    assert abs(np.median(x) - 0.7) < 0.05


def test_environment_irradiance_quadrature():
    # Lambertian (kd = 1) triangle, B = 1: L = (1/pi) * integral of L_env cos over the
    # hemisphere. The quadrature below restates the equirectangular mapping
    # (theta from +y, phi = atan2(x, -z) + pi) independently.
    rng = np.random.default_rng(8)
    env = S.lognormal_env(rng, 16, 8, sigma=0.6)
    sc = S.single_triangle(8, 8)
    sc.face_params = np.array([[1, 1, 1, 0, 0.5]], np.float32)
    sc.light_pos = np.zeros((0, 3), np.float32)
    sc.light_intensity = np.zeros((0, 3), np.float32)
    sc.env = env
    osc = O.OracleScene(sc)
    V = sc.vertices.astype(np.float64)
    n = np.cross(V[1] - V[0], V[2] - V[0])
    n /= np.linalg.norm(n)          # faces the camera at +z
    H, W = env.shape[:2]
    sub = 16
    acc = np.zeros(3)
    for r in range(H):
        for c in range(W):
            th = (r + (np.arange(sub) + 0.5) / sub) * np.pi / H
            ph = (c + (np.arange(sub) + 0.5) / sub) * 2 * np.pi / W
            T, P = np.meshgrid(th, ph, indexing="ij")
            wi = np.stack([-np.sin(T) * np.sin(P), np.cos(T), np.sin(T) * np.cos(P)], -1)
            cos = np.maximum(0, wi @ n)
            acc += env[r, c] * (cos * np.sin(T)).sum() * (np.pi / H / sub) * (2 * np.pi / W / sub)
    exp = acc / np.pi
    prm = O.params(1, 31)
    Ls = np.array([O.trace_screen(osc, prm, 0, 4.2, 4.3, c0=7, c1=s) for s in range(6000)])
    mean, se = Ls.mean(0), Ls.std(0) / math.sqrt(len(Ls))
    assert np.all(np.abs(mean - exp) < 4 * se + 1e-6), (mean, exp, se)


# ---------------------------------------------------------------------------- interior gradient vs FD
def _book_scene(brdf="ggx"):
    """Two quads meeting at a right angle (a concave corner), lit by a light and an environment."""
    V = np.array([[-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0],
                  [-1, -1, 0], [1, -1, 0], [1, -1, 2], [-1, -1, 2]], np.float64)
    V[4:, 1] += 1e-3
    F = np.array([[0, 1, 2], [0, 2, 3], [4, 6, 5], [4, 7, 6]], np.int32)
    rng = np.random.default_rng(9)
    P = np.c_[rng.uniform(0.3, 0.9, (4, 3)), rng.uniform(0.1, 0.6, 4), rng.uniform(0.15, 0.5, 4)].astype(np.float32)
    vs = [S.View((0.3, 1.2, 3.0), (0.0, -0.4, 0.4), (0.0, 1.0, 0.0), 50.0, 16, 16, 1)]
    return S.Scene("book", V.astype(np.float32), F, P, brdf, light_pos=np.array([[0.2, 0.5, 1.2]], np.float32),
                   light_intensity=np.array([[2.0, 1.5, 1.0]], np.float32),
                   env=S.lognormal_env(rng, 16, 8, sigma=0.5), views=vs)


@pytest.mark.parametrize("brdf,B", [("ggx", 1), ("ggx", 3), ("beckmann", 3)])
def test_interior_gradient_matches_tape_replay_fd(brdf, B):
    sc = _book_scene(brdf)
    V0 = sc.vertices.astype(np.float64)
    P0 = sc.face_params.astype(np.float64)
    prm = O.params(B, 1234)
    w = np.array([0.3, -0.7, 0.5])
    checked = 0
    for (px, py, c1) in [(5.3, 9.1, 0), (8.7, 11.2, 1), (10.1, 6.4, 2), (6.6, 12.8, 3), (9.9, 13.3, 4)]:
        osc = O.OracleScene(sc, vertices=V0, face_params=P0)
        rgb, dv, df = O.trace_screen(osc, prm, 0, px, py, c0=11, c1=c1, grad_w=w)
        _, tape = O.trace_screen_taped(osc, prm, 0, px, py, c0=11, c1=c1)
        rgb2 = O.trace_screen_taped(osc, prm, 0, px, py, c0=11, c1=c1, tape=tape)
        np.testing.assert_array_equal(rgb, rgb2)
        if not np.any(dv) and not np.any(df):
            continue
        h = 1e-6
        for (vi, k) in [(i, k) for i in range(len(V0)) for k in range(3) if dv[i, k] != 0]:
            Vp, Vm = V0.copy(), V0.copy()
            Vp[vi, k] += h
            Vm[vi, k] -= h
            fp = O.trace_screen_taped(O.OracleScene(sc, vertices=Vp, face_params=P0), prm, 0, px, py, 11, c1, tape=tape)
            fm = O.trace_screen_taped(O.OracleScene(sc, vertices=Vm, face_params=P0), prm, 0, px, py, 11, c1, tape=tape)
            fd = (w @ fp - w @ fm) / (2 * h)
            assert abs(fd - dv[vi, k]) < 1e-5 * max(1.0, abs(fd)), (vi, k, fd, dv[vi, k])
            checked += 1
        for (fi, k) in [(i, k) for i in range(len(P0)) for k in range(5) if df[i, k] != 0]:
            Pp, Pm = P0.copy(), P0.copy()
            Pp[fi, k] += h
            Pm[fi, k] -= h
            fp = O.trace_screen_taped(O.OracleScene(sc, vertices=V0, face_params=Pp), prm, 0, px, py, 11, c1, tape=tape)
            fm = O.trace_screen_taped(O.OracleScene(sc, vertices=V0, face_params=Pm), prm, 0, px, py, 11, c1, tape=tape)
            fd = (w @ fp - w @ fm) / (2 * h)
            assert abs(fd - df[fi, k]) < 1e-5 * max(1.0, abs(fd)), (fi, k, fd, df[fi, k])
            checked += 1
    assert checked > 20


# ---------------------------------------------------------------------------- edge term
def test_edge_term_matches_area_derivative_of_single_triangle():
    # I_p = integral over (pixel ∩ projected triangle) of L(s) ds (background is black).
    # Its derivative by central differences of a polygon-clipped quadrature, minus
    # the interior term integrated by the same quadrature, is the boundary term the
    # edge estimator must reproduce in expectation.
    sc = S.single_triangle(10, 10)
    v = sc.views[0]
    V0 = sc.vertices.astype(np.float64)
    rng = np.random.default_rng(12)
    wpix = rng.normal(size=(v.height * v.width, 3))
    prm = O.params(1, 0, edge_mode=0, edge_spp=64)

    def J(Vx, interior=False):
        osc = O.OracleScene(sc, vertices=Vx)
        tri2d = G.project(v, Vx)
        tot, gint = 0.0, np.zeros_like(Vx)
        for y in range(v.height):
            for x in range(v.width):
                P = G.clip_polygon(tri2d, x, y, x + 1, y + 1)
                if len(P) < 3:
                    continue
                pts, wts = G.polygon_quadrature(P, subdiv=1)
                wp = wpix[y * v.width + x]
                for (sx, sy), q in zip(pts, wts):
                    if interior:
                        _, dv, _ = O.trace_screen(osc, prm, 0, sx, sy, grad_w=wp * q)
                        gint += dv
                    else:
                        tot += q * (wp @ O.trace_screen(osc, prm, 0, sx, sy))
        return gint if interior else tot

    h = 1e-6
    fd = np.zeros_like(V0)
    for i in range(3):
        for k in range(3):
            Vp, Vm = V0.copy(), V0.copy()
            Vp[i, k] += h
            Vm[i, k] -= h
            fd[i, k] = (J(Vp) - J(Vm)) / (2 * h)
    expected_edge = fd - J(V0, interior=True)
    ests = []
    for seed in range(8):
        dv, _ = O.edge_grad(O.OracleScene(sc), O.params(1, 1000 + seed, edge_mode=0, edge_spp=2048), wpix)
        ests.append(dv)
    ests = np.array(ests)
    mean, se = ests.mean(0), ests.std(0, ddof=1) / math.sqrt(len(ests))
    err = np.abs(mean - expected_edge)
    assert np.all(err < 4 * se + 2e-3 * np.abs(expected_edge).max()), (mean, expected_edge, se)
    # and the estimate is not trivially small
    assert np.abs(expected_edge).max() > 10 * se.max()


@pytest.mark.slow
def test_edge_plus_interior_matches_crn_finite_difference():
    # Small convex mesh, B = 1, one point light, every edge sampled: the sum of the
    # edge and interior estimates has the derivative of the expected image along a
    # random vertex direction as its mean; central differences with common random
    # numbers estimate the same derivative.
    V, F = S.icosphere(1)
    rng = np.random.default_rng(13)
    P = S.random_face_params(rng, len(F))
    vs = S.ring_views(1, 16, 64)
    sc = S.Scene("ico1", V.astype(np.float32), F, P, light_pos=np.array([[0.0, 2.1, 2.1]], np.float32),
                 light_intensity=np.array([[9.0, 9.0, 9.0]], np.float32), views=vs)
    V0 = sc.vertices.astype(np.float64)
    delta = rng.normal(size=V0.shape)
    wimg = rng.normal(size=(sc.n_pixels, 3))
    pix = O.all_pixels(sc)
    grads, fds = [], []
    h = 2e-3
    for seed in range(8):
        prm = O.params(1, 500 + seed, edge_mode=1, edge_spp=64)
        osc = O.OracleScene(sc, vertices=V0)
        dv, _, _ = O.grad_pixels(osc, prm, pix, wimg)
        ev, _ = O.edge_grad(osc, prm, wimg)
        grads.append(((dv + ev) * delta).sum())
        ip, _ = O.render_pixels(O.OracleScene(sc, vertices=V0 + h * delta), prm, pix)
        im, _ = O.render_pixels(O.OracleScene(sc, vertices=V0 - h * delta), prm, pix)
        fds.append(((ip - im) * wimg).sum() / (2 * h))
    g, f = np.array(grads), np.array(fds)
    se = math.sqrt(g.var(ddof=1) / len(g) + f.var(ddof=1) / len(f))
    assert abs(g.mean() - f.mean()) < 3 * se + 1e-3 * abs(f.mean()), (g.mean(), f.mean(), se)


# ---------------------------------------------------------------------------- mesh colors r > 0
def _texel_index(r, t, alpha, beta):
    i = min(max(int(math.floor(r * alpha)), 0), r)
    j = min(max(int(math.floor(r * beta)), 0), r - i)
    return (t * (r + 1) * (r + 2) + i * (2 * r - i + 3)) // 2 + j


def test_mesh_colors_uniform_texels_equal_per_face():
    sc = S.tiny(res=24, spp=2)
    r = 2
    n = (r + 1) * (r + 2) // 2
    P = np.repeat(sc.face_params, n, axis=0)
    ref, _ = O.render_pixels(O.OracleScene(sc), O.params(2, 3), O.all_pixels(sc))
    sc2 = S.tiny(res=24, spp=2)
    sc2.color_res = r
    got, _ = O.render_pixels(O.OracleScene(sc2, face_params=P), O.params(2, 3), O.all_pixels(sc2))
    np.testing.assert_array_equal(got, ref)


def test_mesh_colors_texel_lookup_on_a_triangle():
    # one Lambertian triangle, r = 3 (10 texels, each its own kd); at screen points
    # of known barycentrics the radiance difference of two kd sets isolates the
    # texel the estimator used: (kd_a - kd_b)[k] / pi * I cos / d^2
    r = 3
    sc = S.single_triangle(16, 16, light_dist=2.5)
    sc.color_res = r
    sc.light_pos = np.array([[0.3, -0.2, 2.4]], np.float32)
    sc.light_intensity = np.array([[5.0, 5.0, 5.0]], np.float32)
    n = (r + 1) * (r + 2) // 2
    rng = np.random.default_rng(21)
    Pa = np.c_[rng.uniform(0.1, 0.9, (n, 3)), np.zeros(n), np.full(n, 0.5)]
    Pb = np.c_[rng.uniform(0.1, 0.9, (n, 3)), np.zeros(n), np.full(n, 0.5)]
    oa, ob = O.OracleScene(sc, face_params=Pa), O.OracleScene(sc, face_params=Pb)
    prm = O.params(1, 5)
    V = sc.vertices.astype(np.float64)
    nrm = np.cross(V[1] - V[0], V[2] - V[0])
    nrm /= np.linalg.norm(nrm)
    seen = set()
    for px in np.linspace(0.25, 15.75, 48):
        for py in np.linspace(0.25, 15.75, 48):
            o, d = G.pixel_ray(sc.views[0], px, py)
            t = ((V[0] - o) @ nrm) / (d @ nrm)
            p = o + t * d
            # weights (w0, alpha, beta) of v0, v1, v2
            alpha, beta = np.linalg.lstsq(np.c_[V[1] - V[0], V[2] - V[0]], p - V[0], rcond=None)[0]
            w0 = 1 - alpha - beta
            if min(w0, alpha, beta) < 1e-3:
                continue
            ra, rb = r * alpha, r * beta
            if min(abs(ra - round(ra)), abs(rb - round(rb))) < 1e-6:
                continue
            k = _texel_index(r, 0, alpha, beta)
            seen.add(k)
            Lp = sc.light_pos[0].astype(np.float64)
            wl = Lp - p
            dist = np.linalg.norm(wl)
            n_ = nrm if nrm @ -d > 0 else -nrm
            exp = (Pa[k, :3] - Pb[k, :3]) / math.pi * 5.0 * max(0.0, n_ @ wl / dist) / dist ** 2
            got = O.trace_screen(oa, prm, 0, px, py) - O.trace_screen(ob, prm, 0, px, py)
            np.testing.assert_allclose(got, exp, rtol=1e-9, atol=1e-13)
    # every texel reachable from the triangle's interior (i + j < r) was used; the
    # others (i + j = r) are met only on the edge alpha + beta = 1
    interior = {_texel_index(r, 0, (i + 0.5) / r, (j + 0.5) / r) for i in range(r) for j in range(r - i)}
    assert seen == interior, (seen, interior)


def test_mesh_colors_texel_gradient_matches_tape_replay_fd():
    sc = _book_scene()
    r = 2
    n = (r + 1) * (r + 2) // 2
    sc.color_res = r
    rng = np.random.default_rng(22)
    P0 = np.repeat(sc.face_params.astype(np.float64), n, axis=0)
    P0[:, :3] = np.clip(P0[:, :3] + rng.normal(0, 0.1, (len(P0), 3)), 0.05, 0.95)
    V0 = sc.vertices.astype(np.float64)
    prm = O.params(3, 99)
    w = np.array([0.4, -0.2, 0.9])
    checked = 0
    for (px, py, c1) in [(5.3, 9.1, 0), (8.7, 11.2, 1), (10.1, 6.4, 2)]:
        osc = O.OracleScene(sc, vertices=V0, face_params=P0)
        _, dv, df = O.trace_screen(osc, prm, 0, px, py, c0=3, c1=c1, grad_w=w)
        _, tape = O.trace_screen_taped(osc, prm, 0, px, py, c0=3, c1=c1)
        h = 1e-6
        for (ti, k) in [(i, k) for i in range(len(P0)) for k in range(5) if df[i, k] != 0]:
            Pp, Pm = P0.copy(), P0.copy()
            Pp[ti, k] += h
            Pm[ti, k] -= h
            fp = O.trace_screen_taped(O.OracleScene(sc, vertices=V0, face_params=Pp), prm, 0, px, py, 3, c1, tape=tape)
            fm = O.trace_screen_taped(O.OracleScene(sc, vertices=V0, face_params=Pm), prm, 0, px, py, 3, c1, tape=tape)
            fd = (w @ fp - w @ fm) / (2 * h)
            assert abs(fd - df[ti, k]) < 1e-5 * max(1.0, abs(fd)), (ti, k, fd, df[ti, k])
            checked += 1
    assert checked > 10


# ---------------------------------------------------------------------------- path signatures
def _fnv(h, x):
    return ((h ^ x) * 0x100000001b3) & 0xffffffffffffffff


def test_path_signature_closed_cases():
    # one Lambertian triangle facing the camera, one point light, one vertex per path:
    # a covered pixel's paths hit face 0 and then either see the light (visibility
    # bit 0) or trace no shadow ray (light behind the face); an uncovered pixel's
    # paths miss. The pixel signature is spp times the path hash, modulo 2^64.
    basis = 0xcbf29ce484222325
    spp = 4
    for light_z, expect_hit in [(2.5, _fnv(_fnv(basis, 0), 1)), (-2.5, _fnv(basis, 0))]:
        sc = S.single_triangle(16, 16, light_dist=2.5)
        sc.light_pos = np.array([[0.0, 0.0, light_z]], np.float32)
        sc.views[0].spp = spp
        sig = O.render_signatures(O.OracleScene(sc), O.params(1, 3), np.array([[0, 8, 8], [0, 0, 0]], np.int32))
        assert int(sig[0]) == (spp * expect_hit) & 0xffffffffffffffff
        assert int(sig[1]) == (spp * _fnv(basis, 0xffffffff)) & 0xffffffffffffffff


def _camera_dirs(v, x, y, seed):
    # per sample: the jittered pinhole direction through pixel (x, y), jitter from the
    # camera counter (pixel_offset + y W + x, sample, 0, 0) of Philox keyed by the seed
    e, t, up = (np.array(a, np.float64) for a in (v.eye, v.target, v.up))
    fwd = (t - e) / np.linalg.norm(t - e)
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    th = np.tan(np.radians(v.fov_y_deg) / 2)
    out = []
    for smp in range(v.spp):
        u = O.philox([v.pixel_offset + y * v.width + x, smp, 0, 0], [seed & 0xffffffff, seed >> 32])
        px, py = x + (int(u[0]) >> 8) / 2.0 ** 24, y + (int(u[1]) >> 8) / 2.0 ** 24
        sx, sy = 2 * px / v.width - 1, 1 - 2 * py / v.height
        d = fwd + right * sx * th * v.width / v.height + upv * sy * th
        out.append(d / np.linalg.norm(d))
    return out


def test_path_signature_holds_the_texel_a_miss_reads_and_the_texel_a_hit_picks():
    # a miss under an environment hashes the equirectangular texel its direction
    # reads (theta from +y, phi = atan2(x, -z) + pi); a hit with mesh colors at
    # r = 2 hashes its texel k = (t (r+1)(r+2) + i (2r - i + 3)) / 2 + j,
    # (i, j) = floor(r (alpha, beta)); both restated here from the camera model
    basis, seed, spp, M = 0xcbf29ce484222325, 3, 6, 0xffffffffffffffff
    sc = S.single_triangle(16, 16, light_dist=2.5)
    sc.light_pos = np.array([[0.0, 0.0, 2.5]], np.float32)
    sc.views[0].spp = spp
    rng = np.random.default_rng(2)
    W, H = 16, 8
    sc.env = rng.lognormal(0, 1, (H, W, 3)).astype(np.float32)
    v = sc.views[0]
    want = 0
    for d in _camera_dirs(v, 0, 0, seed):
        phi = np.arctan2(d[0], -d[2]) + np.pi
        col = min(int(phi / (2 * np.pi) * W), W - 1)
        row = min(int(np.arccos(np.clip(d[1], -1, 1)) / np.pi * H), H - 1)
        want += _fnv(_fnv(basis, 0xffffffff), row * W + col)
    sig = O.render_signatures(O.OracleScene(sc), O.params(1, seed), np.array([[0, 0, 0]], np.int32))
    assert int(sig[0]) == want & M

    # mesh colors at r = 2 under the point light alone (no environment, so no NEE texel draw)
    sc.env = None
    r = 2
    n_tex = (r + 1) * (r + 2) // 2
    sc.color_res = r
    sc.face_params = np.repeat(sc.face_params, n_tex, axis=0)
    V = sc.vertices.astype(np.float64)
    e1, e2 = V[1] - V[0], V[2] - V[0]
    want, ks = 0, set()
    for d in _camera_dirs(v, 8, 8, seed):
        p = np.array(v.eye) + d * (-v.eye[2] / d[2])          # the triangle lies in z = 0
        a, b = np.linalg.solve(np.c_[e1[:2], e2[:2]], (p - V[0])[:2])
        i = min(max(int(np.floor(r * a)), 0), r)
        j = min(max(int(np.floor(r * b)), 0), r - i)
        k = (0 * (r + 1) * (r + 2) + i * (2 * r - i + 3)) // 2 + j
        ks.add(k)
        want += _fnv(_fnv(_fnv(basis, 0), k), 1)
    sig = O.render_signatures(O.OracleScene(sc), O.params(1, seed), np.array([[0, 8, 8]], np.int32))
    assert int(sig[0]) == want & M


def test_path_signature_depends_on_decisions_only():
    # with ks = 0 the lobe probability is the same for any albedo, so changing kd
    # changes the pixel values but no decision: equal signatures; moving the
    # mesh changes the faces hit: different signatures
    sc = S.tiny(res=16, spp=2)
    P = sc.face_params.copy()
    P[:, 3] = 0.0
    P2 = P.copy()
    P2[:, :3] = np.clip(P2[:, :3] * 0.5 + 0.2, 0, 1)
    pix = O.all_pixels(sc)
    prm = O.params(3, 17)
    a = O.render_signatures(O.OracleScene(sc, face_params=P), prm, pix)
    b = O.render_signatures(O.OracleScene(sc, face_params=P2), prm, pix)
    va, _ = O.render_pixels(O.OracleScene(sc, face_params=P), prm, pix)
    vb, _ = O.render_pixels(O.OracleScene(sc, face_params=P2), prm, pix)
    np.testing.assert_array_equal(a, b)
    assert np.abs(va - vb).max() > 1e-3
    V2 = sc.vertices.astype(np.float64) * 1.05
    c = O.render_signatures(O.OracleScene(sc, vertices=V2, face_params=P), prm, pix)
    assert (c != a).mean() > 0.2


# ---------------------------------------------------------------------------- RGB specular (7 parameters)
def _rgb_params(P5, ks_rgb):
    return np.c_[P5[:, :3], ks_rgb, P5[:, 4]].astype(np.float64)


@pytest.mark.parametrize("brdf", ["ggx", "beckmann"])
def test_rgb_specular_normal_incidence_closed_form(brdf):
    # light at the eye, ray along the view axis onto a triangle facing the camera:
    # wi = wo = n, so D = 1 / (pi alpha^2), G1 = 1 and L_c = (kd_c / pi + ks_c / (4 pi alpha^2)) I / d^2
    sc = S.single_triangle(16, 16)
    sc.brdf = brdf
    sc.light_pos = np.array([sc.views[0].eye], np.float32)
    sc.light_intensity = np.array([[2.0, 3.0, 4.0]], np.float32)
    kd, ks, alpha = np.array([0.3, 0.5, 0.2]), np.array([0.6, 0.1, 0.35]), 0.4
    P = np.array([np.r_[kd, ks, alpha]])
    got = O.trace_screen(O.OracleScene(sc, face_params=P), O.params(1, 0), 0, 8.0, 8.0)
    d = float(np.linalg.norm(np.array(sc.views[0].eye, np.float64)))
    exp = (kd / math.pi + ks / (4 * math.pi * alpha ** 2)) * np.array([2.0, 3.0, 4.0]) / d ** 2
    np.testing.assert_allclose(got, exp, rtol=1e-12)


def test_rgb_specular_with_equal_channels_equals_scalar_specular():
    sc = S.tiny(res=16, spp=2)
    P5 = sc.face_params.astype(np.float64)
    P7 = _rgb_params(P5, np.repeat(P5[:, 3:4], 3, axis=1))
    pix = O.all_pixels(sc)
    a, _ = O.render_pixels(O.OracleScene(sc, face_params=P5), O.params(3, 4), pix)
    b, _ = O.render_pixels(O.OracleScene(sc, face_params=P7), O.params(3, 4), pix)
    np.testing.assert_array_equal(a, b)
    w = np.random.default_rng(1).normal(size=a.shape)
    _, f5, _ = O.grad_pixels(O.OracleScene(sc, face_params=P5), O.params(3, 4), pix, w)
    _, f7, _ = O.grad_pixels(O.OracleScene(sc, face_params=P7), O.params(3, 4), pix, w)
    # the scalar specular's derivative is the sum of the three channels'
    np.testing.assert_allclose(f7[:, 3:6].sum(1), f5[:, 3], rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(f7[:, [0, 1, 2, 6]], f5[:, [0, 1, 2, 4]], rtol=1e-9, atol=1e-14)


def test_rgb_specular_gradient_matches_tape_replay_fd():
    sc = _book_scene()
    rng = np.random.default_rng(23)
    P0 = _rgb_params(sc.face_params.astype(np.float64), rng.uniform(0.05, 0.6, (len(sc.faces), 3)))
    V0 = sc.vertices.astype(np.float64)
    prm = O.params(3, 77)
    w = np.array([0.4, -0.3, 0.8])
    checked = 0
    for (px, py, c1) in [(5.3, 9.1, 0), (8.7, 11.2, 1), (10.1, 6.4, 2)]:
        osc = O.OracleScene(sc, vertices=V0, face_params=P0)
        _, dv, df = O.trace_screen(osc, prm, 0, px, py, c0=5, c1=c1, grad_w=w)
        _, tape = O.trace_screen_taped(osc, prm, 0, px, py, c0=5, c1=c1)
        h = 1e-6
        for (ti, k) in [(i, k) for i in range(len(P0)) for k in range(7) if df[i, k] != 0]:
            Pp, Pm = P0.copy(), P0.copy()
            Pp[ti, k] += h
            Pm[ti, k] -= h
            fp = O.trace_screen_taped(O.OracleScene(sc, vertices=V0, face_params=Pp), prm, 0, px, py, 5, c1, tape=tape)
            fm = O.trace_screen_taped(O.OracleScene(sc, vertices=V0, face_params=Pm), prm, 0, px, py, 5, c1, tape=tape)
            fd = (w @ fp - w @ fm) / (2 * h)
            assert abs(fd - df[ti, k]) < 1e-5 * max(1.0, abs(fd)), (ti, k, fd, df[ti, k])
            checked += 1
    assert checked > 12
