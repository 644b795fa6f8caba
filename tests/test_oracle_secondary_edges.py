"""Pins of the oracle's secondary-visibility edge term (boundary term at every path vertex).

At a path vertex the estimator integrates f cos L_in over incoming directions;
L_in jumps where a direction crosses a mesh edge that occludes what lies
behind it. Moving the mesh moves those jumps, and the boundary (edge) term
accounts for it. The pins below check the oracle's estimate of it against
values that neither the oracle nor the CUDA library computes:

* a closed form: a Lambertian floor under a uniform environment, shadowed by a
  floating triangle, has L_o = kd L0 (1 - P/pi) with P the triangle's projected
  solid angle (Lambert's polygon formula), so every pixel's derivative with
  respect to every vertex follows from Gauss quadrature over the pixel and
  central differences;
* a two-bounce quadrature: the same floor lit only from below the horizon, so
  all its light arrives after one reflection off the floating triangle's
  underside (itself lit by the environment around the floor). The pixel value is
  then a smooth integral over the triangle of the underside's closed-form
  radiance, which Gauss quadrature evaluates to high accuracy.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2012_03939_gb300 import scenes as S
from tests import _geom as G


def _ray_tri(o, d, a, b, c):
    """Möller-Trumbore for many rays (o [3], d [N,3]) against one triangle: t [N] (inf on a miss)."""
    e1, e2 = b - a, c - a
    pv = np.cross(d, e2)
    det = pv @ e1
    inv = 1.0 / det
    tv = o - a
    u = (pv @ tv) * inv
    qv = np.cross(tv, e1)
    v = (d @ qv) * inv
    t = (qv @ e2) * inv
    ok = (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0)
    return np.where(ok, t, np.inf)


def _projected_solid_angle(p, n, poly):
    """Lambert's formula: projected solid angle of a polygon above the horizon, seen from points p [N,3]."""
    tot = np.zeros(len(p))
    k = len(poly)
    for i in range(k):
        a, b = poly[i] - p, poly[(i + 1) % k] - p
        c = np.cross(a, b)
        cn = np.linalg.norm(c, axis=1)
        theta = np.arctan2(cn, np.einsum("ij,ij->i", a, b))
        tot += theta * np.einsum("ij,ij->i", n, c) / cn
    return np.abs(tot) / 2


def _occluder_scene(spp=1):
    V = np.array([[-3, 0, -3], [3, 0, -3], [3, 0, 3], [-3, 0, 3],
                  [-0.45, 0.30, -0.30], [0.50, 0.38, -0.15], [0.05, 0.33, 0.55]], np.float64)
    F = np.array([[0, 2, 1], [0, 3, 2], [4, 5, 6]], np.int32)
    P = np.array([[0.7, 0.5, 0.3, 0.0, 0.5], [0.7, 0.5, 0.3, 0.0, 0.5], [0.5, 0.5, 0.5, 0.0, 0.5]], np.float32)
    env = np.ones((4, 8, 3), np.float32)
    vs = [S.View((0.9, 2.2, 1.6), (0.0, 0.0, 0.1), (0.0, 1.0, 0.0), 40.0, 12, 12, spp)]
    return S.Scene("occluder", V.astype(np.float32), F, P, "ggx", env=env, views=vs, max_bounces=1)


def _pixel_rays(v, pix, n_gauss):
    """Eye and unit directions of an n x n Gauss-Legendre rule over every listed pixel: d [pixels * n^2, 3]."""
    gx, gw = np.polynomial.legendre.leggauss(n_gauss)
    gx, gw = (gx + 1) / 2, gw / 2
    ux, uy = np.meshgrid(gx, gx)
    eye, fwd, right, up, th = G.camera_frame(v)
    px = (pix[:, 1:2] + ux.ravel()[None, :]).ravel()
    py = (pix[:, 2:3] + uy.ravel()[None, :]).ravel()
    sx = 2 * px / v.width - 1
    sy = 1 - 2 * py / v.height
    d = fwd[None, :] + right[None, :] * (sx * th * v.width / v.height)[:, None] + up[None, :] * (sy * th)[:, None]
    return eye, d / np.linalg.norm(d, axis=1, keepdims=True), np.outer(gw, gw).ravel()


def _floor_hits(V, o, d):
    """Hit points and normals (facing the ray's origin) of rays on the two floor triangles of V."""
    floor = [V[[0, 2, 1]], V[[0, 3, 2]]]
    ts = np.stack([_ray_tri(o, d, *tri) for tri in floor])
    k = np.argmin(ts, 0)
    t = ts[k, np.arange(len(d))]
    assert np.all(np.isfinite(t))
    p = o + d * t[:, None]
    n = np.stack([np.cross(tri[1] - tri[0], tri[2] - tri[0]) for tri in floor])[k]
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    n *= np.where(np.einsum("ij,ij->i", n, d) < 0, 1.0, -1.0)[:, None]
    return p, n


def _free_pixels(sc):
    v = sc.views[0]
    occ = G.project(v, sc.vertices[4:7].astype(np.float64))
    out = []
    for y in range(v.height):
        for x in range(v.width):
            if len(G.clip_polygon(occ, x - 0.05, y - 0.05, x + 1.05, y + 1.05)) < 3:
                out.append((0, x, y))
    return np.array(out, np.int32)


def _closed_form_pixels(sc, V, pix, n_gauss=8):
    """Pixel means of kd L0 (1 - P/pi) over each pixel (Gauss-Legendre), camera rays on the floor of V."""
    eye, d, wpx = _pixel_rays(sc.views[0], pix, n_gauss)
    p, n = _floor_hits(V, eye, d)
    occ = V[4:7]
    assert np.all(occ[None, :, 1] - p[:, None, 1] > 0.2)
    L = (1.0 - _projected_solid_angle(p, n, occ) / math.pi).reshape(len(pix), -1) @ wpx
    return L[:, None] * sc.face_params[0, :3].astype(np.float64)[None, :]


def test_closed_form_occluded_floor_value():
    # the forward estimator itself reproduces the closed form (B = 1: one vertex,
    # environment NEE). A uniform environment is sampled uniformly over the sphere,
    # so one sample is 4 kd cos(theta) on the upper hemisphere and 0 below: its
    # standard deviation is at most sqrt(5/3) kd.
    spp = 1 << 15
    sc = _occluder_scene(spp=spp)
    pix = _free_pixels(sc)[::5]
    exp = _closed_form_pixels(sc, sc.vertices.astype(np.float64), pix)
    got, _ = O.render_pixels(O.OracleScene(sc), O.params(1, 3), pix)
    se = math.sqrt(5.0 / 3.0) * sc.face_params[0, :3] / math.sqrt(spp)
    assert np.all(np.abs(got - exp) < 4 * se), (got, exp, se)
    assert exp.min() < 0.8 * exp.max()     # the pixels include the penumbra


@pytest.mark.parametrize("sampling,edge_mode", [(1, 0), (2, 0), (2, 1)])
def test_secondary_edge_gradient_matches_closed_form(sampling, edge_mode):
    # sampling 1: one edge picked uniformly; 2: picked through the edge hierarchy
    # (edge_mode 1: every edge is a candidate, so the normal cones drop nothing;
    # the scene has no shading discontinuity, so the expectation is the same)
    sc = _occluder_scene(spp=512)
    pix = _free_pixels(sc)
    V0 = sc.vertices.astype(np.float64)
    rng = np.random.default_rng(31)
    w = rng.normal(size=(len(pix), 3))
    h = 1e-5
    exp = np.zeros_like(V0)
    for vi in range(len(V0)):
        for k in range(3):
            Vp, Vm = V0.copy(), V0.copy()
            Vp[vi, k] += h
            Vm[vi, k] -= h
            exp[vi, k] = ((_closed_form_pixels(sc, Vp, pix) - _closed_form_pixels(sc, Vm, pix)) * w).sum() / (2 * h)
    ests, plain = [], []
    osc = O.OracleScene(sc)
    for seed in range(8):
        dv, _, _ = O.grad_pixels(osc, O.params(1, 700 + seed, edge_mode=edge_mode, secondary=sampling), pix, w)
        ests.append(dv)
        if seed < 2:
            plain.append(O.grad_pixels(osc, O.params(1, 700 + seed), pix, w)[0])
    ests = np.array(ests)
    mean, se = ests.mean(0), ests.std(0, ddof=1) / math.sqrt(len(ests))
    scale = np.abs(exp).max()
    assert np.all(np.abs(mean - exp) < 4 * se + 2e-3 * scale), (mean, exp, se)
    # the occluder's vertices receive their whole gradient from the boundary term:
    # without it the estimate is exactly zero there
    assert np.abs(exp[4:]).max() > 0.2 * scale
    assert np.all(np.array(plain)[:, 4:] == 0)



def _duffy_rule(n):
    """Barycentric points (alpha, beta) and weights (summing to 1/2) of an n x n Gauss rule on the unit triangle."""
    g, w = np.polynomial.legendre.leggauss(n)
    g, w = (g + 1) / 2, w / 2
    u, v = np.meshgrid(g, g, indexing="ij")
    wu, wv = np.meshgrid(w, w, indexing="ij")
    return u.ravel(), (v * (1 - u)).ravel(), (wu * wv * (1 - u)).ravel()


def _underside_scene(spp=1, L0=100.0):
    V = np.array([[-1.5, 0, -1.5], [1.5, 0, -1.5], [1.5, 0, 1.5], [-1.5, 0, 1.5],
                  [-0.45, 0.6, -0.30], [0.50, 0.6, -0.15], [0.05, 0.6, 0.55]], np.float64)
    F = np.array([[0, 2, 1], [0, 3, 2], [4, 5, 6]], np.int32)
    P = np.array([[0.7, 0.5, 0.3, 0.0, 0.5], [0.7, 0.5, 0.3, 0.0, 0.5], [0.4, 0.6, 0.8, 0.0, 0.5]], np.float32)
    env = np.zeros((4, 8, 3), np.float32)
    env[2:] = L0                     # rows below the horizon (theta > pi/2) only
    vs = [S.View((0.9, 2.2, 1.6), (0.0, 0.0, 0.1), (0.0, 1.0, 0.0), 40.0, 12, 12, spp)]
    return S.Scene("underside", V.astype(np.float32), F, P, "ggx", env=env, views=vs, max_bounces=2)


def _floor_pixels(sc):
    v = sc.views[0]
    V = sc.vertices.astype(np.float64)
    occ = G.project(v, V[4:7])
    floor = G.project(v, V[0:4])
    out = []
    for y in range(v.height):
        for x in range(v.width):
            inside = abs(G.polygon_area(G.clip_polygon(floor, x - 0.05, y - 0.05, x + 1.05, y + 1.05)) - 1.21) < 1e-9
            if inside and len(G.clip_polygon(occ, x - 0.05, y - 0.05, x + 1.05, y + 1.05)) < 3:
                out.append((0, x, y))
    return np.array(out, np.int32)


def _two_bounce_pixels(sc, V, pix, L0=100.0, n_gauss=4, n_tri=12):
    """Pixel means of the B = 2 estimator's expectation: floor point p receives, from every point q
    of the triangle's underside, L1(q) = kd_o L0 (1 - P_floor(q)/pi) (the environment below the
    horizon that the floor does not hide), times the geometry term cos_p cos_q / r^2."""
    kd_f = sc.face_params[0, :3].astype(np.float64)
    kd_o = sc.face_params[2, :3].astype(np.float64)
    floor = [V[[0, 2, 1]], V[[0, 3, 2]]]
    a, b, c = V[4], V[5], V[6]
    al, be, wq = _duffy_rule(n_tri)
    q = a + al[:, None] * (b - a) + be[:, None] * (c - a)
    m = np.cross(b - a, c - a)
    area2 = np.linalg.norm(m)
    nq = m / area2
    if nq[1] > 0:
        nq = -nq                          # the underside faces the floor
    nqs = np.broadcast_to(nq, q.shape)
    for tri in floor:
        assert np.all((tri[None, :, :] - q[:, None, :]) @ nq > 0.1)
    L1 = 1.0 - sum(_projected_solid_angle(q, nqs, tri) for tri in floor) / math.pi   # times kd_o L0
    wq = wq * area2                       # dA = |m| d(alpha) d(beta)
    eye, d, wpx = _pixel_rays(sc.views[0], pix, n_gauss)
    p, npf = _floor_hits(V, eye, d)
    dv = q[None, :, :] - p[:, None, :]                      # [pixel points, q points, 3]
    r2 = np.einsum("ijk,ijk->ij", dv, dv)
    r = np.sqrt(r2)
    cp = np.einsum("ijk,ik->ij", dv, npf) / r
    cq = -(dv @ nq) / r
    assert np.all(cp > 0) and np.all(cq > 0)
    E = ((cp * cq / r2 * L1[None, :]) @ wq).reshape(len(pix), -1) @ wpx
    return E[:, None] * (kd_f * kd_o * L0 / math.pi)[None, :]


def test_two_bounce_quadrature_value():
    spp = 1 << 14
    sc = _underside_scene(spp=spp)
    pix = _floor_pixels(sc)[::4]
    exp = _two_bounce_pixels(sc, sc.vertices.astype(np.float64), pix)
    vals = np.array([O.render_pixels(O.OracleScene(sc), O.params(2, 40 + s), pix)[0] for s in range(4)])
    mean, se = vals.mean(0), vals.std(0, ddof=1) / 2
    assert np.all(np.abs(mean - exp) < 4 * se + 1e-3 * exp.max()), (mean, exp, se)
    assert exp.min() > 0.02


@pytest.mark.parametrize("sampling", [1, 2])
def test_secondary_edge_gradient_two_bounces_matches_quadrature(sampling):
    # every bit of the floor's light takes two bounces, so the gradient exercises
    # side paths that continue to a shaded vertex (edges seen from the floor) and
    # edges seen from the triangle's underside (the floor's boundary), with the
    # vertex-motion part chained back through the earlier vertex
    sc = _underside_scene(spp=4096)
    pix = _floor_pixels(sc)
    V0 = sc.vertices.astype(np.float64)
    rng = np.random.default_rng(32)
    w = rng.normal(size=(len(pix), 3))
    h = 1e-5
    exp = np.zeros_like(V0)
    for vi in range(len(V0)):
        for k in range(3):
            Vp, Vm = V0.copy(), V0.copy()
            Vp[vi, k] += h
            Vm[vi, k] -= h
            exp[vi, k] = ((_two_bounce_pixels(sc, Vp, pix) - _two_bounce_pixels(sc, Vm, pix)) * w).sum() / (2 * h)
    osc = O.OracleScene(sc)
    ests = np.array([O.grad_pixels(osc, O.params(2, 800 + s, secondary=sampling), pix, w)[0] for s in range(8)])
    mean, se = ests.mean(0), ests.std(0, ddof=1) / math.sqrt(len(ests))
    scale = np.abs(exp).max()
    assert np.all(np.abs(mean - exp) < 4 * se + 2e-3 * scale), (mean, exp, se)
    # the pin tells the full estimator from one without the boundary term
    plain = np.array([O.grad_pixels(osc, O.params(2, 800 + s), pix, w)[0] for s in range(4)]).mean(0)
    assert (np.abs(plain - exp) / (se + 1e-3 * scale)).max() > 10, (plain, exp, se)


# ---------------------------------------------------------------------------- edge hierarchy (importance pick)
def _tangent_frames(sc, n, seed):
    """Points just off random faces of the mesh with the face normal: (p, n) pairs."""
    rng = np.random.default_rng(seed)
    V = sc.vertices.astype(np.float64)
    out = []
    for f in rng.integers(0, len(sc.faces), size=n):
        a, b, c = V[sc.faces[f]]
        u, v = rng.random(2)
        if u + v > 1:
            u, v = 1 - u, 1 - v
        m = np.cross(b - a, c - a)
        m /= np.linalg.norm(m)
        out.append((a + u * (b - a) + v * (c - a) + 1e-4 * m, m * rng.choice([-1.0, 1.0])))
    return out


def _edges_and_faces(sc):
    """Edges in edge order (sorted vertex pairs) with their two faces (-1 if fewer)."""
    F = sc.faces
    pairs = {}
    for f in range(len(F)):
        for a, b in ((F[f, 0], F[f, 1]), (F[f, 1], F[f, 2]), (F[f, 2], F[f, 0])):
            pairs.setdefault((min(a, b), max(a, b)), []).append(f)
    keys = sorted(pairs)
    return np.array(keys), [pairs[k] for k in keys]


@pytest.mark.parametrize("edge_mode", [0, 1])
def test_hierarchy_pick_probabilities(edge_mode):
    # every edge the sample can use -- a part above the tangent plane and, when
    # sampling silhouettes, one face seeing the vertex and the other not -- can
    # be picked (so the estimator stays unbiased); the mass never exceeds one; a
    # pick returns the probability the enumeration gives; picks follow it
    sc = S.small_variant(S.make("env"), n_views=1, max_res=8, spp=1)
    osc = O.OracleScene(sc)
    V = sc.vertices.astype(np.float64)
    ev, ef = _edges_and_faces(sc)
    tri = V[sc.faces]
    un = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    un /= np.linalg.norm(un, axis=1, keepdims=True)
    for k, (p, n) in enumerate(_tangent_frames(sc, 6, 4)):
        bnd = 1e-5 * (1 + np.abs(p).max())
        pmf = O.sec_edge_pmf(osc, p, n, bnd, edge_mode)
        assert len(pmf) == len(ev) and pmf.sum() <= 1 + 1e-12
        usable = np.maximum((V[ev[:, 0]] - p) @ n, (V[ev[:, 1]] - p) @ n) > bnd
        if edge_mode == 0:
            side = np.einsum("ij,ij->i", un, p - tri[:, 0])
            sil = np.array([len(fs) != 2 or (side[fs[0]] > bnd and side[fs[1]] < -bnd) or
                            (side[fs[0]] < -bnd and side[fs[1]] > bnd) for fs in ef])
            usable &= sil
            assert (pmf[~sil] == 0).mean() > 0.5     # the cones rule most of the rest out
        assert np.all(pmf[usable] > 0)
        if k < 2:
            N = 40000
            e, pr = O.sec_edge_picks(osc, 11, k, 1, 0, p, n, bnd, np.random.default_rng(k).integers(0, 1 << 32, N),
                                     edge_mode)
            ok = e >= 0
            np.testing.assert_allclose(pr[ok], pmf[e[ok]], rtol=1e-12)
            cnt = np.bincount(e[ok], minlength=len(pmf)).astype(np.float64)
            # chi^2 over 40 groups of edges of equal probability mass (most edges are rare)
            order = np.argsort(pmf)
            grp = np.minimum((np.cumsum(pmf[order]) / pmf.sum() * 40).astype(int), 39)
            exp_g = np.bincount(grp, weights=N * pmf[order], minlength=40)
            got_g = np.bincount(grp, weights=cnt[order], minlength=40)
            chi2 = ((got_g - exp_g) ** 2 / exp_g).sum()
            assert chi2 < 39 + 6 * math.sqrt(2 * 39), chi2
            assert abs(cnt.sum() - N * pmf.sum()) < 6 * math.sqrt(N)


def test_hierarchy_pick_lands_on_usable_edges_more_often():
    # the chance that a pick can become a sample -- a silhouette seen from the
    # vertex with a part above its tangent plane -- averaged over vertices of
    # the self-occluding torus knot: the hierarchy (boxes below the plane and
    # cones without silhouettes dropped, near edges favoured) against the
    # uniform pick, computed exactly from the probabilities
    sc = S.small_variant(S.make("env"), n_views=1, max_res=8, spp=1)
    osc = O.OracleScene(sc)
    V = sc.vertices.astype(np.float64)
    ev, ef = _edges_and_faces(sc)
    tri = V[sc.faces]
    un = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    un /= np.linalg.norm(un, axis=1, keepdims=True)
    f0 = np.array([fs[0] for fs in ef])
    f1 = np.array([fs[1] for fs in ef])
    tree, unif = [], []
    for p, n in _tangent_frames(sc, 30, 9):
        bnd = 1e-5 * (1 + np.abs(p).max())
        side = np.einsum("ij,ij->i", un, p - tri[:, 0])
        sil = ((side[f0] > bnd) & (side[f1] < -bnd)) | ((side[f0] < -bnd) & (side[f1] > bnd))
        usable = sil & (np.maximum((V[ev[:, 0]] - p) @ n, (V[ev[:, 1]] - p) @ n) > bnd)
        tree.append(O.sec_edge_pmf(osc, p, n, bnd)[usable].sum())
        unif.append(usable.mean())
    assert np.mean(tree) > 3 * np.mean(unif) > 0, (np.mean(tree), np.mean(unif))


def _py_tree(sc):
    """The edge hierarchy restated in numpy from its definition (blocks of G edges in edge order under a
    complete binary tree; boxes, summed lengths and normal cones)."""
    V = sc.vertices.astype(np.float64)
    ev, ef = _edges_and_faces(sc)
    tri = V[sc.faces]
    un = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    un /= np.linalg.norm(un, axis=1, keepdims=True)
    E = len(ev)
    G = max(4, -(-E // (1 << 14)))
    nleaf = -(-E // G)
    L = 0
    while (1 << L) < nleaf:
        L += 1
    nn = 2 << L
    lo = np.full((nn, 3), np.inf)
    hi = np.full((nn, 3), -np.inf)
    S = np.zeros(nn)
    ax = np.zeros((nn, 3))
    ct = np.full(nn, -2.0)
    for i in range(nleaf):
        k = (1 << L) + i
        es = range(i * G, min(E, (i + 1) * G))
        P = V[ev[list(es)].ravel()]
        lo[k], hi[k] = P.min(0), P.max(0)
        S[k] = sum(np.linalg.norm(V[ev[e, 1]] - V[ev[e, 0]]) for e in es)
        if any(len(ef[e]) != 2 for e in es):
            continue
        normals = np.array([un[f] for e in es for f in ef[e]])
        a = normals.sum(0)
        if np.linalg.norm(a) <= 1e-6:
            continue
        a /= np.linalg.norm(a)
        c = (normals @ a).min()
        ax[k], ct[k] = a, (c if c > 0 else -2.0)
    for k in range((1 << L) - 1, 0, -1):
        a, b = 2 * k, 2 * k + 1
        lo[k], hi[k], S[k] = np.minimum(lo[a], lo[b]), np.maximum(hi[a], hi[b]), S[a] + S[b]
        if not (S[a] > 0) or not (S[b] > 0):
            o = a if S[a] > 0 else b
            ax[k], ct[k] = ax[o], ct[o]
            continue
        if ct[a] < -1.5 or ct[b] < -1.5:
            continue
        s = ax[a] + ax[b]
        if np.linalg.norm(s) <= 1e-6:
            continue
        s /= np.linalg.norm(s)
        ang = lambda x: math.acos(max(-1.0, min(1.0, x)))
        th = max(ang(s @ ax[a]) + ang(ct[a]), ang(s @ ax[b]) + ang(ct[b]))
        ax[k], ct[k] = s, (math.cos(th) if th < math.pi / 2 else -2.0)
    return dict(G=G, L=L, nleaf=nleaf, E=E, lo=lo, hi=hi, S=S, ax=ax, ct=ct)


def _py_weight(t, k, p, n, bnd, sil):
    if not (t["S"][k] > 0):
        return 0.0
    lo, hi = t["lo"][k], t["hi"][k]
    top = np.where(n > 0, hi - p, lo - p) @ n
    if not (top > bnd):
        return 0.0
    if sil and t["ct"][k] > -1.5:
        v = p - 0.5 * (lo + hi)
        r, D = 0.5 * np.linalg.norm(hi - lo), np.linalg.norm(v)
        if D > r:
            cp = t["ax"][k] @ v / D
            sp = math.sqrt(max(0.0, 1 - cp * cp))
            cq = t["ct"][k]
            sq = math.sqrt(max(0.0, 1 - cq * cq))
            cmin = -1.0 if cp <= -cq else cp * cq - sp * sq
            cmax = 1.0 if cp >= cq else cp * cq + sp * sq
            if D * cmin - r > -bnd or D * cmax + r < bnd:
                return 0.0
    d = np.maximum(lo - p, np.maximum(0.0, p - hi))
    return t["S"][k] / max(max(d @ d, 0.25 * (hi - lo) @ (hi - lo)), 1e-30)


@pytest.mark.parametrize("name", ["occluder", "edges"])
def test_hierarchy_matches_a_restatement_of_its_definition(name):
    # probabilities and picks from an independent numpy statement of the tree,
    # its weights and its counters (Philox words of the vertex's draws)
    sc = _occluder_scene() if name == "occluder" else S.small_variant(S.make("edges"), 1, 8, 1)
    t = _py_tree(sc)
    osc = O.OracleScene(sc)
    key = np.array([11 & 0xffffffff, 0], np.uint32)
    for k_frame, (p, n) in enumerate(_tangent_frames(sc, 4, 12)):
        bnd = 1e-5 * (1 + np.abs(p).max())
        for mode in (0, 1):
            # probabilities: products of the branch ratios along each leaf's path
            pmf = np.zeros(t["E"])
            for leaf in range(t["nleaf"]):
                k, pr = (1 << t["L"]) + leaf, 1.0
                while k > 1:
                    par = k // 2
                    wa, wb = _py_weight(t, 2 * par, p, n, bnd, mode == 0), _py_weight(t, 2 * par + 1, p, n, bnd,
                                                                                      mode == 0)
                    pr *= (wa if k % 2 == 0 else wb) / (wa + wb) if wa + wb > 0 else 0.0
                    k = par
                first = leaf * t["G"]
                cnt = min(t["G"], t["E"] - first)
                pmf[first:first + cnt] = pr / cnt
            got = O.sec_edge_pmf(osc, p, n, bnd, mode)
            np.testing.assert_allclose(got, pmf, rtol=1e-9, atol=1e-15)
        # picks: the descent with one Philox word per level, then the leaf word
        N = 64
        uleaf = np.random.default_rng(k_frame).integers(0, 1 << 32, N)
        e_or, pr_or = O.sec_edge_picks(osc, 11, 3, 1, 0, p, n, bnd, uleaf)
        for i in range(N):
            k, pr, u = 1, 1.0, None
            for j in range(t["L"]):
                if j % 4 == 0:
                    u = O.philox([i, 3, (1 << 4) | (4 + j // 4), 0], key)
                wa, wb = _py_weight(t, 2 * k, p, n, bnd, True), _py_weight(t, 2 * k + 1, p, n, bnd, True)
                if not (wa + wb > 0):
                    k = -1
                    break
                if (int(u[j % 4]) >> 8) * 2.0 ** -24 < wa / (wa + wb):
                    k, pr = 2 * k, pr * wa / (wa + wb)
                else:
                    k, pr = 2 * k + 1, pr * wb / (wa + wb)
            if k < 0:
                assert e_or[i] == -1
                continue
            first = (k - (1 << t["L"])) * t["G"]
            cnt = min(t["G"], t["E"] - first)
            assert e_or[i] == first + ((int(uleaf[i]) >> 8) * cnt >> 24)
            assert abs(pr_or[i] - pr / cnt) <= 1e-9 * pr / cnt
