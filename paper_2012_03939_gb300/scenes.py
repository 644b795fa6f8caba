"""Seeded synthetic scenes (inputs only).

This module produces plain scene data -- mesh vertices and faces, per-face
Torrance-Sparrow parameters, point lights, an equirectangular HDR environment
map and pinhole views -- for the five workloads the library is measured on.
It contains none of the rendering arithmetic (no camera model, no BRDF, no
sampling, no intersection): both the CUDA path and the FP64 CPU oracle read
the arrays it returns, and nothing else is shared between them.

The scenes stand in for the paper's simulated captures (textured meshes seen by
32 cameras on a Fibonacci sphere with two point lights per view, 128x128
targets; Sec. 4, "Simulated results"), which are not available here.

Every array is derived from ``numpy.random.default_rng(seed)`` so a scene is a
pure function of its name and seed.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

BASE_SEED = 2012_03939


@dataclasses.dataclass
class View:
    eye: tuple
    target: tuple
    up: tuple
    fov_y_deg: float
    width: int
    height: int
    spp: int
    pixel_offset: int = 0
    lights: tuple = ()              # the view's own point lights: ((x, y, z), (I_r, I_g, I_b)) pairs, at most 2


@dataclasses.dataclass
class Scene:
    name: str
    vertices: np.ndarray            # float32 [V,3]
    faces: np.ndarray               # int32 [F,3], counter-clockwise seen from outside
    face_params: np.ndarray         # float32 [F,5]: kd_r, kd_g, kd_b, ks, roughness
    brdf: str = "ggx"               # "ggx" | "beckmann"
    light_pos: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 3), np.float32))
    light_intensity: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 3), np.float32))
    env: Optional[np.ndarray] = None  # float32 [H,W,3] equirectangular radiance
    views: List[View] = dataclasses.field(default_factory=list)
    max_bounces: int = 2
    edge_term: bool = False
    seed: int = BASE_SEED
    target_vertices: Optional[np.ndarray] = None  # perturbed copy used to render a target
    color_res: int = 0              # mesh-colors resolution r: face_params has F*(r+1)(r+2)/2 texel rows
    smooth_normals: bool = False    # shading normals interpolated from vertex normals (flat face normals if False)
    fresnel: int = 0                # 0: Fresnel factor held at ks; 1: Schlick's approximation with F0 = ks

    @property
    def n_pixels(self) -> int:
        return int(sum(v.width * v.height for v in self.views))

    def subset_views(self, idx) -> "Scene":
        """Same scene restricted to the views ``idx`` (pixel offsets repacked)."""
        s = dataclasses.replace(self)
        vs = [dataclasses.replace(self.views[i]) for i in idx]
        _pack_offsets(vs)
        s.views = vs
        return s


def _pack_offsets(views: List[View]) -> None:
    off = 0
    for v in views:
        v.pixel_offset = off
        off += v.width * v.height


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------

def icosphere(subdiv: int):
    """Unit icosphere: 12 * 4^s ... V = 10*4^s + 2, F = 20*4^s."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(v, np.float64) / np.linalg.norm(v) for v in verts]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(verts, np.float64), np.array(faces, np.int32)


def uv_sphere(n_lon: int, n_bands: int):
    """Latitude/longitude sphere with pole fans: F = 2*n_lon*(n_bands-1)."""
    verts = [(0.0, 1.0, 0.0)]
    for i in range(1, n_bands):
        th = math.pi * i / n_bands
        for j in range(n_lon):
            ph = 2 * math.pi * j / n_lon
            verts.append((math.sin(th) * math.cos(ph), math.cos(th), -math.sin(th) * math.sin(ph)))
    verts.append((0.0, -1.0, 0.0))
    V = np.array(verts, np.float64)
    south = len(verts) - 1

    def ring(i, j):  # i in [1, n_bands-1]
        return 1 + (i - 1) * n_lon + (j % n_lon)

    F = []
    j = np.arange(n_lon)
    F.append(np.stack([np.zeros(n_lon, int), ring(1, j), ring(1, j + 1)], 1))
    for i in range(1, n_bands - 1):
        a, b, c, d = ring(i, j), ring(i + 1, j), ring(i + 1, j + 1), ring(i, j + 1)
        F.append(np.stack([a, b, c], 1))
        F.append(np.stack([a, c, d], 1))
    F.append(np.stack([np.full(n_lon, south), ring(n_bands - 1, j + 1), ring(n_bands - 1, j)], 1))
    return V, np.concatenate(F).astype(np.int32)


def torus_knot(p: int, q: int, n_seg: int, n_ring: int, tube: float = 0.42, scale: float = 1.0 / 3.2):
    """Tube of radius ``tube`` around the (p, q) torus knot, F = 2*n_seg*n_ring."""
    phi = 2 * math.pi * np.arange(n_seg) / n_seg

    def curve(ph):
        r = 2.0 + np.cos(q * ph)
        return np.stack([r * np.cos(p * ph), r * np.sin(p * ph), -np.sin(q * ph)], -1)

    c = curve(phi)
    tan = curve(phi + 1e-4) - curve(phi - 1e-4)
    tan /= np.linalg.norm(tan, axis=1, keepdims=True)
    ref = np.stack([np.cos(q * phi) * np.cos(p * phi), np.cos(q * phi) * np.sin(p * phi), -np.sin(q * phi)], -1)
    nrm = ref - (ref * tan).sum(1, keepdims=True) * tan
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    bin_ = np.cross(tan, nrm)
    a = 2 * math.pi * np.arange(n_ring) / n_ring
    V = (c[:, None, :] + tube * (np.cos(a)[None, :, None] * nrm[:, None, :]
                                  + np.sin(a)[None, :, None] * bin_[:, None, :]))
    V = V.reshape(-1, 3) * scale
    i = np.arange(n_seg)[:, None]
    j = np.arange(n_ring)[None, :]
    v00 = i * n_ring + j
    v10 = ((i + 1) % n_seg) * n_ring + j
    v11 = ((i + 1) % n_seg) * n_ring + (j + 1) % n_ring
    v01 = i * n_ring + (j + 1) % n_ring
    F = np.concatenate([np.stack([v00, v10, v11], -1).reshape(-1, 3),
                        np.stack([v00, v11, v01], -1).reshape(-1, 3)])
    return V.astype(np.float64), F.astype(np.int32)


def _orient_outward(V, F):
    """Flip faces whose normal points toward the centroid (star-shaped meshes)."""
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(b - a, c - a)
    cen = (a + b + c) / 3 - V.mean(0)
    flip = (n * cen).sum(1) < 0
    F = F.copy()
    F[flip] = F[flip][:, [0, 2, 1]]
    return F


def sinusoid_displace(V, rng, n_terms=8, amp=0.05):
    """Radial displacement r = 1 + (amp/n) * sum_k sin(w_k . p + phase_k)."""
    dirs = rng.normal(size=(n_terms, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    freq = rng.integers(1, 4, size=n_terms)
    phase = rng.uniform(0, 2 * math.pi, size=n_terms)
    p = V / np.linalg.norm(V, axis=1, keepdims=True)
    s = np.sin(p @ (dirs * freq[:, None]).T + phase).sum(1)
    return p * (1.0 + amp / n_terms * s)[:, None]


def _gradient_noise(P, rng, table=256):
    """3-D lattice gradient noise with quintic fade (after Perlin, SIGGRAPH 2002)."""
    g = rng.normal(size=(table, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    perm = rng.permutation(table)
    Pi = np.floor(P).astype(np.int64)
    f = P - Pi

    def h(ix, iy, iz):
        return perm[(perm[(perm[ix % table] + iy) % table] + iz) % table]

    def fade(t):
        return t * t * t * (t * (t * 6 - 15) + 10)

    out = 0.0
    u = fade(f)
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                gi = h(Pi[:, 0] + dx, Pi[:, 1] + dy, Pi[:, 2] + dz)
                d = f - np.array([dx, dy, dz])
                w = ((u[:, 0] if dx else 1 - u[:, 0]) * (u[:, 1] if dy else 1 - u[:, 1])
                     * (u[:, 2] if dz else 1 - u[:, 2]))
                out = out + w * (g[gi] * d).sum(1)
    return out


def fractal_displace(V, rng, octaves=6, amp=0.05, base_freq=2.0):
    p = V / np.linalg.norm(V, axis=1, keepdims=True)
    s = np.zeros(len(p))
    a, f, norm = 1.0, base_freq, 0.0
    for _ in range(octaves):
        s += a * _gradient_noise(p * f + 17.0, rng)
        norm += a
        a *= 0.5
        f *= 2.0
    s = s / norm
    s = s / max(np.abs(s).max(), 1e-12)
    return p * (1.0 + amp * s)[:, None]


# ----------------------------------------------------------------------------
# materials, lights, environment, cameras
# ----------------------------------------------------------------------------

def random_face_params(rng, n_faces):
    P = np.empty((n_faces, 5), np.float32)
    P[:, 0:3] = rng.uniform(0.1, 0.9, size=(n_faces, 3))
    P[:, 3] = 0.04
    P[:, 4] = rng.uniform(0.1, 0.6, size=n_faces)
    return P


def lognormal_env(rng, w, h, sigma=1.5):
    return np.exp(rng.normal(0.0, sigma, size=(h, w, 3))).astype(np.float32)


def ring_views(n, res, spp, radius=3.0, fov=45.0):
    vs = []
    for i in range(n):
        a = 2 * math.pi * i / n
        vs.append(View((radius * math.sin(a), 0.0, radius * math.cos(a)), (0.0, 0.0, 0.0),
                       (0.0, 1.0, 0.0), fov, res, res, spp))
    _pack_offsets(vs)
    return vs


def fibonacci_dirs(n):
    g = math.pi * (3.0 - math.sqrt(5.0))
    out = []
    for i in range(n):
        y = 1 - 2 * (i + 0.5) / n
        r = math.sqrt(max(0.0, 1 - y * y))
        out.append((r * math.cos(g * i), y, r * math.sin(g * i)))
    return out


def fibonacci_views(n, widths, heights, spps, radius=3.0, fov=45.0):
    vs = []
    for i, d in enumerate(fibonacci_dirs(n)):
        up = (0.0, 1.0, 0.0) if abs(d[1]) < 0.95 else (0.0, 0.0, 1.0)
        vs.append(View(tuple(radius * c for c in d), (0.0, 0.0, 0.0), up, fov,
                       int(widths[i]), int(heights[i]), int(spps[i])))
    _pack_offsets(vs)
    return vs


def with_view_lights(views, intensity=(4.0, 4.0, 4.0), offset=0.35):
    """Copies of ``views`` lit as the paper's captures (Sec. 4): one point light at the camera and one
    displaced from it along the camera's right (tangent) direction by ``offset``."""
    out = []
    for v in views:
        eye = np.asarray(v.eye, np.float64)
        fwd = np.asarray(v.target, np.float64) - eye
        right = np.cross(fwd, np.asarray(v.up, np.float64))
        right /= np.linalg.norm(right)
        I = tuple(float(x) for x in intensity)
        lights = ((tuple(float(x) for x in eye), I), (tuple(float(x) for x in eye + offset * right), I))
        out.append(dataclasses.replace(v, lights=lights))
    return out


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

def tiny(seed=BASE_SEED + 0, res=64, spp=4):
    """Icosphere subdivision 2 (320 faces), one light at distance 3, one 64x64 view, 4 spp, 2 bounces."""
    rng = np.random.default_rng(seed)
    V, F = icosphere(2)
    P = random_face_params(rng, len(F))
    noisy = V + rng.normal(0, 0.01, size=V.shape)
    s = 3.0 / math.sqrt(2.0)
    return Scene("tiny", _f32(V), F, P, "ggx",
                 light_pos=_f32([[0.0, s, s]]), light_intensity=_f32([[9.0, 9.0, 9.0]]),
                 views=ring_views(1, res, spp), max_bounces=2, edge_term=True, seed=seed,
                 target_vertices=_f32(noisy))


def edges(seed=BASE_SEED + 1, res=128, spp=16, n_views=16):
    """Displaced icosphere subdivision 4 (5120 faces), 3 lights, 16 ring views 128x128, 16 spp, 3 bounces."""
    rng = np.random.default_rng(seed)
    V, F = icosphere(4)
    V = sinusoid_displace(V, rng)
    P = random_face_params(rng, len(F))
    d = rng.normal(size=(3, 3))
    d[:, 1] = np.abs(d[:, 1])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return Scene("edges", _f32(V), F, P, "ggx", light_pos=_f32(3.0 * d),
                 light_intensity=_f32(np.full((3, 3), 6.0)),
                 views=ring_views(n_views, res, spp), max_bounces=3, edge_term=True, seed=seed)


def env(seed=BASE_SEED + 2, res=256, spp=4, n_views=32):
    """Torus knot (2,3) with 50,000 faces under a 256x128 lognormal environment, 32 views 256x256, 4 spp, 4 bounces."""
    rng = np.random.default_rng(seed)
    V, F = torus_knot(2, 3, 500, 50)
    P = random_face_params(rng, len(F))
    n = n_views
    return Scene("env", _f32(V), F, P, "ggx", env=lognormal_env(rng, 256, 128),
                 views=fibonacci_views(n, [res] * n, [res] * n, [spp] * n), max_bounces=4,
                 edge_term=False, seed=seed)


def batched(seed=BASE_SEED + 3, n_views=64, n_lon=500, n_bands=201):
    """Displaced UV sphere (200,000 faces), 512x256 environment, 64 views with width and height drawn from
    {64,128,256,512} and spp from {1,4,16}, 3 bounces."""
    rng = np.random.default_rng(seed)
    V, F = uv_sphere(n_lon, n_bands)
    V = sinusoid_displace(V, rng)
    P = random_face_params(rng, len(F))
    e = lognormal_env(rng, 512, 256)
    ws = rng.choice([64, 128, 256, 512], size=n_views)
    hs = rng.choice([64, 128, 256, 512], size=n_views)
    ss = rng.choice([1, 4, 16], size=n_views)
    return Scene("batched", _f32(V), F, P, "ggx", env=e, views=fibonacci_views(n_views, ws, hs, ss),
                 max_bounces=3, edge_term=True, seed=seed)


def scale(seed=BASE_SEED + 4, n_views=100, res=512, spp=16, n_lon=1000, n_bands=501):
    """Fractal-noise displaced UV sphere (1,000,000 faces), 1024x512 environment plus 2 point lights,
    100 views 512x512, 16 spp, 5 bounces."""
    rng = np.random.default_rng(seed)
    V, F = uv_sphere(n_lon, n_bands)
    V = fractal_displace(V, rng)
    P = random_face_params(rng, len(F))
    e = lognormal_env(rng, 1024, 512)
    d = rng.normal(size=(2, 3))
    d[:, 1] = np.abs(d[:, 1])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return Scene("scale", _f32(V), F, P, "ggx", env=e, light_pos=_f32(3.0 * d),
                 light_intensity=_f32(np.full((2, 3), 6.0)),
                 views=fibonacci_views(n_views, [res] * n_views, [res] * n_views, [spp] * n_views),
                 max_bounces=5, edge_term=True, seed=seed)


def _grid_quad(origin, u, v, n):
    """n x n quads spanning origin + [0,1] u + [0,1] v, two triangles each, normal along u x v."""
    origin, u, v = (np.asarray(a, np.float64) for a in (origin, u, v))
    g = np.arange(n + 1) / n
    P = origin + g[:, None, None] * u + g[None, :, None] * v
    idx = np.arange((n + 1) * (n + 1)).reshape(n + 1, n + 1)
    a, b, c, d = idx[:-1, :-1], idx[1:, :-1], idx[1:, 1:], idx[:-1, 1:]
    F = np.concatenate([np.stack([a, b, c], -1).reshape(-1, 3), np.stack([a, c, d], -1).reshape(-1, 3)])
    return P.reshape(-1, 3), F


def color_bleed(seed=BASE_SEED + 5, res=64, spp=16, n=8, plane_kd=((0.8, 0.1, 0.1), (0.1, 0.1, 0.8), (0.8, 0.8, 0.8))):
    """Three intersecting planes -- red wall, blue wall, white floor -- seen from the open side, as in the
    paper's study of global illumination on material estimation (Sec. 3.3, colour bleeding).
    face_plane gives each face's plane (0 red, 1 blue, 2 floor)."""
    walls = [((0, 0, 0), (0, 2, 0), (0, 0, 2)),     # x = 0, red, normal +x
             ((0, 0, 0), (2, 0, 0), (0, 2, 0)),     # z = 0, blue, normal +z
             ((0, 0, 0), (0, 0, 2), (2, 0, 0))]     # y = 0, white floor, normal +y
    Vs, Fs, plane = [], [], []
    off = 0
    for k, (o, u, v) in enumerate(walls):
        P, F = _grid_quad(o, u, v, n)
        Vs.append(P)
        Fs.append(F + off)
        plane.append(np.full(len(F), k))
        off += len(P)
    V = np.concatenate(Vs)
    F = np.concatenate(Fs).astype(np.int32)
    plane = np.concatenate(plane)
    P = np.zeros((len(F), 5), np.float32)
    P[:, :3] = np.asarray(plane_kd, np.float32)[plane]
    P[:, 3] = 0.0
    P[:, 4] = 0.5
    vs = []
    for i, (ex, ez) in enumerate([(3.6, 3.0), (3.0, 3.6), (3.4, 3.4), (4.0, 2.6)]):
        vs.append(View((ex, 2.2, ez), (0.6, 0.5, 0.6), (0.0, 1.0, 0.0), 45.0, res, res, spp))
    _pack_offsets(vs)
    sc = Scene("color_bleed", _f32(V), F, P, "ggx", light_pos=_f32([[1.3, 1.6, 1.3]]),
               light_intensity=_f32([[4.0, 4.0, 4.0]]), views=vs, max_bounces=3, seed=seed)
    sc.face_plane = plane
    return sc


WORKLOADS = {"tiny": tiny, "edges": edges, "env": env, "batched": batched, "scale": scale, "color_bleed": color_bleed}


def make(name: str, **kw) -> Scene:
    return WORKLOADS[name](**kw)


def single_triangle(width=16, height=16, light_dist=1000.0):
    """One Lambertian triangle facing a camera, lit by a distant point light along the view axis."""
    V = _f32([[-0.6, -0.5, 0.0], [0.7, -0.4, 0.0], [0.05, 0.65, 0.0]])
    F = np.array([[0, 1, 2]], np.int32)
    P = _f32([[0.8, 0.5, 0.3, 0.0, 0.5]])
    I = light_dist * light_dist
    vs = [View((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 30.0, width, height, 1)]
    _pack_offsets(vs)
    return Scene("triangle", V, F, P, "ggx", light_pos=_f32([[0.0, 0.0, light_dist]]),
                 light_intensity=_f32([[I, I, I]]), views=vs, max_bounces=1)


def small_variant(sc: Scene, n_views: int = 2, max_res: int = 48, spp: Optional[int] = None) -> Scene:
    """A few views of ``sc`` at reduced (ragged) resolution, for oracle-sized parity runs."""
    s = dataclasses.replace(sc)
    vs = []
    for i, v in enumerate(sc.views[:n_views]):
        w = min(v.width, max_res - 3 * i)
        h = min(v.height, max_res - 5 * i - 1)
        vs.append(dataclasses.replace(v, width=w, height=h, spp=spp or v.spp))
    _pack_offsets(vs)
    s.views = vs
    return s
