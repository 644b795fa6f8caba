"""ctypes binding of the FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg import this package. The CUDA library never does, and this package never
imports the CUDA library. See ``oracle.cpp`` for the estimator it computes and
the paper sections it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with g++ (plain C++17, no vendor code)."""
    src = os.path.join(HERE, "oracle.cpp")
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(HERE, "oracle.h"))):
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                               src, "-o", LIB_PATH + ".tmp"])
        os.replace(LIB_PATH + ".tmp", LIB_PATH)
    return LIB_PATH


class _Scene(C.Structure):
    _fields_ = [("n_vertices", C.c_int), ("n_faces", C.c_int), ("vertices", C.c_void_p),
                ("faces", C.c_void_p), ("face_params", C.c_void_p), ("brdf", C.c_int),
                ("n_lights", C.c_int), ("light_pos", C.c_void_p), ("light_intensity", C.c_void_p),
                ("env_width", C.c_int), ("env_height", C.c_int), ("env_rgb", C.c_void_p),
                ("color_res", C.c_int), ("param_width", C.c_int), ("smooth_normals", C.c_int),
                ("fresnel", C.c_int)]


class _View(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3),
                ("fov_y_deg", C.c_float), ("width", C.c_int), ("height", C.c_int), ("spp", C.c_int),
                ("pixel_offset", C.c_longlong), ("n_lights", C.c_int), ("light_pos", (C.c_float * 3) * 2),
                ("light_intensity", (C.c_float * 3) * 2)]


class _Params(C.Structure):
    _fields_ = [("max_bounces", C.c_int), ("seed", C.c_ulonglong), ("edge_mode", C.c_int),
                ("edge_spp", C.c_int), ("n_threads", C.c_int), ("secondary", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.orc_render_pixels.restype = C.c_longlong
        L.orc_render_pixels.argtypes = [P, P, C.c_int, P, P, C.c_int, P]
        L.orc_render_signatures.restype = C.c_longlong
        L.orc_render_signatures.argtypes = [P, P, C.c_int, P, P, C.c_int, P]
        L.orc_grad_pixels.restype = C.c_longlong
        L.orc_grad_pixels.argtypes = [P, P, C.c_int, P, P, C.c_int, P, P, P]
        L.orc_edge_grad.restype = C.c_longlong
        L.orc_edge_grad.argtypes = [P, P, C.c_int, P, P, P]
        L.orc_shadow_edge_grad.restype = C.c_longlong
        L.orc_shadow_edge_grad.argtypes = [P, P, C.c_int, P, P, P]
        L.orc_edge_candidates.restype = C.c_int
        L.orc_edge_candidates.argtypes = [P, P, P, P]
        L.orc_trace_screen.restype = C.c_longlong
        L.orc_trace_screen.argtypes = [P, P, P, C.c_double, C.c_double, C.c_uint32, C.c_uint32,
                                       C.c_uint32, P, P, P, P]
        L.orc_trace_screen_taped.restype = C.c_longlong
        L.orc_trace_screen_taped.argtypes = [P, P, P, C.c_double, C.c_double, C.c_uint32, C.c_uint32,
                                             C.c_uint32, C.c_int, P, P, P]
        L.orc_microfacet.restype = None
        L.orc_microfacet.argtypes = [C.c_int, C.c_double, C.c_double, P, P]
        L.orc_closest_hit.restype = None
        L.orc_closest_hit.argtypes = [P, P, C.c_int, C.c_int, P, P]
        L.orc_brdf_eval.restype = None
        L.orc_brdf_eval.argtypes = [C.c_int, C.c_int, P, P, P, P, P]
        L.orc_brdf_pdf.restype = C.c_double
        L.orc_brdf_pdf.argtypes = [C.c_int, P, P, P, P]
        L.orc_brdf_sample.restype = C.c_double
        L.orc_brdf_sample.argtypes = [C.c_int, P, P, P, C.c_double, C.c_double, C.c_double, P]
        L.orc_philox.restype = None
        L.orc_philox.argtypes = [P, P, P]
        L.orc_env_alias.restype = C.c_int
        L.orc_env_alias.argtypes = [P, C.c_int, C.c_int, P, P, P]
        L.orc_alias_pick.restype = C.c_int
        L.orc_alias_pick.argtypes = [P, P, C.c_int, C.c_uint32, C.c_uint32]
        L.orc_mesh_color_index.restype = C.c_longlong
        L.orc_mesh_color_index.argtypes = [C.c_int, C.c_longlong, C.c_double, C.c_double]
        L.orc_sec_edge_pmf.restype = C.c_int
        L.orc_sec_edge_pmf.argtypes = [P, P, P, C.c_double, C.c_int, P]
        L.orc_sec_edge_picks.restype = C.c_int
        L.orc_sec_edge_picks.argtypes = [P, C.c_ulonglong, C.c_uint32, C.c_int, C.c_uint32, P, P, C.c_double,
                                         C.c_int, P, C.c_int, P, P]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class OracleScene:
    """Holds ctypes views of a ``scenes.Scene`` (arrays kept alive here)."""

    def __init__(self, sc, vertices=None, face_params=None):
        # float32 scene data converts exactly; callers may pass float64 (finite differences)
        self.V = np.ascontiguousarray(sc.vertices if vertices is None else vertices, np.float64)
        self.F = np.ascontiguousarray(sc.faces, np.int32)
        self.P = np.ascontiguousarray(sc.face_params if face_params is None else face_params, np.float64)
        self.LP = np.ascontiguousarray(sc.light_pos, np.float64).reshape(-1, 3)
        self.LI = np.ascontiguousarray(sc.light_intensity, np.float64).reshape(-1, 3)
        self.E = None if sc.env is None else np.ascontiguousarray(sc.env, np.float32)
        self.s = _Scene(len(self.V), len(self.F), _ptr(self.V).value, _ptr(self.F).value, _ptr(self.P).value,
                        0 if sc.brdf == "ggx" else 1, len(self.LP), _ptr(self.LP).value, _ptr(self.LI).value,
                        0 if self.E is None else self.E.shape[1], 0 if self.E is None else self.E.shape[0],
                        None if self.E is None else _ptr(self.E).value, int(getattr(sc, "color_res", 0)),
                        self.P.shape[1], int(bool(getattr(sc, "smooth_normals", False))),
                        int(getattr(sc, "fresnel", 0)))
        self.views = (_View * len(sc.views))()
        for i, v in enumerate(sc.views):
            lights = list(getattr(v, "lights", ()) or ())
            lp = ((C.c_float * 3) * 2)(*[(C.c_float * 3)(*l[0]) for l in lights])
            li = ((C.c_float * 3) * 2)(*[(C.c_float * 3)(*l[1]) for l in lights])
            self.views[i] = _View((C.c_float * 3)(*v.eye), (C.c_float * 3)(*v.target), (C.c_float * 3)(*v.up),
                                  v.fov_y_deg, v.width, v.height, v.spp, v.pixel_offset, len(lights), lp, li)
        self.n_views = len(sc.views)
        self.nv, self.nf = len(self.V), len(self.F)
        self.ntex = len(self.P)          # texels (= faces at mesh-colors resolution 0)
        self.np = self.P.shape[1]        # parameters per texel: 5 (scalar specular) or 7 (RGB specular)


def params(max_bounces, seed, edge_mode=0, edge_spp=0, n_threads=0, secondary=0):
    """secondary: 0 off, 1 secondary edge picked uniformly, 2 picked through the edge hierarchy."""
    return _Params(max_bounces, seed, edge_mode, edge_spp, n_threads, secondary)


def sec_edge_pmf(osc: OracleScene, p, n, bnd, edge_mode=0):
    """Pick probability of every edge (edge order) at vertex p, tangent-plane normal n, band bnd."""
    p = np.ascontiguousarray(p, np.float64)
    n = np.ascontiguousarray(n, np.float64)
    out = np.zeros(3 * osc.nf, np.float64)
    ne = lib().orc_sec_edge_pmf(C.byref(osc.s), _ptr(p), _ptr(n), bnd, edge_mode, _ptr(out))
    if ne < 0:
        raise ValueError("oracle rejected the input")
    return out[:ne]


def sec_edge_picks(osc: OracleScene, seed, c1, b, stream, p, n, bnd, uleaf, edge_mode=0):
    """Hierarchy picks at one vertex, pick i with counters (i, c1): (edge or -1, probability) arrays."""
    p = np.ascontiguousarray(p, np.float64)
    n = np.ascontiguousarray(n, np.float64)
    u = np.ascontiguousarray(uleaf, np.uint32)
    e = np.zeros(len(u), np.int32)
    pr = np.zeros(len(u), np.float64)
    if lib().orc_sec_edge_picks(C.byref(osc.s), seed, c1, b, stream, _ptr(p), _ptr(n), bnd, edge_mode, _ptr(u),
                                len(u), _ptr(e), _ptr(pr)) < 0:
        raise ValueError("oracle rejected the input")
    return e, pr


def render_pixels(osc: OracleScene, prm, pix):
    pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 3)
    out = np.zeros((len(pix), 3), np.float64)
    seg = lib().orc_render_pixels(C.byref(osc.s), osc.views, osc.n_views, C.byref(prm), _ptr(pix), len(pix),
                                  _ptr(out))
    if seg < 0:
        raise ValueError("oracle rejected the input")
    return out, seg


def render_signatures(osc: OracleScene, prm, pix):
    """Per listed pixel: the sum (mod 2^64) of its samples' path-decision hashes."""
    pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 3)
    out = np.zeros(len(pix), np.uint64)
    seg = lib().orc_render_signatures(C.byref(osc.s), osc.views, osc.n_views, C.byref(prm), _ptr(pix), len(pix),
                                      _ptr(out))
    if seg < 0:
        raise ValueError("oracle rejected the input")
    return out


def all_pixels(sc):
    out = []
    for vi, v in enumerate(sc.views):
        yy, xx = np.mgrid[0:v.height, 0:v.width]
        out.append(np.stack([np.full(xx.size, vi), xx.ravel(), yy.ravel()], 1))
    return np.concatenate(out).astype(np.int32)


def pixel_index(sc, pix):
    """Packed image row of each (view, x, y)."""
    offs = np.array([v.pixel_offset for v in sc.views])
    ws = np.array([v.width for v in sc.views])
    return offs[pix[:, 0]] + pix[:, 2] * ws[pix[:, 0]] + pix[:, 1]


def grad_pixels(osc: OracleScene, prm, pix, dLdI):
    pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 3)
    w = np.ascontiguousarray(dLdI, np.float64).reshape(-1, 3)
    dv = np.zeros((osc.nv, 3), np.float64)
    df = np.zeros((osc.ntex, osc.np), np.float64)
    seg = lib().orc_grad_pixels(C.byref(osc.s), osc.views, osc.n_views, C.byref(prm), _ptr(pix), len(pix),
                                _ptr(w), _ptr(dv), _ptr(df))
    if seg < 0:
        raise ValueError("oracle rejected the input")
    return dv, df, seg


def edge_grad(osc: OracleScene, prm, dLdI_full):
    w = np.ascontiguousarray(dLdI_full, np.float64).reshape(-1, 3)
    dv = np.zeros((osc.nv, 3), np.float64)
    seg = lib().orc_edge_grad(C.byref(osc.s), osc.views, osc.n_views, C.byref(prm), _ptr(w), _ptr(dv))
    if seg < 0:
        raise ValueError("oracle rejected the input")
    return dv, seg


def shadow_edge_grad(osc: OracleScene, prm, dLdI_full):
    w = np.ascontiguousarray(dLdI_full, np.float64).reshape(-1, 3)
    dv = np.zeros((osc.nv, 3), np.float64)
    seg = lib().orc_shadow_edge_grad(C.byref(osc.s), osc.views, osc.n_views, C.byref(prm), _ptr(w), _ptr(dv))
    if seg < 0:
        raise ValueError("oracle rejected the input")
    return dv, seg


def edge_candidates(osc: OracleScene, prm, view_index=0):
    v = C.byref(osc.views[view_index])
    n = lib().orc_edge_candidates(C.byref(osc.s), v, C.byref(prm), None)
    out = np.zeros((max(n, 0), 2), np.int32)
    lib().orc_edge_candidates(C.byref(osc.s), v, C.byref(prm), _ptr(out))
    return out


def trace_screen(osc: OracleScene, prm, view_index, px, py, c0=0, c1=0, stream=0, grad_w=None):
    rgb = np.zeros(3, np.float64)
    dv = df = gw = None
    if grad_w is not None:
        gw = np.ascontiguousarray(grad_w, np.float64)
        dv = np.zeros((osc.nv, 3), np.float64)
        df = np.zeros((osc.ntex, osc.np), np.float64)
    seg = lib().orc_trace_screen(C.byref(osc.s), C.byref(osc.views[view_index]), C.byref(prm), px, py, c0, c1,
                                 stream, _ptr(rgb), _ptr(gw), _ptr(dv), _ptr(df))
    if seg < 0:
        raise ValueError("oracle rejected the input")
    return (rgb, dv, df) if grad_w is not None else rgb


def trace_screen_taped(osc: OracleScene, prm, view_index, px, py, c0=0, c1=0, stream=0, tape=None):
    """Without ``tape``: record and return (rgb, tape). With ``tape``: replay it and return rgb."""
    rgb = np.zeros(3, np.float64)
    if tape is None:
        buf = np.zeros(4096, np.float64)
        n = C.c_int(len(buf))
        seg = lib().orc_trace_screen_taped(C.byref(osc.s), C.byref(osc.views[view_index]), C.byref(prm), px, py,
                                           c0, c1, stream, 1, _ptr(buf), C.byref(n), _ptr(rgb))
        if seg < 0:
            raise ValueError("oracle tape record failed (%d)" % seg)
        return rgb, buf[:n.value].copy()
    buf = np.ascontiguousarray(tape, np.float64)
    n = C.c_int(len(buf))
    seg = lib().orc_trace_screen_taped(C.byref(osc.s), C.byref(osc.views[view_index]), C.byref(prm), px, py,
                                       c0, c1, stream, 2, _ptr(buf), C.byref(n), _ptr(rgb))
    if seg < 0:
        raise ValueError("oracle tape replay out of step (%d)" % seg)
    return rgb


def microfacet(brdf, alpha, c):
    D = C.c_double()
    G = C.c_double()
    lib().orc_microfacet(brdf, alpha, c, C.byref(D), C.byref(G))
    return D.value, G.value


def closest_hit(osc: OracleScene, rays, exclude=-1):
    rays = np.ascontiguousarray(rays, np.float64).reshape(-1, 7)
    tri = np.zeros(len(rays), np.int32)
    t = np.zeros(len(rays), np.float64)
    lib().orc_closest_hit(C.byref(osc.s), _ptr(rays), len(rays), exclude, _ptr(tri), _ptr(t))
    return tri, t


def brdf_eval(brdf, p5, n, wi, wo, fresnel=0):
    """f(wi, wo) (RGB); fresnel: 0 = Fresnel factor held at ks, 1 = Schlick with F0 = ks."""
    out = np.zeros(3)
    a = [np.ascontiguousarray(x, np.float64) for x in (p5, n, wi, wo)]
    lib().orc_brdf_eval(brdf, int(fresnel), *[_ptr(x) for x in a], _ptr(out))
    return out


def brdf_pdf(brdf, p5, n, wi, wo):
    a = [np.ascontiguousarray(x, np.float64) for x in (p5, n, wi, wo)]
    return lib().orc_brdf_pdf(brdf, *[_ptr(x) for x in a])


def brdf_sample(brdf, p5, n, wo, ul, u1, u2):
    wi = np.zeros(3)
    a = [np.ascontiguousarray(x, np.float64) for x in (p5, n, wo)]
    pdf = lib().orc_brdf_sample(brdf, *[_ptr(x) for x in a], ul, u1, u2, _ptr(wi))
    return wi, pdf


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def env_alias(rgb):
    rgb = np.ascontiguousarray(rgb, np.float32)
    h, w = rgb.shape[:2]
    prob = np.zeros(w * h)
    alias = np.zeros(w * h, np.int32)
    pmf = np.zeros(w * h)
    if lib().orc_env_alias(_ptr(rgb), w, h, _ptr(prob), _ptr(alias), _ptr(pmf)):
        raise ValueError("environment has no positive weight")
    return prob, alias, pmf


def alias_pick(prob, alias, u0, u1):
    return lib().orc_alias_pick(_ptr(prob), _ptr(alias), len(prob), int(u0), int(u1))


def mesh_color_index(r, t, alpha, beta):
    return lib().orc_mesh_color_index(r, t, alpha, beta)
