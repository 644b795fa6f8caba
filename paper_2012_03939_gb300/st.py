"""Thin Python binding of libst (argument marshalling only).

Every step of the forward and adjoint path trace runs in the CUDA library
declared by ``include/st.h``; this module only converts torch tensors and
Python objects into the C structures and raw pointers that library takes. There
is no CPU fallback: if ``libst.so`` is missing or cannot be loaded the import of
the library fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libst.so")

ST_OK = 0
STATUS = {0: "ST_OK", 1: "ST_ERR_INVALID_ARG", 2: "ST_ERR_OOM", 3: "ST_ERR_CUDA", 4: "ST_ERR_TIMEOUT",
          5: "ST_ERR_STATE", 6: "ST_ERR_UNSUPPORTED", 7: "ST_ERR_DEVICE"}
MODE_BATCHED, MODE_PER_VIEW = 0, 1
EDGE_SILHOUETTE, EDGE_ALL = 0, 1
EDGE_TERM_PRIMARY, EDGE_TERM_SECONDARY, EDGE_TERM_SHADOW = 1, 2, 4
BVH_PLOC, BVH_LBVH = 0, 1
FRESNEL_HELD, FRESNEL_SCHLICK = 0, 1

EXPORTED = ["st_scene_create", "st_scene_destroy", "st_refit", "st_rebuild", "st_set_face_params", "st_render",
            "st_render_backward", "st_trace_closest", "st_get_stats", "st_debug_bvh", "st_build_bvh_noalloc",
            "st_measure_l2_read", "st_inject_fault", "st_last_error"]


class StError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class PointLight(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("intensity", C.c_float * 3)]


class EnvMap(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("rgb", C.c_void_p)]


MAX_VIEW_LIGHTS = 2
SEC_PICK_TREE, SEC_PICK_UNIFORM = 0, 1
MAX_VIEWS = 65535


class View(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3), ("fov_y_deg", C.c_float),
                ("width", C.c_int), ("height", C.c_int), ("spp", C.c_int), ("pixel_offset", C.c_longlong),
                ("n_lights", C.c_int), ("lights", PointLight * MAX_VIEW_LIGHTS)]


class SceneDesc(C.Structure):
    _fields_ = [("n_vertices", C.c_int), ("n_faces", C.c_int), ("vertices", C.c_void_p), ("faces", C.c_void_p),
                ("face_params", C.c_void_p), ("brdf", C.c_int), ("n_point_lights", C.c_int),
                ("point_lights", C.c_void_p), ("env", C.c_void_p), ("color_res", C.c_int), ("bvh_builder", C.c_int),
                ("rgb_specular", C.c_int), ("smooth_normals", C.c_int), ("fresnel", C.c_int)]


class RenderOpts(C.Structure):
    _fields_ = [("edge_term", C.c_int), ("edge_mode", C.c_int), ("edge_spp", C.c_int), ("mode", C.c_int),
                ("use_graph", C.c_int), ("chunk_paths", C.c_int), ("time_kernels", C.c_int),
                ("count_visits", C.c_int), ("persist_blocks", C.c_int), ("path_signatures", C.c_void_p),
                ("sec_pick", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("paths", C.c_longlong), ("extension_rays", C.c_longlong), ("shadow_rays", C.c_longlong),
                ("edge_samples", C.c_longlong), ("node_visits", C.c_longlong), ("tri_tests", C.c_longlong),
                ("extend_launches", C.c_int), ("extend_ms", C.c_double), ("device_error", C.c_int),
                ("bvh_nodes", C.c_int), ("scratch_bytes", C.c_longlong), ("kernel_launches", C.c_int),
                ("bvh4_nodes", C.c_int), ("secondary_samples", C.c_longlong),
                ("shadow_node_visits", C.c_longlong), ("shadow_tri_tests", C.c_longlong),
                ("shadow_launches", C.c_int), ("shadow_ms", C.c_double), ("busy_ms", C.c_double),
                ("host_syncs", C.c_int)]


_lib = None


def lib():
    """Load libst.so (built by ``paper_2012_03939_gb300.build``); raise if it is absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libst.so is not built (run paper_2012_03939_gb300.build.build()); "
                              "there is no fallback path")
        L = C.CDLL(LIB_PATH)
        P, I, U = C.c_void_p, C.c_int, C.c_ulonglong
        L.st_scene_create.argtypes = [P, P, P]
        L.st_scene_destroy.argtypes = [P]
        L.st_refit.argtypes = [P, P, P]
        L.st_rebuild.argtypes = [P, P, P]
        L.st_set_face_params.argtypes = [P, P, P]
        L.st_render.argtypes = [P, P, I, I, I, U, P, P, P]
        L.st_render_backward.argtypes = [P, P, I, I, I, U, P, P, P, P, P]
        L.st_trace_closest.argtypes = [P, P, I, I, P, P, P]
        L.st_get_stats.argtypes = [P, P]
        L.st_debug_bvh.argtypes = [P, P, P]
        L.st_build_bvh_noalloc.argtypes = [P, P, I, I, P, P, P, P]
        L.st_measure_l2_read.argtypes = [C.c_longlong, I, P, P]
        L.st_inject_fault.argtypes = [I, I]
        L.st_last_error.restype = C.c_char_p
        L.st_last_error.argtypes = []
        for name in EXPORTED[:-1]:
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(status):
    if status != ST_OK:
        raise StError(status, lib().st_last_error().decode())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def make_views(views, default_spp=0):
    """ctypes array of View from ``scenes.View`` objects (or View structures)."""
    arr = (View * len(views))()
    for i, v in enumerate(views):
        if isinstance(v, View):
            arr[i] = v
        else:
            lights = list(getattr(v, "lights", ()) or ())
            if len(lights) > MAX_VIEW_LIGHTS:
                raise ValueError("at most %d lights per view" % MAX_VIEW_LIGHTS)
            pl = (PointLight * MAX_VIEW_LIGHTS)(*[PointLight((C.c_float * 3)(*l[0]), (C.c_float * 3)(*l[1]))
                                                  for l in lights])
            arr[i] = View((C.c_float * 3)(*v.eye), (C.c_float * 3)(*v.target), (C.c_float * 3)(*v.up),
                          v.fov_y_deg, v.width, v.height, v.spp, v.pixel_offset, len(lights), pl)
    return arr


def n_pixels(views) -> int:
    return int(max(v.pixel_offset + v.width * v.height for v in views))


def make_opts(**kw) -> RenderOpts:
    """st_render_opts with the library's defaults, fields overridden by keyword. Names accepted for mode
    ("batched", "per_view"), edge_mode ("silhouette", "all") and sec_pick ("tree": the edge hierarchy, "uniform");
    edge_term is an OR of EDGE_TERM_PRIMARY, EDGE_TERM_SECONDARY and EDGE_TERM_SHADOW."""
    o = RenderOpts(0, EDGE_SILHOUETTE, 0, MODE_BATCHED, 1, 0, 0, 0, 0, None, SEC_PICK_TREE)
    for k, v in kw.items():
        if k == "mode" and isinstance(v, str):
            v = {"batched": MODE_BATCHED, "per_view": MODE_PER_VIEW}[v]
        if k == "sec_pick" and isinstance(v, str):
            v = {"tree": SEC_PICK_TREE, "uniform": SEC_PICK_UNIFORM}[v]
        if k == "edge_mode" and isinstance(v, str):
            v = {"silhouette": EDGE_SILHOUETTE, "all": EDGE_ALL}[v]
        setattr(o, k, int(v))
    return o


class Scene:
    """A mesh scene on the current CUDA device (owns a library scene handle). color_res: mesh-colors resolution
    (face_params then holds a row per texel); bvh_builder: "ploc" or "lbvh"; smooth_normals: shading normals
    interpolated from vertex normals (recomputed by refit and rebuild) instead of flat face normals; fresnel:
    "held" (0: the specular lobe scaled by ks at every angle) or "schlick" (1: Schlick's factor, F0 = ks)."""

    def __init__(self, vertices: torch.Tensor, faces: torch.Tensor, face_params: torch.Tensor, brdf: str = "ggx",
                 light_pos=None, light_intensity=None, env: Optional[np.ndarray] = None, stream=None,
                 color_res: int = 0, bvh_builder: str = "ploc", smooth_normals: bool = False, fresnel=0):
        dev = torch.device("cuda", torch.cuda.current_device())
        self.vertices = vertices.detach().to(dev, torch.float32).contiguous()
        self.faces = faces.detach().to(dev, torch.int32).contiguous()
        self.face_params = face_params.detach().to(dev, torch.float32).contiguous()
        if self.face_params.dim() != 2 or self.face_params.shape[1] not in (5, 7):
            raise ValueError("face_params must be [texels, 5] (scalar specular) or [texels, 7] (RGB specular)")
        self.nv, self.nf = self.vertices.shape[0], self.faces.shape[0]
        self.ntex = self.face_params.shape[0]      # texels: faces * (r+1)(r+2)/2
        lp = np.zeros((0, 3), np.float32) if light_pos is None else np.asarray(light_pos, np.float32).reshape(-1, 3)
        li = np.zeros((0, 3), np.float32) if light_intensity is None else np.asarray(light_intensity,
                                                                                    np.float32).reshape(-1, 3)
        self._lights = (PointLight * max(len(lp), 1))()
        for j in range(len(lp)):
            self._lights[j] = PointLight((C.c_float * 3)(*lp[j]), (C.c_float * 3)(*li[j]))
        # the environment may be a host array or a CUDA tensor [H, W, 3]; either is passed by pointer
        if env is None:
            self._env_arr = None
        elif isinstance(env, torch.Tensor) and env.is_cuda:
            self._env_arr = env.detach().to(dev, torch.float32).contiguous()
        else:
            self._env_arr = np.ascontiguousarray(env, np.float32)
        self._env = None
        if self._env_arr is not None:
            ptr = self._env_arr.data_ptr() if isinstance(self._env_arr, torch.Tensor) else self._env_arr.ctypes.data
            self._env = EnvMap(self._env_arr.shape[1], self._env_arr.shape[0], ptr)
        desc = SceneDesc(self.nv, self.nf, self.vertices.data_ptr(), self.faces.data_ptr(),
                         self.face_params.data_ptr(), {"ggx": 0, "beckmann": 1}[brdf], len(lp),
                         C.addressof(self._lights), None if self._env is None else C.addressof(self._env),
                         int(color_res), {"ploc": BVH_PLOC, "lbvh": BVH_LBVH}[bvh_builder],
                         1 if self.face_params.shape[1] == 7 else 0, int(bool(smooth_normals)),
                         {"held": FRESNEL_HELD, "schlick": FRESNEL_SCHLICK}.get(fresnel, fresnel))
        h = C.c_void_p()
        _check(lib().st_scene_create(C.byref(desc), _stream(stream), C.byref(h)))
        self.handle = h

    @classmethod
    def from_scene(cls, sc, vertices=None, device="cuda", **kw):
        V = torch.as_tensor(sc.vertices if vertices is None else vertices, dtype=torch.float32, device=device)
        return cls(V, torch.as_tensor(sc.faces, device=device), torch.as_tensor(sc.face_params, device=device),
                   sc.brdf, sc.light_pos, sc.light_intensity, sc.env, color_res=getattr(sc, "color_res", 0),
                   smooth_normals=bool(getattr(sc, "smooth_normals", False)), fresnel=int(getattr(sc, "fresnel", 0)),
                   **kw)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().st_scene_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def refit(self, vertices: torch.Tensor, stream=None):
        v = vertices.detach().to(torch.float32).contiguous()
        _check(lib().st_refit(self.handle, v.data_ptr(), _stream(stream)))
        self.vertices.copy_(v)

    def rebuild(self, vertices: torch.Tensor, stream=None):
        v = vertices.detach().to(torch.float32).contiguous()
        _check(lib().st_rebuild(self.handle, v.data_ptr(), _stream(stream)))
        self.vertices.copy_(v)

    def set_face_params(self, p: torch.Tensor, stream=None):
        p = p.detach().to(torch.float32).contiguous()
        _check(lib().st_set_face_params(self.handle, p.data_ptr(), _stream(stream)))
        self.face_params.copy_(p)

    def render(self, views, max_bounces: int, seed: int, opts: Optional[RenderOpts] = None, out=None,
               default_spp: int = 0, stream=None, signatures: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Forward render into ``out`` [N, 3]; with ``signatures`` (int64 [N] on the device), also each pixel's
        path-signature sum (the uint64 bit pattern)."""
        vs = make_views(views)
        if out is None:
            out = torch.zeros((n_pixels(views), 3), dtype=torch.float32, device=self.vertices.device)
        if signatures is not None:
            if signatures.dtype != torch.int64 or signatures.numel() < n_pixels(views) or not signatures.is_cuda:
                raise ValueError("signatures must be a CUDA int64 tensor with a row per pixel")
            o = make_opts() if opts is None else RenderOpts.from_buffer_copy(opts)
            o.path_signatures = signatures.data_ptr()
            opts = o
        _check(lib().st_render(self.handle, vs, len(vs), default_spp, max_bounces, seed,
                               None if opts is None else C.byref(opts), out.data_ptr(), _stream(stream)))
        return out

    def backward(self, views, max_bounces: int, seed: int, dLdI: torch.Tensor, opts: Optional[RenderOpts] = None,
                 d_vertices=None, d_face_params=None, want_vertices=True, want_params=True, default_spp: int = 0,
                 stream=None):
        vs = make_views(views)
        dLdI = dLdI.detach().to(torch.float32).contiguous()
        if want_vertices and d_vertices is None:
            d_vertices = torch.zeros((self.nv, 3), dtype=torch.float32, device=dLdI.device)
        if want_params and d_face_params is None:
            d_face_params = torch.zeros((self.ntex, self.face_params.shape[1]), dtype=torch.float32,
                                        device=dLdI.device)
        _check(lib().st_render_backward(self.handle, vs, len(vs), default_spp, max_bounces, seed,
                                        None if opts is None else C.byref(opts), dLdI.data_ptr(),
                                        None if d_vertices is None else d_vertices.data_ptr(),
                                        None if d_face_params is None else d_face_params.data_ptr(),
                                        _stream(stream)))
        return d_vertices, d_face_params

    def trace_closest(self, rays: torch.Tensor, exclude: int = -1, stream=None):
        rays = rays.detach().to(torch.float32).contiguous()
        n = rays.shape[0]
        tri = torch.empty(n, dtype=torch.int32, device=rays.device)
        t = torch.empty(n, dtype=torch.float32, device=rays.device)
        _check(lib().st_trace_closest(self.handle, rays.data_ptr(), n, exclude, tri.data_ptr(), t.data_ptr(),
                                      _stream(stream)))
        return tri, t

    def stats(self) -> dict:
        s = Stats()
        _check(lib().st_get_stats(self.handle, C.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def debug_bvh(self):
        nodes = np.zeros((max(self.nf - 1, 1), 16), np.float32)
        leaf = np.zeros(self.nf, np.int32)
        _check(lib().st_debug_bvh(self.handle, nodes.ctypes.data, leaf.ctypes.data))
        return nodes[: self.nf - 1], leaf


FAULT_ALLOC, FAULT_COPY = 1, 2


def inject_fault(site, nth: int = 0):
    """Arm the library's host-side fault injection: the nth next device allocation ("alloc") or host<->device
    copy ("copy") fails as the CUDA call would have; nth < 0 disarms the site."""
    site = {"alloc": FAULT_ALLOC, "copy": FAULT_COPY}.get(site, site)
    _check(lib().st_inject_fault(int(site), int(nth)))


def measure_l2_read(bytes_=32 << 20, passes=64, stream=None) -> float:
    """L2-resident read bandwidth in GB/s (library measurement utility)."""
    g = C.c_double()
    _check(lib().st_measure_l2_read(bytes_, passes, _stream(stream), C.byref(g)))
    return g.value


class STRender(torch.autograd.Function):
    """images = R(vertices, face_params; views). Backward replays the forward's seed (path replay)."""

    @staticmethod
    def forward(ctx, vertices, face_params, scene: Scene, views, max_bounces: int, seed: int,
                opts: Optional[RenderOpts] = None, bwd_opts: Optional[RenderOpts] = None):
        scene.refit(vertices)
        scene.set_face_params(face_params)
        img = scene.render(views, max_bounces, seed, opts)
        ctx.scene, ctx.views, ctx.B, ctx.seed, ctx.bwd_opts = scene, views, max_bounces, seed, bwd_opts
        ctx.needs = (ctx.needs_input_grad[0], ctx.needs_input_grad[1])
        return img

    @staticmethod
    def backward(ctx, gI):
        dV, dF = ctx.scene.backward(ctx.views, ctx.B, ctx.seed, gI, ctx.bwd_opts, want_vertices=ctx.needs[0],
                                    want_params=ctx.needs[1])
        return dV, dF, None, None, None, None, None, None


def render(vertices, face_params, scene: Scene, views, max_bounces: int, seed: int, opts=None, bwd_opts=None):
    return STRender.apply(vertices, face_params, scene, views, max_bounces, seed, opts, bwd_opts)
