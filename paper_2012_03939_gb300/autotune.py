"""Autotuner for the wavefront launch parameters (host policy over the C ABI).

Two knobs decide how the batched path trace maps onto the GPU: the number of
paths in flight per wavefront chunk (queue capacity; larger chunks fill the
152 SMs with fewer launches but hold more scratch) and the resident blocks per
SM of the persistent stage kernels. ``tune`` times one forward + backward call
of the caller's workload for each candidate with CUDA events and keeps the
fastest; results are cached in a JSON file keyed by the workload signature
(face count, view sizes and spp, bounces, edge options) and the device name,
so a later call with the same workload costs nothing. The candidates change
only scheduling: every candidate yields the bitwise identical image.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Dict, Optional, Sequence

import torch

from . import st as _st

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "st_autotune.json")
CHUNKS = (1 << 20, 1 << 21, 1 << 22, 1 << 23, 1 << 24, 1 << 25)
PERSIST = (0, 2)


def signature(scene: "_st.Scene", views, max_bounces: int, edge_term: int, edge_mode: int) -> str:
    h = hashlib.sha256()
    h.update(("%d|%d|%d|%d|%s|" % (scene.nf, max_bounces, edge_term, edge_mode,
                                    torch.cuda.get_device_name())).encode())
    for v in views:
        h.update(("%d,%d,%d;" % (v.width, v.height, v.spp)).encode())
    return h.hexdigest()[:24]


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(scene: "_st.Scene", views, max_bounces: int, seed: int = 1, edge_term: int = 1, edge_mode: int = 0,
         cache_path: Optional[str] = DEFAULT_CACHE, chunks: Sequence[int] = CHUNKS,
         persist: Sequence[int] = PERSIST, repeats: int = 2) -> Dict[str, int]:
    """Return {"chunk_paths": ..., "persist_blocks": ..., "ms": ...} for this workload (cached)."""
    key = signature(scene, views, max_bounces, edge_term, edge_mode)
    cache = _load(cache_path) if cache_path else {}
    if key in cache:
        return dict(cache[key], cached=True)
    n = _st.n_pixels(views)
    dev = scene.vertices.device
    img = torch.zeros((n, 3), dtype=torch.float32, device=dev)
    g = torch.full((n, 3), 1e-3, dtype=torch.float32, device=dev)
    dV = torch.zeros((scene.nv, 3), dtype=torch.float32, device=dev)
    dF = torch.zeros(tuple(scene.face_params.shape), dtype=torch.float32, device=dev)
    best = None
    results = []
    for ch in chunks:
        for pb in persist:
            fo = _st.make_opts(chunk_paths=ch, persist_blocks=pb)
            bo = _st.make_opts(chunk_paths=ch, persist_blocks=pb, edge_term=edge_term, edge_mode=edge_mode)
            scene.render(views, max_bounces, seed, fo, out=img)        # capture + warm
            scene.backward(views, max_bounces, seed, g, bo, d_vertices=dV, d_face_params=dF)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(repeats):
                scene.render(views, max_bounces, seed, fo, out=img)
                scene.backward(views, max_bounces, seed, g, bo, d_vertices=dV, d_face_params=dF)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / repeats
            results.append((ms, ch, pb))
            if best is None or ms < best[0]:
                best = (ms, ch, pb)
    out = {"chunk_paths": best[1], "persist_blocks": best[2], "ms": round(best[0], 3),
           "tried": [[round(m, 3), c, p] for m, c, p in results]}
    if cache_path:
        cache = _load(cache_path)
        cache[key] = out
        os.makedirs(os.path.dirname(cache_path) or ".", exist_ok=True)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return dict(out, cached=False)
