"""Adam over vertex positions and per-face parameters through the path tracer.

The paper refines a mesh and its per-facet material by stochastic gradient
descent on an image MSE (Sec. 3.2 "Vertex optimization" with the loss over
views c_i; Sec. 3.3 for the material loss), here with Adam over random
minibatches of views. Each iteration renders the minibatch with the current
vertices (the BVH is refit on the device first), takes the MSE against the
target images, runs the adjoint (path replay with the same seed, interior and
edge terms) and applies one Adam step. Parameters are clamped to their valid
range after each step. State (vertices, parameters, optimiser moments, RNG
position) checkpoints to a torch file and resumes bit for bit.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import torch

from . import st as _st


@dataclasses.dataclass
class AdamConfig:
    max_bounces: int = 3
    minibatch: int = 8
    lr_vertices: float = 1e-3
    lr_params: float = 2e-2
    edge_term: int = 1
    edge_mode: int = 0
    seed: int = 12345


def clamp_params_(P: torch.Tensor) -> torch.Tensor:
    """Clamp texel parameters in place to their valid range, by layout: 5 per texel (kd rgb, ks, roughness) or
    7 (kd rgb, ks rgb, roughness). Albedos and specular values to [0, 1], roughness (the last column) to
    [0.01, 1]."""
    if P.dim() != 2 or P.shape[1] not in (5, 7):
        raise ValueError("texel parameters must be [texels, 5] or [texels, 7]")
    r = P.shape[1] - 1
    P[:, :r].clamp_(0.0, 1.0)
    P[:, r].clamp_(0.01, 1.0)
    return P


class Reconstruction:
    """Holds the scene, the optimised tensors and the Adam state."""

    def __init__(self, scene: "_st.Scene", views, targets: torch.Tensor, vertices: torch.Tensor,
                 face_params: torch.Tensor, cfg: AdamConfig):
        self.scene, self.views, self.targets, self.cfg = scene, list(views), targets, cfg
        self.V = vertices.detach().clone().requires_grad_(True)
        self.P = face_params.detach().clone().requires_grad_(True)
        self.opt = torch.optim.Adam([{"params": [self.V], "lr": cfg.lr_vertices},
                                     {"params": [self.P], "lr": cfg.lr_params}])
        self.it = 0
        self.fopts = _st.make_opts()
        self.bopts = _st.make_opts(edge_term=cfg.edge_term, edge_mode=cfg.edge_mode)
        # per-view offsets in the full target image
        self.rows = [(v.pixel_offset, v.pixel_offset + v.width * v.height) for v in self.views]

    def _batch(self) -> List[int]:
        rng = np.random.default_rng(self.cfg.seed * 1000003 + self.it)
        return sorted(int(i) for i in rng.choice(len(self.views), size=min(self.cfg.minibatch, len(self.views)),
                                                 replace=False))

    def step(self) -> torch.Tensor:
        """One iteration; returns the minibatch loss as a 0-d device tensor (no host sync)."""
        idx = self._batch()
        # repack the minibatch's views contiguously for the render call
        vs, tg, off = [], [], 0
        for i in idx:
            v = dataclasses.replace(self.views[i], pixel_offset=off) if dataclasses.is_dataclass(self.views[i]) \
                else self.views[i]
            vs.append(v)
            a, b = self.rows[i]
            tg.append(self.targets[a:b])
            off += b - a
        target = torch.cat(tg)
        self.opt.zero_grad(set_to_none=True)
        img = _st.render(self.V, self.P, self.scene, vs, self.cfg.max_bounces,
                         self.cfg.seed + 7919 * self.it, self.fopts, self.bopts)
        loss = torch.mean((img - target) ** 2)
        loss.backward()
        self.opt.step()
        with torch.no_grad():
            clamp_params_(self.P)
        self.it += 1
        return loss.detach()

    def state_dict(self):
        return {"V": self.V.detach().clone(), "P": self.P.detach().clone(), "opt": self.opt.state_dict(),
                "it": self.it}

    def load_state_dict(self, sd):
        with torch.no_grad():
            self.V.copy_(sd["V"])
            self.P.copy_(sd["P"])
        self.opt.load_state_dict(sd["opt"])
        self.it = sd["it"]

    def save(self, path: str):
        torch.save(self.state_dict(), path)

    def load(self, path: str):
        self.load_state_dict(torch.load(path, map_location=self.V.device))


def render_targets(sc, vertices: Optional[np.ndarray] = None, max_bounces: int = 3, seed: int = 99) -> torch.Tensor:
    """Target images of every view of ``sc`` rendered from ``vertices`` (default: the scene's own)."""
    scene = _st.Scene.from_scene(sc, vertices=vertices)
    img = scene.render(sc.views, max_bounces, seed).clone()
    torch.cuda.synchronize()
    scene.close()
    return img
