"""The reconstruction loop of Sec. 4 (Algorithm 1) on the device.

Each iteration renders the chosen views, computes Eq. 17's loss and backpropagates it (rasterizer.py), records the
densification statistics from dL/ds, densifies / prunes and resets opacities on their schedules, and advances Adam
one step. Every step runs in the CUDA library; this module owns the buffers and the schedule.

The optimiser state is one row of P = 11 + 3K raw floats per Gaussian (mean, log-scale, quaternion, logit-opacity,
SH), with Adam moments of the same layout; the renderer reads the activated arrays the Adam step publishes. As in the
3DGS loop the paper follows, an iteration that densifies does not also take an optimiser step (the rows it would
update have just been rebuilt), and the prune by screen-space size only starts after the first opacity reset.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import _cabi as C
from .rasterizer import Rasterizer, Settings


@dataclasses.dataclass
class TrainConfig:
    lr_means: float = 1.6e-4      # times the scene extent (3DGS convention)
    lr_scales: float = 5e-3
    lr_quats: float = 1e-3
    lr_opacity: float = 5e-2
    lr_sh_dc: float = 2.5e-3
    lr_sh_rest: float = 2.5e-3 / 20
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15
    densify_from: int = 500
    densify_until: int = 15000
    densify_interval: int = 100
    opacity_reset_interval: int = 3000
    grad_threshold: float = 2e-4
    percent_dense: float = 0.01
    min_opacity: float = 0.005
    max_scale_frac: float = 0.1
    max_screen_radius: float = 20.0
    loss: str = "dssim"          # "dssim" (Eq. 17, lambda below) or "l1"
    ssim_lambda: float = 0.2

    def adam(self, extent: float) -> C.omnigs_adam_config:
        a = C.omnigs_adam_config()
        a.lr_means, a.lr_scales, a.lr_quats = self.lr_means * extent, self.lr_scales, self.lr_quats
        a.lr_opacity, a.lr_sh_dc, a.lr_sh_rest = self.lr_opacity, self.lr_sh_dc, self.lr_sh_rest
        a.beta1, a.beta2, a.eps = self.beta1, self.beta2, self.eps
        return a

    def densify(self, extent: float, screen_limit: bool = True) -> C.omnigs_densify_config:
        d = C.omnigs_densify_config()
        d.grad_threshold, d.percent_dense, d.extent = self.grad_threshold, self.percent_dense, extent
        d.min_opacity, d.max_scale_frac = self.min_opacity, self.max_scale_frac
        d.max_screen_radius = self.max_screen_radius if screen_limit else float("inf")
        return d


def raw_rows(means, scales, quats, opacity, sh) -> np.ndarray:
    """[n, 11 + 3K] raw rows from activated parameters (host arrays)."""
    n = means.shape[0]
    o = np.clip(np.asarray(opacity, np.float64), 1e-6, 1 - 1e-6)
    return np.concatenate([means, np.log(scales), quats, np.log(o / (1 - o))[:, None], sh.reshape(n, -1)],
                          axis=1).astype(np.float32)


class GaussianModel:
    """Raw rows, Adam moments, activated arrays and densification statistics of n Gaussians on the device."""

    def __init__(self, rows: torch.Tensor, K: int):
        self.K = K
        self.P = 11 + 3 * K
        self._set_rows(rows.contiguous(), torch.zeros_like(rows), torch.zeros_like(rows))

    @classmethod
    def from_scene(cls, scene, device="cuda"):
        rows = raw_rows(*scene.arrays())
        return cls(torch.from_numpy(rows).to(device), scene.sh.shape[1])

    @property
    def n(self) -> int:
        return int(self.params.shape[0])

    def _set_rows(self, params, m, v):
        self.params, self.m, self.v = params, m, v
        n, dev = params.shape[0], params.device
        self.means = torch.empty((n, 3), device=dev)
        self.scales = torch.empty((n, 3), device=dev)
        self.quats = torch.empty((n, 4), device=dev)
        self.opacity = torch.empty((n,), device=dev)
        self.sh = torch.empty((n, self.K, 3), device=dev)
        self.accum = torch.zeros((n,), device=dev)
        self.count = torch.zeros((n,), dtype=torch.int32, device=dev)
        self.max_radius = torch.zeros((n,), device=dev)
        C.omnigs_publish_params(n, self.K, self.params, self.means, self.scales, self.quats, self.opacity, self.sh)

    def activated(self):
        return self.means, self.scales, self.quats, self.opacity, self.sh


class Trainer:
    def __init__(self, model: GaussianModel, settings: Settings, cfg: TrainConfig | None = None,
                 extent: float = 5.0, seed: int = 0):
        self.model = model
        self.s = settings
        self.cfg = cfg or TrainConfig()
        self.extent = extent
        self.iteration = 0
        self.adam_steps = 0
        self.r = Rasterizer(settings, device=model.params.device)
        self.gen = torch.Generator(device=model.params.device)
        self.gen.manual_seed(seed)
        self._dssim_scratch = None
        self.history = []

    def _loss(self, target):
        if self.cfg.loss == "dssim":
            if self._dssim_scratch is None:
                self._dssim_scratch = torch.empty(C.omnigs_dssim_scratch_size(self.r.cfg), dtype=torch.uint8,
                                                  device=target.device)
            C.omnigs_dssim_loss(self.r.cfg, self.cfg.ssim_lambda, self.r.rgb, target, self.r.dL_drgb, self.r.loss,
                                self._dssim_scratch)
        else:
            self.r.l1_loss(target)
        return self.r.loss

    def densify_and_prune(self):
        mdl = self.model
        n = mdl.n
        normals = torch.randn((n, 2, 3), device=mdl.params.device, generator=self.gen)
        cap = max(2 * n, 1)
        P = mdl.P
        po = torch.empty((cap, P), device=mdl.params.device)
        mo, vo = torch.empty_like(po), torch.empty_like(po)
        n_out = torch.zeros(1, dtype=torch.int64, device=mdl.params.device)
        ws = torch.empty(max(C.omnigs_densify_workspace_size(n), 256), dtype=torch.uint8, device=mdl.params.device)
        # as in the 3DGS loop, the screen-size prune starts after the first opacity reset
        screen_limit = self.iteration > self.cfg.opacity_reset_interval
        C.omnigs_densify(n, mdl.K, self.cfg.densify(self.extent, screen_limit), mdl.params, mdl.m, mdl.v, mdl.accum,
                         mdl.count, mdl.max_radius, normals, po, mo, vo, n_out, ws)
        k = int(n_out.item())
        mdl._set_rows(po[:k].clone(), mo[:k].clone(), vo[:k].clone())
        return k

    def step(self, viewmats, target):
        """One iteration of Algorithm 1 on the views `viewmats` [V, 4, 4] against `target` [V, 3, H, W]."""
        self.iteration += 1
        it, cfg, mdl = self.iteration, self.cfg, self.model
        self.r.forward(*mdl.activated(), viewmats)
        loss = self._loss(target)
        grads = self.r.backward()
        C.omnigs_densify_stats(self.r.cfg, mdl.n, self.r.splats, self.r.grads2d, mdl.accum, mdl.count,
                               mdl.max_radius)
        densified = False
        if it <= cfg.densify_until:
            if it >= cfg.densify_from and it % cfg.densify_interval == 0:
                self.densify_and_prune()
                densified = True
            if it % cfg.opacity_reset_interval == 0:
                C.omnigs_reset_opacity(mdl.n, mdl.K, 0.01, mdl.params, mdl.m, mdl.v, mdl.opacity)
        if not densified:
            self.adam_steps += 1
            C.omnigs_adam_step(mdl.n, mdl.K, cfg.adam(self.extent), self.adam_steps, mdl.params, mdl.m, mdl.v,
                               grads["means"], grads["scales"], grads["quats"], grads["opacity"], grads["sh"],
                               mdl.means, mdl.scales, mdl.quats, mdl.opacity, mdl.sh)
        return loss
