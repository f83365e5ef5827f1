"""Autotuner for the tile size and the blend schedule of a workload.

The tile side (8, 16 or 32 px) trades binning and sorting work (instances grow roughly with 1 / tile^2 of the
covered area) against blending work (a larger tile walks longer lists per pixel); the blend schedule (2, 4 or 8 pixels
per thread) trades per-entry sharing against threads per tile (at 8 one warp covers a 16 x 16 tile). The best choice depends on the scene, the poses and
the resolution, so the tuner times each candidate on the caller's own data, with CUDA events on the current stream,
and keeps the fastest per workload key (Gaussian count bucket, views, resolution, SH degree, mode).

Changing the tile size changes which splats a pixel examines: a splat whose 3-sigma square is the binding limit
(high opacity) can reach pixels outside its instance box when the tile grows, exactly as in the tiled renderer the
paper builds on. Images therefore agree across tile sizes only up to those pixels; the blend schedule never changes
the forward result (and the gradients only by the order of float additions).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import torch

from . import _cabi as C
from .rasterizer import Rasterizer, Settings

CANDIDATES = [(8, 2), (16, 2), (16, 4), (16, 8), (32, 2), (32, 4), (32, 8)]


@dataclass
class Choice:
    tile: int
    pixels_per_thread: int
    ms: float
    table: dict  # (tile, ppt) -> ms


def workload_key(n: int, settings: Settings, mode: str) -> tuple:
    bucket = 0 if n <= 0 else int(round(math.log2(n) * 2))  # half-octave buckets of the Gaussian count
    return (bucket, settings.num_views, settings.width, settings.height, settings.sh_degree, mode)


class Autotuner:
    def __init__(self, candidates=CANDIDATES, warmup: int = 2, iters: int = 5):
        self.candidates = list(candidates)
        self.warmup, self.iters = warmup, iters
        self.cache: dict = {}

    def _valid(self, settings: Settings, tile: int) -> bool:
        return settings.width % tile == 0 and settings.height % tile == 0

    def tune(self, params, viewmats, settings: Settings, mode: str = "train", target=None) -> Choice:
        """Times every valid candidate on (params, viewmats) and returns the fastest.

        mode "train": forward + L1 loss (against `target`, or the first candidate's own image) + backward;
        mode "render": forward only."""
        n = int(params[0].shape[0])
        key = workload_key(n, settings, mode)
        if key in self.cache:
            return self.cache[key]
        table = {}
        for tile, ppt in self.candidates:
            if not self._valid(settings, tile):
                continue
            try:
                ms, target = self._time(params, viewmats, replace(settings, tile=tile, pixels_per_thread=ppt), mode,
                                        target)
            except (C.OmnigsError, torch.cuda.OutOfMemoryError):
                torch.cuda.empty_cache()
                continue  # e.g. more instances than one workspace can index at this tile size
            if ms is not None:
                table[(tile, ppt)] = ms
        if not table:
            raise RuntimeError("no autotuning candidate ran")
        (tile, ppt), ms = min(table.items(), key=lambda kv: kv[1])
        choice = Choice(tile, ppt, ms, table)
        self.cache[key] = choice
        return choice

    def _time(self, params, viewmats, s: Settings, mode: str, target):
        probe = Rasterizer(s, device=params[0].device)
        probe.forward(*params, viewmats)
        if mode == "train" and target is None:
            target = probe.rgb.clone()
        r = Rasterizer(s, device=params[0].device, capacity=int(probe.count * 1.1) + 4096, grow=False)
        del probe

        def step():
            r.forward(*params, viewmats)
            if mode == "train":
                r.l1_loss(target)
                r.backward()

        for _ in range(self.warmup):
            step()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(self.iters):
            step()
        e1.record()
        torch.cuda.synchronize()
        try:
            r.check()
        except C.OmnigsError:
            return None, target  # capacity overflow in the timed loop: not a timing of the full work
        return e0.elapsed_time(e1) / self.iters, target

    def settings(self, params, viewmats, settings: Settings, mode: str = "train", target=None) -> Settings:
        c = self.tune(params, viewmats, settings, mode, target)
        return replace(settings, tile=c.tile, pixels_per_thread=c.pixels_per_thread)
