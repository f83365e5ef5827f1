"""Streamed training or rendering steps whose inputs come from pinned host memory and whose results go back to it.

Each step copies its inputs (the Gaussian parameters, the camera poses and the target images) host -> device, runs
forward, loss and backward, and copies the loss and every gradient device -> host. The copies of step k + 1 (in) and
of step k - 1 (out) run on two copy streams while step k computes: the device holds two input slots and two output
slots, and CUDA events order each slot's copy against the compute that reads or writes it. Every step's copies are
still made in full; only their overlap with the neighbouring steps' compute is new.

With graph=True (a Rasterizer built with grow=False, and the same shapes every step) the compute of each slot is
captured once in a CUDA graph after its first, eager, run and replayed from then on: the same kernels on the slot's
buffers without the per-launch host cost.
"""
from __future__ import annotations

from typing import Callable, Sequence

import torch

from .rasterizer import Rasterizer


class StreamedSteps:
    """Double-buffered fwd + loss + bwd steps of one Rasterizer.

    loss_fn(rasterizer, target) computes the loss into rasterizer.loss and its image gradient into
    rasterizer.dL_drgb on the current stream (e.g. lambda r, t: r.l1_loss(t)). loss_fn=None: the L1 loss, computed
    by the forward blend itself (Rasterizer.forward with l1_target).
    """

    def __init__(self, rasterizer: Rasterizer, loss_fn: Callable[[Rasterizer, torch.Tensor], object] | None,
                 graph: bool = False):
        if graph and rasterizer.grow:
            raise ValueError("graph=True needs a Rasterizer built with grow=False (no host synchronisation)")
        self.r = rasterizer
        self.loss_fn = loss_fn
        self.graph = graph
        self.graphs = [None, None]    # captured compute of each slot
        dev = rasterizer.device
        self.h2d = torch.cuda.Stream(dev)
        self.d2h = torch.cuda.Stream(dev)
        self.inputs = [None, None]    # device input slots
        self.outputs = [None, None]   # device result slots (gradients + loss)
        self.in_ready = [torch.cuda.Event(), torch.cuda.Event()]
        self.in_free = [None, None]   # compute done reading the slot
        self.out_ready = [torch.cuda.Event(), torch.cuda.Event()]
        self.out_free = [None, None]  # device -> host copy of the slot done
        self.k = 0

    def _alloc(self, s: int, host_in: Sequence[torch.Tensor]):
        dev = self.r.device
        if self.inputs[s] is None or any(d.shape != h.shape for d, h in zip(self.inputs[s], host_in)):
            self.inputs[s] = [torch.empty(h.shape, dtype=h.dtype, device=dev) for h in host_in]
            self.graphs = [None, None]  # new buffers (and possibly new shapes inside the Rasterizer): capture again

    def _out_slot(self, s: int, means: torch.Tensor, sh: torch.Tensor):
        dev = self.r.device
        n, K = int(means.shape[0]), int(sh.shape[1])
        shapes = dict(means=(n, 3), scales=(n, 3), quats=(n, 4), opacity=(n,), sh=(n, K, 3), screen=(n, 2))
        o = self.outputs[s]
        if o is None or any(tuple(o[k].shape) != v for k, v in shapes.items()):
            o = {k: torch.empty(v, dtype=torch.float32, device=dev) for k, v in shapes.items()}
            o["loss"] = torch.empty(1, dtype=torch.float32, device=dev)
            self.outputs[s] = o
            self.graphs[s] = None
        return o

    def _compute(self, s: int):
        means, scales, quats, opacity, sh, viewmats, target = self.inputs[s]
        if self.loss_fn is None:
            self.r.forward(means, scales, quats, opacity, sh, viewmats, l1_target=target)
        else:
            self.r.forward(means, scales, quats, opacity, sh, viewmats)
            self.loss_fn(self.r, target)
        o = self.outputs[s]
        self.r.backward(out=o)
        o["loss"].copy_(self.r.loss)

    def begin(self):
        """Order the copy streams after everything the current stream has enqueued (e.g. a start event)."""
        cur = torch.cuda.current_stream(self.r.device)
        self.h2d.wait_stream(cur)
        self.d2h.wait_stream(cur)

    def submit(self, host_in: Sequence[torch.Tensor], host_out: dict) -> torch.cuda.Event:
        """Enqueue one step. host_in = (means, scales, quats, opacity, sh, viewmats, target), pinned host tensors;
        host_out maps the gradient names of Rasterizer.GRAD_NAMES and "loss" to pinned host tensors of matching
        shapes. Returns the event that completes when the results are in host_out."""
        s = self.k % 2
        cur = torch.cuda.current_stream(self.r.device)
        self._alloc(s, host_in)
        with torch.cuda.stream(self.h2d):
            if self.in_free[s] is not None:
                self.h2d.wait_event(self.in_free[s])
            for d, h in zip(self.inputs[s], host_in):
                d.copy_(h, non_blocking=True)
            self.in_ready[s].record(self.h2d)
        cur.wait_event(self.in_ready[s])
        o = self._out_slot(s, self.inputs[s][0], self.inputs[s][4])
        if self.out_free[s] is not None:
            cur.wait_event(self.out_free[s])
        if self.graphs[s] is not None:
            self.graphs[s].replay()
        else:
            self._compute(s)
            if self.graph:  # record the same work once for the next uses of this slot (capture runs nothing)
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g):
                    self._compute(s)
                self.graphs[s] = g
        self.in_free[s] = torch.cuda.Event()
        self.in_free[s].record(cur)
        self.out_ready[s].record(cur)
        with torch.cuda.stream(self.d2h):
            self.d2h.wait_event(self.out_ready[s])
            for k, h in host_out.items():
                h.copy_(o[k], non_blocking=True)
            done = torch.cuda.Event()
            done.record(self.d2h)
        self.out_free[s] = done
        self.k += 1
        return done

    def end(self):
        """Make the current stream wait for every enqueued copy (e.g. before an end event)."""
        cur = torch.cuda.current_stream(self.r.device)
        cur.wait_stream(self.h2d)
        cur.wait_stream(self.d2h)
