"""Frame-level driver of the C ABI: owns the device buffers of one frame shape and chains the calls.

forward:  omnigs_preprocess -> omnigs_bin -> omnigs_sort -> omnigs_render_fwd        (Sec. 3.2-3.3)
loss:     omnigs_l1_loss                                                              (Eq. 17, L1 term)
backward: omnigs_render_bwd -> omnigs_preprocess_bwd                                  (Sec. 3.4)

torch provides the memory and the stream; every arithmetic step runs in libomnigs. A Rasterizer keeps the state of
its last forward until the matching backward, so one Rasterizer serves one frame in flight at a time.
"""
from __future__ import annotations

import dataclasses
import math

import torch

from . import _cabi as C


@dataclasses.dataclass
class Settings:
    width: int
    height: int
    tile: int = 16
    num_views: int = 1
    sh_degree: int = 3
    near_r: float = 0.2
    bg: tuple = (0.0, 0.0, 0.0)
    pixels_per_thread: int = 0  # forward blend schedule (2, 4 or 8); 0 = the library's choice
    pinhole: tuple | None = None  # (fx, fy, cx, cy) for the pinhole camera of Eq. 2; None = equirectangular
    adjoint_pixels_per_thread: int = 0  # schedule of the blend adjoint (2, 4 or 8); 0 = the library's choice

    def config(self):
        return C.make_config(self.width, self.height, self.tile, self.num_views, self.sh_degree, self.near_r, self.bg,
                             self.pixels_per_thread, self.pinhole, self.adjoint_pixels_per_thread)

    @property
    def tiles(self) -> int:
        return (self.width // self.tile) * (self.height // self.tile)


def _empty(shape, dtype, device):
    return torch.empty(shape, dtype=dtype, device=device)


class Rasterizer:
    """Buffers for n Gaussians rendered into `num_views` equirectangular views.

    capacity: room for tile instances. With `grow=True` (default) the forward pass reads the instance count back
    (one synchronisation) and re-bins with a larger capacity when needed. With `grow=False` the pass never
    synchronises (it can be captured in a CUDA graph); an overflow is then reported by `check()`.
    alloc: optional allocator `(shape, dtype, device) -> tensor` for every device buffer (default torch.empty);
    forward_only: leave out the buffers of the backward pass (the adjoint's outputs and dL/dC).
    """

    def __init__(self, settings: Settings, device="cuda", capacity: int = 1 << 20, grow: bool = True,
                 headroom: float = 1.25, alloc=None, forward_only: bool = False):
        C.load()
        self._empty = alloc if alloc is not None else _empty
        self.forward_only = forward_only
        self.s = settings
        self.cfg = settings.config()
        self.device = torch.device(device)
        self.capacity = int(capacity)
        self.grow = grow
        self.headroom = headroom
        self.n = -1
        self.count = None
        V, H, W = settings.num_views, settings.height, settings.width
        self.rgb = self._empty((V, 3, H, W), torch.float32, self.device)
        self.T = self._empty((V, H, W), torch.float32, self.device)
        self.ncontrib = self._empty((V, H, W), torch.int32, self.device)
        self.count_out = None  # set to an int32 [V, H, W] tensor to receive per-pixel contributor counts
        self.dL_drgb = None if forward_only else self._empty((V, 3, H, W), torch.float32, self.device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.ranges = self._empty((V * settings.tiles * 2,), torch.int32, self.device)
        self._alloc_instances(self.capacity)

    # ---------------------------------------------------------------- buffers
    def _alloc_instances(self, capacity: int):
        self.capacity = int(capacity)
        cap = max(self.capacity, 1)
        self.keys = self._empty((cap,), torch.int64, self.device)
        self.ws = None

    def _ensure(self, n: int, K: int):
        V = self.s.num_views
        if n != self.n:
            self.n = n
            m = max(V * n, 1)
            self.splats = self._empty((m, C.SPLAT_FLOATS), torch.float32, self.device)
            self.order = self._empty((m,), torch.int32, self.device)
            if not self.forward_only:
                self.grads2d = self._empty((m, C.GRAD_FLOATS), torch.float32, self.device)
                self.d_means = self._empty((max(n, 1), 3), torch.float32, self.device)
                self.d_scales = self._empty((max(n, 1), 3), torch.float32, self.device)
                self.d_quats = self._empty((max(n, 1), 4), torch.float32, self.device)
                self.d_opacity = self._empty((max(n, 1),), torch.float32, self.device)
                self.d_screen = self._empty((max(n, 1), 2), torch.float32, self.device)
            self.ws = None
        if not self.forward_only and (getattr(self, "d_sh", None) is None or self.d_sh.shape[0] != max(n, 1)
                                      or self.d_sh.shape[1] != K):
            self.d_sh = self._empty((max(n, 1), K, 3), torch.float32, self.device)
        if self.ws is None:
            nbytes = C.omnigs_workspace_size(self.cfg, max(n, 0), self.capacity)
            if nbytes == 0:
                raise C.OmnigsError(C.OMNIGS_E_INVALID, "omnigs_workspace_size")
            self.ws = self._empty((nbytes,), torch.uint8, self.device)

    # ---------------------------------------------------------------- forward
    def forward(self, means, scales, quats, opacity, sh, viewmats, stream=None, l1_target=None):
        """Render every view. Inputs are contiguous float32 device tensors; returns rgb [V, 3, H, W] (a buffer of
        this Rasterizer, overwritten by the next forward). With l1_target (a [V, 3, H, W] float32 device tensor) the
        L1 loss is computed by the blend itself (omnigs_render_fwd_l1): self.loss and self.dL_drgb are then set as
        l1_loss(l1_target) would set them, without a second pass over the image."""
        if l1_target is not None:
            if self.forward_only or self.count_out is not None:
                raise ValueError("l1_target needs a Rasterizer with gradients and without per-pixel counts")
            self._check_target(l1_target)
        n = int(means.shape[0])
        K = int(sh.shape[1]) if n > 0 else (self.s.sh_degree + 1) ** 2
        self._ensure(n, K)
        self._params = (means, scales, quats, opacity, sh, viewmats)
        # (omnigs_preprocess then omnigs_bin, in one call: with the equirectangular camera the projection also
        # writes the depth sort's keys)
        C.omnigs_preprocess_bin(self.cfg, n, means, scales, quats, opacity, sh, viewmats, self.splats, self.order,
                                self.keys, self.capacity, self.ws, stream)
        if self.grow:
            self.count = C.omnigs_instance_count(self.ws, stream)
            if self.count > self.capacity:
                self._alloc_instances(int(math.ceil(self.count * self.headroom)))
                self._ensure(n, K)
                C.omnigs_bin(self.cfg, n, self.splats, self.order, self.keys, self.capacity, self.ws, stream)
        C.omnigs_sort(self.cfg, n, self.capacity, self.keys, self.ranges, self.ws, stream)
        if l1_target is not None:
            C.omnigs_render_fwd_l1(self.cfg, n, self.splats, self.ranges, self.keys, self.order, l1_target,
                                   self.rgb, self.T, self.ncontrib, self.dL_drgb, self.loss, self.ws, stream)
        else:
            C.omnigs_render_fwd(self.cfg, n, self.splats, self.ranges, self.keys, self.order, self.rgb, self.T,
                                self.ncontrib, self.count_out, stream)
        return self.rgb

    def _check_target(self, target) -> None:
        """The loss kernels read a [V, 3, H, W] float32 image through a raw pointer: anything else is refused here."""
        if (not isinstance(target, torch.Tensor) or target.dtype != torch.float32 or not target.is_cuda
                or tuple(target.shape) != tuple(self.rgb.shape) or not target.is_contiguous()):
            raise ValueError(f"target must be a contiguous float32 CUDA tensor of shape {tuple(self.rgb.shape)}")

    def l1_loss(self, target, stream=None, rows=None):
        """mean |rgb - target| (device scalar) and its gradient in self.dL_drgb; with rows = (begin, end) only those
        image rows count (the others get a zero gradient)."""
        self._check_target(target)
        if rows is None:
            C.omnigs_l1_loss(self.cfg, self.rgb, target, self.dL_drgb, self.loss, self.ws, stream)
        else:
            C.omnigs_l1_loss_rows(self.cfg, rows[0], rows[1], self.rgb, target, self.dL_drgb, self.loss, self.ws,
                                  stream)
        return self.loss

    # ---------------------------------------------------------------- backward
    def backward_2d(self, dL_drgb=None, stream=None):
        """Blend adjoint only: per-(view, Gaussian) splat gradients [V * n, 12]."""
        g = self.dL_drgb if dL_drgb is None else dL_drgb
        C.omnigs_render_bwd(self.cfg, self.n, self.splats, self.ranges, self.keys, self.order, self.T, self.ncontrib,
                            g, self.grads2d, stream)
        return self.grads2d

    GRAD_NAMES = ("means", "scales", "quats", "opacity", "sh", "screen")

    def backward(self, dL_drgb=None, stream=None, out=None):
        """Gradients of the loss with respect to means, scales, quats, opacity, sh, and dL/ds (screen space).
        They go to this Rasterizer's buffers, or to the device tensors of `out` (a dict with the keys of
        GRAD_NAMES, shaped like those buffers)."""
        self.backward_2d(dL_drgb, stream)
        means, scales, quats, opacity, sh, viewmats = self._params
        g = dict(means=self.d_means, scales=self.d_scales, quats=self.d_quats, opacity=self.d_opacity, sh=self.d_sh,
                 screen=self.d_screen)
        if out is not None:
            for k in self.GRAD_NAMES:
                if tuple(out[k].shape) != tuple(g[k].shape) or out[k].dtype != torch.float32 or not out[k].is_cuda:
                    raise ValueError(f"out[{k!r}] must be a float32 device tensor of shape {tuple(g[k].shape)}")
            g = {k: out[k] for k in self.GRAD_NAMES}
        C.omnigs_preprocess_bwd(self.cfg, self.n, means, scales, quats, opacity, sh, viewmats, self.grads2d,
                                g["means"], g["scales"], g["quats"], g["opacity"], g["sh"], g["screen"], stream)
        return g

    def check(self, stream=None) -> None:
        """Raise if a device-side error (capacity overflow) was recorded since the last check (synchronises)."""
        st = C.omnigs_last_error(self.ws, stream)
        if st != C.OMNIGS_OK:
            raise C.OmnigsError(st, "device")

    def instance_count(self, stream=None) -> int:
        return C.omnigs_instance_count(self.ws, stream)

    def sorted_splats(self, count: int):
        """Splat index (v * n + g) of every sorted instance position [0, count) (host copy, for inspection)."""
        keys = self.keys[:count].cpu().numpy().view("uint64")
        order = self.order.cpu().numpy().view("uint32").astype("int64")
        rb = C.rank_bits(self.n)
        tiles = self.s.tiles
        view = (keys >> rb).astype("int64") // tiles
        return order[view * self.n + (keys & ((1 << rb) - 1)).astype("int64")]


class OmniRender(torch.autograd.Function):
    """Differentiable equirectangular render: (means, scales, quats, opacity, sh) -> rgb [V, 3, H, W].

    `rasterizer` is a Rasterizer whose frame state stays untouched between this forward and its backward."""

    @staticmethod
    def forward(ctx, means, scales, quats, opacity, sh, viewmats, rasterizer):
        rgb = rasterizer.forward(means.contiguous(), scales.contiguous(), quats.contiguous(), opacity.contiguous(),
                                 sh.contiguous(), viewmats.contiguous())
        ctx.rasterizer = rasterizer
        return rgb.clone()

    @staticmethod
    def backward(ctx, grad_rgb):
        g = ctx.rasterizer.backward(grad_rgb.contiguous())
        return (g["means"].clone(), g["scales"].clone(), g["quats"].clone(), g["opacity"].clone(), g["sh"].clone(),
                None, None)


def render(means, scales, quats, opacity, sh, viewmats, rasterizer: Rasterizer):
    """Functional, autograd-aware form of Rasterizer.forward."""
    return OmniRender.apply(means, scales, quats, opacity, sh, viewmats, rasterizer)
