"""ctypes binding of `libomnigs.so` (declared in include/omnigs.h), with the same entry-point names.

This layer only marshals arguments: torch tensors become device pointers, the current torch CUDA stream becomes
the stream argument. All computation happens in the CUDA library; if it is missing, importing this module fails.
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libomnigs.so")

OMNIGS_OK, OMNIGS_E_INVALID, OMNIGS_E_CAPACITY, OMNIGS_E_CUDA, OMNIGS_E_TIMEOUT = range(5)


class OmnigsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


class omnigs_config(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("num_views", ctypes.c_int32), ("sh_degree", ctypes.c_int32), ("near_r", ctypes.c_float),
                ("bg", ctypes.c_float * 3), ("pixels_per_thread", ctypes.c_int32), ("camera", ctypes.c_int32),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("adjoint_pixels_per_thread", ctypes.c_int32)]

CAMERA_EQUIRECT, CAMERA_PINHOLE = 0, 1


class omnigs_adam_config(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in ("lr_means", "lr_scales", "lr_quats", "lr_opacity", "lr_sh_dc",
                                              "lr_sh_rest", "beta1", "beta2", "eps")]


class omnigs_densify_config(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in ("grad_threshold", "percent_dense", "extent", "min_opacity",
                                              "max_scale_frac", "max_screen_radius")]


class omnigs_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


SPLAT_FLOATS = 12  # sizeof(omnigs_splat) / 4
GRAD_FLOATS = 12   # sizeof(omnigs_splat_grad) / 4


def rank_bits(n: int) -> int:
    """Bits of the depth rank in an instance key (max(1, ceil(log2(n))))."""
    return max(1, (max(int(n), 1) - 1).bit_length())

_lib = None


def load() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build() or "
                              f"python paper_2404_03202_gb300/build.py)")
        lib = ctypes.CDLL(LIB_PATH)
        P, i64, st = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        cfgp = ctypes.POINTER(omnigs_config)
        lib.omnigs_version.restype = ctypes.c_int
        lib.omnigs_status_string.argtypes = [st]
        lib.omnigs_status_string.restype = ctypes.c_char_p
        lib.omnigs_workspace_size.argtypes = [cfgp, i64, i64]
        lib.omnigs_workspace_size.restype = ctypes.c_size_t
        lib.omnigs_preprocess.argtypes = [cfgp, i64, P, P, P, P, P, P, P, P]
        lib.omnigs_bin.argtypes = [cfgp, i64, P, P, P, i64, P, P]
        lib.omnigs_preprocess_bin.argtypes = [cfgp, i64, P, P, P, P, P, P, P, P, P, i64, P, P]
        lib.omnigs_sort.argtypes = [cfgp, i64, i64, P, P, P, P]
        lib.omnigs_render_fwd.argtypes = [cfgp, i64, P, P, P, P, P, P, P, P, P]
        lib.omnigs_render_fwd_l1.argtypes = [cfgp, i64, P, P, P, P, P, P, P, P, P, P, P, P]
        lib.omnigs_l1_loss.argtypes = [cfgp, P, P, P, P, P, P]
        lib.omnigs_l1_loss_rows.argtypes = [cfgp, ctypes.c_int32, ctypes.c_int32, P, P, P, P, P, P]
        lib.omnigs_l1_loss_static.argtypes = [cfgp, P, P, P, P, P]
        lib.omnigs_dssim_scratch_size.argtypes = [cfgp]
        lib.omnigs_dssim_scratch_size.restype = ctypes.c_size_t
        lib.omnigs_dssim_loss.argtypes = [cfgp, ctypes.c_float, P, P, P, P, P, P]
        lib.omnigs_l1_loss_static.restype = st
        lib.omnigs_render_bwd.argtypes = [cfgp, i64, P, P, P, P, P, P, P, P, P]
        lib.omnigs_preprocess_bwd.argtypes = [cfgp, i64, P, P, P, P, P, P, P, P, P, P, P, P, P, P]
        lib.omnigs_instance_count.argtypes = [P, ctypes.POINTER(i64), P]
        lib.omnigs_last_error.argtypes = [P, P]
        i32 = ctypes.c_int32
        lib.omnigs_adam_step.argtypes = [i64, i32, ctypes.POINTER(omnigs_adam_config), i64] + [P] * 13 + [P]
        lib.omnigs_publish_params.argtypes = [i64, i32] + [P] * 6 + [P]
        lib.omnigs_densify_stats.argtypes = [cfgp, i64, P, P, P, P, P, P]
        lib.omnigs_densify_workspace_size.argtypes = [i64]
        lib.omnigs_densify_workspace_size.restype = ctypes.c_size_t
        lib.omnigs_densify.argtypes = [i64, i32, ctypes.POINTER(omnigs_densify_config)] + [P] * 12 + [P]
        lib.omnigs_reset_opacity.argtypes = [i64, i32, ctypes.c_float, P, P, P, P, P]
        f32 = ctypes.c_float
        lib.omnigs_equirect_crop.argtypes = [i32, i32, i32, P, P, i32, i32, f32, f32, f32, f32, P, P]
        lib.omnigs_profiler_enable.argtypes = [ctypes.c_int]
        lib.omnigs_profiler_collect.argtypes = [ctypes.POINTER(omnigs_kernel_time), ctypes.c_int]
        lib.omnigs_profiler_collect.restype = ctypes.c_int
        for name in ("omnigs_preprocess", "omnigs_bin", "omnigs_preprocess_bin", "omnigs_sort", "omnigs_render_fwd", "omnigs_render_fwd_l1",
                     "omnigs_l1_loss",
                     "omnigs_l1_loss_rows", "omnigs_dssim_loss", "omnigs_adam_step", "omnigs_publish_params",
                     "omnigs_densify_stats", "omnigs_densify", "omnigs_reset_opacity", "omnigs_equirect_crop",
                     "omnigs_render_bwd", "omnigs_preprocess_bwd", "omnigs_instance_count", "omnigs_last_error",
                     "omnigs_profiler_enable"):
            getattr(lib, name).restype = st
        _lib = lib
    return _lib


def status_string(status: int) -> str:
    return load().omnigs_status_string(int(status)).decode()


def _check(status: int, where: str) -> None:
    if status != OMNIGS_OK:
        raise OmnigsError(status, where)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_config(width: int, height: int, tile: int = 16, num_views: int = 1, sh_degree: int = 3,
                near_r: float = 0.2, bg=(0.0, 0.0, 0.0), pixels_per_thread: int = 0, pinhole=None,
                adjoint_pixels_per_thread: int = 0) -> omnigs_config:
    """pinhole: None for the equirectangular camera, else (fx, fy, cx, cy) in pixels (Eq. 2). pixels_per_thread and
    adjoint_pixels_per_thread: schedules of the forward blend and of its adjoint (0: the library's choice)."""
    c = omnigs_config()
    c.width, c.height, c.tile, c.num_views, c.sh_degree, c.near_r = width, height, tile, num_views, sh_degree, near_r
    c.pixels_per_thread = pixels_per_thread
    c.adjoint_pixels_per_thread = adjoint_pixels_per_thread
    if pinhole is not None:
        c.camera = CAMERA_PINHOLE
        c.fx, c.fy, c.cx, c.cy = (float(x) for x in pinhole)
    for i in range(3):
        c.bg[i] = float(bg[i])
    return c


# ------------------------------------------------------------------ entry points (same names as the C ABI)

def omnigs_version() -> int:
    return load().omnigs_version()


def omnigs_workspace_size(cfg: omnigs_config, n: int, capacity: int) -> int:
    return int(load().omnigs_workspace_size(ctypes.byref(cfg), n, capacity))


def omnigs_preprocess(cfg, n, means, scales, quats, opacity, sh, viewmats, splats, stream=None):
    _check(load().omnigs_preprocess(ctypes.byref(cfg), n, _ptr(means), _ptr(scales), _ptr(quats), _ptr(opacity),
                                    _ptr(sh), _ptr(viewmats), _ptr(splats), _stream(stream)), "omnigs_preprocess")


def omnigs_bin(cfg, n, splats, order, keys, capacity, workspace, stream=None):
    _check(load().omnigs_bin(ctypes.byref(cfg), n, _ptr(splats), _ptr(order), _ptr(keys), capacity, _ptr(workspace),
                             _stream(stream)), "omnigs_bin")


def omnigs_preprocess_bin(cfg, n, means, scales, quats, opacity, sh, viewmats, splats, order, keys, capacity,
                          workspace, stream=None):
    _check(load().omnigs_preprocess_bin(ctypes.byref(cfg), n, _ptr(means), _ptr(scales), _ptr(quats), _ptr(opacity),
                                        _ptr(sh), _ptr(viewmats), _ptr(splats), _ptr(order), _ptr(keys), capacity,
                                        _ptr(workspace), _stream(stream)), "omnigs_preprocess_bin")


def omnigs_sort(cfg, n, capacity, keys, ranges, workspace, stream=None):
    _check(load().omnigs_sort(ctypes.byref(cfg), n, capacity, _ptr(keys), _ptr(ranges), _ptr(workspace),
                              _stream(stream)), "omnigs_sort")


def omnigs_render_fwd(cfg, n, splats, ranges, keys, order, out_rgb, out_T, out_ncontrib, out_count=None, stream=None):
    _check(load().omnigs_render_fwd(ctypes.byref(cfg), n, _ptr(splats), _ptr(ranges), _ptr(keys), _ptr(order),
                                    _ptr(out_rgb), _ptr(out_T), _ptr(out_ncontrib), _ptr(out_count), _stream(stream)),
           "omnigs_render_fwd")


def omnigs_render_fwd_l1(cfg, n, splats, ranges, keys, order, target, out_rgb, out_T, out_ncontrib, dL_drgb, loss,
                         workspace, stream=None):
    _check(load().omnigs_render_fwd_l1(ctypes.byref(cfg), n, _ptr(splats), _ptr(ranges), _ptr(keys), _ptr(order),
                                       _ptr(target), _ptr(out_rgb), _ptr(out_T), _ptr(out_ncontrib), _ptr(dL_drgb),
                                       _ptr(loss), _ptr(workspace), _stream(stream)), "omnigs_render_fwd_l1")


def omnigs_l1_loss(cfg, rgb, target, dL_drgb, loss, workspace, stream=None):
    _check(load().omnigs_l1_loss(ctypes.byref(cfg), _ptr(rgb), _ptr(target), _ptr(dL_drgb), _ptr(loss),
                                 _ptr(workspace), _stream(stream)), "omnigs_l1_loss")


def omnigs_l1_loss_rows(cfg, row_begin, row_end, rgb, target, dL_drgb, loss, workspace, stream=None):
    _check(load().omnigs_l1_loss_rows(ctypes.byref(cfg), int(row_begin), int(row_end), _ptr(rgb), _ptr(target),
                                      _ptr(dL_drgb), _ptr(loss), _ptr(workspace), _stream(stream)),
           "omnigs_l1_loss_rows")


def omnigs_dssim_scratch_size(cfg) -> int:
    return int(load().omnigs_dssim_scratch_size(ctypes.byref(cfg)))


def omnigs_dssim_loss(cfg, lam, rgb, target, dL_drgb, loss, scratch, stream=None):
    _check(load().omnigs_dssim_loss(ctypes.byref(cfg), float(lam), _ptr(rgb), _ptr(target), _ptr(dL_drgb),
                                    _ptr(loss), _ptr(scratch), _stream(stream)), "omnigs_dssim_loss")


def omnigs_l1_loss_static(cfg, rgb, target, dL_drgb, loss, stream=None):
    """omnigs_l1_loss without a workspace (no device allocation anywhere); see include/omnigs.h for its limit."""
    _check(load().omnigs_l1_loss_static(ctypes.byref(cfg), _ptr(rgb), _ptr(target), _ptr(dL_drgb), _ptr(loss),
                                        _stream(stream)), "omnigs_l1_loss_static")


def omnigs_render_bwd(cfg, n, splats, ranges, keys, order, out_T, ncontrib, dL_drgb, grads, stream=None):
    _check(load().omnigs_render_bwd(ctypes.byref(cfg), n, _ptr(splats), _ptr(ranges), _ptr(keys), _ptr(order),
                                    _ptr(out_T), _ptr(ncontrib), _ptr(dL_drgb), _ptr(grads), _stream(stream)),
           "omnigs_render_bwd")


def omnigs_preprocess_bwd(cfg, n, means, scales, quats, opacity, sh, viewmats, grads, d_means, d_scales, d_quats,
                          d_opacity, d_sh, d_screen, stream=None):
    _check(load().omnigs_preprocess_bwd(ctypes.byref(cfg), n, _ptr(means), _ptr(scales), _ptr(quats), _ptr(opacity),
                                        _ptr(sh), _ptr(viewmats), _ptr(grads), _ptr(d_means), _ptr(d_scales),
                                        _ptr(d_quats), _ptr(d_opacity), _ptr(d_sh), _ptr(d_screen), _stream(stream)),
           "omnigs_preprocess_bwd")


def omnigs_instance_count(workspace, stream=None) -> int:
    out = ctypes.c_int64(0)
    _check(load().omnigs_instance_count(_ptr(workspace), ctypes.byref(out), _stream(stream)), "omnigs_instance_count")
    return int(out.value)


def omnigs_last_error(workspace, stream=None) -> int:
    """Returns the status code (does not raise)."""
    return int(load().omnigs_last_error(_ptr(workspace), _stream(stream)))


def omnigs_profiler_enable(enable: bool) -> None:
    _check(load().omnigs_profiler_enable(1 if enable else 0), "omnigs_profiler_enable")


def omnigs_profiler_collect(max_kernels: int = 64) -> list:
    arr = (omnigs_kernel_time * max_kernels)()
    k = load().omnigs_profiler_collect(arr, max_kernels)
    return [(arr[i].name.decode(), int(arr[i].launches), float(arr[i].total_ms)) for i in range(min(k, max_kernels))]


# ------------------------------------------------------------------ reconstruction loop (Algorithm 1)

def omnigs_adam_step(n, K, cfg, step, params, m, v, d_means, d_scales, d_quats, d_opacity, d_sh, means, scales,
                     quats, opacity, sh, stream=None):
    _check(load().omnigs_adam_step(n, K, ctypes.byref(cfg), int(step), _ptr(params), _ptr(m), _ptr(v),
                                   _ptr(d_means), _ptr(d_scales), _ptr(d_quats), _ptr(d_opacity), _ptr(d_sh),
                                   _ptr(means), _ptr(scales), _ptr(quats), _ptr(opacity), _ptr(sh), _stream(stream)),
           "omnigs_adam_step")


def omnigs_publish_params(n, K, params, means, scales, quats, opacity, sh, stream=None):
    _check(load().omnigs_publish_params(n, K, _ptr(params), _ptr(means), _ptr(scales), _ptr(quats), _ptr(opacity),
                                        _ptr(sh), _stream(stream)), "omnigs_publish_params")


def omnigs_densify_stats(cfg, n, splats, grads, accum, count, max_radius, stream=None):
    _check(load().omnigs_densify_stats(ctypes.byref(cfg), n, _ptr(splats), _ptr(grads), _ptr(accum), _ptr(count),
                                       _ptr(max_radius), _stream(stream)), "omnigs_densify_stats")


def omnigs_densify_workspace_size(n) -> int:
    return int(load().omnigs_densify_workspace_size(n))


def omnigs_densify(n, K, cfg, params, m, v, accum, count, max_radius, normals, params_out, m_out, v_out, n_out,
                   workspace, stream=None):
    _check(load().omnigs_densify(n, K, ctypes.byref(cfg), _ptr(params), _ptr(m), _ptr(v), _ptr(accum), _ptr(count),
                                 _ptr(max_radius), _ptr(normals), _ptr(params_out), _ptr(m_out), _ptr(v_out),
                                 _ptr(n_out), _ptr(workspace), _stream(stream)), "omnigs_densify")


def omnigs_reset_opacity(n, K, value, params, m, v, opacity=None, stream=None):
    _check(load().omnigs_reset_opacity(n, K, float(value), _ptr(params), _ptr(m), _ptr(v), _ptr(opacity),
                                       _stream(stream)), "omnigs_reset_opacity")


def omnigs_equirect_crop(V, eq_width, eq_height, equirect, rotations, width, height, fx, fy, cx, cy, out, stream=None):
    _check(load().omnigs_equirect_crop(V, eq_width, eq_height, _ptr(equirect), _ptr(rotations), width, height,
                                       float(fx), float(fy), float(cx), float(cy), _ptr(out), _stream(stream)),
           "omnigs_equirect_crop")
