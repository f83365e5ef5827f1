"""FP64 CPU oracle of equirectangular Gaussian splatting (OmniGS, arXiv 2404.03202).

TEST INFRASTRUCTURE. Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline / reference leg of `bench.py` may
import this package. It shares no code with the CUDA path (`paper_2404_03202_gb300`): the arithmetic lives in
`omnigs_oracle.c` (plain C, double precision, single thread), and this file only marshals numpy arrays to it and
chains its stages in the paper's order (Sec. 3.2 projection, Sec. 3.3 tile binning / sort by t_r / blending,
Sec. 3.4 gradients).

Every function is pinned by `tests/test_oracle_pins.py` against closed forms, library routines, brute force and
finite differences (see that file for which pin covers which function).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "omnigs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

R_LEN = 19
(R_PX, R_PY, R_DEPTH, R_C0, R_C1, R_C2, R_OPAC, R_RED, R_GREEN, R_BLUE, R_RADIUS, R_COV00, R_COV01, R_COV11,
 R_RMARGIN, R_FLAGS, R_RX, R_RY, R_Q) = range(R_LEN)
SPLAT_COLS = [R_PX, R_PY, R_C0, R_C1, R_C2, R_OPAC, R_RED, R_GREEN, R_BLUE]
G_LEN = 9


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (gcc), in place."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.orc_project.argtypes = [P, i32, i32, P, P, P]
        lib.orc_jacobian.argtypes = [P, i32, i32, P]
        lib.orc_sh_basis.argtypes = [i32, P, P, P]
        lib.orc_quat_to_rot.argtypes = [P, P]
        lib.orc_preprocess.argtypes = [i64, i32, i32, i32, i32, f64, P, P, P, P, P, P, P]
        lib.orc_rect.argtypes = [f64, f64, i32, i32, i32, i32, i32, P]
        lib.orc_count_instances.argtypes = [i32, i64, i32, i32, i32, P, P, P, P]
        lib.orc_count_instances.restype = i64
        lib.orc_bin_sort.argtypes = [i32, i64, i32, i32, i32, P, P, P, P, P, P, P, P]
        lib.orc_bin_sort.restype = i64
        lib.orc_blend_fwd.argtypes = [i32, i64, i32, i32, i32, P, P, P, P, f64, P, P, P, P, P]
        lib.orc_blend_bwd.argtypes = [i32, i64, i32, i32, i32, P, P, P, P, P, P]
        lib.orc_set_camera.argtypes = [i32, f64, f64, f64, f64]
        lib.orc_preprocess_bwd.argtypes = [i64, i32, i32, i32, i32, f64, P, P, P, P, P, P, P, P, P, P, P, P, P]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def pinhole(fx: float, fy: float, cx: float, cy: float) -> dict:
    """A pinhole camera (Eq. 2) for the `camera` argument of the stage functions (None = equirectangular)."""
    return dict(fx=float(fx), fy=float(fy), cx=float(cx), cy=float(cy))


def _camera(camera):
    lib = _load()
    if camera is None:
        lib.orc_set_camera(0, 0.0, 0.0, 0.0, 0.0)
    else:
        lib.orc_set_camera(1, camera["fx"], camera["fy"], camera["cx"], camera["cy"])


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------------ single-point maths (Eqs. 3-5, 10-16, Sec. 3.1)

def project(t, width: int, height: int):
    """Eqs. 3-5 for one camera-space point: returns (lon, lat), s, p."""
    lib = _load()
    t = _f64(t)
    ll, s, p = np.zeros(2), np.zeros(2), np.zeros(2)
    lib.orc_project(_p(t), width, height, _p(ll), _p(s), _p(p))
    return ll, s, p


def jacobian(t, width: int, height: int) -> np.ndarray:
    """Eqs. 10-16: the 2x3 Jacobian dp/dt."""
    lib = _load()
    t = _f64(t)
    J = np.zeros(6)
    lib.orc_jacobian(_p(t), width, height, _p(J))
    return J.reshape(2, 3)


def sh_basis(degree: int, d):
    """Real orthonormal SH values Y[16] and their gradients dY[16, 3] at unit direction d."""
    lib = _load()
    d = _f64(d)
    Y, dY = np.zeros(16), np.zeros((16, 3))
    lib.orc_sh_basis(degree, _p(d), _p(Y), _p(dY))
    return Y, dY


def quat_to_rot(q) -> np.ndarray:
    lib = _load()
    q = _f64(q)
    R = np.zeros(9)
    lib.orc_quat_to_rot(_p(q), _p(R))
    return R.reshape(3, 3)


def rect(px: float, py: float, rx: int, ry: int, width: int, height: int, tile: int, camera=None):
    """Tile rectangle (x0, nx, y0, ny) of the instance box (half-extents rx, ry) of one splat."""
    lib = _load()
    _camera(camera)
    out = np.zeros(4, dtype=np.int64)
    lib.orc_rect(float(px), float(py), int(rx), int(ry), width, height, tile, _p(out))
    return tuple(int(x) for x in out)


# ------------------------------------------------------------------ stages

def preprocess(scene, viewmats, width: int, height: int, near: float = 0.2, camera=None) -> np.ndarray:
    """Per-(view, Gaussian) records [V * N, R_LEN] (field order: see R_* constants)."""
    lib = _load()
    _camera(camera)
    means, scales, quats, opacity, sh = (_f32(a) for a in scene.arrays())
    vm = _f32(viewmats).reshape(-1, 16)
    V, n = vm.shape[0], means.shape[0]
    rec = np.zeros((V * n, R_LEN))
    lib.orc_preprocess(n, V, width, height, scene.sh_degree, near, _p(means), _p(scales), _p(quats), _p(opacity),
                       _p(sh), _p(vm), _p(rec))
    return rec


def splats_from_records(rec: np.ndarray) -> dict:
    """Screen-space splat fields from preprocess records (double precision; rx, ry and the square's radius int32)."""
    return dict(px=rec[:, R_PX], py=rec[:, R_PY], c0=rec[:, R_C0], c1=rec[:, R_C1], c2=rec[:, R_C2],
                opacity=rec[:, R_OPAC], r=rec[:, R_RED], g=rec[:, R_GREEN], b=rec[:, R_BLUE],
                depth=rec[:, R_DEPTH], rx=rec[:, R_RX].astype(np.int32), ry=rec[:, R_RY].astype(np.int32),
                radius=rec[:, R_RADIUS].astype(np.int32), q=rec[:, R_Q])


def splat_q(splats: dict) -> np.ndarray:
    """q = 2 ln(255 o) of each splat (the alpha >= 1/255 level of its ellipse): the stored value when the dict has
    one (preprocess records), else computed from the opacity (hand-made splats)."""
    if "q" in splats:
        return _f64(splats["q"])
    o = _f64(splats["opacity"])
    with np.errstate(divide="ignore"):
        return np.maximum(2.0 * np.log(255.0 * o), 0.0)


def count_instances(splats: dict, V: int, width: int, height: int, tile: int, camera=None) -> int:
    """Number of (Gaussian, tile) instances: every tile of every instance box (Sec. 3.3)."""
    lib = _load()
    _camera(camera)
    px, py = _f64(splats["px"]), _f64(splats["py"])
    rx, ry = _i32(splats["rx"]), _i32(splats["ry"])
    return int(lib.orc_count_instances(V, px.shape[0] // V, width, height, tile, _p(px), _p(py), _p(rx), _p(ry)))


def bin_sort(splats: dict, V: int, width: int, height: int, tile: int, tile_mask=None, camera=None):
    """Instances (one per Gaussian and tile of its instance box) sorted by (view, tile, t_r, Gaussian): returns ranges
    [V*tiles, 2] and the list of (v*N + g). With `tile_mask` ([V*tiles] bool), only the lists of the masked tiles are
    built."""
    lib = _load()
    _camera(camera)
    px, py, depth = _f64(splats["px"]), _f64(splats["py"]), _f64(splats["depth"])
    rx, ry = _i32(splats["rx"]), _i32(splats["ry"])
    n = px.shape[0] // V
    tiles = (width // tile) * (height // tile)
    mask = None if tile_mask is None else np.ascontiguousarray(tile_mask, dtype=np.uint8)
    ranges = np.zeros((V * tiles, 2), dtype=np.int64)
    total = int(lib.orc_bin_sort(V, n, width, height, tile, _p(px), _p(py), _p(rx), _p(ry), _p(depth), _p(ranges),
                                 None, None if mask is None else _p(mask)))
    lst = np.zeros(max(total, 1), dtype=np.int64)
    lib.orc_bin_sort(V, n, width, height, tile, _p(px), _p(py), _p(rx), _p(ry), _p(depth), _p(ranges), _p(lst),
                     None if mask is None else _p(mask))
    return ranges, lst[:total]


def _splat9(splats: dict) -> np.ndarray:
    return np.ascontiguousarray(np.stack([_f64(splats[k]) for k in ("px", "py", "c0", "c1", "c2", "opacity", "r", "g", "b")], axis=1))


def blend_fwd(splats: dict, ranges, lst, V: int, width: int, height: int, tile: int, bg=(0.0, 0.0, 0.0),
              eps: float = 1e-5, camera=None):
    """Eqs. 6-8 per pixel over its tile list. Returns rgb [V,3,H,W], T [V,H,W], n_contrib, near-threshold flags; the
    per-pixel number of contributors of the last call is kept in blend_fwd.last_count."""
    lib = _load()
    _camera(camera)
    sp = _splat9(splats)
    n = sp.shape[0] // V
    bgv = _f64(bg)
    rgb = np.zeros((V, 3, height, width))
    T = np.zeros((V, height, width))
    nc = np.zeros((V, height, width), dtype=np.int32)
    near = np.zeros((V, height, width), dtype=np.uint8)
    count = np.zeros((V, height, width), dtype=np.int32)
    lib.orc_blend_fwd(V, n, width, height, tile, _p(bgv), _p(sp), _p(_i64(ranges)), _p(_i64(lst)), eps, _p(rgb), _p(T),
                      _p(nc), _p(near), _p(count))
    blend_fwd.last_count = count
    return rgb, T, nc, near


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def blend_bwd(splats: dict, ranges, lst, dL_drgb, V: int, width: int, height: int, tile: int, bg=(0.0, 0.0, 0.0),
              camera=None):
    """Exact adjoint of blend_fwd: per-(view, Gaussian) [V*N, 9] = dL/d(px, py, c0, c1, c2, opacity, r, g, b)."""
    lib = _load()
    _camera(camera)
    sp = _splat9(splats)
    n = sp.shape[0] // V
    bgv = _f64(bg)
    g = _f64(dL_drgb)
    out = np.zeros((V * n, G_LEN))
    lib.orc_blend_bwd(V, n, width, height, tile, _p(bgv), _p(sp), _p(_i64(ranges)), _p(_i64(lst)), _p(g), _p(out))
    return out


def preprocess_bwd(scene, viewmats, grad2d, width: int, height: int, near: float = 0.2, camera=None) -> dict:
    """Chain rule from screen-space gradients back to means, scales, quats, opacity and SH (Eqs. 18-20)."""
    lib = _load()
    _camera(camera)
    means, scales, quats, opacity, sh = (_f32(a) for a in scene.arrays())
    vm = _f32(viewmats).reshape(-1, 16)
    V, n = vm.shape[0], means.shape[0]
    K = sh.shape[1]
    out = dict(means=np.zeros((n, 3)), scales=np.zeros((n, 3)), quats=np.zeros((n, 4)), opacity=np.zeros(n),
               sh=np.zeros((n, K, 3)), screen=np.zeros((n, 2)))
    g2 = _f64(grad2d)
    lib.orc_preprocess_bwd(n, V, width, height, scene.sh_degree, near, _p(means), _p(scales), _p(quats), _p(opacity),
                           _p(sh), _p(vm), _p(g2), _p(out["means"]), _p(out["scales"]), _p(out["quats"]),
                           _p(out["opacity"]), _p(out["sh"]), _p(out["screen"]))
    return out


# ------------------------------------------------------------------ the whole path

def render(scene, viewmats, width: int, height: int, tile: int = 16, bg=(0.0, 0.0, 0.0), near: float = 0.2,
           eps: float = 1e-5, camera=None) -> dict:
    """Forward render of every view: projection, binning, sort by t_r, blending."""
    V = np.asarray(viewmats).reshape(-1, 16).shape[0]
    rec = preprocess(scene, viewmats, width, height, near, camera)
    sp = splats_from_records(rec)
    ranges, lst = bin_sort(sp, V, width, height, tile, camera=camera)
    rgb, T, nc, nearf = blend_fwd(sp, ranges, lst, V, width, height, tile, bg, eps, camera)
    return dict(rec=rec, splats=sp, ranges=ranges, list=lst, rgb=rgb, T=T, n_contrib=nc, near=nearf)


def render_grad(scene, viewmats, dL_drgb, width: int, height: int, tile: int = 16, bg=(0.0, 0.0, 0.0),
                near: float = 0.2, fwd: dict | None = None, camera=None) -> dict:
    """Gradients of sum(dL_drgb * render(...)) with respect to every Gaussian parameter."""
    V = np.asarray(viewmats).reshape(-1, 16).shape[0]
    if fwd is None:
        fwd = render(scene, viewmats, width, height, tile, bg, near, camera=camera)
    g2 = blend_bwd(fwd["splats"], fwd["ranges"], fwd["list"], dL_drgb, V, width, height, tile, bg, camera)
    out = preprocess_bwd(scene, viewmats, g2, width, height, near, camera)
    out["grad2d"] = g2
    return out
