"""CPU checks of the C ABI library: it loads, exports every function include/omnigs.h declares, answers the calls
that need no GPU, and the host-side sort plan covers every key bit (no CUDA call is made here)."""
import ctypes
import importlib.util
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "omnigs.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    path = __graft_entry__._load_build_module().build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(omnigs_\w+)\s*\(", text)))


def test_header_declares_the_stage_calls():
    names = declared_functions()
    for n in ["omnigs_preprocess", "omnigs_bin", "omnigs_sort", "omnigs_render_fwd", "omnigs_render_bwd",
              "omnigs_preprocess_bwd", "omnigs_l1_loss", "omnigs_workspace_size", "omnigs_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    lib.omnigs_version.restype = ctypes.c_int
    assert lib.omnigs_version() >= 100
    lib.omnigs_status_string.restype = ctypes.c_char_p
    lib.omnigs_status_string.argtypes = [ctypes.c_int]
    assert lib.omnigs_status_string(2) == b"instance capacity exceeded"
    assert lib.omnigs_status_string(99) == b"unknown status"
    # invalid arguments are rejected before any CUDA call
    lib.omnigs_preprocess.argtypes = [ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 8
    assert lib.omnigs_preprocess(None, 10, *([None] * 8)) == 1
    lib.omnigs_last_error.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.omnigs_last_error(None, None) == 1


def test_config_layout_and_schedule_validation(lib):
    """omnigs_config is 64 bytes (the header's field order); invalid blend and adjoint schedules, cameras and image
    sizes beyond 65536 pixels (instance-box half-extents are 16-bit) are rejected on the host."""
    spec = importlib.util.spec_from_file_location("omnigs_cabi_layout", os.path.join(ROOT, "paper_2404_03202_gb300",
                                                                                      "_cabi.py"))
    text = open(spec.origin).read()
    fields = re.findall(r'\("(\w+)", ctypes\.c_(\w+)(?: \* 3)?\)', text.split("class omnigs_config")[1].split("class ")[0])
    assert [f for f, _ in fields] == ["width", "height", "tile", "num_views", "sh_degree", "near_r", "bg",
                                      "pixels_per_thread", "camera", "fx", "fy", "cx", "cy",
                                      "adjoint_pixels_per_thread"]

    class Cfg(ctypes.Structure):
        _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("tile", ctypes.c_int32),
                    ("num_views", ctypes.c_int32), ("sh_degree", ctypes.c_int32), ("near_r", ctypes.c_float),
                    ("bg", ctypes.c_float * 3), ("pixels_per_thread", ctypes.c_int32), ("camera", ctypes.c_int32),
                    ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                    ("adjoint_pixels_per_thread", ctypes.c_int32)]

    assert ctypes.sizeof(Cfg) == 64
    lib.omnigs_workspace_size.argtypes = [ctypes.POINTER(Cfg), ctypes.c_int64, ctypes.c_int64]
    lib.omnigs_workspace_size.restype = ctypes.c_size_t
    for tile, ppt in [(8, 4), (8, 8), (16, 3), (16, 1), (32, 16)]:
        c = Cfg(256, 128, tile, 1, 3, 0.2, (ctypes.c_float * 3)(0, 0, 0), ppt)
        assert lib.omnigs_workspace_size(ctypes.byref(c), 10, 100) == 0, (tile, ppt)
        c = Cfg(256, 128, tile, 1, 3, 0.2, (ctypes.c_float * 3)(0, 0, 0), 0, 0, 0.0, 0.0, 0.0, 0.0, ppt)
        assert lib.omnigs_workspace_size(ctypes.byref(c), 10, 100) == 0, ("adjoint", tile, ppt)
    for tile, ppt in [(8, 2), (16, 8), (32, 4)]:
        c = Cfg(256, 128, tile, 1, 3, 0.2, (ctypes.c_float * 3)(0, 0, 0), 0, 0, 0.0, 0.0, 0.0, 0.0, ppt)
        assert lib.omnigs_workspace_size(ctypes.byref(c), 10, 100) > 0, ("adjoint", tile, ppt)
    for w, h in [(65536 + 16, 128), (256, 65536 + 16), (250, 128)]:
        c = Cfg(w, h, 16, 1, 3, 0.2, (ctypes.c_float * 3)(0, 0, 0), 0)
        assert lib.omnigs_workspace_size(ctypes.byref(c), 10, 100) == 0, (w, h)
    for cam, fx, fy in [(2, 100.0, 100.0), (1, 0.0, 100.0), (1, 100.0, -1.0), (1, float("nan"), 100.0)]:
        c = Cfg(256, 128, 16, 1, 3, 0.2, (ctypes.c_float * 3)(0, 0, 0), 0, cam, fx, fy, 128.0, 64.0)
        assert lib.omnigs_workspace_size(ctypes.byref(c), 10, 100) == 0, (cam, fx, fy)


def test_fused_calls_reject_invalid_arguments_on_the_host(lib):
    """omnigs_preprocess_bin and omnigs_render_fwd_l1 validate their arguments before any CUDA call: no config, and
    a valid config with a missing workspace or target."""
    P = ctypes.c_void_p
    lib.omnigs_preprocess_bin.argtypes = [P, ctypes.c_int64] + [P] * 9 + [ctypes.c_int64, P, P]
    lib.omnigs_render_fwd_l1.argtypes = [P, ctypes.c_int64] + [P] * 12
    assert lib.omnigs_preprocess_bin(None, 10, *([None] * 9), 100, None, None) == 1
    assert lib.omnigs_render_fwd_l1(None, 10, *([None] * 12)) == 1
    cfg = (ctypes.c_int32 * 16)()
    for i, v in enumerate([256, 128, 16, 1, 3]):
        cfg[i] = v
    ctypes.cast(ctypes.byref(cfg, 20), ctypes.POINTER(ctypes.c_float))[0] = 0.2  # near_r
    buf = (ctypes.c_float * 128)()
    p = ctypes.c_void_p((ctypes.addressof(buf) + 255) // 256 * 256)  # 256-byte aligned: only the tested argument fails
    # n = 10 with every array given but no workspace; a negative capacity
    assert lib.omnigs_preprocess_bin(ctypes.byref(cfg), 10, *([p] * 9), 100, None, None) == 1
    assert lib.omnigs_preprocess_bin(ctypes.byref(cfg), 10, *([p] * 9), -1, p, None) == 1
    # render_fwd_l1: no target, then no workspace
    args = [p] * 4 + [None] + [p] * 5
    assert lib.omnigs_render_fwd_l1(ctypes.byref(cfg), 10, *args, p, None) == 1
    args = [p] * 10
    assert lib.omnigs_render_fwd_l1(ctypes.byref(cfg), 10, *args, None, None) == 1
