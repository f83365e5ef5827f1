"""Helpers shared by the GPU tests: moving seeded inputs to the device and comparing against the oracle."""
import numpy as np
import torch

SPLAT_KEYS = ("px", "py", "c0", "c1", "c2", "opacity", "r", "g", "b", "depth")


def pack_splats(sp: dict) -> np.ndarray:
    """Generator splat fields -> the [m, 12] float32 layout of omnigs_splat (radius stored as int32 bits)."""
    m = len(sp["px"])
    out = np.zeros((m, 12), np.float32)
    for i, k in enumerate(SPLAT_KEYS):
        out[:, i] = np.asarray(sp[k], np.float32)
    out[:, 10] = np.asarray(sp["radius"], np.int32).view(np.float32)
    return out


def unpack_splats(arr: np.ndarray) -> dict:
    d = {k: arr[:, i].copy() for i, k in enumerate(SPLAT_KEYS)}
    d["radius"] = arr[:, 10].copy().view(np.int32)
    return d


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def scene_to_device(scene):
    return [dev(a) for a in scene.arrays()]


def normwise(got, ref):
    ref = np.asarray(ref, np.float64)
    got = np.asarray(got, np.float64)
    den = np.linalg.norm(ref)
    return np.linalg.norm(got - ref) / (den if den > 0 else 1.0)


def assert_grad_close(got, ref, name, rel=1e-4):
    """Normwise relative error <= rel, and elementwise |g - g*| <= rel * max|g*| (atomics reorder sums)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    nw = normwise(got, ref)
    scale = np.abs(ref).max() if ref.size else 0.0
    el = np.abs(got - ref).max() / scale if scale > 0 else np.abs(got).max()
    assert nw <= rel and el <= rel, f"{name}: normwise {nw:.3e}, elementwise/max {el:.3e}"
    return nw, el
