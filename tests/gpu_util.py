"""Helpers shared by the GPU tests: moving seeded inputs to the device and comparing against the oracle."""
import numpy as np
import torch

SPLAT_KEYS = ("px", "py", "c0", "c1", "c2", "depth")  # columns 0-5; 6: rx | ry << 16; 7: q; 8-11: COLOUR_KEYS
COLOUR_KEYS = ("opacity", "r", "g", "b")


def pack_splats(sp: dict) -> np.ndarray:
    """Generator splat fields -> the [m, 12] float32 layout of omnigs_splat (px, py, c0, c1, c2, depth, rx | ry << 16
    stored as uint32 bits, q = 2 ln(255 o) (the dict's own when it has one), opacity, r, g, b)."""
    import oracle
    m = len(sp["px"])
    out = np.zeros((m, 12), np.float32)
    for i, k in enumerate(SPLAT_KEYS):
        out[:, i] = np.asarray(sp[k], np.float32)
    for i, k in enumerate(COLOUR_KEYS):
        out[:, 8 + i] = np.asarray(sp[k], np.float32)
    rx, ry = np.asarray(sp["rx"], np.int64), np.asarray(sp["ry"], np.int64)
    assert rx.min(initial=0) >= 0 and rx.max(initial=0) <= 65535 and ry.min(initial=0) >= 0 and ry.max(initial=0) <= 65535
    out[:, 6] = (rx | (ry << 16)).astype(np.uint32).view(np.float32)
    out[:, 7] = oracle.splat_q(sp).astype(np.float32)
    return out


def unpack_splats(arr: np.ndarray) -> dict:
    d = {k: arr[:, i].copy() for i, k in enumerate(SPLAT_KEYS)}
    d.update({k: arr[:, 8 + i].copy() for i, k in enumerate(COLOUR_KEYS)})
    radii = arr[:, 6].copy().view(np.uint32)
    d["rx"] = (radii & 0xFFFF).astype(np.int32)
    d["ry"] = (radii >> 16).astype(np.int32)
    d["q"] = arr[:, 7].copy()
    return d


def to64(sp: dict) -> dict:
    """Splat fields in double precision (integer fields unchanged)."""
    return {k: (np.asarray(v, np.float64) if np.asarray(v).dtype.kind == "f" else v) for k, v in sp.items()}


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


def _box_margin(px, py, rx, ry, W, H):
    """How far (px) the box [floor(p) -+ r] is from the pinhole's frustum-cull decision (hitting or missing the
    image): small values are decisions that FP32 and FP64 may take differently."""
    ix, iy = np.floor(px), np.floor(py)
    gaps = [np.abs(ix + rx + 0.5), np.abs(ix - rx - W + 0.5), np.abs(iy + ry + 0.5), np.abs(iy - ry - H + 0.5)]
    return np.minimum.reduce(gaps)


def check_preprocess_pinhole(got: dict, rec: np.ndarray, opacity_expected: np.ndarray, W: int, H: int, intr):
    """check_preprocess for a pinhole camera (Eq. 2): FP32 carries p - c to ~1e-7 of its size, so the position
    tolerance (2e-6 of W, H) applies to centres within one image width / height of the principal point c, and the
    rest are compared relative to |p - c|. Returns (summary, number of far centres checked)."""
    import oracle
    cx, cy = intr[2], intr[3]
    dx, dy = rec[:, oracle.R_PX] - cx, rec[:, oracle.R_PY] - cy
    on = (np.abs(dx) < W) & (np.abs(dy) < H)
    far = ~on & (rec[:, oracle.R_RX] > 0) & (got["rx"] > 0)
    gp = np.stack([got["px"] - cx, got["py"] - cy], 1)[far]
    rp = np.stack([dx, dy], 1)[far]
    if far.any():
        assert (np.abs(gp - rp).max(1) / np.abs(rp).max(1)).max() <= 2e-6
    summary = check_preprocess({k: v[on] for k, v in got.items()}, rec[on], opacity_expected[on], W, H, pinhole=True)
    return summary, int(far.sum())


def check_preprocess(got: dict, rec: np.ndarray, opacity_expected: np.ndarray, W: int, H: int, near: float = 0.2,
                     pinhole: bool = False):
    """FP32 preprocess output against the oracle's FP64 records of the same (view, Gaussian) rows.

    Culling agrees except within 1e-6 (relative) of the near distance; p within 2e-6 W (H) px, the angle carrying a
    few ulp (longitude differences taken across the seam); conic within 1e-4 of its norm; rgb within 1e-5; opacity
    copied exactly; q = 2 ln(255 o) within 1e-5; the instance box (rx, ry) exact unless one of its ceil() arguments
    lies within 1e-4 of an integer. Returns a summary."""
    import oracle
    ref = oracle.splats_from_records(rec)
    near_edge = np.abs(ref["depth"] - near) < 1e-6 * near
    alive = ref["rx"] > 0
    if pinhole:
        # frustum-cull decisions within a pixel of the image border (through floor(p) or r) may differ
        mism = (got["rx"] > 0) != alive
        g_m = _box_margin(got["px"], got["py"], got["rx"], got["ry"], W, H)
        r_m = _box_margin(ref["px"], ref["py"], ref["rx"], ref["ry"], W, H)
        border = mism & (np.where(got["rx"] > 0, g_m, r_m) <= 1.5)
        near_edge = near_edge | border
    assert np.array_equal((got["rx"] > 0)[~near_edge], alive[~near_edge])
    a = alive & (got["rx"] > 0)
    np.testing.assert_allclose(got["depth"], ref["depth"], rtol=2e-6, atol=1e-6)
    dpx = (got["px"][a] - ref["px"][a] + W / 2) % W - W / 2
    dpy = got["py"][a] - ref["py"][a]
    assert np.abs(dpx).max(initial=0) <= 2e-6 * W and np.abs(dpy).max(initial=0) <= 2e-6 * H
    cg = np.stack([got["c0"], got["c1"], got["c2"]], 1)[a]
    cr = np.stack([ref["c0"], ref["c1"], ref["c2"]], 1)[a]
    cerr = (np.abs(cg - cr).max(1) / np.abs(cr).max(1)).max(initial=0)
    assert cerr <= 1e-4
    rgb_err = max(np.abs(got[k][a] - ref[k][a]).max(initial=0) for k in ("r", "g", "b"))
    assert rgb_err <= 1e-5
    assert np.array_equal(got["opacity"][a], opacity_expected[a])
    np.testing.assert_allclose(got["q"][a], ref["q"][a], rtol=1e-5, atol=1e-5)
    margin_ok = rec[:, oracle.R_RMARGIN][a] > 1e-4 * np.maximum(1.0, ref["radius"][a])
    assert np.array_equal(got["rx"][a][margin_ok], ref["rx"][a][margin_ok])
    assert np.array_equal(got["ry"][a][margin_ok], ref["ry"][a][margin_ok])
    return dict(alive=int(a.sum()), dpx=float(np.abs(dpx).max(initial=0)), dpy=float(np.abs(dpy).max(initial=0)),
                conic=float(cerr), rgb=float(rgb_err))


def gpu_lists(r, count):
    """The GPU's tile ranges [V * tiles, 2] and sorted splat list (v * n + g) of a rasterizer after bin + sort."""
    ranges = r.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
    return ranges, r.sorted_splats(count)


def check_gpu_lists(r, count, sp, V, W, H, T, camera=None, tiles=None, ref=None):
    """GPU tile lists against the oracle's instance-box lists of the same float32 splats, by the validity rules of
    tests/tile_check.py (q as the float32 value both sides read). Returns the check's counts."""
    import oracle
    from tests import tile_check
    sp64 = to64(sp)
    ranges_ref, list_ref = ref if ref is not None else oracle.bin_sort(sp64, V, W, H, T, tile_mask=None, camera=camera)
    ranges, lst = gpu_lists(r, count)
    q = pack_splats(sp)[:, 7].astype(np.float64)
    st = tile_check.check_tile_lists(sp64, V, W, H, T, ranges, lst, ranges_ref, list_ref, tiles=tiles, camera=camera,
                                     q=q)
    if tiles is None:
        assert count == st["kept"], (count, st)
    return st


def last_contributor(ranges, lst, n_contrib, V, W, H, T):
    """Splat (v * n + g) of every pixel's last contributor, -1 where none: n_contrib is the position after it in the
    pixel's tile list, so this compares contributors between lists that differ in entries no pixel uses."""
    TX, TY = W // T, H // T
    ys, xs = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    tile = (np.arange(V)[:, None, None] * (TX * TY) + (ys // T) * TX + xs // T)
    nc = np.asarray(n_contrib, np.int64).reshape(V, H, W)
    pos = np.asarray(ranges, np.int64)[tile, 0] + nc - 1
    lst = np.asarray(lst, np.int64)
    return np.where(nc > 0, lst[np.clip(pos, 0, max(len(lst) - 1, 0))] if len(lst) else -1, -1)
