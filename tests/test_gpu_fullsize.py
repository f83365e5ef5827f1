"""GPU path vs the FP64 oracle at the full benchmark sizes, on sampled outputs (gpu).

Workloads, each in the launch configuration the benchmark times (capacity sized from a probe, no host
synchronisation inside the frame):
  * egocentric: 1,000,000 Gaussians in a 10 x 3 x 8 m room, 8 poses near its centre, 2048 x 1024, 16 x 16 tiles,
    the library's blend schedule;
  * training: 300,000 Gaussians in a 0.5-20 m shell around one identity pose, 2048 x 1024, 16 x 16 tiles;
  * roaming: 3,000,000 Gaussians along a 60 m corridor of 5 rooms, 16 poses on its centre line, 4096 x 2048,
    32 x 32 tiles at 4 pixels per thread (the schedule the autotuner picks for it);
  * egocentric cube map: the room's 8 poses split into 6 90-degree pinhole faces each (Eq. 2), 48 views of
    512 x 512, 16 x 16 tiles.

Each stage is checked where the oracle computes the exact answer:
  * preprocess: 3,000 sampled Gaussians in every view (the tolerances of the small parity tests);
  * bin + sort + ranges: the oracle's own splats (rounded to float32) fed to both sides; the GPU's instance count at
    most the oracle's box count, and the lists of every sampled tile valid against the oracle's box lists
    (tests/tile_check.py). Sampled tiles: whole views, and in the other views random tiles, seam columns, pole rows
    and full-width bands of tile rows;
  * render_fwd: every pixel of the sampled tiles: |dC| <= 1e-5 and |dT| <= 1e-5 outside near-threshold pixels (at
    most 1e-3 of them), the same last contributor and contributor count;
  * render_bwd: the 2D gradients of every splat whose instance box lies inside the sampled tiles of its view (so the
    oracle sees every pixel it touches), normwise and elementwise <= 1e-4, with the number of splats that receive a
    gradient printed and bounded below;
  * preprocess_bwd: 3,000 sampled Gaussians from a full-size random upstream gradient, <= 1e-4;
  * L1 loss: the full 8-view image against float64 numpy.
The oracle runs view by view, so its memory stays at one view's records and lists.
"""
import functools
import time

import numpy as np
import pytest
import torch

import oracle
import synth
from tests import tile_check
from tests.gpu_util import (assert_grad_close, check_preprocess, check_preprocess_pinhole, dev, last_contributor,
                            pack_splats, scene_to_device, to64, unpack_splats)

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2404_03202_gb300 as og  # noqa: E402
from paper_2404_03202_gb300 import _cabi as C  # noqa: E402

CUBE = (256.0, 256.0, 256.0, 256.0)
# full: views whose every tile is checked; bands: (view, first tile row, end tile row) checked across the full width;
# min_visible: the least number of splats that must receive a gradient among those compared
WORKLOADS = {
    "egocentric": dict(W=2048, H=1024, tile=16, ppt=0, pinhole=None, full=(0, 1, 2), bands=(), min_visible=10_000),
    "training": dict(W=2048, H=1024, tile=16, ppt=0, pinhole=None, full=(0,), bands=(), min_visible=10_000),
    "roaming": dict(W=4096, H=2048, tile=32, ppt=4, pinhole=None, full=(), bands=((0, 16, 48), (15, 0, 8)),
                    min_visible=1_000),
    "cubemap": dict(W=512, H=512, tile=16, ppt=0, pinhole=CUBE, full=(0, 1, 2, 3, 4, 5), bands=(), min_visible=5_000),
}


@functools.lru_cache(maxsize=1)
def _workload(name):
    if name == "egocentric":
        return synth.room_scene(1_000_000, 0), synth.room_viewmats(8, 1000)
    if name == "training":
        return synth.shell_scene(300_000, 2, r_min=0.5, r_max=20.0), synth.identity_viewmats(1)
    if name == "roaming":
        return synth.corridor_scene(3_000_000, 0), synth.corridor_viewmats(16, 1000)
    return synth.room_scene(1_000_000, 0), synth.cube_face_viewmats(synth.room_viewmats(8, 1000))


def _camera(wl):
    return oracle.pinhole(*wl["pinhole"]) if wl["pinhole"] else None


def _rasterizer(wl, V, capacity):
    s = og.Settings(width=wl["W"], height=wl["H"], tile=wl["tile"], num_views=V, sh_degree=3,
                    pixels_per_thread=wl["ppt"], pinhole=wl["pinhole"])
    return og.Rasterizer(s, capacity=int(capacity * 1.05) + 4096, grow=False)


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_preprocess_sampled_full_size(name):
    wl = WORKLOADS[name]
    W, H = wl["W"], wl["H"]
    sc, vm = _workload(name)
    V, n = vm.shape[0], sc.n
    r = _rasterizer(wl, V, 1)
    r._ensure(n, sc.sh.shape[1])
    C.omnigs_preprocess(r.cfg, n, *scene_to_device(sc), dev(vm), r.splats)
    idx = np.sort(np.random.default_rng(1).choice(n, 3000, replace=False))
    rows = (np.arange(V)[:, None] * n + idx[None, :]).reshape(-1)
    got = unpack_splats(r.splats[torch.from_numpy(rows).cuda()].cpu().numpy())
    rec = oracle.preprocess(sc.subset(idx), vm, W, H, camera=_camera(wl))
    opac = np.tile(sc.opacity[idx], V).astype(np.float32)
    if wl["pinhole"]:
        summary, far = check_preprocess_pinhole(got, rec, opac, W, H, wl["pinhole"])
        summary["far"] = far
    else:
        summary = check_preprocess(got, rec, opac, W, H)
    print(f"{name} preprocess sample: {summary}")
    assert summary["alive"] > (0.05 if wl["pinhole"] else 0.5) * len(rows)


def _oracle_splats(sc, vm, wl):
    """The oracle's splats of every view in the float32 layout both sides read, computed one view at a time."""
    n, V = sc.n, vm.shape[0]
    packed = np.empty((V * n, 12), np.float32)
    for v in range(V):
        rec = oracle.preprocess(sc, vm[v:v + 1], wl["W"], wl["H"], camera=_camera(wl))
        packed[v * n:(v + 1) * n] = pack_splats(oracle.splats_from_records(rec))
    return packed


def _view_slice(packed, v, n):
    sp = to64(unpack_splats(packed[v * n:(v + 1) * n]))
    return sp, packed[v * n:(v + 1) * n, 7].astype(np.float64)


def _sampled_tiles(wl, v, rng):
    """[TY, TX] mask of the tiles of view v whose lists and pixels are checked."""
    W, H, T = wl["W"], wl["H"], wl["tile"]
    TX, TY = W // T, H // T
    if v in wl["full"]:
        return np.ones((TY, TX), bool)
    m = np.zeros((TY, TX), bool)
    m.reshape(-1)[rng.choice(TX * TY, min(40, TX * TY), replace=False)] = True
    if not wl["pinhole"]:
        m[rng.choice(TY, 6, replace=False), 0] = True          # seam: first and last tile columns
        m[rng.choice(TY, 6, replace=False), TX - 1] = True
        m[0, rng.choice(TX, 4, replace=False)] = True           # pole rows
        m[TY - 1, rng.choice(TX, 4, replace=False)] = True
    for bv, y0, y1 in wl["bands"]:
        if bv == v:
            m[y0:y1, :] = True
    return m


def _inside(sp, mask, T):
    """Splats whose every instance tile lies in the mask (the oracle then sees every pixel they reach). The mask is a
    whole view, or full-width bands of tile rows plus scattered tiles: a splat is inside when the rows of its box
    are full rows of the mask."""
    TY = mask.shape[0]
    alive = np.asarray(sp["rx"]) > 0
    if mask.all():
        return np.nonzero(alive)[0]
    full_row = mask.all(axis=1)
    before = np.concatenate([[0], np.cumsum(~full_row)])  # rows that are not full, before each row
    iy = np.floor(np.asarray(sp["py"], np.float64)).astype(np.int64)
    ry = np.asarray(sp["ry"], np.int64)
    y0 = np.clip(np.floor_divide(iy - ry, T), 0, TY - 1)
    y1 = np.clip(np.floor_divide(iy + ry, T), 0, TY - 1)
    return np.nonzero(alive & (before[y1 + 1] - before[y0] == 0))[0]


def _gpu_view_lists(r, v, n, tiles_v, tiles_per_view):
    """GPU ranges ([tiles_per_view, 2], zero outside tiles_v) and splat list (g within the view) of view v's tiles."""
    ranges = r.ranges.view(-1, 2)[v * tiles_per_view:(v + 1) * tiles_per_view].cpu().numpy().view(np.uint32)
    ranges = ranges.astype(np.int64)
    a, b = ranges[tiles_v, 0], ranges[tiles_v, 1]
    lens = b - a
    pos = np.repeat(a, lens) + np.arange(int(lens.sum())) - np.repeat(np.cumsum(lens) - lens, lens)
    keys = r.keys[torch.from_numpy(pos).cuda()].cpu().numpy().view(np.uint64)
    rb = C.rank_bits(n)
    assert np.array_equal((keys >> np.uint64(rb)).astype(np.int64), np.repeat(v * tiles_per_view + tiles_v, lens))
    rank = (keys & np.uint64((1 << rb) - 1)).astype(np.int64)
    order = r.order[v * n:(v + 1) * n].cpu().numpy().view(np.uint32).astype(np.int64)
    lst = order[rank] - v * n
    out = np.zeros_like(ranges)
    off = np.cumsum(lens) - lens
    out[tiles_v, 0], out[tiles_v, 1] = off, off + lens
    return out, lst


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_tiles_sampled_full_size(name):
    wl = WORKLOADS[name]
    W, H, T = wl["W"], wl["H"], wl["tile"]
    TX, TY = W // T, H // T
    TILES = TX * TY
    cam = _camera(wl)
    sc, vm = _workload(name)
    V, n = vm.shape[0], sc.n
    t0 = time.time()
    packed = _oracle_splats(sc, vm, wl)
    box_total = sum(oracle.count_instances(_view_slice(packed, v, n)[0], 1, W, H, T, camera=cam) for v in range(V))

    r = _rasterizer(wl, V, box_total)
    r._ensure(n, sc.sh.shape[1])
    r.splats.copy_(dev(packed))
    C.omnigs_bin(r.cfg, n, r.splats, r.order, r.keys, r.capacity, r.ws)
    C.omnigs_sort(r.cfg, n, r.capacity, r.keys, r.ranges, r.ws)
    r.count_out = torch.empty_like(r.ncontrib)
    C.omnigs_render_fwd(r.cfg, n, r.splats, r.ranges, r.keys, r.order, r.rgb, r.T, r.ncontrib, r.count_out)
    torch.cuda.synchronize()
    r.check()
    count = r.instance_count()
    assert 0 < count <= box_total
    print(f"{name}: {count} instances, {box_total} box instances (oracle)")

    rng = np.random.default_rng(7)
    adj = {}  # view -> (splat fields, oracle ranges, oracle list, splats inside the sampled tiles)
    near_all = np.zeros((V, H, W), np.uint8)
    stats = dict(entries=0, dropped=0, pixels=0, masked=0, err=0.0)
    for v in range(V):
        sp, q = _view_slice(packed, v, n)
        mask = _sampled_tiles(wl, v, rng)
        tiles_v = np.nonzero(mask.reshape(-1))[0]
        ranges_o, list_o = oracle.bin_sort(sp, 1, W, H, T, tile_mask=mask.reshape(-1), camera=cam)
        ranges_g, list_g = _gpu_view_lists(r, v, n, tiles_v, TILES)
        st = tile_check.check_tile_lists(sp, 1, W, H, T, ranges_g, list_g, ranges_o, list_o, tiles=tiles_v,
                                         camera=cam, q=q)
        stats["entries"] += st["kept"]
        stats["dropped"] += st["dropped"]
        # forward on every pixel of the sampled tiles
        rgb_o, T_o, nc_o, near_o = oracle.blend_fwd(sp, ranges_o, list_o, 1, W, H, T, eps=1e-5, camera=cam)
        count_o = oracle.blend_fwd.last_count
        near_all[v] = near_o[0]
        pix = np.repeat(mask[:, None, :, None], T, 1).repeat(T, 3).reshape(H, W)
        ok = pix & ((near_o[0] & 1) == 0)
        err = np.abs(r.rgb[v].cpu().numpy() - rgb_o[0]).max(axis=0)[ok]
        stats["pixels"] += int(pix.sum())
        stats["masked"] += int(pix.sum() - ok.sum())
        stats["err"] = max(stats["err"], float(err.max()))
        assert err.max() <= 1e-5, (v, err.max())
        assert np.abs(r.T[v].cpu().numpy() - T_o[0])[ok].max() <= 1e-5
        nc_g = r.ncontrib[v].cpu().numpy()
        last_g = last_contributor(ranges_g, list_g, nc_g[None], 1, W, H, T)[0]
        last_o = last_contributor(ranges_o, list_o, nc_o, 1, W, H, T)[0]
        assert np.array_equal(last_g[ok], last_o[ok])
        assert np.array_equal(r.count_out[v].cpu().numpy()[ok], count_o[0][ok])
        if v in wl["full"] or any(b[0] == v for b in wl["bands"]):
            adj[v] = (sp, ranges_o, list_o, _inside(sp, mask, T))
    assert stats["masked"] <= 1e-3 * stats["pixels"]
    print(f"{name}: lists of {stats['entries']} entries valid ({stats['dropped']} box pairs left out); "
          f"render_fwd on {stats['pixels']} pixels, max|dC| {stats['err']:.3e}, masked {stats['masked']}; "
          f"oracle {time.time() - t0:.0f} s")

    # adjoint of the splats whose every tile is sampled; near-threshold pixels carry no upstream gradient
    g = np.random.default_rng(5).standard_normal((V, 3, H, W), dtype=np.float32)
    g *= (near_all == 0)[:, None]
    got_all = r.backward_2d(dev(g))
    compared = visible = 0
    fields = ["px", "py", "c0", "c1", "c2", "opacity", "r", "g", "b"]
    got, ref = [], []
    for v, (sp, ranges_o, list_o, chosen) in adj.items():
        ref_v = oracle.blend_bwd(sp, ranges_o, list_o, g[v:v + 1].astype(np.float64), 1, W, H, T, camera=cam)
        got.append(got_all[torch.from_numpy(v * n + chosen).cuda()].cpu().numpy()[:, :9])
        ref.append(ref_v[chosen])
        compared += len(chosen)
    got, ref = np.concatenate(got), np.concatenate(ref)
    visible = int((np.abs(ref).max(axis=1) > 0).sum())
    assert visible >= wl["min_visible"], visible
    for j, field in enumerate(fields):
        nw, el = assert_grad_close(got[:, j], ref[:, j], field)
        print(f"{name} render_bwd {field} ({compared} splats, {visible} with a gradient): normwise {nw:.2e} "
              f"elementwise {el:.2e}")


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_preprocess_bwd_sampled_full_size(name):
    wl = WORKLOADS[name]
    sc, vm = _workload(name)
    V, n = vm.shape[0], sc.n
    rng = np.random.default_rng(17)
    g2 = np.zeros((V * n, 12), np.float32)
    g2[:, :9] = rng.standard_normal((V * n, 9), dtype=np.float32)
    g2[:, 2:5] *= 10.0
    r = _rasterizer(wl, V, 1)
    r._ensure(n, sc.sh.shape[1])
    params = scene_to_device(sc)
    r.grads2d.copy_(dev(g2))
    C.omnigs_preprocess_bwd(r.cfg, n, *params, dev(vm), r.grads2d, r.d_means, r.d_scales, r.d_quats, r.d_opacity,
                            r.d_sh, r.d_screen)
    torch.cuda.synchronize()
    idx = np.sort(rng.choice(n, 3000, replace=False))
    rows = (np.arange(V)[:, None] * n + idx[None, :]).reshape(-1)
    ref = oracle.preprocess_bwd(sc.subset(idx), vm, g2[rows, :9].astype(np.float64), wl["W"], wl["H"],
                                camera=_camera(wl))
    for field, got in [("means", r.d_means), ("scales", r.d_scales), ("quats", r.d_quats),
                       ("opacity", r.d_opacity), ("sh", r.d_sh), ("screen", r.d_screen)]:
        nw, el = assert_grad_close(got.cpu().numpy()[idx], ref[field], field)
        print(f"{name} preprocess_bwd {field}: normwise {nw:.2e} elementwise {el:.2e}")


def test_l1_full_size_eight_views():
    wl = WORKLOADS["egocentric"]
    W, H, V = wl["W"], wl["H"], 8
    rgb = synth.random_image(V, W, H, 21)
    tgt = synth.random_image(V, W, H, 22)
    r = _rasterizer(wl, V, 1)
    r._ensure(1, 16)
    r.rgb.copy_(dev(rgb))
    loss = r.l1_loss(dev(tgt)).item()
    d = rgb.astype(np.float64) - tgt
    ref = np.abs(d).mean()
    assert abs(loss - ref) <= 1e-6 * ref
    assert np.array_equal(r.dL_drgb.cpu().numpy(), (np.sign(d) / d.size).astype(np.float32))
