"""GPU path vs the FP64 oracle at the full benchmark sizes, on sampled outputs (gpu).

Workloads, in the launch configuration the benchmark times (capacity sized from a probe, no host synchronisation
inside the frame, the library's default blend schedule):
  * egocentric: 1,000,000 Gaussians in a 10 x 3 x 8 m room, 8 poses near its centre, 2048 x 1024, 16 x 16 tiles;
  * training: 300,000 Gaussians uniform in a 0.5-20 shell around one identity pose, 2048 x 1024, 16 x 16 tiles.

Each stage is checked where the oracle can compute the exact answer one output at a time:
  * preprocess: a sample of Gaussians in every view (same tolerances as the small parity tests);
  * bin + sort + ranges: the oracle's own splats (rounded to float32) fed to both sides; the total instance count
    and the sorted list of every sampled tile (random tiles, seam columns, pole rows, and two full-width bands of
    tile rows) bit-exact;
  * render_fwd: every pixel of the sampled tiles, |dC| <= 1e-5 outside near-threshold pixels;
  * render_bwd: the 2D gradients of the splats whose tile rectangle lies inside a band (so the oracle sees every
    pixel they touch), normwise and elementwise <= 1e-4;
  * preprocess_bwd: a sample of Gaussians from a full-size random upstream gradient, <= 1e-4;
  * L1 loss: the full image against float64 numpy.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import (assert_grad_close, check_preprocess, dev, pack_splats, scene_to_device, to64,
                            unpack_splats)

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2404_03202_gb300 as og  # noqa: E402
from paper_2404_03202_gb300 import _cabi as C  # noqa: E402

W, H, TILE = 2048, 1024, 16
TX, TY = W // TILE, H // TILE
TILES = TX * TY


def _workload(name):
    if name == "egocentric":
        return synth.room_scene(1_000_000, 0), synth.room_viewmats(8, 1000)
    return synth.shell_scene(300_000, 2, r_min=0.5, r_max=20.0), synth.identity_viewmats(1)


def _rasterizer(V, capacity):
    s = og.Settings(width=W, height=H, tile=TILE, num_views=V, sh_degree=3)
    return og.Rasterizer(s, capacity=int(capacity * 1.05) + 4096, grow=False)


@pytest.mark.parametrize("name", ["egocentric", "training"])
def test_preprocess_sampled_full_size(name):
    sc, vm = _workload(name)
    V, n = vm.shape[0], sc.n
    r = _rasterizer(V, 1)
    r._ensure(n, sc.sh.shape[1])
    C.omnigs_preprocess(r.cfg, n, *scene_to_device(sc), dev(vm), r.splats)
    idx = np.sort(np.random.default_rng(1).choice(n, 3000, replace=False))
    rows = (np.arange(V)[:, None] * n + idx[None, :]).reshape(-1)
    got = unpack_splats(r.splats[torch.from_numpy(rows).cuda()].cpu().numpy())
    rec = oracle.preprocess(sc.subset(idx), vm, W, H)
    summary = check_preprocess(got, rec, np.tile(sc.opacity[idx], V).astype(np.float32), W, H)
    print(f"{name} preprocess sample: {summary}")
    assert summary["alive"] > 0.5 * len(rows)


def _tile_sample(sp, V, n, rng):
    """Sampled tiles per view, plus two full-width bands of tile rows (the horizon of the first view, the top pole of
    the last); the splats whose tile rectangle lies inside a band have every pixel they touch sampled."""
    mask = np.zeros((V, TY, TX), bool)
    for v in range(V):
        flat = mask[v].reshape(-1)
        flat[rng.choice(TILES, 40, replace=False)] = True
        mask[v, rng.choice(TY, 6, replace=False), 0] = True        # seam: first and last tile columns
        mask[v, rng.choice(TY, 6, replace=False), TX - 1] = True
        mask[v, 0, rng.choice(TX, 4, replace=False)] = True        # pole rows
        mask[v, TY - 1, rng.choice(TX, 4, replace=False)] = True
    bands = [(0, TY // 2 - 6, TY // 2 + 6), (V - 1, 0, 8)]
    chosen = []
    for v, y0, y1 in bands:
        mask[v, y0:y1, :] = True
        ry, py = sp["ry"][v * n:(v + 1) * n], sp["py"][v * n:(v + 1) * n]
        near_band = (sp["rx"][v * n:(v + 1) * n] > 0) & (py - ry >= y0 * TILE - 2 * TILE) & (py + ry < y1 * TILE + 2 * TILE)
        for g in np.nonzero(near_band)[0]:  # a loose pre-filter; the oracle's rectangle decides
            i = v * n + g
            _, _, ry0, rny = oracle.rect(float(sp["px"][i]), float(sp["py"][i]), int(sp["rx"][i]), int(sp["ry"][i]),
                                         W, H, TILE)
            if y0 <= ry0 and ry0 + rny <= y1:
                chosen.append(i)
    return mask.reshape(-1), np.array(sorted(set(chosen)), np.int64)


@pytest.mark.parametrize("name", ["egocentric", "training"])
def test_tiles_sampled_full_size(name):
    sc, vm = _workload(name)
    V, n = vm.shape[0], sc.n
    # the oracle's splats, rounded to the float32 layout both sides read
    packed = pack_splats(oracle.splats_from_records(oracle.preprocess(sc, vm, W, H)))
    sp32 = unpack_splats(packed)
    sp64 = to64(sp32)
    total = oracle.count_instances(sp64, V, W, H, TILE)

    r = _rasterizer(V, total)
    r._ensure(n, sc.sh.shape[1])
    r.splats.copy_(dev(packed))
    C.omnigs_bin(r.cfg, n, r.splats, r.order, r.keys, r.capacity, r.ws)
    C.omnigs_sort(r.cfg, n, r.capacity, r.keys, r.ranges, r.ws)
    r.count_out = torch.empty_like(r.ncontrib)
    C.omnigs_render_fwd(r.cfg, n, r.splats, r.ranges, r.keys, r.order, r.rgb, r.T, r.ncontrib, r.count_out)
    torch.cuda.synchronize()
    r.check()
    assert r.instance_count() == total

    rng = np.random.default_rng(7)
    tmask, chosen = _tile_sample(sp64, V, n, rng)
    ranges_o, list_o = oracle.bin_sort(sp64, V, W, H, TILE, tmask)
    # sorted lists of the sampled tiles, decoded from the GPU keys: splat = order[v n + rank]
    ranges_g = r.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
    tiles = np.nonzero(tmask)[0]
    lens_g = ranges_g[tiles, 1] - ranges_g[tiles, 0]
    lens_o = ranges_o[tiles, 1] - ranges_o[tiles, 0]
    assert np.array_equal(lens_g, lens_o)
    pos = np.concatenate([np.arange(a, b) for a, b in ranges_g[tiles]])
    keys = r.keys[torch.from_numpy(pos).cuda()].cpu().numpy().view(np.uint64)
    order = r.order.cpu().numpy().view(np.uint32).astype(np.int64)
    rb = C.rank_bits(n)
    view = np.repeat(tiles // TILES, lens_g)
    assert np.array_equal((keys >> np.uint64(rb)).astype(np.int64), np.repeat(tiles, lens_g))
    got_list = order[view * n + (keys & np.uint64((1 << rb) - 1)).astype(np.int64)]
    exp_list = np.concatenate([list_o[a:b] for a, b in ranges_o[tiles]])
    assert np.array_equal(got_list, exp_list)
    print(f"{name}: {total} instances; {len(tiles)} sampled tiles with {len(exp_list)} entries bit-exact")

    # forward on every pixel of the sampled tiles
    rgb_o, T_o, nc_o, near_o = oracle.blend_fwd(sp64, ranges_o, list_o, V, W, H, TILE, eps=1e-5)
    count_o = oracle.blend_fwd.last_count
    pix = np.repeat(tmask.reshape(V, TY, 1, TX, 1), TILE, 2).repeat(TILE, 4).reshape(V, H, W)
    ok = pix & ((near_o & 1) == 0)
    assert 1 - ok.sum() / pix.sum() <= 1e-3
    err = np.abs(r.rgb.cpu().numpy() - rgb_o).max(axis=1)[ok]
    print(f"{name} render_fwd: {pix.sum()} pixels, max|dC| {err.max():.3e}, masked {1 - ok.sum() / pix.sum():.2e}")
    assert err.max() <= 1e-5
    assert np.abs(r.T.cpu().numpy() - T_o)[ok].max() <= 1e-5
    assert np.array_equal(r.ncontrib.cpu().numpy()[ok], nc_o[ok])
    assert np.array_equal(r.count_out.cpu().numpy()[ok], count_o[ok])

    # adjoint of the splats whose every tile is sampled
    g = synth.random_image_grad(V, W, H, 5)
    g[np.repeat((near_o != 0)[:, None], 3, axis=1)] = 0.0
    got = r.backward_2d(dev(g))[torch.from_numpy(chosen).cuda()].cpu().numpy()
    ref = oracle.blend_bwd(sp64, ranges_o, list_o, g.astype(np.float64), V, W, H, TILE)[chosen]
    visible = int((np.abs(ref).max(axis=1) > 0).sum())
    assert visible >= 100, visible  # enough of the band's splats escape occlusion to carry a gradient
    for j, field in enumerate(["px", "py", "c0", "c1", "c2", "opacity", "r", "g", "b"]):
        nw, el = assert_grad_close(got[:, j], ref[:, j], field)
        print(f"{name} render_bwd {field} ({len(chosen)} splats, {visible} with a gradient): normwise {nw:.2e} "
              f"elementwise {el:.2e}")


@pytest.mark.parametrize("name", ["egocentric", "training"])
def test_preprocess_bwd_sampled_full_size(name):
    sc, vm = _workload(name)
    V, n = vm.shape[0], sc.n
    rng = np.random.default_rng(17)
    g2 = np.zeros((V * n, 12), np.float32)
    g2[:, :9] = rng.normal(size=(V * n, 9)).astype(np.float32)
    g2[:, 2:5] *= 10.0
    r = _rasterizer(V, 1)
    r._ensure(n, sc.sh.shape[1])
    params = scene_to_device(sc)
    r.grads2d.copy_(dev(g2))
    C.omnigs_preprocess_bwd(r.cfg, n, *params, dev(vm), r.grads2d, r.d_means, r.d_scales, r.d_quats, r.d_opacity,
                            r.d_sh, r.d_screen)
    torch.cuda.synchronize()
    idx = np.sort(rng.choice(n, 3000, replace=False))
    rows = (np.arange(V)[:, None] * n + idx[None, :]).reshape(-1)
    ref = oracle.preprocess_bwd(sc.subset(idx), vm, g2[rows, :9].astype(np.float64), W, H)
    for field, got in [("means", r.d_means), ("scales", r.d_scales), ("quats", r.d_quats),
                       ("opacity", r.d_opacity), ("sh", r.d_sh), ("screen", r.d_screen)]:
        nw, el = assert_grad_close(got.cpu().numpy()[idx], ref[field], field)
        print(f"{name} preprocess_bwd {field}: normwise {nw:.2e} elementwise {el:.2e}")


def test_l1_full_size_eight_views():
    V = 8
    rgb = synth.random_image(V, W, H, 21)
    tgt = synth.random_image(V, W, H, 22)
    r = _rasterizer(V, 1)
    r._ensure(1, 16)
    r.rgb.copy_(dev(rgb))
    loss = r.l1_loss(dev(tgt)).item()
    d = rgb.astype(np.float64) - tgt
    ref = np.abs(d).mean()
    assert abs(loss - ref) <= 1e-6 * ref
    assert np.array_equal(r.dL_drgb.cpu().numpy(), (np.sign(d) / d.size).astype(np.float32))
