"""The pinhole camera of Eq. 2 through the same C ABI, against the FP64 oracle (gpu).

Same tolerances as the equirectangular parity tests: tile lists on identical splats valid against the oracle's
instance-box lists (tests/tile_check.py, columns clipped, no seam), images within 1e-5 outside near-threshold
pixels, gradients within 1e-4 (normwise and elementwise).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import (assert_grad_close, check_gpu_lists, check_preprocess_pinhole, dev, gpu_lists, last_contributor,
                            normwise, pack_splats, scene_to_device, to64, unpack_splats)

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2404_03202_gb300 as og  # noqa: E402
from paper_2404_03202_gb300 import _cabi as C  # noqa: E402

W, H = 256, 160
INTR = (180.0, 170.0, 128.0, 80.0)
CAM = oracle.pinhole(*INTR)


def _settings(V=1, tile=16, bg=(0.0, 0.0, 0.0), ppt=0):
    return og.Settings(width=W, height=H, tile=tile, num_views=V, sh_degree=3, bg=bg, pixels_per_thread=ppt,
                       adjoint_pixels_per_thread=ppt,
                       pinhole=INTR)


def _front_scene(n, seed):
    """Gaussians in front of the camera (+z), some beyond the field of view and beyond the Jacobian clamp."""
    sc = synth.shell_scene(n, seed, r_min=0.5, r_max=6.0, log_scale_mean=-3.0)
    m = sc.means.astype(np.float64)
    m[:, 2] = np.abs(m[:, 2]) + 0.3
    sc.means[:] = m.astype(np.float32)
    return sc


def test_preprocess_matches_oracle():
    sc = _front_scene(8000, 1)
    sc.scales[1::2] *= 8.0  # broad Gaussians: some centred far off the image still reach it
    vm = np.concatenate([synth.identity_viewmats(1), synth.random_viewmats(1, 2, max_offset=0.1)])
    r = og.Rasterizer(_settings(V=2))
    r._ensure(sc.n, 16)
    C.omnigs_preprocess(r.cfg, sc.n, *scene_to_device(sc), dev(vm), r.splats)
    got = unpack_splats(r.splats.cpu().numpy())
    rec = oracle.preprocess(sc, vm, W, H, camera=CAM)
    summary, far = check_preprocess_pinhole(got, rec, np.tile(sc.opacity, 2), W, H, INTR)
    print("pinhole preprocess:", summary, "far centres", far)
    assert far > 100
    assert summary["alive"] > 2000


def _offscreen_splats(V, n, seed):
    sp = synth.random_splats(V, n, W, H, seed=seed, max_radius=30, seam_frac=0.0)
    rng = np.random.default_rng(seed + 1)
    off = rng.uniform(size=V * n) < 0.15  # centres off the image, boxes reaching back in
    sp["px"][off] = np.where(rng.uniform(size=off.sum()) < 0.5, -rng.uniform(1, 25, off.sum()),
                             W + rng.uniform(1, 25, off.sum())).astype(np.float32)
    return sp


@pytest.mark.parametrize("tile", [16, 8])
def test_bin_sort_valid(tile):
    V, n = 2, 4000
    sp = _offscreen_splats(V, n, 3 + tile)
    s = _settings(V=V, tile=tile)
    r = og.Rasterizer(s, capacity=1 << 18)
    r._ensure(n, 16)
    r.splats.copy_(dev(pack_splats(sp)))
    C.omnigs_bin(r.cfg, n, r.splats, r.order, r.keys, r.capacity, r.ws)
    C.omnigs_sort(r.cfg, n, r.capacity, r.keys, r.ranges, r.ws)
    cnt = r.instance_count()
    st = check_gpu_lists(r, cnt, sp, V, W, H, tile, camera=CAM)
    print(f"pinhole bin tile {tile}: {st}")
    assert st["dropped"] > 0


def _fwd(sp, V, tile=16, bg=(0.0, 0.0, 0.0), ppt=0):
    s = _settings(V=V, tile=tile, bg=bg, ppt=ppt)
    r = og.Rasterizer(s, capacity=1 << 18)
    n = len(sp["px"]) // V
    r._ensure(n, 16)
    r.splats.copy_(dev(pack_splats(sp)))
    C.omnigs_bin(r.cfg, n, r.splats, r.order, r.keys, r.capacity, r.ws)
    C.omnigs_sort(r.cfg, n, r.capacity, r.keys, r.ranges, r.ws)
    C.omnigs_render_fwd(r.cfg, n, r.splats, r.ranges, r.keys, r.order, r.rgb, r.T, r.ncontrib)
    torch.cuda.synchronize()
    sp64 = to64(sp)
    ranges, lst = oracle.bin_sort(sp64, V, W, H, tile, camera=CAM)
    rgb, T, nc, near = oracle.blend_fwd(sp64, ranges, lst, V, W, H, tile, bg=bg, eps=1e-5, camera=CAM)
    # n_contrib is a position in the pixel's tile list: compare the splat it points at
    r.last_splat = last_contributor(*gpu_lists(r, r.instance_count()), r.ncontrib.cpu().numpy(), V, W, H, tile)
    return r, (rgb, T, last_contributor(ranges, lst, nc, V, W, H, tile), near), (ranges, lst, sp64)


@pytest.mark.parametrize("ppt", [4, 2, 8])
def test_render_fwd_and_bwd_match_oracle(ppt):
    V = 2
    sp = _offscreen_splats(V, 2500, 11)
    bg = (0.2, 0.3, 0.4)
    r, (rgb, T, last, near), (ranges, lst, sp64) = _fwd(sp, V, bg=bg, ppt=ppt)
    mask = (near & 1) == 0
    err = np.abs(r.rgb.cpu().numpy() - rgb).max(axis=1)[mask]
    print(f"pinhole render_fwd: max|dC| {err.max():.2e}, masked {1 - mask.mean():.1e}")
    assert 1 - mask.mean() <= 1e-3 and err.max() <= 1e-5
    assert np.array_equal(r.last_splat[mask], last[mask])
    g = synth.random_image_grad(V, W, H, 12)
    g[np.repeat((near != 0)[:, None], 3, axis=1)] = 0.0
    got = r.backward_2d(dev(g)).cpu().numpy()
    ref = oracle.blend_bwd(sp64, ranges, lst, g.astype(np.float64), V, W, H, 16, bg, camera=CAM)
    for j, name in enumerate(["px", "py", "c0", "c1", "c2", "opacity", "r", "g", "b"]):
        assert_grad_close(got[:, j], ref[:, j], name)


def test_preprocess_bwd_matches_oracle():
    sc = _front_scene(3000, 21)
    vm = np.concatenate([synth.identity_viewmats(1), synth.random_viewmats(1, 22, max_offset=0.1)])
    rng = np.random.default_rng(23)
    g2 = np.zeros((2 * sc.n, 12), np.float32)
    g2[:, :9] = rng.normal(size=(2 * sc.n, 9))
    g2[:, 2:5] *= 10.0
    r = og.Rasterizer(_settings(V=2))
    r._ensure(sc.n, 16)
    params = scene_to_device(sc)
    r.grads2d.copy_(dev(g2))
    C.omnigs_preprocess_bwd(r.cfg, sc.n, *params, dev(vm), r.grads2d, r.d_means, r.d_scales, r.d_quats, r.d_opacity,
                            r.d_sh, r.d_screen)
    ref = oracle.preprocess_bwd(sc, vm, g2[:, :9].astype(np.float64), W, H, camera=CAM)
    for name, got in [("means", r.d_means), ("scales", r.d_scales), ("quats", r.d_quats), ("opacity", r.d_opacity),
                      ("sh", r.d_sh), ("screen", r.d_screen)]:
        nw, el = assert_grad_close(got.cpu().numpy(), ref[name], name)
        print(f"pinhole preprocess_bwd {name}: normwise {nw:.1e} elementwise {el:.1e}")


def test_end_to_end_against_oracle():
    sc = _front_scene(6000, 31)
    vm = synth.identity_viewmats(1)
    r = og.Rasterizer(_settings())
    img = r.forward(*scene_to_device(sc), dev(vm)).cpu().numpy()
    f = oracle.render(sc, vm, W, H, 16, eps=1e-3, camera=CAM)
    mask = (f["near"] & 1) == 0
    err = np.abs(img - f["rgb"]).max(axis=1)[mask]
    print(f"pinhole e2e: max|dC| {err.max():.2e}, p99.9 {np.quantile(err, 0.999):.2e}")
    assert np.quantile(err, 0.999) <= 1e-4 and err.max() <= 2e-6 * W * 4
    g = synth.random_image_grad(1, W, H, 32)
    g[np.repeat((f["near"] != 0)[:, None], 3, axis=1)] = 0.0
    grads = r.backward(dev(g))
    ref = oracle.render_grad(sc, vm, g.astype(np.float64), W, H, 16, fwd=f, camera=CAM)
    for name in ["means", "scales", "quats", "opacity", "sh"]:
        nw = normwise(grads[name].cpu().numpy(), ref[name])
        print(f"pinhole e2e grad {name}: normwise {nw:.2e}")
        assert nw <= 1e-4, name


def test_views_that_see_nothing_or_everything():
    """Three pinhole views of front-facing Gaussians: the first looks at them, the second away from them (every splat
    culled: no instance, background only), the third at them again. The depth sort ranks only what each view sees,
    so the views must not disturb one another: images against the oracle, and the lists of the oracle's own splats
    binned in one 3-view launch valid against its box lists."""
    sc = _front_scene(3000, 41)
    back = synth.identity_viewmats(1)
    back[0, :3, :3] = np.diag([-1.0, 1.0, -1.0])  # yaw by pi: everything behind the camera
    vm = np.concatenate([synth.identity_viewmats(1), back, synth.random_viewmats(1, 42, max_offset=0.05)])
    vm[2, :3, :3] = np.eye(3)
    bg = (0.1, 0.2, 0.3)
    r = og.Rasterizer(_settings(V=3, bg=bg))
    img = r.forward(*scene_to_device(sc), dev(vm)).cpu().numpy()
    f = oracle.render(sc, vm, W, H, 16, bg=bg, eps=1e-3, camera=CAM)
    assert (f["splats"]["rx"].reshape(3, -1)[1] == 0).all() and (f["splats"]["rx"].reshape(3, -1)[0] > 0).sum() > 500
    assert np.array_equal(img[1], np.broadcast_to(np.array(bg, np.float32)[:, None, None], img[1].shape))
    cnt = r.instance_count()
    ranges = r.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
    tiles = (W // 16) * (H // 16)
    assert (ranges[tiles:2 * tiles] == 0).all()
    assert cnt > 0
    # the oracle's splats (rounded to the float32 layout) binned by the GPU in one 3-view launch
    sp32 = unpack_splats(pack_splats(f["splats"]))
    rb = og.Rasterizer(_settings(V=3), capacity=1 << 20)
    rb._ensure(sc.n, 16)
    rb.splats.copy_(dev(pack_splats(sp32)))
    C.omnigs_bin(rb.cfg, sc.n, rb.splats, rb.order, rb.keys, rb.capacity, rb.ws)
    C.omnigs_sort(rb.cfg, sc.n, rb.capacity, rb.keys, rb.ranges, rb.ws)
    cb = rb.instance_count()
    st = check_gpu_lists(rb, cb, sp32, 3, W, H, 16, camera=CAM)
    assert (gpu_lists(rb, cb)[0][tiles:2 * tiles] == 0).all() and st["kept"] > 0
    mask = (f["near"] & 1) == 0
    err = np.abs(img - f["rgb"]).max(axis=1)[mask]
    assert np.quantile(err, 0.999) <= 1e-4 and err.max() <= 2e-6 * W * 4
