"""GPU path vs the FP64 oracle, stage by stage and end to end, through the C ABI (marked gpu).

Tolerances (written in each test):
  * tile lists, given identical splats: valid against the oracle's instance-box lists (tests/tile_check.py: an
    order-preserving subsequence, every left-out pair out of reach by half the stated widening, every kept pair within
    it), and equal to them, ranges included, where the binning keeps whole rows; the depth order bit-exact;
  * blended images: |dC| <= 1e-5 per channel, given identical splats, outside pixels where a skip / stop decision
    lies within 1e-5 (relative) of its threshold (the oracle flags them; at most 1e-3 of the pixels);
  * blend and preprocess gradients: normwise relative error <= 1e-4 and elementwise <= 1e-4 * max|g*|;
  * preprocess outputs (FP32 vs FP64 from identical parameters): see test_preprocess_matches_oracle.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import (assert_grad_close, check_gpu_lists, check_preprocess, dev, gpu_lists, last_contributor,
                            pack_splats, scene_to_device, to64, unpack_splats)

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2404_03202_gb300 as og  # noqa: E402
from paper_2404_03202_gb300 import _cabi as C  # noqa: E402


def _settings(W, H, tile=16, V=1, deg=3, bg=(0.0, 0.0, 0.0), ppt=0):
    """ppt: the schedule of both the forward blend and its adjoint (0: the library's choices)."""
    return og.Settings(width=W, height=H, tile=tile, num_views=V, sh_degree=deg, bg=bg, pixels_per_thread=ppt,
                       adjoint_pixels_per_thread=ppt)


def _run_splats(sp_packed, s: og.Settings, capacity=1 << 16):
    """bin + sort + render_fwd on given splats (numpy [V*n, 12])."""
    r = og.Rasterizer(s, capacity=capacity)
    m = sp_packed.shape[0]
    n = m // s.num_views
    r._ensure(n, (s.sh_degree + 1) ** 2)
    r.splats.copy_(dev(sp_packed))
    C.omnigs_bin(r.cfg, n, r.splats, r.order, r.keys, r.capacity, r.ws)
    cnt = r.instance_count()
    if cnt > r.capacity:
        r._alloc_instances(cnt)
        r._ensure(n, (s.sh_degree + 1) ** 2)
        r.splats.copy_(dev(sp_packed))
        C.omnigs_bin(r.cfg, n, r.splats, r.order, r.keys, r.capacity, r.ws)
    C.omnigs_sort(r.cfg, n, r.capacity, r.keys, r.ranges, r.ws)
    r.count_out = torch.empty_like(r.ncontrib)
    C.omnigs_render_fwd(r.cfg, n, r.splats, r.ranges, r.keys, r.order, r.rgb, r.T, r.ncontrib, r.count_out)
    torch.cuda.synchronize()
    assert r.check() is None
    return r, cnt


# ------------------------------------------------------------------ S1 preprocess

@pytest.mark.parametrize("deg", [3, 1])
def test_preprocess_matches_oracle(deg):
    W, H = 512, 256
    sc = synth.shell_scene(10000, seed=1, sh_degree=deg)
    vm = np.concatenate([synth.identity_viewmats(1), synth.random_viewmats(2, 5)])
    s = _settings(W, H, V=3, deg=deg)
    r = og.Rasterizer(s)
    params = scene_to_device(sc)
    r._ensure(sc.n, sc.sh.shape[1])
    C.omnigs_preprocess(r.cfg, sc.n, *params, dev(vm), r.splats)
    got = unpack_splats(r.splats.cpu().numpy())
    rec = oracle.preprocess(sc, vm, W, H)
    summary = check_preprocess(got, rec, np.tile(sc.opacity, vm.shape[0]).astype(np.float32), W, H)
    print(f"preprocess: {summary}")
    assert summary["alive"] > 0.5 * len(rec)


# ------------------------------------------------------------------ S2-S4 bin, sort, ranges

@pytest.mark.parametrize("tile,V,n,W,H", [(16, 2, 3000, 256, 128), (8, 1, 1500, 256, 128), (32, 3, 1000, 256, 128),
                                         (16, 1, 60000, 512, 256), (8, 2, 20000, 128, 64),
                                         (16, 4096, 300, 64, 32), (16, 2, 3000, 4096, 64), (16, 2, 3000, 64, 2304),
                                         (8, 3, 200, 256, 128)])
def test_bin_sort_valid(tile, V, n, W, H):
    """Includes lists longer than one shared-memory chunk (sorted in chunks and merged) and many depth ties. With
    4096 views of 300 splats the (view, depth, splat index) key needs 12 + 32 + 21 bits, so the depth sort carries
    the index as a value instead of inside the key. 4096 x 64 px on 16 px tiles has the most tile columns (256) of
    the instance order bucketed by (view, tile row); 64 x 2304 px (144 tile rows) and 200 splats a view (a 256-splat
    block spans three views) take the radix sort over all tile-key bits instead."""
    sp = synth.random_splats(V, n, W, H, seed=100 + tile, max_radius=30)
    packed = pack_splats(sp)
    s = _settings(W, H, tile=tile, V=V)
    r, cnt = _run_splats(packed, s)
    st = check_gpu_lists(r, cnt, sp, V, W, H, tile)
    print(f"bin tile {tile}, {V} x {n}: {st}")
    assert st["dropped"] > 0 and st["kept_checked"] > 0
    # the depth order behind the ranks: per view, by (t_r, splat index)
    order = r.order.cpu().numpy().view(np.uint32).astype(np.int64).reshape(V, n)
    for v in range(V):
        d = sp["depth"][v * n:(v + 1) * n]
        assert np.array_equal(order[v] - v * n, np.lexsort((np.arange(n), d)))


def test_bin_sort_valid_when_rows_overflow_the_row_store():
    """The instance capacity set to the count itself, with splats of one or two tiles per box row: the box rows
    outnumber what the row store holds (capacity / 2 + 1 rows), so bin_count stores the first blocks' rows and the
    fallback emission derives and ranks the other blocks' rows again. The lists stay valid and complete."""
    W, H, V, n, T = 512, 256, 2, 4000, 16
    sp = synth.random_splats(V, n, W, H, seed=77, max_radius=6, wide_frac=0.0)
    ry = np.asarray(sp["ry"], np.int64)
    iy = np.floor(np.asarray(sp["py"], np.float64)).astype(np.int64)
    y0 = np.maximum(np.floor_divide(iy - ry, T), 0)
    y1 = np.minimum(np.floor_divide(iy + ry, T), H // T - 1)
    rows = int(np.where(np.asarray(sp["rx"]) > 0, np.maximum(y1 - y0 + 1, 0), 0).sum())
    r, cnt = _run_splats(pack_splats(sp), _settings(W, H, tile=T, V=V), capacity=1)
    assert r.capacity == cnt and rows > cnt // 2 + 1, (rows, cnt)
    st = check_gpu_lists(r, cnt, sp, V, W, H, T)
    print(f"row store overflow: {rows} box rows, {cnt} instances: {st}")


def _whole_row_splats(V, n, W, H, seed):
    """Boxes wider than the image and, for the rest, needle conics (det = 5e-4 c0 c2, either sign of c1): the
    binning keeps every tile of every box."""
    sp = synth.random_splats(V, n, W, H, seed=seed, max_radius=30, wide_frac=0.4)
    c0, c2 = sp["c0"].astype(np.float64), sp["c2"].astype(np.float64)
    sign = np.where(np.random.default_rng(seed).uniform(size=len(c0)) < 0.5, -1.0, 1.0)
    sp["c1"] = (sign * np.sqrt(c0 * c2 * (1.0 - 5e-4))).astype(np.float32)
    return sp


@pytest.mark.parametrize("tile", [16, 8])
def test_bin_sort_exact_where_rows_are_whole(tile):
    """Where no pair may be left out, the lists and ranges equal the oracle's box lists exactly."""
    W, H, V, n = 256, 128, 2, 2000
    sp = _whole_row_splats(V, n, W, H, 60 + tile)
    r, cnt = _run_splats(pack_splats(sp), _settings(W, H, tile=tile, V=V), capacity=1 << 20)
    ranges_ref, list_ref = oracle.bin_sort(sp, V, W, H, tile)
    ranges, lst = gpu_lists(r, cnt)
    assert cnt == len(list_ref)
    assert np.array_equal(ranges, ranges_ref)
    assert np.array_equal(lst, list_ref)


def test_row_culling_hand_computed():
    """One circle of radius sqrt(q / c0) = 12 px (q = 9, c0 = c2 = 1/16) at (108.4, 50) on 16 px tiles, given a box
    of half-extent 60 (tile rows 0-6, columns 3-10). Grown by the stated widening (q = 9.01: radius 12.007) and one
    pixel, the circle's widest chord in tile row 3 (pixel centres 48.5 .. 63.5) spans 95.39 .. 121.41, which reaches
    columns 5 (last centre 95.5) to 7; in tile row 2 (centres 32.5 .. 47.5) the widest chord, at y = 47.5, less one
    pixel starts at 108.4 - sqrt(144.16 - 2.5^2) - 1 = 95.66 > 95.5, so the row keeps columns 6-7; no other row of
    the box is within reach."""
    W, H, T = 256, 128, 16
    sp = dict(px=np.float32([108.4]), py=np.float32([50.0]), c0=np.float32([1 / 16]), c1=np.float32([0.0]),
              c2=np.float32([1 / 16]), opacity=np.float32([np.exp(4.5) / 255]), r=np.float32([1]), g=np.float32([1]),
              b=np.float32([1]), depth=np.float32([1]), rx=np.int32([60]), ry=np.int32([60]), q=np.float32([9.0]))
    r, cnt = _run_splats(pack_splats(sp), _settings(W, H, tile=T))
    ranges, lst = gpu_lists(r, cnt)
    TX = W // T
    kept = sorted(int(t) for t in np.nonzero(ranges[:, 1] > ranges[:, 0])[0])
    assert kept == [2 * TX + 6, 2 * TX + 7, 3 * TX + 5, 3 * TX + 6, 3 * TX + 7]
    assert cnt == 5 and (lst == 0).all()


def test_sort_many_ties_and_all_columns():
    """Every splat at one depth (order decided by index alone) and some wider than the image."""
    W, H, V, n = 128, 64, 2, 800
    sp = synth.random_splats(V, n, W, H, seed=9, max_radius=20, wide_frac=0.2)
    sp["depth"][:] = np.float32(3.0)
    r, cnt = _run_splats(pack_splats(sp), _settings(W, H, V=V))
    st = check_gpu_lists(r, cnt, sp, V, W, H, 16)
    assert st["whole_row_pairs"] > 0


# ------------------------------------------------------------------ S5 render forward

def _row_cull_splats(V, n, W, H, seed):
    """Large, strongly sheared ellipses (correlations up to and past the 1 - 1e-3 determinant guard), opacities down
    to just above 1/255 (q near 0), centres on pixel centres and tile corners; the nearest (first in depth order) are
    the largest, so that one CTA's splats span several thousand box rows (past the 2048 whose bucket offsets bin_count
    keeps in shared memory; the rest take its global-memory fix-up)."""
    rng = np.random.default_rng(seed)
    m = V * n
    sx, sy = rng.uniform(0.4, 50.0, m), rng.uniform(0.4, 50.0, m)
    rho = rng.choice([0.0, 0.5, -0.9, 0.99, 0.9994, -0.9996, 0.99999, rng.uniform(-1, 1)], m)
    s00, s11, s01 = sx * sx, sy * sy, rho * sx * sy
    det = s00 * s11 - s01 * s01
    o = rng.choice([1.0 / 255 + 1e-6, 0.01, 0.3, 0.99], m)
    q = np.maximum(2 * np.log(255 * o), 0.0)
    px = rng.uniform(0, W, m)
    py = rng.uniform(0, H, m)
    k = rng.uniform(size=m)
    px[k < 0.2] = np.floor(px[k < 0.2]) + 0.5
    px[(k >= 0.2) & (k < 0.3)] = 16.0 * rng.integers(0, W // 16, ((k >= 0.2) & (k < 0.3)).sum())
    py[k >= 0.8] = 16.0 * rng.integers(0, H // 16, (k >= 0.8).sum())
    rx = np.minimum(np.ceil(np.sqrt(q * s00) * (1 + 1e-4) + 1e-3), 3000).astype(np.int32)
    ry = np.minimum(np.ceil(np.sqrt(q * s11) * (1 + 1e-4) + 1e-3), 3000).astype(np.int32)
    return dict(px=px.astype(np.float32), py=py.astype(np.float32), c0=(s11 / det).astype(np.float32),
                c1=(-s01 / det).astype(np.float32), c2=(s00 / det).astype(np.float32), opacity=o.astype(np.float32),
                r=np.full(m, 0.5, np.float32), g=np.full(m, 0.5, np.float32), b=np.full(m, 0.5, np.float32),
                depth=(1.0 / (sx * sy)).astype(np.float32), rx=rx, ry=ry, q=q.astype(np.float32))


@pytest.mark.parametrize("tile", [16, 8])
def test_bin_sort_row_culling_edges(tile):
    """Tile lists under the per-row column culling, valid against the oracle's box lists, on splats that stress its
    decision procedure."""
    W, H, V, n = 512, 256, 2, 3000
    sp = _row_cull_splats(V, n, W, H, 40 + tile)
    r, cnt = _run_splats(pack_splats(sp), _settings(W, H, tile=tile, V=V), capacity=1 << 20)
    st = check_gpu_lists(r, cnt, sp, V, W, H, tile)
    print(f"row culling edges, tile {tile}: {st}")
    assert st["dropped"] > 0 and st["whole_row_pairs"] > 0


def _fwd_compare(sp, V, W, H, tile, bg=(0.0, 0.0, 0.0), ppt=0):
    r, cnt = _run_splats(pack_splats(sp), _settings(W, H, tile=tile, V=V, bg=bg, ppt=ppt))
    sp64 = to64(sp)
    ranges, lst = oracle.bin_sort(sp64, V, W, H, tile)
    rgb, T, nc, near = oracle.blend_fwd(sp64, ranges, lst, V, W, H, tile, bg=bg, eps=1e-5)
    # n_contrib is a position in the pixel's tile list: compare the splat it points at
    r.last_splat = last_contributor(*gpu_lists(r, cnt), r.ncontrib.cpu().numpy(), V, W, H, tile)
    last_ref = last_contributor(ranges, lst, nc, V, W, H, tile)
    return r, (rgb, T, last_ref, near), (ranges, lst, sp64)


@pytest.mark.parametrize("tile,V,ppt", [(16, 2, 4), (16, 2, 2), (16, 2, 8), (8, 1, 2), (32, 1, 4), (32, 1, 2),
                                        (32, 1, 8)])
def test_render_fwd_matches_oracle(tile, V, ppt):
    W, H = 256, 128
    sp = synth.random_splats(V, 2500, W, H, seed=200 + tile, max_radius=24)
    bg = (0.25, 0.5, 0.75)
    r, (rgb, T, last, near), _ = _fwd_compare(sp, V, W, H, tile, bg, ppt)
    mask = (near & 1) == 0
    frac = 1.0 - mask.mean()
    got = r.rgb.cpu().numpy()
    err = np.abs(got - rgb).max(axis=1)[mask]
    print(f"render_fwd tile {tile}: max|dC| {err.max():.3e}, masked {frac:.2e}, mean T {T.mean():.3f}")
    assert frac <= 1e-3
    assert err.max() <= 1e-5
    assert np.abs(r.T.cpu().numpy() - T)[mask].max() <= 1e-5
    assert np.array_equal(r.last_splat[mask], last[mask])
    assert np.array_equal(r.count_out.cpu().numpy()[mask], oracle.blend_fwd.last_count[mask])


def test_render_fwd_opaque_stacks_stop_rule():
    """Dense opaque splats: most pixels stop at T < 1e-4 (the 0.9999 rule)."""
    W, H, V = 128, 64, 1
    sp = synth.random_splats(V, 3000, W, H, seed=3, max_radius=16, opacity_range=(0.9, 1.0), cull_frac=0.0)
    r, (rgb, T, last, near), _ = _fwd_compare(sp, V, W, H, 16)
    mask = (near & 1) == 0
    assert (T[mask] < 1e-2).mean() > 0.5
    assert np.abs(r.rgb.cpu().numpy() - rgb).max(axis=1)[mask].max() <= 1e-5
    assert np.array_equal(r.last_splat[mask], last[mask])


# ------------------------------------------------------------------ S7 render backward

@pytest.mark.parametrize("tile,V,opac,ppt", [(16, 2, (0.05, 0.99), 4), (16, 2, (0.05, 0.99), 2), (8, 1, (0.5, 1.0), 2),
                                             (16, 2, (0.5, 1.0), 8), (32, 1, (0.05, 0.99), 4), (32, 1, (0.5, 1.0), 2),
                                             (32, 1, (0.05, 0.99), 8)])
def test_render_bwd_matches_oracle(tile, V, opac, ppt):
    W, H = 256, 128
    sp = synth.random_splats(V, 2000, W, H, seed=300 + tile, max_radius=24, opacity_range=opac)
    bg = (0.1, 0.2, 0.3)
    r, (rgb, T, _, near), (ranges, lst, sp64) = _fwd_compare(sp, V, W, H, tile, bg, ppt)
    g = synth.random_image_grad(V, W, H, 7)
    g[np.repeat((near != 0)[:, None], 3, axis=1)] = 0.0  # pixels near a decision threshold carry no gradient
    ref = oracle.blend_bwd(sp64, ranges, lst, g.astype(np.float64), V, W, H, tile, bg)
    got = r.backward_2d(dev(g)).cpu().numpy()
    for j, name in enumerate(["px", "py", "c0", "c1", "c2", "opacity", "r", "g", "b"]):
        nw, el = assert_grad_close(got[:, j], ref[:, j], name)
        print(f"render_bwd tile {tile} {name}: normwise {nw:.2e} elementwise {el:.2e}")
    assert np.all(got[:, 9:] == 0)


# ------------------------------------------------------------------ S8 preprocess backward

@pytest.mark.parametrize("deg", [3, 0])
def test_preprocess_bwd_matches_oracle(deg):
    W, H = 512, 256
    sc = synth.shell_scene(4000, seed=11, sh_degree=deg)
    vm = np.concatenate([synth.identity_viewmats(1), synth.random_viewmats(1, 12)])
    V = vm.shape[0]
    rng = np.random.default_rng(13)
    g2 = rng.normal(size=(V * sc.n, 9))
    g2[:, 2:5] *= 10.0  # conic gradients are larger in practice (dL/dconic ~ dx^2 dL/dpower)
    s = _settings(W, H, V=V, deg=deg)
    r = og.Rasterizer(s)
    params = scene_to_device(sc)
    r._ensure(sc.n, sc.sh.shape[1])
    grads = np.zeros((V * sc.n, 12), np.float32)
    grads[:, :9] = g2
    r.grads2d.copy_(dev(grads))
    r._params = (*params, dev(vm))
    C.omnigs_preprocess_bwd(r.cfg, sc.n, *params, dev(vm), r.grads2d, r.d_means, r.d_scales, r.d_quats,
                            r.d_opacity, r.d_sh, r.d_screen)
    ref = oracle.preprocess_bwd(sc, vm, grads[:, :9].astype(np.float64), W, H)
    for name, got in [("means", r.d_means), ("scales", r.d_scales), ("quats", r.d_quats), ("opacity", r.d_opacity),
                      ("sh", r.d_sh), ("screen", r.d_screen)]:
        nw, el = assert_grad_close(got.cpu().numpy(), ref[name], name, rel=1e-4)
        print(f"preprocess_bwd {name}: normwise {nw:.2e} elementwise {el:.2e}")


@pytest.mark.parametrize("n,V", [(4000, 3), (600, 37)])
def test_preprocess_bwd_sparse_upstream_gradient(n, V):
    """Most (view, Gaussian) pairs of a real step pass no gradient (occluded or off every pixel). Here 60 % of the
    rows are zero, 15 % carry one field only (each of the nine in turn), and the first 50 Gaussians get none in any
    view; 37 views cross the 32-view chunks of the kernel's live-view mask."""
    W, H = 512, 256
    sc = synth.shell_scene(n, seed=17, sh_degree=3)
    vm = np.concatenate([synth.identity_viewmats(1), synth.random_viewmats(V - 1, 19)])
    rng = np.random.default_rng(23)
    g2 = rng.normal(size=(V * n, 9))
    g2[:, 2:5] *= 10.0
    u = rng.random(V * n)
    g2[u < 0.6] = 0.0
    one = (u >= 0.6) & (u < 0.75)
    keep = np.arange(V * n) % 9
    g2[one] *= (np.arange(9)[None, :] == keep[one, None])
    g2.reshape(V, n, 9)[:, :50] = 0.0
    s = _settings(W, H, V=V, deg=3)
    r = og.Rasterizer(s)
    params = scene_to_device(sc)
    r._ensure(n, sc.sh.shape[1])
    grads = np.zeros((V * n, 12), np.float32)
    grads[:, :9] = g2
    r.grads2d.copy_(dev(grads))
    C.omnigs_preprocess_bwd(r.cfg, n, *params, dev(vm), r.grads2d, r.d_means, r.d_scales, r.d_quats,
                            r.d_opacity, r.d_sh, r.d_screen)
    ref = oracle.preprocess_bwd(sc, vm, grads[:, :9].astype(np.float64), W, H)
    for name, got in [("means", r.d_means), ("scales", r.d_scales), ("quats", r.d_quats), ("opacity", r.d_opacity),
                      ("sh", r.d_sh), ("screen", r.d_screen)]:
        g = got.cpu().numpy()
        assert_grad_close(g, ref[name], name, rel=1e-4)
        assert not np.any(g.reshape(n, -1)[:50]), name  # no gradient in any view: exactly zero


# ------------------------------------------------------------------ S6 loss

def test_l1_loss_matches_numpy():
    W, H, V = 256, 128, 2
    rgb = synth.random_image(V, W, H, 1)
    tgt = synth.random_image(V, W, H, 2)
    tgt[0, 0, :4, :4] = rgb[0, 0, :4, :4]  # equal entries: zero gradient
    r = og.Rasterizer(_settings(W, H, V=V))
    r._ensure(1, 16)
    r.rgb.copy_(dev(rgb))
    loss = r.l1_loss(dev(tgt)).item()
    d = rgb.astype(np.float64) - tgt
    assert abs(loss - np.abs(d).mean()) <= 1e-6 * np.abs(d).mean()
    exp = np.sign(d) / d.size
    assert np.array_equal(r.dL_drgb.cpu().numpy(), exp.astype(np.float32))


@pytest.mark.parametrize("rows", [(0, 128), (0, 112), (16, 100)])
def test_l1_loss_over_a_band_of_rows(rows):
    """Loss restricted to image rows [begin, end) (the masked bottom band of Sec. 5.2), against float64 numpy."""
    W, H, V = 256, 128, 2
    rgb = synth.random_image(V, W, H, 3)
    tgt = synth.random_image(V, W, H, 4)
    r = og.Rasterizer(_settings(W, H, V=V))
    r._ensure(1, 16)
    r.rgb.copy_(dev(rgb))
    loss = r.l1_loss(dev(tgt), rows=rows).item()
    a, b = rows
    d = rgb.astype(np.float64)[:, :, a:b] - tgt[:, :, a:b]
    assert abs(loss - np.abs(d).mean()) <= 1e-6 * np.abs(d).mean()
    exp = np.zeros_like(rgb)
    exp[:, :, a:b] = (np.sign(d) / d.size).astype(np.float32)
    assert np.array_equal(r.dL_drgb.cpu().numpy(), exp)


def test_l1_loss_rows_rejects_empty_or_outside_bands():
    r = og.Rasterizer(_settings(64, 32))
    r._ensure(1, 16)
    x = torch.zeros_like(r.rgb)
    for rows in [(5, 5), (-1, 10), (0, 33), (20, 10)]:
        with pytest.raises(og.OmnigsError) as ei:
            r.l1_loss(x, rows=rows)
        assert ei.value.status == C.OMNIGS_E_INVALID
