"""Whole GPU path vs the FP64 oracle from identical 3D parameters, edge cases, autograd and graph capture (gpu).

End to end the GPU rounds p to float32 (half an ulp of W) before blending and the oracle does not, so agreement is
bounded by |dC/dp| * dp rather than by the blend's own 1e-5: with the 0.3 px^2 dilation every 2D Gaussian has
sigma >= sqrt(0.3) px, so |dG/dp| <= exp(-1/2) / sqrt(0.3) ~ 1.1 per px, and the per-pixel error stays within
~1e-6 * W summed over the few splats that matter. The asserts below use that bound with the pixel mask of the
oracle's near-threshold flags (eps 1e-3, matching the FP32 alpha error of ~1e-4 relative). The gradients, with the
near-threshold pixels' upstream gradient set to zero, are held to 1e-4 normwise per parameter tensor.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import dev, normwise, scene_to_device

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2404_03202_gb300 as og  # noqa: E402
from paper_2404_03202_gb300 import _cabi as C  # noqa: E402


def _settings(W, H, tile=16, V=1, deg=3, bg=(0.0, 0.0, 0.0)):
    return og.Settings(width=W, height=H, tile=tile, num_views=V, sh_degree=deg, bg=bg)


def test_end_to_end_config1_forward_backward():
    """10,000 Gaussians in a 0.5-5 shell, identity pose, 512x256, 16x16 tiles, dL/dC ~ N(0, 1)."""
    W, H = 512, 256
    sc = synth.shell_scene(10000, seed=1)
    vm = synth.identity_viewmats(1)
    r = og.Rasterizer(_settings(W, H))
    params = scene_to_device(sc)
    rgb = r.forward(*params, dev(vm)).cpu().numpy()
    f = oracle.render(sc, vm, W, H, 16, eps=1e-3)
    mask = (f["near"] & 1) == 0
    err = np.abs(rgb - f["rgb"]).max(axis=1)
    print(f"e2e fwd: instances gpu {r.count} oracle {len(f['list'])}; max|dC| {err[mask].max():.3e} "
          f"p99.9 {np.quantile(err[mask], 0.999):.3e} mean {err[mask].mean():.3e} masked {1 - mask.mean():.2e}")
    # the oracle lists every tile of every instance box; the GPU leaves out pairs out of reach
    assert 0.5 * len(f["list"]) <= r.count <= len(f["list"])
    assert 1 - mask.mean() <= 1e-2
    assert err[mask].max() <= 2e-6 * W * 4
    assert np.quantile(err[mask], 0.999) <= 1e-4
    g = synth.random_image_grad(1, W, H, 2)
    g[np.repeat((f["near"] != 0)[:, None], 3, axis=1)] = 0.0
    grads = r.backward(dev(g))
    ref = oracle.render_grad(sc, vm, g.astype(np.float64), W, H, 16, fwd=f)
    for name in ["means", "scales", "quats", "opacity", "sh", "screen"]:
        got = grads[name].cpu().numpy()
        nw = normwise(got, ref[name])
        print(f"e2e grad {name}: normwise {nw:.2e}")
        assert nw <= 1e-4, name


def test_autograd_function_matches_direct_backward():
    W, H = 256, 128
    sc = synth.shell_scene(3000, seed=4)
    vm = synth.random_viewmats(2, 9)
    r1 = og.Rasterizer(_settings(W, H, V=2))
    ps = [p.clone().requires_grad_(True) for p in scene_to_device(sc)]
    out = og.render(*ps, dev(vm), r1)
    g = torch.randn_like(out)
    grads = torch.autograd.grad(out, ps, g)
    r2 = og.Rasterizer(_settings(W, H, V=2))
    r2.forward(*[p.detach() for p in ps], dev(vm))
    direct = r2.backward(g.contiguous())
    for got, name in zip(grads, ["means", "scales", "quats", "opacity", "sh"]):
        assert normwise(got.cpu().numpy(), direct[name].cpu().numpy()) <= 1e-5, name


def test_empty_scene_renders_background():
    W, H = 128, 64
    bg = (0.2, 0.4, 0.6)
    r = og.Rasterizer(_settings(W, H, bg=bg))
    z = torch.zeros((0, 3), device="cuda")
    rgb = r.forward(z, z.clone(), torch.zeros((0, 4), device="cuda"), torch.zeros((0,), device="cuda"),
                    torch.zeros((0, 16, 3), device="cuda"), dev(synth.identity_viewmats(1)))
    torch.cuda.synchronize()
    assert r.count == 0
    assert torch.allclose(rgb, torch.tensor(bg, device="cuda").view(1, 3, 1, 1).expand_as(rgb))
    assert (r.T == 1).all() and (r.ncontrib == 0).all()


def test_empty_scene_with_the_fused_loss():
    """No Gaussians: the fused blend writes the background, its L1 loss against a target and the sign gradient."""
    W, H = 128, 64
    bg = (0.2, 0.4, 0.6)
    r = og.Rasterizer(_settings(W, H, bg=bg))
    z = torch.zeros((0, 3), device="cuda")
    tgt = dev(synth.random_image(1, W, H, 4))
    rgb = r.forward(z, z.clone(), torch.zeros((0, 4), device="cuda"), torch.zeros((0,), device="cuda"),
                    torch.zeros((0, 16, 3), device="cuda"), dev(synth.identity_viewmats(1)), l1_target=tgt)
    torch.cuda.synchronize()
    d = np.broadcast_to(np.asarray(bg, np.float32).reshape(1, 3, 1, 1), (1, 3, H, W)).astype(np.float64) \
        - tgt.cpu().numpy()
    assert r.count == 0 and torch.equal(rgb, torch.tensor(bg, device="cuda").view(1, 3, 1, 1).expand_as(rgb))
    assert abs(r.loss.item() - np.abs(d).mean()) <= 1e-6 * np.abs(d).mean()
    assert np.array_equal(r.dL_drgb.cpu().numpy(), (np.sign(d) / d.size).astype(np.float32))


def test_all_culled_inside_near_sphere():
    W, H = 128, 64
    sc = synth.shell_scene(500, seed=2, r_min=0.01, r_max=0.15)
    r = og.Rasterizer(_settings(W, H, bg=(1.0, 0.0, 0.0)))
    rgb = r.forward(*scene_to_device(sc), dev(synth.identity_viewmats(1)))
    torch.cuda.synchronize()
    assert r.count == 0 and (rgb[0, 0] == 1).all() and (rgb[0, 1:] == 0).all()


def test_capacity_overflow_is_reported():
    W, H = 256, 128
    sc = synth.shell_scene(5000, seed=3)
    r = og.Rasterizer(_settings(W, H), capacity=1000, grow=False)
    r.forward(*scene_to_device(sc), dev(synth.identity_viewmats(1)))
    with pytest.raises(og.OmnigsError) as ei:
        r.check()
    assert ei.value.status == C.OMNIGS_E_CAPACITY
    r.check()  # cleared after reporting
    assert r.instance_count() > 1000


def test_invalid_arguments_rejected():
    with pytest.raises(og.OmnigsError) as ei:
        og.Rasterizer(_settings(250, 128))._ensure(10, 16)  # width not a multiple of the tile
    assert ei.value.status == C.OMNIGS_E_INVALID
    cfg = C.make_config(256, 128, tile=12)
    assert C.omnigs_workspace_size(cfg, 10, 100) == 0
    cfg = C.make_config(256, 128, sh_degree=4)
    assert C.omnigs_workspace_size(cfg, 10, 100) == 0
    cfg = C.make_config(256, 128, tile=8, pixels_per_thread=4)  # 16 threads per 8x8 tile: not a whole warp
    assert C.omnigs_workspace_size(cfg, 10, 100) == 0
    cfg = C.make_config(256, 128, pixels_per_thread=3)
    assert C.omnigs_workspace_size(cfg, 10, 100) == 0


def test_graph_capture_matches_eager():
    """The forward + L1 + backward chain without host synchronisation replays from a CUDA graph."""
    W, H, V = 256, 128, 2
    sc = synth.shell_scene(4000, seed=8)
    vm = dev(synth.random_viewmats(V, 1))
    params = scene_to_device(sc)
    tgt = dev(synth.random_image(V, W, H, 3))
    r = og.Rasterizer(_settings(W, H, V=V))
    r.forward(*params, vm)
    cap = int(r.count * 1.5) + 1024
    g = og.Rasterizer(_settings(W, H, V=V), capacity=cap, grow=False)

    def step():
        g.forward(*params, vm)
        g.l1_loss(tgt)
        return g.backward()

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()  # warm-up outside capture (sets kernel attributes)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        out = step()
    graph.replay()
    torch.cuda.synchronize()
    g.check()
    eager_rgb = r.forward(*params, vm).clone()
    r.l1_loss(tgt)
    eager = r.backward()
    torch.cuda.synchronize()
    assert torch.equal(g.rgb, eager_rgb)
    assert abs(g.loss.item() - r.loss.item()) <= 1e-6 * abs(r.loss.item())
    for k in ["means", "scales", "quats", "opacity", "sh", "screen"]:
        assert normwise(out[k].cpu().numpy(), eager[k].cpu().numpy()) <= 1e-5, k


def test_profiler_collects_kernel_times():
    W, H = 128, 64
    sc = synth.shell_scene(1000, seed=5)
    r = og.Rasterizer(_settings(W, H))
    C.omnigs_profiler_enable(True)
    try:
        r.forward(*scene_to_device(sc), dev(synth.identity_viewmats(1)))
        r.l1_loss(torch.zeros_like(r.rgb))
        r.backward()
        times = C.omnigs_profiler_collect()
    finally:
        C.omnigs_profiler_enable(False)
    names = {t[0] for t in times}
    # 1000 splats (a 256-splat block spans two views at most) and 8 x 4 tiles: the bucketed order; the projection
    # writes the depth sort's keys itself (omnigs_preprocess_bin), so there is no separate depth_keys stage
    for k in ["preprocess_fwd", "depth_sort", "bin_count", "bin_emit", "tile_count", "tile_scatter",
              "tile_ranges", "render_fwd", "l1_loss", "render_bwd", "preprocess_bwd"]:
        assert k in names, k
    assert "depth_keys" not in names
    assert all(t[2] >= 0 for t in times)
    # fewer than 256 splats: the radix sort over the tile bits
    r = og.Rasterizer(_settings(W, H))
    C.omnigs_profiler_enable(True)
    try:
        r.forward(*scene_to_device(synth.shell_scene(200, seed=6)), dev(synth.identity_viewmats(1)))
        torch.cuda.synchronize()
        names = {t[0] for t in C.omnigs_profiler_collect()}
    finally:
        C.omnigs_profiler_enable(False)
    assert {"sort_upsweep", "sort_downsweep", "tile_ranges"} <= names and "tile_scatter" not in names


@pytest.mark.parametrize("tile,ppt", [(16, 4), (16, 2), (16, 8), (32, 4), (8, 2)])
def test_forward_with_fused_l1_matches_forward_then_l1(tile, ppt):
    """omnigs_render_fwd_l1 against omnigs_render_fwd followed by omnigs_l1_loss: the image, T, n_contrib and the
    gradient bit for bit, the loss (the same sum in another order) within 1e-6 relative, and against float64 numpy
    over the rendered image; pixels equal to the target get a zero gradient. The graph-captured fused step repeats
    the loss exactly."""
    W, H, V = 256, 128, 2
    sc = synth.shell_scene(6000, seed=11)
    vm = dev(synth.random_viewmats(V, 4))
    params = scene_to_device(sc)
    s = og.Settings(width=W, height=H, tile=tile, num_views=V, sh_degree=3, pixels_per_thread=ppt)
    a = og.Rasterizer(s)
    rgb = a.forward(*params, vm).clone()
    tgt = dev(synth.random_image(V, W, H, 12))
    tgt[0, :, :8, :8] = rgb[0, :, :8, :8]  # equal pixels: zero gradient
    a.l1_loss(tgt)
    b = og.Rasterizer(s, capacity=int(a.count * 1.5) + 1024, grow=False)
    b.forward(*params, vm, l1_target=tgt)
    torch.cuda.synchronize()
    b.check()
    assert torch.equal(b.rgb, a.rgb) and torch.equal(b.T, a.T) and torch.equal(b.ncontrib, a.ncontrib)
    assert torch.equal(b.dL_drgb, a.dL_drgb)
    assert not torch.any(b.dL_drgb[0, :, :8, :8])
    d = rgb.cpu().numpy().astype(np.float64) - tgt.cpu().numpy()
    ref = np.abs(d).mean()
    print(f"fused L1 {tile}x{tile}/{ppt}: {b.loss.item():.9g} unfused {a.loss.item():.9g} float64 {ref:.9g}")
    assert abs(b.loss.item() - a.loss.item()) <= 1e-6 * ref
    assert abs(b.loss.item() - ref) <= 1e-6 * ref

    def step():
        b.forward(*params, vm, l1_target=tgt)
        return b.backward()

    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        step()
    torch.cuda.current_stream().wait_stream(st)
    torch.cuda.synchronize()
    first = b.loss.clone()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(b.loss, first)


def test_fused_l1_rejects_a_forward_only_rasterizer_and_a_mismatched_target():
    W, H = 64, 32
    sc = synth.shell_scene(200, seed=2)
    params, vm = scene_to_device(sc), dev(synth.identity_viewmats(1))
    r = og.Rasterizer(_settings(W, H), forward_only=True)
    with pytest.raises(ValueError):
        r.forward(*params, vm, l1_target=torch.zeros(1, 3, H, W, device="cuda"))
    g = og.Rasterizer(_settings(W, H))
    for bad in (torch.zeros(2, 3, H, W, device="cuda"), torch.zeros(1, 3, H, W, device="cuda", dtype=torch.float64),
                torch.zeros(1, 3, W, H, device="cuda").transpose(2, 3), torch.zeros(1, 3, H, W)):
        with pytest.raises(ValueError):
            g.forward(*params, vm, l1_target=bad)
        g.forward(*params, vm)
        with pytest.raises(ValueError):
            g.l1_loss(bad)


@pytest.mark.parametrize("camera", ["equirect", "pinhole"])
def test_preprocess_bin_equals_preprocess_then_bin(camera):
    """omnigs_preprocess_bin (the projection also writing the depth sort's keys, equirectangular camera) against
    omnigs_preprocess followed by omnigs_bin: splats, order, the instance count and, after omnigs_sort, the sorted
    keys and the tile ranges bit for bit; and the same capacity-overflow error."""
    W, H, V = 256, 128, 3
    sc = synth.shell_scene(5000, seed=21)
    vm = dev(synth.random_viewmats(V, 9))
    params = scene_to_device(sc)
    pin = (200.0, 200.0, 128.0, 64.0) if camera == "pinhole" else None
    s = og.Settings(width=W, height=H, tile=16, num_views=V, sh_degree=3, pinhole=pin)
    a = og.Rasterizer(s)
    a.forward(*params, vm)  # sizes the buffers (capacity) and the workspace
    cap = int(a.count * 1.2) + 64
    outs = []
    for fused in (False, True):
        r = og.Rasterizer(s, capacity=cap, grow=False)
        r._ensure(sc.n, sc.sh.shape[1])
        r.order.fill_(-1)  # (pinhole: the entries past a view's ranked splats are left as they are)
        if fused:
            C.omnigs_preprocess_bin(r.cfg, sc.n, *params, vm, r.splats, r.order, r.keys, r.capacity, r.ws)
        else:
            C.omnigs_preprocess(r.cfg, sc.n, *params, vm, r.splats)
            C.omnigs_bin(r.cfg, sc.n, r.splats, r.order, r.keys, r.capacity, r.ws)
        count = C.omnigs_instance_count(r.ws)
        C.omnigs_sort(r.cfg, sc.n, r.capacity, r.keys, r.ranges, r.ws)  # (the bucketed bin leaves keys to the sort)
        outs.append((r.splats.clone(), r.order.clone(), count, r.keys[:count].clone(), r.ranges.clone()))
    (s0, o0, c0, k0, g0), (s1, o1, c1, k1, g1) = outs
    assert torch.equal(s0, s1) and torch.equal(o0, o1) and c0 == c1 == a.count
    assert torch.equal(k0, k1) and torch.equal(g0, g1)
    small = og.Rasterizer(s, capacity=max(a.count // 2, 1), grow=False)
    small._ensure(sc.n, sc.sh.shape[1])
    C.omnigs_preprocess_bin(small.cfg, sc.n, *params, vm, small.splats, small.order, small.keys, small.capacity,
                            small.ws)
    with pytest.raises(og.OmnigsError) as ei:
        small.check()
    assert ei.value.status == C.OMNIGS_E_CAPACITY
