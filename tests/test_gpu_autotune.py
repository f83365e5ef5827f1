"""Autotuner of the tile size and blend schedule (gpu)."""

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2404_03202_gb300 as og  # noqa: E402
from paper_2404_03202_gb300.autotune import CANDIDATES, Autotuner  # noqa: E402


def test_tuner_times_every_candidate_and_caches_the_fastest():
    sc = synth.room_scene(20000, 5)
    params = [torch.from_numpy(a).cuda() for a in sc.arrays()]
    vm = torch.from_numpy(synth.room_viewmats(2, 6)).cuda()
    base = og.Settings(width=512, height=256, num_views=2, sh_degree=3)
    tuner = Autotuner(warmup=1, iters=2)
    c = tuner.tune(params, vm, base, "train")
    assert set(c.table) == set(CANDIDATES)
    assert c.ms == min(c.table.values()) and c.table[(c.tile, c.pixels_per_thread)] == c.ms
    assert tuner.tune(params, vm, base, "train") is c  # cached per workload
    s = tuner.settings(params, vm, base, "train")
    assert (s.tile, s.pixels_per_thread) == (c.tile, c.pixels_per_thread)


def test_blend_schedule_leaves_the_forward_bit_identical():
    sc = synth.room_scene(20000, 7)
    params = [torch.from_numpy(a).cuda() for a in sc.arrays()]
    vm = torch.from_numpy(synth.room_viewmats(2, 8)).cuda()
    for tile in (16, 32):
        imgs = []
        for ppt in (2, 4):
            s = og.Settings(width=512, height=256, tile=tile, num_views=2, sh_degree=3, pixels_per_thread=ppt)
            r = og.Rasterizer(s)
            imgs.append(r.forward(*params, vm).clone())
        assert torch.equal(imgs[0], imgs[1]), tile


def test_tile_size_changes_only_pixels_reached_outside_a_splats_box():
    """Across tile sizes the images agree except where a splat's 3-sigma square limits its box (high opacity):
    with every opacity below 0.35 the alpha >= 1/255 region lies inside the box, so all tile sizes agree."""
    sc = synth.room_scene(20000, 9)
    sc.opacity[:] = np.minimum(sc.opacity, 0.34)
    params = [torch.from_numpy(a).cuda() for a in sc.arrays()]
    vm = torch.from_numpy(synth.room_viewmats(1, 10)).cuda()
    out = []
    for tile in (8, 16, 32):
        r = og.Rasterizer(og.Settings(width=512, height=256, tile=tile, num_views=1, sh_degree=3))
        out.append(r.forward(*params, vm).clone())
    assert torch.equal(out[0], out[1]) and torch.equal(out[1], out[2])
