"""The workspace-free L1 entry point (omnigs_l1_loss_static) against the regular one (gpu).

omnigs_l1_loss_static exists for callers that cannot allocate device memory or pass the library a workspace, for
example a host application that owns the CUDA allocator. It keeps its partial sums in a fixed array inside the
library. This file is collected last so that a run stopping at its first failure has run every other test first;
it passes alone in a fresh process (where the entry point's first call does its one-time address lookup) and after
the other tests.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2404_03202_gb300 import _cabi as C  # noqa: E402


def _regular(cfg, rgb, tgt):
    ws = torch.empty(C.omnigs_workspace_size(cfg, 0, 0), dtype=torch.uint8, device="cuda")
    dL = torch.empty_like(rgb)
    loss = torch.zeros(1, device="cuda")
    C.omnigs_l1_loss(cfg, rgb, tgt, dL, loss, ws)
    return loss, dL


def _static(cfg, rgb, tgt):
    dL = torch.empty_like(rgb)
    loss = torch.zeros(1, device="cuda")
    C.omnigs_l1_loss_static(cfg, rgb, tgt, dL, loss)
    return loss, dL


def test_static_l1_matches_regular_on_two_calls_in_a_row():
    """Two consecutive calls with different inputs and sizes: the second must not see the first's partial sums."""
    for V, W, H, seed in [(2, 512, 256, 1), (1, 256, 128, 2)]:
        cfg = C.make_config(W, H, num_views=V)
        rgb = torch.from_numpy(synth.random_image(V, W, H, seed)).cuda()
        tgt = torch.from_numpy(synth.random_image(V, W, H, seed + 10)).cuda()
        loss_r, dL_r = _regular(cfg, rgb, tgt)
        loss_s, dL_s = _static(cfg, rgb, tgt)
        torch.cuda.synchronize()
        # same per-element gradient; the loss differs only in the order of float additions (relative 1e-6)
        assert torch.equal(dL_s, dL_r)
        assert abs(loss_s.item() - loss_r.item()) <= 1e-6 * abs(loss_r.item())
        ref = np.abs(rgb.cpu().numpy().astype(np.float64) - tgt.cpu().numpy()).mean()
        assert abs(loss_s.item() - ref) <= 1e-6 * ref


def test_static_l1_matches_regular_on_eight_full_views():
    """8 views of 2048 x 1024: 768 blocks of the static path, each spanning parts of several views."""
    V, W, H = 8, 2048, 1024
    cfg = C.make_config(W, H, num_views=V)
    g = torch.Generator(device="cuda").manual_seed(3)
    rgb = torch.rand((V, 3, H, W), device="cuda", generator=g)
    tgt = torch.rand((V, 3, H, W), device="cuda", generator=g)
    loss_r, dL_r = _regular(cfg, rgb, tgt)
    loss_s, dL_s = _static(cfg, rgb, tgt)
    torch.cuda.synchronize()
    assert torch.equal(dL_s, dL_r)
    assert abs(loss_s.item() - loss_r.item()) <= 1e-6 * abs(loss_r.item())


def test_static_l1_at_the_size_limit():
    """3 x 8192 x 10912 = 268,173,312 floats, the largest 16-row multiple within the 268,435,456-float limit (4093
    blocks), is accepted and matches the regular path; 16 more rows are rejected before anything runs."""
    W, H = 8192, 10912
    cfg = C.make_config(W, H, num_views=1)
    g = torch.Generator(device="cuda").manual_seed(4)
    rgb = torch.rand((1, 3, H, W), device="cuda", generator=g)
    tgt = torch.rand((1, 3, H, W), device="cuda", generator=g)
    loss_s, dL_s = _static(cfg, rgb, tgt)
    loss_r, dL_r = _regular(cfg, rgb, tgt)
    torch.cuda.synchronize()
    assert torch.equal(dL_s, dL_r)
    assert abs(loss_s.item() - loss_r.item()) <= 1e-6 * abs(loss_r.item())
    del dL_s, dL_r
    with pytest.raises(C.OmnigsError) as ei:
        C.omnigs_l1_loss_static(C.make_config(W, H + 16, num_views=1), rgb, tgt, rgb, loss_s)
    assert ei.value.status == C.OMNIGS_E_INVALID


def test_static_l1_rejects_what_the_regular_path_rejects():
    x = torch.zeros(4, device="cuda")
    for cfg in [C.make_config(65536, 32768, num_views=1),   # 3 * 65536 * 32768 floats > 268,435,456
                C.make_config(131072, 16, num_views=1),      # wider than 65536 px
                C.make_config(64, 32, num_views=5000),       # more than 4096 views
                C.make_config(64, 32, sh_degree=4)]:         # no such SH degree
        with pytest.raises(C.OmnigsError) as ei:
            C.omnigs_l1_loss_static(cfg, x, x, x, x)
        assert ei.value.status == C.OMNIGS_E_INVALID
