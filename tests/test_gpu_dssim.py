"""Eq. 17 with its D-SSIM term on the GPU against the FP64 oracle (gpu).

Tolerances: the moments are FP32 sums of 121 products of shifted values (|x'| <= 1/2), so a per-pixel SSIM error of
~1e-5 is expected where a window's variance is small against C2; the loss is a mean over many pixels (relative
1e-5 asserted), and the gradient's terms of size 1/C2 cancel to O(1), so it is held to normwise 1e-4 and
elementwise 1e-4 of its largest entry.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import ssim as oracle_ssim
from tests.gpu_util import dev, normwise

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2404_03202_gb300 import _cabi as C  # noqa: E402


def _smooth(V, W, H, seed):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W]
    img = np.empty((V, 3, H, W), np.float32)
    for v in range(V):
        for c in range(3):
            fx, fy, ph = rng.uniform(3, 15), rng.uniform(3, 15), rng.uniform(0, 6)
            img[v, c] = 0.5 + 0.35 * np.sin(xx / fx + ph) * np.cos(yy / fy) + 0.02 * rng.normal(size=(H, W))
    return np.clip(img, 0, 1).astype(np.float32)


def _run(rgb, tgt, lam, tile=16):
    V, _, H, W = rgb.shape
    cfg = C.make_config(W, H, tile=tile, num_views=V)
    scratch = torch.empty(C.omnigs_dssim_scratch_size(cfg), dtype=torch.uint8, device="cuda")
    dL = torch.empty(rgb.shape, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, device="cuda")
    C.omnigs_dssim_loss(cfg, lam, dev(rgb), dev(tgt), dL, loss, scratch)
    torch.cuda.synchronize()
    return loss.item(), dL.cpu().numpy()


@pytest.mark.parametrize("kind,W,H,tile,lam", [("smooth", 112, 48, 16, 0.2), ("noise", 80, 40, 8, 0.2),
                                               ("smooth", 256, 128, 16, 1.0), ("noise", 64, 32, 16, 0.0)])
def test_dssim_matches_oracle(kind, W, H, tile, lam):
    """Ragged tiles (112 = 3.5 x 32 columns, 40 = 2.5 x 16 rows), lambda 0 (plain L1) to 1 (pure D-SSIM)."""
    V = 2
    if kind == "smooth":
        rgb = _smooth(V, W, H, 1)
        tgt = np.clip(rgb + 0.05 * np.random.default_rng(2).normal(size=rgb.shape), 0, 1).astype(np.float32)
    else:
        rgb, tgt = synth.random_image(V, W, H, 3), synth.random_image(V, W, H, 4)
    loss, g = _run(rgb, tgt, lam, tile)
    ref_loss, ref_g = oracle_ssim.loss_and_grad(rgb.astype(np.float64), tgt.astype(np.float64), lam)
    nw = normwise(g, ref_g)
    el = np.abs(g - ref_g).max() / np.abs(ref_g).max()
    print(f"dssim {kind} {W}x{H} lambda {lam}: loss rel {abs(loss - ref_loss) / ref_loss:.2e}, grad normwise {nw:.2e}, "
          f"elementwise {el:.2e}")
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    assert nw <= 1e-4 and el <= 1e-4


def test_dssim_full_size_view():
    """One 2048 x 1024 view (the benchmark's resolution), full gradient."""
    W, H = 2048, 1024
    rgb = _smooth(1, W, H, 5)
    tgt = np.clip(rgb + 0.05 * np.random.default_rng(6).normal(size=rgb.shape), 0, 1).astype(np.float32)
    loss, g = _run(rgb, tgt, 0.2)
    ref_loss, ref_g = oracle_ssim.loss_and_grad(rgb.astype(np.float64), tgt.astype(np.float64), 0.2)
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    assert normwise(g, ref_g) <= 1e-4


def test_identical_images_give_zero_loss_and_gradient():
    rgb = _smooth(1, 64, 32, 7)
    loss, g = _run(rgb, rgb.copy(), 0.2)
    assert abs(loss) < 1e-6 and np.abs(g).max() < 1e-6 / rgb.size * 1e3


def test_dssim_rejects_bad_lambda():
    cfg = C.make_config(64, 32)
    x = torch.zeros(4, device="cuda")
    s = torch.empty(C.omnigs_dssim_scratch_size(cfg), dtype=torch.uint8, device="cuda")
    for lam in (-0.1, 1.5, float("nan")):
        with pytest.raises(C.OmnigsError) as ei:
            C.omnigs_dssim_loss(cfg, lam, x, x, x, x, s)
        assert ei.value.status == C.OMNIGS_E_INVALID
