"""Perspective crops of equirectangular images (Sec. 5.4) on the GPU against the FP64 oracle (gpu).

Tolerance: FP32 atan2f / asinf place a sample within ~1e-6 px of the FP64 position; on images whose values change by
at most ~1 per pixel the crop then agrees to 2e-5.
"""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import synth
from oracle import crop as OC
from tests.gpu_util import dev

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2404_03202_gb300 import _cabi as C  # noqa: E402


def test_crop_matches_oracle():
    V, We, He = 3, 128, 64
    img = synth.random_image(V, We, He, 3)
    rots = np.stack([np.eye(3), Rotation.random(random_state=4).as_matrix(),
                     Rotation.from_euler("y", 175, degrees=True).as_matrix()]).astype(np.float32)  # the last looks at the seam
    W, H, fx, fy, cx, cy = 48, 36, 24.0, 24.0, 24.0, 18.0
    out = torch.empty((V, 3, H, W), device="cuda")
    C.omnigs_equirect_crop(V, We, He, dev(img), dev(rots), W, H, fx, fy, cx, cy, out)
    got = out.cpu().numpy()
    for v in range(V):
        ref = OC.crop(img[v], rots[v].astype(np.float64), W, H, fx, fy, cx, cy)
        err = np.abs(got[v] - ref).max()
        print(f"crop view {v}: max abs {err:.2e}")
        assert err <= 2e-5


def test_crop_rejects_bad_intrinsics():
    x = torch.zeros(12, device="cuda")
    for fx in (0.0, -1.0, float("inf")):
        with pytest.raises(C.OmnigsError):
            C.omnigs_equirect_crop(1, 4, 2, x, x, 2, 2, fx, 1.0, 1.0, 1.0, x)
