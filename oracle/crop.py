"""FP64 oracle of the perspective crop of an equirectangular image (Sec. 5.4: rendered equirectangular views are
cropped into perspective images before they are compared with perspective renders), for tests only.

TEST INFRASTRUCTURE: only the test-suite uses this module; the product path never does. It shares no code with the
CUDA sources.

Readings (the paper names the operation, not its sampling): the crop is a pinhole image (Eq. 2 intrinsics fx, fy,
cx, cy) looking along R^T of the equirectangular camera's axes, i.e. the pixel centre (x + 0.5, y + 0.5) has the
camera-frame direction d = R^T ((x + 0.5 - cx) / fx, (y + 0.5 - cy) / fy, 1); its longitude and latitude (Eq. 3) give
the equirectangular position p (Eqs. 4-5), sampled bilinearly between pixel centres with the columns wrapping around
the seam and the rows clamped at the poles.
"""
from __future__ import annotations

import numpy as np


def crop(equirect: np.ndarray, rot: np.ndarray, width: int, height: int, fx: float, fy: float, cx: float,
         cy: float) -> np.ndarray:
    """equirect [3, He, We], rot [3, 3] -> [3, height, width]."""
    img = np.asarray(equirect, np.float64)
    _, He, We = img.shape
    R = np.asarray(rot, np.float64)
    out = np.zeros((3, height, width))
    for y in range(height):
        for x in range(width):
            d = R.T @ np.array([(x + 0.5 - cx) / fx, (y + 0.5 - cy) / fy, 1.0])
            lon = np.arctan2(d[0], d[2])
            lat = np.arcsin(np.clip(d[1] / np.linalg.norm(d), -1.0, 1.0))
            u = (lon / np.pi + 1.0) * We / 2.0 - 0.5   # continuous column, pixel centres at integers
            v = (2.0 * lat / np.pi + 1.0) * He / 2.0 - 0.5
            x0, y0 = int(np.floor(u)), int(np.floor(v))
            fu, fv = u - x0, v - y0
            acc = np.zeros(3)
            for dy, wy in ((0, 1.0 - fv), (1, fv)):
                yy = min(max(y0 + dy, 0), He - 1)
                for dx, wx in ((0, 1.0 - fu), (1, fu)):
                    xx = (x0 + dx) % We
                    acc += wx * wy * img[:, yy, xx]
            out[:, y, x] = acc
    return out
