"""FP64 oracle of the photometric loss with its D-SSIM term (Eq. 17), for tests only.

TEST INFRASTRUCTURE: only the test-suite and the benchmark's CPU-baseline leg use this module; the product path
never does. It shares no code with the CUDA sources.

Eq. 17 mixes an L1 term and a D-SSIM term: L = (1 - lambda) L1 + lambda (1 - SSIM). The paper defers the SSIM
details to 3DGS; the readings here follow that renderer's conventions:
  * SSIM per colour channel with an 11 x 11 Gaussian window of standard deviation 1.5 (normalised to sum 1), applied
    as a "same"-size filter with zero padding outside the image;
  * C1 = 0.01^2, C2 = 0.03^2 (data range 1);
  * SSIM = mean over views, channels and pixels of
        ((2 mu_x mu_y + C1)(2 sigma_xy + C2)) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2)),
    mu = G * x, sigma_x^2 = G * x^2 - mu_x^2, sigma_xy = G * (x y) - mu_x mu_y;
  * lambda = 0.2 unless given.
The gradient with respect to the rendered image x is the chain rule through the filtered moments, written out below.
"""
from __future__ import annotations

import numpy as np

C1 = 0.01 ** 2
C2 = 0.03 ** 2
WINDOW = 11
SIGMA = 1.5


def gaussian_window(size: int = WINDOW, sigma: float = SIGMA) -> np.ndarray:
    """Normalised 1D Gaussian taps; the 2D window is their outer product."""
    r = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-(r * r) / (2.0 * sigma * sigma))
    return g / g.sum()


def filter_same(img: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Separable "same" filter of the last two axes with taps g (odd length), zero padding outside the image."""
    k = len(g) // 2
    H, W = img.shape[-2:]
    p = np.pad(img, [(0, 0)] * (img.ndim - 2) + [(k, k), (k, k)])
    rows = sum(g[t] * p[..., :, t:t + W] for t in range(len(g)))          # along x
    return sum(g[t] * rows[..., t:t + H, :] for t in range(len(g)))         # along y


def ssim_map(x: np.ndarray, y: np.ndarray, g: np.ndarray | None = None):
    """Per-pixel SSIM of x against y ([..., H, W]) and the filtered moments it is built from."""
    g = gaussian_window() if g is None else g
    mx, my = filter_same(x, g), filter_same(y, g)
    exx, eyy, exy = filter_same(x * x, g), filter_same(y * y, g), filter_same(x * y, g)
    a1 = 2 * mx * my + C1
    a2 = 2 * (exy - mx * my) + C2
    b1 = mx * mx + my * my + C1
    b2 = (exx - mx * mx) + (eyy - my * my) + C2
    s = a1 * a2 / (b1 * b2)
    return s, dict(mx=mx, my=my, a1=a1, a2=a2, b1=b1, b2=b2)


def loss_and_grad(x: np.ndarray, y: np.ndarray, lam: float = 0.2):
    """Eq. 17 for rendered images x and targets y ([V, 3, H, W]): (loss, dL/dx)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    n = x.size
    g = gaussian_window()
    s, m = ssim_map(x, y, g)
    d = x - y
    loss = (1 - lam) * np.abs(d).mean() + lam * (1.0 - s.mean())
    # dS/d(mu_x), dS/d(E[x^2]), dS/d(E[xy]) per output pixel
    ds_dmx = s * (2 * m["my"] / m["a1"] - 2 * m["my"] / m["a2"] - 2 * m["mx"] / m["b1"] + 2 * m["mx"] / m["b2"])
    ds_dexx = -s / m["b2"]
    ds_dexy = 2 * s / m["a2"]
    # each moment is a symmetric zero-padded filter, so its adjoint is the same filter
    dmean_dx = (filter_same(ds_dmx, g) + 2 * x * filter_same(ds_dexx, g) + y * filter_same(ds_dexy, g)) / n
    grad = (1 - lam) * np.sign(d) / n - lam * dmean_dx
    return float(loss), grad
