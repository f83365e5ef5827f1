"""Pins of the D-SSIM loss oracle (Eq. 17 with its SSIM term), CPU only."""
import numpy as np
from scipy.signal import correlate2d

from oracle import ssim as S

RNG = np.random.default_rng(12)


def test_window_is_a_normalised_gaussian():
    g = S.gaussian_window()
    assert len(g) == 11 and abs(g.sum() - 1) < 1e-15 and np.argmax(g) == 5
    assert np.allclose(g, g[::-1])
    assert abs(np.log(g[5] / g[6]) - 1 / (2 * 1.5 ** 2)) < 1e-12  # sigma = 1.5


def test_separable_filter_equals_2d_correlation_with_zero_padding():
    img = RNG.uniform(size=(20, 27))
    g = S.gaussian_window()
    ref = correlate2d(img, np.outer(g, g), mode="same", boundary="fill", fillvalue=0.0)
    np.testing.assert_allclose(S.filter_same(img, g), ref, atol=1e-14)


def test_identical_images_have_ssim_one_and_zero_ssim_gradient():
    x = RNG.uniform(size=(1, 3, 16, 24))
    s, _ = S.ssim_map(x, x)
    np.testing.assert_allclose(s, 1.0, atol=1e-12)
    loss, grad = S.loss_and_grad(x, x, lam=1.0)
    assert abs(loss) < 1e-12 and np.abs(grad).max() < 1e-12  # SSIM is maximal at x = y


def test_constant_images_closed_form_in_the_interior():
    """Away from the border sigma = 0, so SSIM = (2ab + C1) / (a^2 + b^2 + C1)."""
    a, b = 0.7, 0.2
    s, _ = S.ssim_map(np.full((30, 30), a), np.full((30, 30), b))
    c1 = 0.01 ** 2  # the reading's constant, written out
    expect = (2 * a * b + c1) / (a * a + b * b + c1)
    np.testing.assert_allclose(s[5:-5, 5:-5], expect, rtol=1e-12)


def test_structure_term_for_an_affine_pair():
    """y = c x + d in a window: sigma_xy = c sigma_x^2 and sigma_y^2 = c^2 sigma_x^2, so the structure factor
    (2 sigma_xy + C2) / (sigma_x^2 + sigma_y^2 + C2) -> 2c / (1 + c^2) for large variance."""
    x = RNG.uniform(size=(40, 40)) * 50.0
    c = 0.5
    s, m = S.ssim_map(x, c * x + 0.1)
    ratio = m["a2"] / m["b2"]
    np.testing.assert_allclose(ratio[5:-5, 5:-5], 2 * c / (1 + c * c), rtol=1e-5)


def test_gradient_matches_central_differences():
    V, H, W = 1, 12, 14
    x = RNG.uniform(size=(V, 3, H, W))
    y = np.clip(x + RNG.normal(scale=0.2, size=x.shape), 0, 1)
    lam = 0.2
    _, grad = S.loss_and_grad(x, y, lam)
    h = 1e-6
    idx = [tuple(RNG.integers([V, 3, H, W])) for _ in range(60)] + [(0, 0, 0, 0), (0, 2, H - 1, W - 1), (0, 1, 0, 7)]
    for i in idx:
        if abs(x[i] - y[i]) < 1e-4:
            continue  # the L1 kink
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd = (S.loss_and_grad(xp, y, lam)[0] - S.loss_and_grad(xm, y, lam)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-7 * max(1e-3, abs(fd)) + 1e-12, (i, fd, grad[i])


def test_lambda_zero_is_plain_l1():
    x = RNG.uniform(size=(2, 3, 8, 8))
    y = RNG.uniform(size=(2, 3, 8, 8))
    loss, grad = S.loss_and_grad(x, y, lam=0.0)
    assert abs(loss - np.abs(x - y).mean()) < 1e-15
    np.testing.assert_allclose(grad, np.sign(x - y) / x.size)


def test_reflected_pair_pins_the_structure_constant():
    """y = 2a - x with the window mean of x equal to a at the centre: mu_x = mu_y = a there, sigma_y = sigma_x and
    sigma_xy = -sigma_x^2, so SSIM = (C2 - 2 v) / (C2 + 2 v) with v the window-weighted variance of x."""
    n, a, eps = 31, 0.5, 0.02
    g = S.gaussian_window()
    w = np.zeros((n, n))
    c = n // 2
    w[c - 5:c + 6, c - 5:c + 6] = np.outer(g, g)  # the window around the centre pixel
    r = RNG.uniform(-1, 1, size=(n, n))
    x = a + eps * (r - (w * r).sum())            # weighted mean exactly a at the centre
    v = (w * (x - a) ** 2).sum()                  # weighted variance there (textbook definition)
    s, _ = S.ssim_map(x, 2 * a - x)
    c2 = 0.03 ** 2  # the reading's constant, written out
    np.testing.assert_allclose(s[c, c], (c2 - 2 * v) / (c2 + 2 * v), rtol=1e-10)
