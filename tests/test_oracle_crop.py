"""Pins of the perspective-crop oracle (Sec. 5.4), CPU only."""
import numpy as np

from oracle import crop as OC

RNG = np.random.default_rng(31)


def test_constant_image_crops_to_the_constant():
    img = np.broadcast_to(np.array([0.2, 0.5, 0.9])[:, None, None], (3, 32, 64))
    out = OC.crop(img, np.eye(3), 16, 12, 8.0, 8.0, 8.0, 6.0)
    np.testing.assert_allclose(out, np.broadcast_to(img[:, :1, :1], out.shape), atol=1e-15)


def test_optical_axis_samples_the_image_centre_column():
    """The crop's centre looks along +z: longitude 0 (column W/2), latitude 0 (row H/2)."""
    We, He = 64, 32
    img = RNG.uniform(size=(3, He, We))
    out = OC.crop(img, np.eye(3), 2, 2, 1.0, 1.0, 1.0, 1.0)  # pixel centre (1.5, 1.5): direction (0.5, 0.5, 1)
    d = np.array([0.5, 0.5, 1.0])
    lon, lat = np.arctan2(d[0], d[2]), np.arcsin(d[1] / np.linalg.norm(d))
    u, v = (lon / np.pi + 1) * We / 2 - 0.5, (2 * lat / np.pi + 1) * He / 2 - 0.5
    x0, y0 = int(u), int(v)
    fu, fv = u - x0, v - y0
    ref = ((1 - fu) * (1 - fv) * img[:, y0, x0] + fu * (1 - fv) * img[:, y0, x0 + 1] + (1 - fu) * fv * img[:, y0 + 1, x0]
           + fu * fv * img[:, y0 + 1, x0 + 1])
    np.testing.assert_allclose(out[:, 1, 1], ref, rtol=1e-12)


def test_a_yaw_of_the_crop_is_a_column_shift_of_the_source():
    """Rotating the crop by 2 pi k / W about y samples the same points of an image rolled by k columns."""
    We, He, k = 64, 32, 8
    img = RNG.uniform(size=(3, He, We))
    a = 2 * np.pi * k / We
    R = np.array([[np.cos(a), 0, -np.sin(a)], [0, 1, 0], [np.sin(a), 0, np.cos(a)]])
    base = OC.crop(img, np.eye(3), 10, 8, 6.0, 6.0, 5.0, 4.0)
    turned = OC.crop(np.roll(img, k, axis=2), R, 10, 8, 6.0, 6.0, 5.0, 4.0)
    np.testing.assert_allclose(turned, base, atol=1e-9)


def test_bilinear_weights_interpolate_a_linear_ramp_exactly():
    """Away from the seam and the poles, a ramp in the column index is reproduced at the sampled position."""
    We, He = 128, 64
    ramp = np.broadcast_to(np.arange(We, dtype=np.float64)[None, None, :], (3, He, We)).copy()
    out = OC.crop(ramp, np.eye(3), 8, 8, 20.0, 20.0, 4.0, 4.0)
    for x in range(8):
        d = np.array([(x + 0.5 - 4.0) / 20.0, 0.0, 1.0])
        u = (np.arctan2(d[0], d[2]) / np.pi + 1) * We / 2 - 0.5
        np.testing.assert_allclose(out[0, 4, x], u, rtol=1e-12)
