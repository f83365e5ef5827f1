"""Pins of the oracle's pinhole camera (Eq. 2, the perspective model the paper contrasts with), CPU only."""
import numpy as np

import oracle
import synth

CAM = oracle.pinhole(fx=90.0, fy=80.0, cx=64.0, cy=40.0)
W, H = 128, 80


def _one(mean, scale, quat=(1, 0, 0, 0), opacity=0.5):
    sh = np.zeros((1, 1, 3), np.float32)
    sh[0, 0] = 0.5
    return synth.Scene(np.array([mean], np.float32), np.array([scale], np.float32), np.array([quat], np.float32),
                       np.array([opacity], np.float32), sh, 0)


def test_projection_and_depth(oracle_lib):
    for X, Y, Z in [(0.3, -0.2, 2.0), (-1.0, 0.5, 4.0), (0.0, 0.0, 1.0)]:
        rec = oracle.preprocess(_one([X, Y, Z], [0.01] * 3), synth.identity_viewmats(1), W, H, camera=CAM)[0]
        X32, Y32, Z32 = (float(np.float32(v)) for v in (X, Y, Z))
        assert abs(rec[oracle.R_PX] - (90.0 * X32 / Z32 + 64.0)) < 1e-12
        assert abs(rec[oracle.R_PY] - (80.0 * Y32 / Z32 + 40.0)) < 1e-12
        assert rec[oracle.R_DEPTH] == Z32  # pinhole Gaussians are ordered by t_z


def test_near_plane_is_on_t_z(oracle_lib):
    for Z, culled in [(0.19, True), (0.21, False), (-1.0, True)]:
        rec = oracle.preprocess(_one([0.05, 0.0, Z], [0.01] * 3), synth.identity_viewmats(1), W, H, camera=CAM)[0]
        assert (rec[oracle.R_RX] == 0) == culled


def test_isotropic_covariance_on_the_axis(oracle_lib):
    """At t = (0, 0, d), J = diag(fx / d, fy / d) rows, so Sigma~ = s^2 diag(fx^2, fy^2) / d^2 + 0.3 I."""
    d, sg = 3.0, 0.05
    rec = oracle.preprocess(_one([0, 0, d], [sg] * 3), synth.identity_viewmats(1), W, H, camera=CAM)[0]
    s32 = float(np.float32(sg))
    np.testing.assert_allclose([rec[oracle.R_COV00], rec[oracle.R_COV01], rec[oracle.R_COV11]],
                               [s32 ** 2 * 90 ** 2 / d ** 2 + 0.3, 0.0, s32 ** 2 * 80 ** 2 / d ** 2 + 0.3], rtol=1e-12,
                               atol=1e-15)


def test_off_screen_jacobian_is_clamped(oracle_lib):
    """Beyond 1.3 half-fields of view the ratio t_x / t_z in J is held at the limit: moving the Gaussian further out
    changes its projected position but not its covariance; inside the limit the covariance still changes."""
    lim = 1.3 * W / (2 * 90.0)

    def cov(k):
        # broad enough that the box still reaches the image from beyond the clamp
        rec = oracle.preprocess(_one([k * lim * 2.0, 0.0, 2.0], [0.6, 0.2, 0.3]), synth.identity_viewmats(1), W, H,
                                camera=CAM)[0]
        return rec[oracle.R_PX], rec[[oracle.R_COV00, oracle.R_COV01, oracle.R_COV11]]

    (p1, c1), (p2, c2) = cov(1.05), cov(1.5)
    assert p1 != p2
    np.testing.assert_allclose(c1, c2, rtol=1e-12)
    (_, c3), (_, c4) = cov(0.95), cov(0.98)
    assert np.abs(c3 - c4).max() > 1e-6 * np.abs(c3).max()


def test_box_off_the_image_is_culled(oracle_lib):
    """A Gaussian whose instance box [floor(p) -+ r] misses the image is culled (it has no tile either way). A tiny
    Gaussian has r_x = r_y = 2 (the 0.3 px^2 dilation sets its footprint), so p_x = -2.5 (box -5..-1) is culled and
    p_x = -1.5 (box -4..0) is kept; likewise p_x = W + 2.3 (box W..W+4) against W + 1.5, and the same for rows."""
    Z = 2.0

    def rec(px, py):
        X, Y = (px - 64.0) * Z / 90.0, (py - 40.0) * Z / 80.0
        return oracle.preprocess(_one([X, Y, Z], [0.002] * 3), synth.identity_viewmats(1), W, H, camera=CAM)[0]

    centre = rec(40.3, 30.6)
    assert centre[oracle.R_RX] == 2 and centre[oracle.R_RY] == 2
    for px, py, culled in [(-2.5, 30.5, True), (-1.5, 30.5, False), (W + 2.3, 30.5, True), (W + 1.5, 30.5, False),
                           (40.5, -2.5, True), (40.5, -1.5, False), (40.5, H + 2.3, True), (40.5, H + 1.5, False)]:
        r = rec(px, py)
        assert abs(r[oracle.R_PX] - px) < 1e-3 or culled  # the centre lands where intended
        assert (r[oracle.R_RX] == 0) == culled, (px, py)


def test_columns_are_clipped_not_wrapped(oracle_lib):
    T = 16
    assert oracle.rect(2.0, 40.0, 10, 3, W, H, T, camera=CAM) == (0, 1, 2, 1)   # pixels -8..12: columns 0 only
    assert oracle.rect(2.0, 40.0, 10, 3, W, H, T) == (-1, 2, 2, 1)              # the equirect camera wraps
    assert oracle.rect(-30.0, 40.0, 10, 3, W, H, T, camera=CAM)[1] == 0         # wholly off screen: no column


def test_no_wrap_across_the_image_edge(oracle_lib):
    """A broad splat at the left edge lights the right edge through the seam of an equirectangular image only."""
    sp = dict(px=np.array([3.0]), py=np.array([40.0]), c0=np.array([1 / 900.0]), c1=np.array([0.0]),
              c2=np.array([1 / 900.0]), opacity=np.array([0.9]), r=np.array([1.0]), g=np.array([1.0]),
              b=np.array([1.0]), depth=np.array([2.0]), rx=np.array([127], np.int32), ry=np.array([30], np.int32))
    lit = {}
    for name, cam in (("pinhole", CAM), ("equirect", None)):
        ranges, lst = oracle.bin_sort(sp, 1, W, H, 16, camera=cam)
        rgb, _, _, _ = oracle.blend_fwd(sp, ranges, lst, 1, W, H, 16, camera=cam)
        lit[name] = rgb[0, 0, 40, W - 1]
    assert lit["pinhole"] < 1e-3 < lit["equirect"]


def test_blend_matches_bruteforce_without_seam(oracle_lib):
    sc = synth.shell_scene(300, seed=3, log_scale_mean=-2.5)
    sc.opacity[:] = np.minimum(sc.opacity, 0.34)
    vm = synth.random_viewmats(1, 4)
    f = oracle.render(sc, vm, W, H, 16, camera=CAM)
    sp = f["splats"]
    ref = np.zeros((3, H, W))
    idx = [i for i in range(sc.n) if sp["rx"][i] > 0]
    idx.sort(key=lambda i: (sp["depth"][i], i))
    for y in range(H):
        for x in range(W):
            T, C = 1.0, np.zeros(3)
            for i in idx:
                dx, dy = sp["px"][i] - (x + 0.5), sp["py"][i] - (y + 0.5)
                power = -0.5 * (sp["c0"][i] * dx * dx + sp["c2"][i] * dy * dy) - sp["c1"][i] * dx * dy
                if power > 0:
                    continue
                a = min(0.99, sp["opacity"][i] * np.exp(power))
                if a < 1 / 255:
                    continue
                if T * (1 - a) < 1e-4:
                    break
                C += a * T * np.array([sp["r"][i], sp["g"][i], sp["b"][i]])
                T *= 1 - a
            ref[:, y, x] = C
    assert len(idx) > 20
    np.testing.assert_allclose(f["rgb"][0], ref, atol=1e-12)


def test_end_to_end_gradient_matches_finite_differences(oracle_lib):
    """Some Gaussians sit beyond the Jacobian clamp (|t_x / t_z| up to 1.5 half-fields of view)."""
    rng = np.random.default_rng(5)
    n = 24
    z = rng.uniform(1.5, 4.0, n)
    means = np.stack([rng.uniform(-1, 1, n) * 1.5 * (W / (2 * 90.0)) * z, rng.uniform(-0.5, 0.5, n) * z, z], 1)
    sc = synth.shell_scene(n, 6, log_scale_mean=-2.2)
    sc.means[:] = means.astype(np.float32)
    # four broad Gaussians beyond the clamp whose footprint still reaches the image
    lim = 1.3 * W / (2 * 90.0)
    for j, (u, v, zj) in enumerate([(1.35, 0.1, 2.0), (-1.4, -0.2, 2.3), (1.5, 0.3, 2.6), (-1.32, 0.0, 2.9)]):
        sc.means[j] = np.array([u * lim * zj, v * zj, zj], np.float32)
        sc.scales[j] = np.array([0.5, 0.4, 0.45], np.float32)
    vm = synth.identity_viewmats(1)
    wgt = synth.random_image_grad(1, W, H, 7).astype(np.float64)
    f = oracle.render(sc, vm, W, H, 16, camera=CAM)
    f["count"] = oracle.blend_fwd.last_count.copy()
    g = oracle.render_grad(sc, vm, wgt, W, H, 16, fwd=f, camera=CAM)
    checked = 0
    for field in ("means", "scales"):
        for idx in np.ndindex(n, 3):
            base = float(getattr(sc, field)[idx])
            h = 1e-5 * (abs(base) if field == "scales" else 1.0)
            vals = []
            for sgn in (1, -1):
                arr = getattr(sc, field)
                old = arr[idx]
                arr[idx] = np.float32(base + sgn * h)
                step = float(arr[idx]) - base
                ff = oracle.render(sc, vm, W, H, 16, camera=CAM)
                ff["count"] = oracle.blend_fwd.last_count.copy()
                vals.append(((ff["rgb"] * wgt).sum(), step, ff))
                arr[idx] = old
            (lp, hp, fp), (lm, hm, fm) = vals
            if not all(np.array_equal(ff[k], f[k]) for ff in (fp, fm) for k in ("n_contrib", "list", "count")):
                continue  # a discrete decision flipped
            fd = (lp - lm) / (hp - hm)
            assert abs(fd - g[field][idx]) <= 2e-4 * max(1.0, abs(fd)), (field, idx, fd, g[field][idx])
            checked += 1
    assert checked >= 60
