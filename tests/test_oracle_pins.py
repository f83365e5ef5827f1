"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Which pin covers which oracle function:
  project (Eqs. 3-5)            closed-form inverse map, seam value, range           test_projection_*
  jacobian (Eqs. 10-16)          central differences of project                       test_jacobian_*
  preprocess: Sigma~ (Eq. 9)     isotropic and axis-aligned closed forms              test_isotropic_*, test_aligned_*
  quat_to_rot                    scipy Rotation                                       test_quaternion_*
  sh_basis                       orthonormality by quadrature, scipy sph_harm_y       test_sh_*
  preprocess: near cull          t_r = 0.19 vs 0.21                                   test_near_cull
  rect / bin_sort                pixel-enumeration brute force of the instance boxes  test_bin_sort_*, test_rect_*
  blend_fwd (Eqs. 6-8)           all-Gaussians brute force, stop rule closed form,    test_blend_*, test_termination_*
                                 background term, yaw = cyclic column shift           test_yaw_*
  blend_bwd, preprocess_bwd      FP64 central finite differences (stage and end-to-end)   test_*_finite_differences
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
import synth

RNG = np.random.default_rng(1234)


def _direction(lon, lat):
    return np.array([np.cos(lat) * np.sin(lon), np.sin(lat), np.cos(lat) * np.cos(lon)])


# ------------------------------------------------------------------ projection (Eqs. 3-5)

def test_projection_closed_form(oracle_lib):
    W, H = 2048, 1024
    for _ in range(200):
        lon = RNG.uniform(-np.pi, np.pi)
        lat = RNG.uniform(-np.pi / 2 + 1e-3, np.pi / 2 - 1e-3)
        d = RNG.uniform(0.3, 50.0)
        ll, s, p = oracle.project(d * _direction(lon, lat), W, H)
        assert abs(ll[0] - lon) < 1e-12 and abs(ll[1] - lat) < 1e-12
        np.testing.assert_allclose(s, [lon / np.pi, 2 * lat / np.pi], atol=1e-13)
        np.testing.assert_allclose(p, [W * (lon + np.pi) / (2 * np.pi), H * (lat + np.pi / 2) / np.pi], atol=1e-9)


def test_projection_seam_and_range(oracle_lib):
    W, H = 512, 256
    # straight behind the camera: atan2(+0, -1) = +pi is mapped to -pi, so p_x = 0 and p_x stays in [0, W)
    _, _, p = oracle.project([0.0, 0.0, -1.0], W, H)
    assert p[0] == 0.0 and p[1] == H / 2
    _, _, p = oracle.project([-1e-9, 0.0, -1.0], W, H)
    assert 0.0 <= p[0] < 1e-6 or W - 1e-6 < p[0] < W
    _, _, p = oracle.project([1e-9, 0.0, -1.0], W, H)
    assert W - 1e-6 < p[0] < W
    # straight ahead, right, up (y is down in the camera frame), down
    assert np.allclose(oracle.project([0, 0, 1], W, H)[2], [W / 2, H / 2])
    assert np.allclose(oracle.project([1, 0, 0], W, H)[2], [3 * W / 4, H / 2])
    assert np.allclose(oracle.project([0, -1, 0], W, H)[2][1], 0.0)
    assert np.allclose(oracle.project([0, 1, 0], W, H)[2][1], H)


# ------------------------------------------------------------------ Jacobian (Eqs. 10-16)

def test_jacobian_matches_finite_differences(oracle_lib):
    W, H = 2048, 1024
    for _ in range(100):
        t = RNG.normal(size=3) * RNG.uniform(0.5, 10)
        if np.hypot(t[0], t[2]) < 0.05 * np.linalg.norm(t):
            continue
        J = oracle.jacobian(t, W, H)
        fd = np.zeros((2, 3))
        for k in range(3):
            h = 1e-6 * np.linalg.norm(t)
            tp, tm = t.copy(), t.copy()
            tp[k] += h
            tm[k] -= h
            pp, pm = oracle.project(tp, W, H)[2], oracle.project(tm, W, H)[2]
            dp = pp - pm
            dp[0] -= W * np.round(dp[0] / W)  # do not difference across the seam
            fd[:, k] = dp / (2 * h)
        np.testing.assert_allclose(J, fd, rtol=1e-6, atol=1e-6 * np.abs(J).max())
        # the second row's last entry is dp_y/dt_z (Eq. 16), not a repeat of dp_y/dt_y
        assert J[0, 1] == 0.0


# ------------------------------------------------------------------ covariance (Eq. 9) closed forms

def _to64(sp):
    return {k: (np.asarray(v, np.float64) if np.asarray(v).dtype.kind == "f" else v) for k, v in sp.items()}


def _one_gaussian(mean, scale, quat, sh_dc=(0.5, 0.5, 0.5), opacity=0.5, degree=0):
    K = (degree + 1) ** 2
    sh = np.zeros((1, K, 3), np.float32)
    sh[0, 0] = sh_dc
    return synth.Scene(np.array([mean], np.float32), np.array([scale], np.float32), np.array([quat], np.float32),
                       np.array([opacity], np.float32), sh, degree)


def test_isotropic_covariance_closed_form(oracle_lib):
    """Sigma = sigma^2 I gives Sigma~ = sigma^2 diag(a^2 / rho^2, b^2 / t_r^2) + 0.3 I, off-diagonal exactly 0."""
    W, H = 2048, 1024
    a, b = W / (2 * np.pi), H / np.pi
    for _ in range(50):
        lon, lat = RNG.uniform(-3, 3), RNG.uniform(-1.4, 1.4)
        tr, sigma = RNG.uniform(1, 10), RNG.uniform(0.01, 0.3)
        vm = synth.random_viewmats(1, int(RNG.integers(1 << 30)), max_offset=0.5)
        Wr, tcw = vm[0, :3, :3].astype(np.float64), vm[0, :3, 3].astype(np.float64)
        t = tr * _direction(lon, lat)
        m = Wr.T @ (t - tcw)
        sc = _one_gaussian(m, [sigma] * 3, [1, 0, 0, 0])
        rec = oracle.preprocess(sc, vm, W, H)[0]
        # the scene stores float32 values; recompute the exact camera-space point from the stored mean
        t32 = Wr @ sc.means[0].astype(np.float64) + tcw
        s32 = float(sc.scales[0, 0])
        rho2 = t32[0] ** 2 + t32[2] ** 2
        tr2 = t32 @ t32
        # the float32 pose is orthonormal only to ~1e-7, which bounds the agreement
        np.testing.assert_allclose(rec[oracle.R_COV00], s32 ** 2 * a * a / rho2 + 0.3, rtol=1e-6)
        np.testing.assert_allclose(rec[oracle.R_COV11], s32 ** 2 * b * b / tr2 + 0.3, rtol=1e-6)
        assert abs(rec[oracle.R_COV01]) < 1e-6 * rec[oracle.R_COV00]
    # with an exact (identity) pose the closed form holds to rounding and the off-diagonal is zero
    for _ in range(20):
        t = RNG.uniform(1, 10) * _direction(RNG.uniform(-3, 3), RNG.uniform(-1.4, 1.4))
        sc = _one_gaussian(t, [0.1] * 3, [1, 0, 0, 0])
        rec = oracle.preprocess(sc, synth.identity_viewmats(1), W, H)[0]
        t32 = sc.means[0].astype(np.float64)
        s32 = float(sc.scales[0, 0])
        np.testing.assert_allclose(rec[oracle.R_COV00], s32 ** 2 * a * a / (t32[0] ** 2 + t32[2] ** 2) + 0.3, rtol=1e-12)
        np.testing.assert_allclose(rec[oracle.R_COV11], s32 ** 2 * b * b / (t32 @ t32) + 0.3, rtol=1e-12)
        assert abs(rec[oracle.R_COV01]) < 1e-12 * rec[oracle.R_COV00]


def test_aligned_covariance_and_quaternion_order(oracle_lib):
    """Straight ahead (lon = lat = 0), J = diag(a/d, b/d); a rotation by theta about the camera's z axis,
    q = (cos theta/2, 0, 0, sin theta/2) in (w, x, y, z) order, turns diag(sx^2, sy^2) by theta."""
    W, H = 1024, 512
    a, b = W / (2 * np.pi), H / np.pi
    for theta in [0.0, 0.3, 1.1, -0.7]:
        d, sx, sy, sz = 3.0, 0.2, 0.05, 0.1
        sc = _one_gaussian([0, 0, d], [sx, sy, sz], [np.cos(theta / 2), 0, 0, np.sin(theta / 2)])
        rec = oracle.preprocess(sc, synth.identity_viewmats(1), W, H)[0]
        c, s = np.cos(theta), np.sin(theta)
        R2 = np.array([[c, -s], [s, c]])
        s32 = sc.scales[0].astype(np.float64)
        q32 = sc.quats[0].astype(np.float64)
        # the float32-stored quaternion is not exactly unit norm; the rotation angle it encodes is exact
        th = 2 * np.arctan2(q32[3], q32[0])
        R2 = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        D = np.diag([a / d, b / d])
        cov = D @ R2 @ np.diag(s32[:2] ** 2) @ R2.T @ D + 0.3 * np.eye(2)
        got = np.array([[rec[oracle.R_COV00], rec[oracle.R_COV01]], [rec[oracle.R_COV01], rec[oracle.R_COV11]]])
        np.testing.assert_allclose(got, cov, rtol=1e-6, atol=1e-9)
        # conic is the inverse, radius = ceil(3 sqrt(lambda_max)) with the 0.1 floor
        conic = np.linalg.inv(cov)
        np.testing.assert_allclose(rec[[oracle.R_C0, oracle.R_C1, oracle.R_C2]], [conic[0, 0], conic[0, 1], conic[1, 1]],
                                   rtol=1e-6)
        lam = np.linalg.eigvalsh(cov).max()
        assert rec[oracle.R_RADIUS] == np.ceil(3 * np.sqrt(lam))
        # instance box: the square narrowed to the box of the alpha >= 1/255 ellipse (opacity 0.5: q = 2 ln 127.5)
        q = 2 * np.log(255 * float(sc.opacity[0]))
        for key, var in ((oracle.R_RX, cov[0, 0]), (oracle.R_RY, cov[1, 1])):
            expect = min(rec[oracle.R_RADIUS], np.ceil(np.sqrt(q * var) * (1 + 1e-4) + 1e-3))
            assert rec[key] == expect


def test_instance_box_is_bounded_by_the_radius(oracle_lib):
    """At opacity 0.99 the alpha >= 1/255 ellipse (q = 2 ln(252.45) = 11.06) reaches past 3 sigma: for an isotropic
    Sigma~ both box half-extents are the 3-sigma radius ceil(3 sqrt(lambda)) of reading 6, not the ellipse's
    ceil(sqrt(q var)); at opacity 0.1 the ellipse's box is the narrower one."""
    W, H = 1024, 512
    for o, binds in ((0.99, True), (0.1, False)):
        sc = _one_gaussian([0, 0, 3.0], [0.05] * 3, [1, 0, 0, 0], opacity=o)
        rec = oracle.preprocess(sc, synth.identity_viewmats(1), W, H)[0]
        lam = max(rec[oracle.R_COV00], rec[oracle.R_COV11])
        r = np.ceil(3 * np.sqrt(lam))
        assert rec[oracle.R_RADIUS] == r
        q = 2 * np.log(255 * float(sc.opacity[0]))
        for key, var in ((oracle.R_RX, rec[oracle.R_COV00]), (oracle.R_RY, rec[oracle.R_COV11])):
            ellipse = np.ceil(np.sqrt(q * var) * (1 + 1e-4) + 1e-3)
            assert (ellipse > r) == binds
            assert rec[key] == min(r, ellipse)


def test_gaussian_on_the_pole_projects_to_finite_values(oracle_lib):
    """A Gaussian straight above the camera (t_x = t_z = 0, lat = pi/2): the projection is finite, and with the pole
    guard so is J (its entries are those at rho = 1e-6 t_r), hence the covariance, conic and box."""
    W, H = 512, 256
    t = np.array([0.0, 2.0, 0.0])
    J = oracle.jacobian(t, W, H)
    assert np.isfinite(J).all()
    sc = _one_gaussian(t, [0.05] * 3, [1, 0, 0, 0])
    rec = oracle.preprocess(sc, synth.identity_viewmats(1), W, H)[0]
    fields = [oracle.R_PX, oracle.R_PY, oracle.R_COV00, oracle.R_COV01, oracle.R_COV11, oracle.R_C0, oracle.R_C1,
              oracle.R_C2, oracle.R_RX, oracle.R_RY]
    assert np.isfinite(rec[fields]).all()
    assert rec[oracle.R_PY] == H


def test_quaternion_matches_scipy(oracle_lib):
    for _ in range(100):
        q = RNG.normal(size=4) * RNG.uniform(0.1, 3)
        R = oracle.quat_to_rot(q)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy is scalar-last
        np.testing.assert_allclose(R, ref, atol=1e-12)


# ------------------------------------------------------------------ SH (Sec. 3.1)

def _sphere_quadrature(n_theta=40, n_phi=80):
    x, w = np.polynomial.legendre.leggauss(n_theta)  # x = cos(theta)
    phi = np.arange(n_phi) * 2 * np.pi / n_phi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=-1).reshape(-1, 3)
    weights = (w[:, None] * np.full(n_phi, 2 * np.pi / n_phi)[None, :]).reshape(-1)
    return dirs, weights


def test_sh_orthonormal(oracle_lib):
    dirs, wts = _sphere_quadrature()
    Y = np.array([oracle.sh_basis(3, d)[0] for d in dirs])
    gram = (Y * wts[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-10)


def test_sh_matches_scipy_real_form(oracle_lib):
    from scipy.special import sph_harm_y
    for _ in range(50):
        d = RNG.normal(size=3)
        d /= np.linalg.norm(d)
        theta, phi = np.arccos(d[2]), np.arctan2(d[1], d[0])
        Y = oracle.sh_basis(3, d)[0]
        k = 0
        for l in range(4):
            for m in range(-l, l + 1):
                c = sph_harm_y(l, abs(m), theta, phi)  # includes the Condon-Shortley phase
                if m < 0:
                    ref = np.sqrt(2) * (-1) ** m * c.imag
                elif m == 0:
                    ref = c.real
                else:
                    ref = np.sqrt(2) * (-1) ** m * c.real
                assert abs(Y[k] - ref) < 1e-12, (l, m)
                k += 1


def test_sh_gradient_matches_finite_differences(oracle_lib):
    for _ in range(20):
        d = RNG.normal(size=3)
        d /= np.linalg.norm(d)
        _, dY = oracle.sh_basis(3, d)
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-6
            fd = (oracle.sh_basis(3, d + e)[0] - oracle.sh_basis(3, d - e)[0]) / 2e-6
            np.testing.assert_allclose(dY[:, k], fd, atol=1e-8)


def test_sh_degree0_colour_closed_form(oracle_lib):
    for dc in [(0.5, -0.2, 1.3), (-3.0, 0.0, 0.7)]:
        sc = _one_gaussian([0.3, -0.2, 2.0], [0.1] * 3, [1, 0, 0, 0], sh_dc=dc)
        rec = oracle.preprocess(sc, synth.identity_viewmats(1), 256, 128)[0]
        expect = np.maximum(0.5 + np.asarray(dc, np.float32).astype(np.float64) / (2 * np.sqrt(np.pi)), 0.0)
        np.testing.assert_allclose(rec[[oracle.R_RED, oracle.R_GREEN, oracle.R_BLUE]], expect, atol=1e-12)


def test_near_cull(oracle_lib):
    for d, culled in [(0.19, True), (0.21, False)]:
        sc = _one_gaussian(d * _direction(0.4, 0.2), [0.01] * 3, [1, 0, 0, 0])
        rec = oracle.preprocess(sc, synth.identity_viewmats(1), 256, 128, near=0.2)[0]
        assert (rec[oracle.R_RADIUS] == 0) == culled


# ------------------------------------------------------------------ binning and sort (Sec. 3.3)

def _brute_force_lists(sp, V, W, H, T):
    """For every tile, the Gaussians whose pixel box (half-extents rx, ry around floor(p), columns taken modulo W,
    rows clipped to the image) touches one of its pixels, ordered by (t_r, index)."""
    TX, TY = W // T, H // T
    lists = [[] for _ in range(V * TX * TY)]
    n = len(sp["px"]) // V
    for i in range(V * n):
        rx, ry = int(sp["rx"][i]), int(sp["ry"][i])
        if rx <= 0:
            continue
        v = i // n
        ix, iy = int(np.floor(sp["px"][i])), int(np.floor(sp["py"][i]))
        cols = {((c % W) // T) for c in range(ix - rx, ix + rx + 1)}
        rows = {y // T for y in range(iy - ry, iy + ry + 1) if 0 <= y < H}
        for ty in rows:
            for tx in cols:
                lists[v * TX * TY + ty * TX + tx].append(i)
    for L in lists:
        L.sort(key=lambda i: (float(sp["depth"][i]), i))
    return lists


def _as_ranges(lists):
    """Per-tile lists -> (ranges [tiles, 2], concatenated list)."""
    sizes = np.array([len(L) for L in lists], np.int64)
    ranges = np.stack([np.cumsum(sizes) - sizes, np.cumsum(sizes)], 1)
    return ranges, np.array([i for L in lists for i in L], np.int64)


def test_bin_sort_matches_bruteforce(oracle_lib):
    """The tile lists are exactly the instance boxes' lists of a pixel-enumeration brute force (columns modulo W,
    rows clipped), ordered by (t_r, index) within every tile, including seam, pole and wider-than-image boxes and
    depth ties; the counting pass agrees with the list."""
    V, W, H, T = 2, 128, 64, 8
    sp = synth.random_splats(V, 150, W, H, seed=7, max_radius=20, wide_frac=0.05)
    ranges, lst = oracle.bin_sort(sp, V, W, H, T)
    ref_ranges, ref_list = _as_ranges(_brute_force_lists(sp, V, W, H, T))
    assert np.array_equal(ranges, ref_ranges) and np.array_equal(lst, ref_list)
    assert oracle.count_instances(sp, V, W, H, T) == len(lst)
    # a tile mask keeps the masked tiles' lists unchanged and empties the rest
    mask = np.random.default_rng(2).uniform(size=len(ranges)) < 0.3
    mr, ml = oracle.bin_sort(sp, V, W, H, T, tile_mask=mask)
    for t in range(len(ranges)):
        got = ml[mr[t, 0]:mr[t, 1]]
        assert np.array_equal(got, lst[ranges[t, 0]:ranges[t, 1]] if mask[t] else got[:0])


def test_rect_cases(oracle_lib):
    W, H, T = 128, 64, 16
    # plain: p = (40.5, 30.2), r = 5 -> pixels 35..45 -> tile columns 2; rows 25..35 -> tile rows 1..2
    assert oracle.rect(40.5, 30.2, 5, 5, W, H, T) == (2, 1, 1, 2)
    # across the seam: p_x = 1.2, r = 4 -> pixel columns -3..5 -> tile columns -1..0, i.e. 7 then 0
    assert oracle.rect(1.2, 30.0, 4, 4, W, H, T) == (-1, 2, 1, 2)
    # wider than the image: every column exactly once, starting at 0
    assert oracle.rect(60.0, 30.0, 70, 70, W, H, T) == (0, 8, 0, 4)
    # pole rows clipped: pixel rows -20..20 -> tile rows 0..1; columns 40..80 -> tiles 2..5
    assert oracle.rect(60.0, 0.3, 20, 20, W, H, T) == (2, 4, 0, 2)
    # anisotropic box: columns from rx = 20 (40..80 -> tiles 2..5), rows from ry = 2 (28..32 -> tiles 1..2)
    assert oracle.rect(60.0, 30.0, 20, 2, W, H, T) == (2, 4, 1, 2)
    assert oracle.rect(60.0, 30.0, 2, 20, W, H, T) == (3, 1, 0, 4)


# ------------------------------------------------------------------ blending (Eqs. 6-8)

def _brute_force_blend(sp, V, W, H, bg):
    """Every Gaussian for every pixel, ordered by (t_r, index), same skip / clamp / stop rules; no tiles."""
    n = len(sp["px"]) // V
    out = np.zeros((V, 3, H, W))
    Tout = np.zeros((V, H, W))
    for v in range(V):
        idx = [v * n + g for g in range(n) if sp["rx"][v * n + g] > 0]
        idx.sort(key=lambda i: (float(sp["depth"][i]), i))
        for y in range(H):
            for x in range(W):
                T, C, Ts = 1.0, np.zeros(3), [1.0]
                for i in idx:
                    dx = sp["px"][i] - (x + 0.5)
                    dy = sp["py"][i] - (y + 0.5)
                    if dx >= W / 2:
                        dx -= W
                    elif dx < -W / 2:
                        dx += W
                    power = -0.5 * (sp["c0"][i] * dx * dx + sp["c2"][i] * dy * dy) - sp["c1"][i] * dx * dy
                    if power > 0:
                        continue
                    alpha = min(0.99, sp["opacity"][i] * np.exp(power))
                    if alpha < 1 / 255:
                        continue
                    Tn = T * (1 - alpha)
                    if Tn < 1e-4:
                        break
                    C += alpha * T * np.array([sp["r"][i], sp["g"][i], sp["b"][i]])
                    T = Tn
                    Ts.append(T)
                assert all(a >= b for a, b in zip(Ts, Ts[1:]))  # transmittance never increases
                out[v, :, y, x] = C + T * np.asarray(bg)
                Tout[v, y, x] = T
    return out, Tout


def test_blend_matches_bruteforce_projected_scene(oracle_lib):
    """Tiny scene through the whole oracle; opacity < 0.35 keeps alpha < 1/255 outside the 3-sigma square, so the
    tile lists lose nothing and the tiled result equals the all-Gaussians blend."""
    W, H, T = 64, 32, 8
    sc = synth.shell_scene(60, seed=3, r_min=0.8, r_max=3.0, log_scale_mean=-1.8)
    sc.opacity[:] = np.minimum(sc.opacity, 0.35)
    vm = synth.random_viewmats(2, 11)
    bg = (0.1, 0.2, 0.3)
    f = oracle.render(sc, vm, W, H, T, bg=bg)
    ref, Tref = _brute_force_blend(f["splats"], 2, W, H, bg)
    np.testing.assert_allclose(f["rgb"], ref, atol=1e-12)
    np.testing.assert_allclose(f["T"], Tref, atol=1e-12)
    assert (f["T"] <= 1).all() and (f["T"] > 0).all()


def test_blend_matches_bruteforce_random_splats(oracle_lib):
    V, W, H, T = 1, 64, 32, 8
    sp = synth.random_splats(V, 80, W, H, seed=5, max_radius=12, opacity_range=(0.05, 0.35), wide_frac=0.05)
    sp64 = _to64(sp)
    # random_splats keeps the 3-sigma ellipse inside the instance box, and alpha < 1/255 beyond 3 sigma here
    ranges, lst = oracle.bin_sort(sp64, V, W, H, T)
    rgb, Tf, nc, near = oracle.blend_fwd(sp64, ranges, lst, V, W, H, T)
    ref, Tref = _brute_force_blend(sp64, V, W, H, (0, 0, 0))
    np.testing.assert_allclose(rgb, ref, atol=1e-12)
    np.testing.assert_allclose(Tf, Tref, atol=1e-12)


def test_instance_box_holds_every_visible_pixel(oracle_lib):
    """Every pixel of the 3-sigma square where alpha >= 1/255 (FP64, brute force over the square) lies in the
    narrowed box (rx, ry), and the box is no more than one pixel wider than that region needs (Sec. 3.3 tiles)."""
    W, H = 256, 128
    sc = synth.shell_scene(400, seed=31, log_scale_mean=-2.5)
    sc.opacity[:] = np.random.default_rng(3).uniform(0.004, 1.0, sc.n).astype(np.float32)  # high opacities too
    rec = oracle.preprocess(sc, synth.random_viewmats(1, 6), W, H)
    sp = oracle.splats_from_records(rec)
    narrower = 0
    for i in np.nonzero(sp["rx"] > 0)[0]:
        r = int(sp["radius"][i])
        ix, iy = int(np.floor(sp["px"][i])), int(np.floor(sp["py"][i]))
        xs = np.arange(ix - r, ix + r + 1) + 0.5
        ys = np.arange(iy - r, iy + r + 1) + 0.5
        dx, dy = sp["px"][i] - xs[None, :], sp["py"][i] - ys[:, None]
        power = -0.5 * (sp["c0"][i] * dx * dx + sp["c2"][i] * dy * dy) - sp["c1"][i] * dx * dy
        vis = sp["opacity"][i] * np.exp(power) >= 1.0 / 255.0
        yy, xx = np.nonzero(vis)
        if len(xx):
            assert np.abs(xx - r).max() <= sp["rx"][i] and np.abs(yy - r).max() <= sp["ry"][i], i
        narrower += int(sp["rx"][i] < r or sp["ry"][i] < r)
    assert narrower > 100  # the narrowing is not vacuous


def test_instance_box_leaves_images_unchanged(oracle_lib):
    """Lists from the narrowed box and from the full 3-sigma square (every tile it touches, brute force) blend to
    identical images: every instance the box leaves out has alpha < 1/255 at every pixel of its tile."""
    W, H, T = 256, 128, 16
    sc = synth.shell_scene(1500, seed=32, log_scale_mean=-2.5)
    sc.opacity[:] = np.random.default_rng(4).uniform(0.004, 1.0, sc.n).astype(np.float32)
    vm = synth.random_viewmats(2, 7)
    f = oracle.render(sc, vm, W, H, T)
    square = dict(f["splats"], rx=f["splats"]["radius"], ry=f["splats"]["radius"])
    ranges, lst = _as_ranges(_brute_force_lists(square, 2, W, H, T))
    assert len(lst) > 1.3 * len(f["list"])  # the square lists are substantially longer
    rgb, Tf, nc, _ = oracle.blend_fwd(square, ranges, lst, 2, W, H, T)
    count_square = oracle.blend_fwd.last_count
    oracle.blend_fwd(f["splats"], f["ranges"], f["list"], 2, W, H, T)
    assert np.array_equal(rgb, f["rgb"]) and np.array_equal(Tf, f["T"])
    assert np.array_equal(count_square, oracle.blend_fwd.last_count)


def test_opacity_below_one_255th_has_no_instance(oracle_lib):
    for o, culled in [(0.0035, True), (0.0040, False)]:
        sc = _one_gaussian([0, 0, 3.0], [0.05] * 3, [1, 0, 0, 0], opacity=o)
        rec = oracle.preprocess(sc, synth.identity_viewmats(1), 256, 128)[0]
        assert (rec[oracle.R_RX] == 0) == culled and (rec[oracle.R_FLAGS] == 1) == culled


def _stack(n_layers, opacity, W=32, H=16, x=5, y=7):
    """`n_layers` identical splats centred exactly on pixel (x, y), at increasing depth."""
    m = n_layers
    return dict(px=np.full(m, x + 0.5), py=np.full(m, y + 0.5), c0=np.full(m, 0.5), c1=np.zeros(m), c2=np.full(m, 0.5),
                opacity=np.full(m, opacity), r=np.linspace(0.1, 0.9, m), g=np.full(m, 0.5), b=np.full(m, 1.0),
                depth=np.arange(1, m + 1, dtype=np.float64), rx=np.full(m, 3, np.int32), ry=np.full(m, 3, np.int32))


def test_termination_closed_form(oracle_lib):
    """alpha = 0.8 at the centre: T = 0.2^k; the 6th layer would give 6.4e-5 < 1e-4 and is not added."""
    W, H, T = 32, 16, 8
    sp = _stack(9, 0.8, W, H)
    ranges, lst = oracle.bin_sort(sp, 1, W, H, T)
    bg = np.array([0.3, 0.6, 0.9])
    rgb, Tf, nc, _ = oracle.blend_fwd(sp, ranges, lst, 1, W, H, T, bg=bg)
    cols = np.stack([sp["r"], sp["g"], sp["b"]], 1)
    expect = sum(0.8 * 0.2 ** k * cols[k] for k in range(5)) + 0.2 ** 5 * bg
    np.testing.assert_allclose(rgb[0, :, 7, 5], expect, atol=1e-14)
    assert abs(Tf[0, 7, 5] - 0.2 ** 5) < 1e-15
    assert nc[0, 7, 5] == 5
    # alpha clamp: opacity 1 gives alpha = 0.99 (T = 0.01), then 0.5 (T = 0.005); the third layer (0.99 again)
    # would leave 5e-5 < 1e-4 and stops the pixel
    sp = _stack(3, 1.0, W, H)
    sp["opacity"][1] = 0.5
    ranges, lst = oracle.bin_sort(sp, 1, W, H, T)
    rgb, Tf, nc, _ = oracle.blend_fwd(sp, ranges, lst, 1, W, H, T)
    assert abs(Tf[0, 7, 5] - 0.005) < 1e-15 and nc[0, 7, 5] == 2
    np.testing.assert_allclose(rgb[0, :, 7, 5], 0.99 * np.array([sp["r"][0], 0.5, 1.0])
                               + 0.01 * 0.5 * np.array([sp["r"][1], 0.5, 1.0]), atol=1e-14)


def test_near_threshold_flag_widens_with_cancelling_exponent_terms(oracle_lib):
    """alpha = (1 + 5e-5) / 255 at pixel (100, 60) from a splat 50 px away along the diagonal: with a diagonal conic
    (c1 = 0, exponent terms of magnitude 5) the pixel is not flagged (5e-5 > 1e-5); with a sheared conic whose terms
    (about 1000 in magnitude) cancel to the same exponent -5, single precision cannot place alpha within 5e-5 of
    1/255, and the pixel is flagged."""
    W, H, T = 256, 128, 16
    d = 50.0
    flags = []
    for c, c1 in [(0.002, 0.0), (0.2, -0.2 * 0.99)]:
        power = -0.5 * d * d * (2 * c + 2 * c1)
        assert abs(power + 5.0) < 1e-12
        o = (1 + 5e-5) / 255 * np.exp(5.0)
        sp = dict(px=np.array([100.5 + d]), py=np.array([60.5 + d]), c0=np.array([c]), c1=np.array([c1]),
                  c2=np.array([c]), opacity=np.array([o]), r=np.ones(1), g=np.ones(1), b=np.ones(1),
                  depth=np.ones(1), rx=np.array([60], np.int32), ry=np.array([60], np.int32))
        ranges, lst = oracle.bin_sort(sp, 1, W, H, T)
        _, _, _, near = oracle.blend_fwd(sp, ranges, lst, 1, W, H, T, eps=1e-5)
        flags.append(int(near[0, 60, 100] & 1))
    assert flags == [0, 1]


def test_yaw_equals_cyclic_column_shift(oracle_lib):
    """Yawing the camera by 2 pi k / W about its y axis shifts longitude by a constant, so the image rolls by k
    columns (Eqs. 3-5); with k a multiple of the tile size the tile lists roll with it."""
    W, H, T = 128, 64, 16
    sc = synth.shell_scene(300, seed=9, log_scale_mean=-2.0)
    base = oracle.render(sc, synth.identity_viewmats(1), W, H, T)["rgb"]
    for k in (16, 48, -32):
        a = 2 * np.pi * k / W
        c, s = np.cos(a), np.sin(a)
        vm = np.eye(4)
        vm[:3, :3] = [[c, 0, s], [0, 1, 0], [-s, 0, c]]
        img = oracle.render(sc, vm[None].astype(np.float32), W, H, T)["rgb"]
        # the float32 pose rounds cos/sin; the shift is exact up to that rounding
        np.testing.assert_allclose(img, np.roll(base, k, axis=-1), atol=5e-5)


# ------------------------------------------------------------------ gradients (Eqs. 18-20)

def _decisions(f):
    return (f["n_contrib"].copy(), f["rec"][:, [oracle.R_RADIUS, oracle.R_RX, oracle.R_RY]].copy(), f["list"].copy())


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def _clamping_splats(n, W, H, seed):
    """Broad splats (sigma = 10 px) near pixel centres with opacity in (0.992, 1): o G exceeds 0.99 on the
    pixels nearest each centre, so alpha sits on its 0.99 clamp there."""
    rng = np.random.default_rng(seed)
    return dict(px=rng.integers(0, W, n) + 0.5 + rng.uniform(-0.05, 0.05, n),
                py=rng.integers(0, H, n) + 0.5 + rng.uniform(-0.05, 0.05, n),
                c0=np.full(n, 0.01), c1=np.zeros(n), c2=np.full(n, 0.01), opacity=rng.uniform(0.992, 1.0, n),
                r=rng.uniform(size=n), g=rng.uniform(size=n), b=rng.uniform(size=n),
                depth=rng.uniform(1, 5, n), rx=np.full(n, 30, np.int32), ry=np.full(n, 30, np.int32))


@pytest.mark.parametrize("case", ["random", "clamped"])
def test_blend_bwd_matches_finite_differences(oracle_lib, case):
    """Stage-level FD; the second case puts alpha on the 0.99 clamp, where its derivative is zero."""
    V, W, H, T = 1, 48, 24, 8
    if case == "random":
        sp = synth.random_splats(V, 30, W, H, seed=21, max_radius=10, wide_frac=0.0, cull_frac=0.0)
    else:
        sp = _clamping_splats(6, W, H, 21)
    sp = _to64(sp)
    ranges, lst = oracle.bin_sort(sp, V, W, H, T)
    wgt = synth.random_image_grad(V, W, H, 4).astype(np.float64)
    bg = (0.2, 0.1, 0.4)
    g = oracle.blend_bwd(sp, ranges, lst, wgt, V, W, H, T, bg)
    fields = ["px", "py", "c0", "c1", "c2", "opacity", "r", "g", "b"]

    def loss(s):
        rgb, _, nc, _ = oracle.blend_fwd(s, ranges, lst, V, W, H, T, bg)
        return float((rgb * wgt).sum()), nc

    _, nc0 = loss(sp)
    checked = skipped = 0
    for j, fld in enumerate(fields):
        for i in range(len(sp["px"])):
            h = 1e-6 * max(1.0, abs(sp[fld][i]))
            sp_p = {k: v.copy() for k, v in sp.items()}
            sp_m = {k: v.copy() for k, v in sp.items()}
            sp_p[fld][i] += h
            sp_m[fld][i] -= h
            lp, ncp = loss(sp_p)
            lm, ncm = loss(sp_m)
            if not (np.array_equal(ncp, nc0) and np.array_equal(ncm, nc0)):
                skipped += 1
                continue
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[i, j]) <= 1e-6 * max(1.0, abs(fd)), (fld, i, fd, g[i, j])
            checked += 1
    assert checked >= 50 and skipped < 0.05 * checked


def test_screen_gradient_matches_finite_differences(oracle_lib):
    """dL/ds (Sec. 4's densification signal), s the screen coordinates of Eq. 4 with p = (s + 1) (W, H) / 2, summed
    over the views: moving s_x by h in every view moves p_x by h W / 2 there (and s_y, p_y by h H / 2). Central
    differences of the blend on a W != H image, the lists held fixed."""
    V, W, H, T = 2, 64, 32, 8
    sc = synth.shell_scene(60, seed=3)
    vm = synth.random_viewmats(V, 7)
    wgt = synth.random_image_grad(V, W, H, 11).astype(np.float64)
    f0 = oracle.render(sc, vm, W, H, T)
    g = oracle.render_grad(sc, vm, wgt, W, H, T, fwd=f0)
    sp, n = f0["splats"], sc.n

    def loss(s):
        rgb, _, nc, _ = oracle.blend_fwd(s, f0["ranges"], f0["list"], V, W, H, T)
        return float((rgb * wgt).sum()), nc

    checked = 0
    for gi in range(n):
        for axis, fld, half in ((0, "px", W / 2), (1, "py", H / 2)):
            h = 1e-7
            sp_p = {k: v.copy() for k, v in sp.items()}
            sp_m = {k: v.copy() for k, v in sp.items()}
            for v in range(V):
                sp_p[fld][v * n + gi] += h * half
                sp_m[fld][v * n + gi] -= h * half
            lp, ncp = loss(sp_p)
            lm, ncm = loss(sp_m)
            if not (np.array_equal(ncp, f0["n_contrib"]) and np.array_equal(ncm, f0["n_contrib"])):
                continue
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g["screen"][gi, axis]) <= 1e-5 * max(1.0, abs(fd)), (gi, fld, fd, g["screen"][gi, axis])
            checked += fd != 0.0
    assert checked >= 20


def test_preprocess_bwd_matches_finite_differences(oracle_lib):
    """Linear functional of the projected fields (p, conic, opacity, colour) over 2 views."""
    W, H = 256, 128
    sc = synth.shell_scene(12, seed=5, log_scale_mean=-1.5)
    vm = synth.random_viewmats(2, 3)
    rec0 = oracle.preprocess(sc, vm, W, H)
    wts = np.random.default_rng(8).normal(size=(rec0.shape[0], 9))
    cols = oracle.SPLAT_COLS
    alive = rec0[:, oracle.R_RX] > 0
    wts[~alive] = 0.0
    grads = oracle.preprocess_bwd(sc, vm, wts, W, H)

    for field, shape in [("means", (12, 3)), ("scales", (12, 3)), ("quats", (12, 4)), ("opacity", (12,)),
                         ("sh", (12, 16, 3))]:
        g = grads[field]
        for idx in np.ndindex(*shape):
            base = float(getattr(sc, field)[idx])
            h = 1e-4 * (abs(base) if field == "scales" else max(1.0, abs(base)))
            lp, hp = _loss_moved(sc, vm, W, H, field, idx, h, cols, wts)
            lm, hm = _loss_moved(sc, vm, W, H, field, idx, -h, cols, wts)
            fd = (lp - lm) / (hp - hm)
            assert abs(fd - g[idx]) <= 2e-5 * max(1.0, abs(fd)) + 1e-6 * np.abs(g).max(), (field, idx, fd, g[idx])


def _loss_moved(sc, vm, W, H, field, idx, h, cols, wts):
    """Loss with one parameter moved by about h. The oracle reads float32 inputs, so the move is applied to a
    float32 copy; the step actually taken (after float32 rounding) is returned with the loss."""
    s = sc.subset(slice(None))
    arr = getattr(s, field)
    old = float(arr[idx])
    arr[idx] = np.float32(old + h)
    rec = oracle.preprocess(s, vm, W, H)
    return float((rec[:, cols] * wts).sum()), float(arr[idx]) - old


def test_render_grad_matches_finite_differences(oracle_lib):
    """End to end: 64 Gaussians, 64x32 image, 2 views, L = sum(w * C). Components whose +-h evaluations change a
    discrete decision (a radius, a tile list, the contributor count of a pixel) are excluded and counted."""
    W, H, T = 64, 32, 16
    sc = synth.shell_scene(64, seed=17, r_min=1.0, r_max=4.0, log_scale_mean=-1.7)
    vm = synth.random_viewmats(2, 23)
    wgt = synth.random_image_grad(2, W, H, 29).astype(np.float64)
    f0 = oracle.render(sc, vm, W, H, T)
    g = oracle.render_grad(sc, vm, wgt, W, H, T, fwd=f0)
    d0 = _decisions(f0)
    rng = np.random.default_rng(0)
    checked = skipped = 0
    worst = 0.0
    for field in ["means", "scales", "quats", "opacity", "sh"]:
        arr = getattr(sc, field)
        idxs = list(np.ndindex(*arr.shape))
        if field == "sh":
            idxs = [idxs[i] for i in rng.choice(len(idxs), 400, replace=False)]
        gmax = np.abs(g[field]).max()
        for idx in idxs:
            vals = []
            ok = True
            for sgn in (1, -1):
                s = sc.subset(slice(None))
                a = getattr(s, field)
                old = float(a[idx])
                h = 1e-5 * (abs(old) if field == "scales" else max(1.0, abs(old)))
                a[idx] = np.float32(old + sgn * h)
                f = oracle.render(s, vm, W, H, T)
                ok &= _same(_decisions(f), d0)
                vals.append((float((f["rgb"] * wgt).sum()), float(a[idx]) - old))
            if not ok:
                skipped += 1
                continue
            fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
            err = abs(fd - g[field][idx])
            worst = max(worst, err / max(gmax, 1e-30))
            assert err <= 1e-4 * max(abs(fd), 1e-3 * gmax), (field, idx, fd, g[field][idx])
            checked += 1
    assert checked > 600 and skipped < 0.1 * checked, (checked, skipped)
