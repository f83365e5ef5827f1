"""Pins of the reconstruction-loop bookkeeping oracle (Sec. 4, Algorithm 1): Adam, densification statistics,
clone / split / prune, opacity reset. CPU only."""
import numpy as np
from scipy.spatial.transform import Rotation

from oracle import train as T

RNG = np.random.default_rng(21)


def _raw(n, K=4, seed=0):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=(n, 4))
    return dict(means=rng.normal(size=(n, 3)), log_scales=rng.normal(-3, 0.5, size=(n, 3)), quats=q,
                logit_opacity=rng.normal(size=n), sh=rng.normal(size=(n, K, 3)))


def _zeros(raw):
    return {k: np.zeros_like(v) for k, v in raw.items()}


def test_adam_with_a_constant_gradient_moves_by_the_learning_rate():
    """With bias correction, a constant gradient gives m_hat = g and v_hat = g^2: every step is -lr sign(g)."""
    raw = _raw(5)
    grads = {k: np.full_like(v, 0.3) for k, v in T.activated(raw).items()}
    grads["means"][:] = -2.0
    cfg = T.AdamConfig()
    m, v = _zeros(raw), _zeros(raw)
    cur = raw
    for step in range(1, 6):
        cur, m, v = T.adam_step(cur, grads, m, v, step, cfg)
    # means: gradient -2 everywhere -> moved by +5 lr
    np.testing.assert_allclose(cur["means"] - raw["means"], 5 * cfg.lr_means, rtol=1e-9)
    # SH band 0 and bands >= 1 use their own rates
    np.testing.assert_allclose(cur["sh"][:, 0] - raw["sh"][:, 0], -5 * cfg.lr_sh_dc, rtol=1e-9)
    np.testing.assert_allclose(cur["sh"][:, 1:] - raw["sh"][:, 1:], -5 * cfg.lr_sh_rest, rtol=1e-9)


def test_adam_first_step_is_the_sign_and_zero_gradient_is_still():
    raw = _raw(4)
    g = {k: RNG.normal(size=v.shape) for k, v in T.activated(raw).items()}
    g["quats"][:] = 0.0
    cfg = T.AdamConfig()
    new, m, v = T.adam_step(raw, g, _zeros(raw), _zeros(raw), 1, cfg)
    rg = T.raw_gradients(raw, g)
    np.testing.assert_allclose(new["log_scales"], raw["log_scales"] - cfg.lr_scales * np.sign(rg["log_scales"]),
                               rtol=1e-9)
    assert np.array_equal(new["quats"], raw["quats"])


def test_raw_gradients_match_finite_differences_of_the_activations():
    raw = _raw(3)
    w = {k: RNG.normal(size=v.shape) for k, v in T.activated(raw).items()}  # L = sum(w * activated)
    g = T.raw_gradients(raw, w)
    h = 1e-6
    for key, act in (("log_scales", "scales"), ("logit_opacity", "opacity")):
        for idx in np.ndindex(*raw[key].shape):
            p, mm = {k: v.copy() for k, v in raw.items()}, {k: v.copy() for k, v in raw.items()}
            p[key][idx] += h
            mm[key][idx] -= h
            fd = ((T.activated(p)[act] * w[act]).sum() - (T.activated(mm)[act] * w[act]).sum()) / (2 * h)
            assert abs(fd - g[key][idx]) < 1e-7 * max(1, abs(fd))


def test_densify_statistics_by_hand():
    V, n, W, H = 2, 3, 200, 100
    rx = np.array([2, 0, 5, 1, 4, 0], np.int32)
    ry = np.array([3, 0, 1, 1, 7, 0], np.int32)
    gx = np.array([0.1, 9.0, 0.0, 0.2, -0.3, 9.0])
    gy = np.array([0.0, 9.0, 0.4, 0.0, 0.1, 9.0])
    acc, cnt, mr = T.densify_stats(rx, ry, gx, gy, W, H, V, n, np.zeros(n), np.zeros(n, np.int64), np.zeros(n))
    # Gaussian 0: views 0 (|(0.1 * 100, 0)| = 10) and 1 (|(0.2 * 100, 0)| = 20)
    assert acc[0] == 30.0 and cnt[0] == 2 and mr[0] == 3
    # Gaussian 1: view 1 only (view 0 has no instance): |(-0.3 * 100, 0.1 * 50)|
    assert abs(acc[1] - np.hypot(30.0, 5.0)) < 1e-12 and cnt[1] == 1 and mr[1] == 7
    # Gaussian 2: view 0 only: |(0, 0.4 * 50)| = 20
    assert acc[2] == 20.0 and cnt[2] == 1 and mr[2] == 5


def _stats(n, hot):
    acc = np.where(hot, 1.0, 0.0)
    return acc, np.ones(n, np.int64), np.zeros(n)


def test_clone_split_and_prune_cases():
    cfg = T.DensifyConfig(grad_threshold=0.5, percent_dense=0.01, extent=10.0, min_opacity=0.01,
                          max_scale_frac=0.1, max_screen_radius=20)
    raw = _raw(6, seed=3)
    raw["log_scales"][:] = np.log(0.05)                  # <= 0.1 = percent_dense * extent: clone size
    raw["log_scales"][1] = np.log([0.5, 0.2, 0.3])       # > 0.1: split size
    raw["logit_opacity"][:] = 0.0                         # opacity 0.5
    raw["logit_opacity"][2] = np.log(0.005 / 0.995)       # opacity 0.005 < 0.01: pruned
    raw["log_scales"][3] = np.log([2.0, 0.1, 0.1])        # 2 > max_scale_frac * extent = 1: pruned
    hot = np.array([True, True, False, False, True, False])
    acc, cnt, mr = _stats(6, hot)
    mr[4] = 25.0                                          # screen radius too large: original pruned, clone kept
    m = {k: np.ones_like(v) for k, v in raw.items()}
    normals = RNG.normal(size=(6, 2, 3))
    out, mo, vo, dec = T.densify(raw, m, m, acc, cnt, mr, normals, cfg)
    assert dec == [(True, False, True), (False, True, False), (False, False, False), (False, False, False),
                   (True, False, False), (False, False, True)]
    # order: 0, clone of 0, children of 1 (x2), clone of 4, 5
    assert out["means"].shape[0] == 6
    np.testing.assert_array_equal(out["means"][[0, 1, 4, 5]], raw["means"][[0, 0, 4, 5]])
    assert np.all(mo["means"][0] == 1) and np.all(mo["means"][1] == 0) and np.all(mo["means"][5] == 1)
    # split children: m + R(q) (S z), scales S / 1.6; R from scipy (scalar-last quaternion)
    q = raw["quats"][1]
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    s = np.exp(raw["log_scales"][1])
    for c in range(2):
        np.testing.assert_allclose(out["means"][2 + c], raw["means"][1] + R @ (s * normals[1, c]), atol=1e-12)
        np.testing.assert_allclose(np.exp(out["log_scales"][2 + c]), s / 1.6, rtol=1e-12)
        np.testing.assert_array_equal(out["sh"][2 + c], raw["sh"][1])


def test_unseen_gaussians_are_never_hot():
    raw = _raw(2)
    acc = np.array([5.0, 5.0])
    cnt = np.array([0, 1])
    out, _, _, dec = T.densify(raw, _zeros(raw), _zeros(raw), acc, cnt, np.zeros(2), np.zeros((2, 2, 3)),
                               T.DensifyConfig(grad_threshold=1.0, extent=1e9))
    assert dec[0][:2] == (False, False) and (dec[1][0] or dec[1][1])


def test_opacity_reset_caps_at_one_percent():
    raw = _raw(50)
    raw["logit_opacity"][:] = np.linspace(-8, 8, 50)
    m = {k: np.ones_like(v) for k, v in raw.items()}
    new, m2, v2 = T.reset_opacity(raw, m, m)
    o = T.sigmoid(new["logit_opacity"])
    assert np.all(o <= 0.01 + 1e-15)
    small = T.sigmoid(raw["logit_opacity"]) < 0.01
    np.testing.assert_array_equal(new["logit_opacity"][small], raw["logit_opacity"][small])
    assert np.all(m2["logit_opacity"] == 0) and np.all(m2["means"] == 1)
