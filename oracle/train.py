"""FP64 oracle of the reconstruction loop's per-iteration bookkeeping (Sec. 4, Algorithm 1), for tests only.

TEST INFRASTRUCTURE: only the test-suite and the benchmark's CPU-baseline leg use this module; the product path
never does. It shares no code with the CUDA sources.

Algorithm 1 densifies by dL/ds, prunes by opacity and by scale, resets large opacities periodically and advances the
optimizer every iteration. The thresholds live in the paper's missing supplement; the readings below follow the 3DGS
conventions the paper says it is similar to:
  * parameters are optimised in raw form: means, log-scales, quaternions (normalised only when used), logit-opacities
    and SH coefficients; rendering sees scales = exp(log-scale) and opacity = sigmoid(logit);
  * Adam (beta1 0.9, beta2 0.999, eps 1e-15) with bias correction, one learning rate per group (means, scales,
    quaternions, opacity, SH band 0, SH bands >= 1);
  * statistics between densifications: for every view in which a Gaussian has tile instances, the norm of its
    screen-space gradient |dL/ds| (s the Eq. 4 coordinates, dL/ds = dL/dp diag(W/2, H/2)) is added to an
    accumulator and a visibility count is incremented; the largest instance half-extent max(rx, ry) seen is kept;
  * densify: a Gaussian whose mean |dL/ds| (accumulator / count) reaches grad_threshold is cloned if its largest
    scale is at most percent_dense * extent, and split into two otherwise. A split child has mean m + R(q) (S z)
    for a standard normal z (given), scales S / 1.6 and the parent's rotation, opacity and SH; the parent is removed;
  * prune: a Gaussian (original, clone or child) goes when its opacity is below min_opacity or its largest scale
    exceeds max_scale_frac * extent; an original also goes when its largest instance half-extent exceeded
    max_screen_radius (clones and children have not been rendered yet);
  * output order: for each original in index order, itself (if kept), then its clone, then its two children;
    Adam moments follow kept originals and are zero for new Gaussians;
  * opacity reset: logit(o) <- min(logit(o), logit(0.01)), with the opacity moments set to zero.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BETA1, BETA2, EPS = 0.9, 0.999, 1e-15


@dataclass
class AdamConfig:
    lr_means: float = 1.6e-4
    lr_scales: float = 5e-3
    lr_quats: float = 1e-3
    lr_opacity: float = 5e-2
    lr_sh_dc: float = 2.5e-3
    lr_sh_rest: float = 2.5e-3 / 20


@dataclass
class DensifyConfig:
    grad_threshold: float = 2e-4
    percent_dense: float = 0.01
    extent: float = 5.0
    min_opacity: float = 0.005
    max_scale_frac: float = 0.1
    max_screen_radius: float = 20.0


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def activated(raw: dict) -> dict:
    """The parameters the renderer sees."""
    return dict(means=raw["means"], scales=np.exp(raw["log_scales"]), quats=raw["quats"],
                opacity=sigmoid(raw["logit_opacity"]), sh=raw["sh"])


def raw_gradients(raw: dict, grads: dict) -> dict:
    """Chain rule from gradients with respect to the rendered parameters to the raw ones."""
    s = np.exp(raw["log_scales"])
    o = sigmoid(raw["logit_opacity"])
    return dict(means=grads["means"], log_scales=grads["scales"] * s, quats=grads["quats"],
                logit_opacity=grads["opacity"] * o * (1 - o), sh=grads["sh"])


def adam_step(raw: dict, grads: dict, m: dict, v: dict, step: int, cfg: AdamConfig):
    """One Adam step (step counts from 1) on the raw parameters; returns new (raw, m, v)."""
    g = raw_gradients(raw, grads)
    lrs = dict(means=cfg.lr_means, log_scales=cfg.lr_scales, quats=cfg.lr_quats, logit_opacity=cfg.lr_opacity)
    out, m2, v2 = {}, {}, {}
    for k in raw:
        mk = BETA1 * m[k] + (1 - BETA1) * g[k]
        vk = BETA2 * v[k] + (1 - BETA2) * g[k] ** 2
        mhat = mk / (1 - BETA1 ** step)
        vhat = vk / (1 - BETA2 ** step)
        if k == "sh":
            lr = np.full(raw[k].shape, cfg.lr_sh_rest)
            lr[:, 0, :] = cfg.lr_sh_dc
        else:
            lr = lrs[k]
        out[k] = raw[k] - lr * mhat / (np.sqrt(vhat) + EPS)
        m2[k], v2[k] = mk, vk
    return out, m2, v2


def densify_stats(rx, ry, grad_px, grad_py, W: int, H: int, V: int, n: int, accum, count, max_radius):
    """Adds one render's statistics (per-(view, Gaussian) instance box and 2D gradient, index v * n + g)."""
    accum, count, max_radius = accum.copy(), count.copy(), max_radius.copy()
    for v in range(V):
        for g in range(n):
            i = v * n + g
            if rx[i] <= 0:
                continue
            accum[g] += np.hypot(grad_px[i] * W / 2.0, grad_py[i] * H / 2.0)
            count[g] += 1
            max_radius[g] = max(max_radius[g], max(rx[i], ry[i]))
    return accum, count, max_radius


def quat_rotation(q) -> np.ndarray:
    q = np.asarray(q, np.float64)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def densify(raw: dict, m: dict, v: dict, accum, count, max_radius, normals, cfg: DensifyConfig):
    """Clone, split and prune (Algorithm 1). normals: [n, 2, 3] standard normal draws for the split children.
    Returns (raw, m, v, decisions) with decisions[g] = (clone, split, keep_original)."""
    n = raw["means"].shape[0]
    out = {k: [] for k in raw}
    mo = {k: [] for k in raw}
    vo = {k: [] for k in raw}
    decisions = []

    def emit(vals, moments):
        for k in raw:
            out[k].append(vals[k])
            mo[k].append(moments[0][k] if moments else np.zeros_like(vals[k]))
            vo[k].append(moments[1][k] if moments else np.zeros_like(vals[k]))

    def pruned(logit_o, log_s):
        o = sigmoid(logit_o)
        return o < cfg.min_opacity or np.exp(log_s).max() > cfg.max_scale_frac * cfg.extent

    for g in range(n):
        p = {k: raw[k][g] for k in raw}
        hot = count[g] > 0 and accum[g] / count[g] >= cfg.grad_threshold  # never seen: never hot
        big = np.exp(p["log_scales"]).max() > cfg.percent_dense * cfg.extent
        clone, split = hot and not big, hot and big
        keep = not split and not pruned(p["logit_opacity"], p["log_scales"]) and not (
            max_radius[g] > cfg.max_screen_radius)
        if keep:
            emit(p, ({k: m[k][g] for k in raw}, {k: v[k][g] for k in raw}))
        if clone and not pruned(p["logit_opacity"], p["log_scales"]):
            emit(dict(p), None)
        if split:
            R = quat_rotation(p["quats"])
            s = np.exp(p["log_scales"])
            for c in range(2):
                child = dict(p)
                child["means"] = p["means"] + R @ (s * normals[g, c])
                child["log_scales"] = np.log(s / 1.6)
                if not pruned(child["logit_opacity"], child["log_scales"]):
                    emit(child, None)
        decisions.append((clone, split, keep))
    pack = lambda d: {k: (np.array(d[k]) if d[k] else np.zeros((0,) + raw[k].shape[1:])) for k in raw}  # noqa: E731
    return pack(out), pack(mo), pack(vo), decisions


def reset_opacity(raw: dict, m: dict, v: dict, value: float = 0.01):
    cap = np.log(value / (1 - value))
    raw = dict(raw, logit_opacity=np.minimum(raw["logit_opacity"], cap))
    m = dict(m, logit_opacity=np.zeros_like(m["logit_opacity"]))
    v = dict(v, logit_opacity=np.zeros_like(v["logit_opacity"]))
    return raw, m, v
