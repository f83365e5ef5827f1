"""Algorithm 1's bookkeeping on the GPU against the FP64 oracle (gpu): Adam, densification statistics,
clone / split / prune, opacity reset, and a short end-to-end training run."""
import numpy as np
import pytest
import torch

import synth
from oracle import train as OT
from tests.gpu_util import dev, pack_splats

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2404_03202_gb300 as og  # noqa: E402
from paper_2404_03202_gb300 import _cabi as C  # noqa: E402
from paper_2404_03202_gb300.trainer import GaussianModel, TrainConfig, Trainer, raw_rows  # noqa: E402

K = 16
P = 11 + 3 * K


def _split(rows):
    r = np.asarray(rows, np.float64)
    n = r.shape[0]
    return dict(means=r[:, 0:3], log_scales=r[:, 3:6], quats=r[:, 6:10], logit_opacity=r[:, 10],
                sh=r[:, 11:].reshape(n, K, 3))


def _join(d):
    n = d["means"].shape[0]
    return np.concatenate([d["means"], d["log_scales"], d["quats"], d["logit_opacity"][:, None],
                           d["sh"].reshape(n, -1)], axis=1)


def _rows(n, seed):
    sc = synth.shell_scene(n, seed)
    return raw_rows(*sc.arrays())


def test_adam_matches_oracle_over_three_steps():
    n = 3000
    rng = np.random.default_rng(1)
    rows = _rows(n, 2)
    params, m, v = dev(rows), torch.zeros((n, P), device="cuda"), torch.zeros((n, P), device="cuda")
    cfg = TrainConfig().adam(1.0)
    out = [torch.empty(s, device="cuda") for s in [(n, 3), (n, 3), (n, 4), (n,), (n, K, 3)]]
    ref, rm, rv = _split(rows), {k: np.zeros_like(x) for k, x in _split(rows).items()}, None
    rv = {k: np.zeros_like(x) for k, x in _split(rows).items()}
    ocfg = OT.AdamConfig(lr_means=cfg.lr_means, lr_scales=cfg.lr_scales, lr_quats=cfg.lr_quats,
                         lr_opacity=cfg.lr_opacity, lr_sh_dc=cfg.lr_sh_dc, lr_sh_rest=cfg.lr_sh_rest)
    for step in (1, 2, 3):
        g = [rng.normal(size=s).astype(np.float32) for s in [(n, 3), (n, 3), (n, 4), (n,), (n, K, 3)]]
        C.omnigs_adam_step(n, K, cfg, step, params, m, v, *[dev(x) for x in g], *out)
        ref, rm, rv = OT.adam_step(ref, dict(means=g[0], scales=g[1], quats=g[2], opacity=g[3], sh=g[4]), rm, rv,
                                   step, ocfg)
    torch.cuda.synchronize()
    got = params.cpu().numpy()
    exp = _join(ref)
    # FP32 against FP64: each step moves a value by at most its learning rate (<= 0.05)
    assert np.abs(got - exp).max() <= 1e-5
    np.testing.assert_allclose(out[1].cpu().numpy(), np.exp(ref["log_scales"]), rtol=1e-5)
    np.testing.assert_allclose(out[3].cpu().numpy(), OT.sigmoid(ref["logit_opacity"]), rtol=1e-5)
    np.testing.assert_allclose(m.cpu().numpy(), _join(rm), rtol=1e-5, atol=1e-7)


def test_densify_stats_match_oracle():
    V, n, W, H = 3, 2000, 256, 128
    sp = synth.random_splats(V, n, W, H, seed=4, max_radius=30)
    g = np.zeros((V * n, 12), np.float32)
    g[:, :2] = np.random.default_rng(5).normal(size=(V * n, 2)) * 1e-4
    s = og.Settings(width=W, height=H, num_views=V)
    r = og.Rasterizer(s)
    r._ensure(n, K)
    acc, cnt, mr = torch.zeros(n, device="cuda"), torch.zeros(n, dtype=torch.int32, device="cuda"), \
        torch.zeros(n, device="cuda")
    C.omnigs_densify_stats(r.cfg, n, dev(pack_splats(sp)), dev(g), acc, cnt, mr)
    C.omnigs_densify_stats(r.cfg, n, dev(pack_splats(sp)), dev(g), acc, cnt, mr)  # accumulates
    ea, ec, em = OT.densify_stats(sp["rx"], sp["ry"], g[:, 0], g[:, 1], W, H, V, n, np.zeros(n),
                                  np.zeros(n, np.int64), np.zeros(n))
    ea, ec, em = OT.densify_stats(sp["rx"], sp["ry"], g[:, 0], g[:, 1], W, H, V, n, ea, ec, em)
    np.testing.assert_allclose(acc.cpu().numpy(), ea, rtol=1e-5)
    assert np.array_equal(cnt.cpu().numpy(), ec) and np.array_equal(mr.cpu().numpy(), em)


def test_densify_and_prune_match_oracle():
    n = 4000
    rng = np.random.default_rng(6)
    rows = _rows(n, 7)
    rows[:, 3:6] = rng.normal(-3.4, 0.8, size=(n, 3))       # largest scales straddle the clone / split boundary
    rows[:, 10] = rng.normal(-2.0, 2.5, size=n)              # some opacities below the prune threshold
    m = rng.normal(size=(n, P)).astype(np.float32)
    v = rng.uniform(size=(n, P)).astype(np.float32)
    accum = rng.uniform(0, 4e-4, size=n).astype(np.float32)
    count = rng.integers(0, 3, size=n).astype(np.int32)
    max_radius = rng.integers(0, 40, size=n).astype(np.float32)
    normals = rng.normal(size=(n, 2, 3)).astype(np.float32)
    tc = TrainConfig()
    extent = 5.0
    out = [torch.empty((2 * n, P), device="cuda") for _ in range(3)]
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(C.omnigs_densify_workspace_size(n), dtype=torch.uint8, device="cuda")
    C.omnigs_densify(n, K, tc.densify(extent), dev(rows), dev(m), dev(v), dev(accum), dev(count), dev(max_radius),
                     dev(normals), *out, n_out, ws)
    k = int(n_out.item())
    ocfg = OT.DensifyConfig(grad_threshold=tc.grad_threshold, percent_dense=tc.percent_dense, extent=extent,
                            min_opacity=tc.min_opacity, max_scale_frac=tc.max_scale_frac,
                            max_screen_radius=tc.max_screen_radius)
    ro, mo, vo, dec = OT.densify(_split(rows), _split(m), _split(v), accum.astype(np.float64), count,
                                 max_radius.astype(np.float64), normals.astype(np.float64), ocfg)
    kinds = np.array(dec)
    print(f"densify: {n} -> {k} rows; clones {kinds[:, 0].sum()}, splits {kinds[:, 1].sum()}, "
          f"kept {kinds[:, 2].sum()}")
    assert kinds[:, 0].sum() > 30 and kinds[:, 1].sum() > 30 and (~kinds[:, 2]).sum() > 30
    assert k == ro["means"].shape[0]
    got = out[0][:k].cpu().numpy()
    np.testing.assert_allclose(got, _join(ro), rtol=1e-5, atol=1e-5)
    np.testing.assert_array_equal(out[1][:k].cpu().numpy(), _join(mo).astype(np.float32))


def test_opacity_reset_matches_oracle():
    n = 1000
    rows = _rows(n, 8)
    rows[:, 10] = np.linspace(-9, 9, n)
    params = dev(rows)
    m, v = torch.ones((n, P), device="cuda"), torch.ones((n, P), device="cuda")
    op = torch.empty(n, device="cuda")
    C.omnigs_reset_opacity(n, K, 0.01, params, m, v, op)
    ref, rm, _ = OT.reset_opacity(_split(rows), _split(np.ones((n, P))), _split(np.ones((n, P))))
    np.testing.assert_allclose(params.cpu().numpy(), _join(ref), rtol=1e-6, atol=1e-6)
    assert np.array_equal(m.cpu().numpy(), _join(rm))
    assert op.max().item() <= 0.01 + 1e-7


def test_short_training_run_reduces_the_loss_and_densifies():
    """Fit a perturbed room to renders of the original from 4 poses (Eq. 17 with D-SSIM): Adam steps lower the
    loss; one densification at the 90th percentile of the recorded mean |dL/ds| adds Gaussians, and training goes
    on from there."""
    W, H, V = 256, 128, 4
    truth = synth.room_scene(6000, 11)
    start = synth.perturbed_copy(truth, 12)
    vm = dev(synth.room_viewmats(V, 13))
    s = og.Settings(width=W, height=H, num_views=V, sh_degree=3)
    gt = og.Rasterizer(s).forward(*[dev(a) for a in truth.arrays()], vm).clone()
    cfg = TrainConfig(densify_from=10 ** 9, opacity_reset_interval=10 ** 9)
    tr = Trainer(GaussianModel.from_scene(start), s, cfg, extent=5.0)
    losses = [tr.step(vm, gt).item() for _ in range(60)]
    mdl = tr.model
    seen = mdl.count.cpu().numpy() > 0
    mean_grad = mdl.accum.cpu().numpy()[seen] / mdl.count.cpu().numpy()[seen]
    tr.cfg.grad_threshold = float(np.quantile(mean_grad, 0.9))
    n_before = mdl.n
    n_after = tr.densify_and_prune()
    losses += [tr.step(vm, gt).item() for _ in range(20)]
    print(f"training: loss {losses[0]:.4f} -> {losses[59]:.4f} -> {losses[-1]:.4f}, Gaussians {n_before} -> "
          f"{n_after}")
    assert losses[59] < 0.85 * losses[0]
    assert n_after > n_before
    # split children land up to a few scales away from their parent, so the loss first rises and then falls again
    assert all(np.isfinite(losses)) and losses[-1] < 0.8 * losses[60]
