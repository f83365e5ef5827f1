"""Double-buffered streamed steps (host inputs in, host results out, copies overlapped with compute) against the same
steps run one at a time (gpu)."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2404_03202_gb300 as og  # noqa: E402
from paper_2404_03202_gb300.streaming import StreamedSteps  # noqa: E402

W, H, V = 256, 128, 2


def _inputs(step):
    """Different parameters, poses and targets for every step."""
    sc = synth.shell_scene(3000, seed=100 + step, log_scale_mean=-2.5)
    vm = synth.random_viewmats(V, 200 + step, max_offset=0.2)
    tgt = np.random.default_rng(300 + step).uniform(0, 1, (V, 3, H, W)).astype(np.float32)
    return [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (*sc.arrays(), vm, tgt)]


@pytest.mark.parametrize("graph,fused", [(False, False), (True, False), (True, True)])
def test_streamed_steps_match_one_at_a_time(graph, fused):
    """With graph=True steps 0 and 1 run eagerly and are captured, steps 2-4 replay the slots' graphs on new inputs.
    fused: loss_fn=None, the L1 loss computed by the forward blend (omnigs_render_fwd_l1)."""
    steps = 5
    s = og.Settings(width=W, height=H, tile=16, num_views=V, sh_degree=3)
    ins = [_inputs(k) for k in range(steps)]
    r = og.Rasterizer(s, capacity=1 << 20, grow=False)
    st = StreamedSteps(r, None if fused else (lambda rr, t: rr.l1_loss(t)), graph=graph)
    outs = []
    for k in range(steps):
        n, K = ins[k][0].shape[0], ins[k][4].shape[1]
        o = {"means": (n, 3), "scales": (n, 3), "quats": (n, 4), "opacity": (n,), "sh": (n, K, 3), "screen": (n, 2),
             "loss": (1,)}
        outs.append({name: torch.empty(shape, dtype=torch.float32).pin_memory() for name, shape in o.items()})
    st.begin()
    for k in range(steps):
        st.submit(ins[k], outs[k])
    st.end()
    torch.cuda.synchronize()
    r.check()

    ref = og.Rasterizer(s, capacity=1 << 20, grow=False)
    for k in range(steps):
        dev = [t.cuda() for t in ins[k]]
        if fused:
            ref.forward(*dev[:6], l1_target=dev[6])
        else:
            ref.forward(*dev[:6])
            ref.l1_loss(dev[6])
        g = ref.backward()
        torch.cuda.synchronize()
        assert outs[k]["loss"].item() == ref.loss.item(), k  # the loss reduction is deterministic
        for name in og.Rasterizer.GRAD_NAMES:
            got, exp = outs[k][name].numpy(), g[name].cpu().numpy()
            scale = max(np.abs(exp).max(), 1e-30)
            assert np.abs(got - exp).max() <= 1e-5 * scale, (k, name)  # the adjoint's atomics reorder sums
    assert len({float(o["loss"].item()) for o in outs}) == steps  # every step saw its own inputs
    assert all(g is not None for g in st.graphs) == graph


def test_graph_mode_needs_a_fixed_capacity():
    s = og.Settings(width=W, height=H, tile=16, num_views=V, sh_degree=3)
    with pytest.raises(ValueError):
        StreamedSteps(og.Rasterizer(s), lambda rr, t: rr.l1_loss(t), graph=True)


def test_backward_into_caller_buffers():
    s = og.Settings(width=W, height=H, tile=16, num_views=V, sh_degree=3)
    dev = [t.cuda() for t in _inputs(0)]
    r = og.Rasterizer(s)
    r.forward(*dev[:6])
    r.l1_loss(dev[6])
    own = {k: v.clone() for k, v in r.backward().items()}
    out = {k: torch.full_like(v, float("nan")) for k, v in own.items()}
    got = r.backward(out=out)
    for k in og.Rasterizer.GRAD_NAMES:
        assert got[k] is out[k]
        np.testing.assert_allclose(out[k].cpu().numpy(), own[k].cpu().numpy(), rtol=1e-5, atol=1e-7 * float(own[k].abs().max()))
    with pytest.raises(ValueError):
        r.backward(out={**out, "means": torch.empty(3, device="cuda")})
