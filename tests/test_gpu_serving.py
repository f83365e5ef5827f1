"""Serving loop on the GPU: requests rendered in the mix of a continuously batched run equal the same requests
rendered alone (gpu)."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2404_03202_gb300 as og  # noqa: E402
from paper_2404_03202_gb300 import serving  # noqa: E402


def _scenes():
    return {"room3k": synth.room_scene(3000, 1), "shell5k": synth.shell_scene(5000, 2),
            "room8k": synth.room_scene(8000, 3)}


def _requests(scenes, n, rate, seed):
    rng = np.random.default_rng(seed)
    names = sorted(scenes)
    res = [(256, 128), (512, 256)]
    poses = synth.room_viewmats(n, seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    return [serving.Request(i, names[rng.integers(len(names))], poses[i], *res[rng.integers(2)], float(t[i]))
            for i in range(n)]


def test_results_identical_alone_and_in_the_mix():
    scenes = _scenes()
    arrays = {k: s.arrays() for k, s in scenes.items()}
    ex = serving.GpuExecutor(arrays, lanes=3)
    sch = serving.Scheduler(ex, lanes=3, max_batch=4)
    reqs = _requests(scenes, 48, 4000.0, 5)
    summary = serving.run_trace(sch, reqs)
    print("serving:", summary)
    assert summary["requests"] == len(reqs) and summary["rejected"] == 0
    assert summary["mean_batch"] > 1.0       # some requests shared a launch
    assert summary["max_in_flight"] > 1      # batches overlapped on the device
    for r in reqs:
        s = og.Settings(width=r.width, height=r.height, tile=16, num_views=1, sh_degree=scenes[r.scene].sh_degree)
        alone = og.Rasterizer(s)
        img = alone.forward(*[torch.from_numpy(a).cuda() for a in scenes[r.scene].arrays()],
                            torch.from_numpy(np.asarray(r.viewmat, np.float32)[None]).cuda())
        assert np.array_equal(img[0].cpu().numpy(), r.result), r.rid


def test_oversize_request_is_rejected_not_run():
    scenes = {"room3k": synth.room_scene(3000, 1).arrays()}
    ex = serving.GpuExecutor(scenes, lanes=1)
    sch = serving.Scheduler(ex, lanes=1, max_batch=2, mem_budget=1 << 20)  # 1 MiB: nothing 512x256 fits
    r = serving.Request(0, "room3k", np.eye(4, dtype=np.float32), 512, 256, 0.0)
    summary = serving.run_trace(sch, [r])
    assert summary["rejected"] == 1 and r.error and r.result is None


def test_reserved_arenas_serve_without_growing_and_close_stops_the_lanes():
    """reserve() sizes every lane's arena for the largest batch: a trace afterwards allocates no arena memory, its
    images equal those of an unreserved executor, and close() ends the waiter threads and frees the arenas."""
    scenes = _scenes()
    arrays = {k: s.arrays() for k, s in scenes.items()}
    res = [(256, 128), (512, 256)]
    ex = serving.GpuExecutor(arrays, lanes=2)
    nbytes = ex.reserve([(nm, wh) for nm in sorted(arrays) for wh in res], 4)
    bufs = [a.buf for a in ex.arenas]
    assert all(b is not None and b.numel() >= nbytes for b in bufs)
    reqs = _requests(scenes, 24, 4000.0, 7)
    serving.run_trace(serving.Scheduler(ex, lanes=2, max_batch=4), reqs)
    assert all(a.buf is b for a, b in zip(ex.arenas, bufs))  # no lane grew its arena
    ref = serving.GpuExecutor(arrays, lanes=1)
    again = _requests(scenes, 24, 4000.0, 7)
    serving.run_trace(serving.Scheduler(ref, lanes=1, max_batch=1), again)
    for a, b in zip(reqs, again):
        assert np.array_equal(a.result, b.result), a.rid
    for e in (ex, ref):
        e.close()
        assert not any(t.is_alive() for t in e._threads) and e.arenas == []


def test_per_lane_host_buffers_deliver_the_same_images():
    """host_buffers='per_lane': each lane reuses one pinned buffer; the images handed to on_result as requests
    complete equal those of the default per-batch buffers (one request at a time)."""
    scenes = _scenes()
    arrays = {k: s.arrays() for k, s in scenes.items()}
    res = [(256, 128), (512, 256)]
    ex = serving.GpuExecutor(arrays, lanes=3, host_buffers="per_lane")
    ex.reserve([(nm, wh) for nm in sorted(arrays) for wh in res], 4)
    got = {}
    sch = serving.Scheduler(ex, lanes=3, max_batch=4, keep_results=False,
                            on_result=lambda r, img: got.__setitem__(r.rid, np.array(img, copy=True)))
    reqs = _requests(scenes, 40, 4000.0, 11)
    summary = serving.run_trace(sch, reqs)
    assert summary["requests"] == len(reqs) and summary["rejected"] == 0 and len(got) == len(reqs)
    ref = serving.GpuExecutor(arrays, lanes=1)
    again = _requests(scenes, 40, 4000.0, 11)
    serving.run_trace(serving.Scheduler(ref, lanes=1, max_batch=1), again)
    for r in again:
        assert np.array_equal(got[r.rid], r.result), r.rid
    for e in (ex, ref):
        e.close()
