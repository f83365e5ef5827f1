"""Continuous-batching scheduler of the serving loop, on the CPU with a simulated device (no CUDA).

The fake executor "renders" a batch in a + b * views simulated seconds and returns, per request, an image that
encodes the request's id, so the tests can check batching, admission by memory, lane limits, ordering and that
every result reaches its own request.
"""
import importlib.util
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _serving():
    # loaded by path: the scheduler needs neither torch's CUDA nor the CUDA library
    spec = importlib.util.spec_from_file_location("omnigs_serving",
                                                  os.path.join(ROOT, "paper_2404_03202_gb300", "serving.py"))
    m = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = m  # dataclasses look their module up while the class is built
    spec.loader.exec_module(m)
    return m


S = _serving()


class SimClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-5)


class FakeExecutor:
    def __init__(self, clock, budget=10_000, base=0.002, per_view=0.001):
        self.clock, self.budget, self.base, self.per_view = clock, budget, base, per_view
        self.launched = []
        self.live_lanes = set()

    def memory_budget(self):
        return self.budget

    def bytes_needed(self, scene, w, h, v):
        return 100 + v * (w * h) // 100

    def launch(self, lane, requests):
        assert lane not in self.live_lanes
        self.live_lanes.add(lane)
        keys = {r.key for r in requests}
        assert len(keys) == 1
        t = self.clock()
        h = {"lane": lane, "end": t + self.base + self.per_view * len(requests), "reqs": requests}
        self.launched.append(h)
        return h

    def done(self, h):
        return self.clock() >= h["end"]

    def collect(self, h):
        self.live_lanes.discard(h["lane"])
        return [np.full((3, 1, 1), r.rid, np.float32) for r in h["reqs"]]


def _trace(n, rate, seed, scenes=("a", "b", "c"), res=((100, 50), (200, 100), (400, 200)), p=(0.3, 0.5, 0.2)):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    out = []
    for i in range(n):
        w, h = res[rng.choice(len(res), p=p)]
        out.append(S.Request(i, str(rng.choice(scenes)), np.eye(4, dtype=np.float32), w, h, float(t[i])))
    return out


def _run(reqs, lanes=3, max_batch=4, budget=10_000, **kw):
    clk = SimClock()
    ex = FakeExecutor(clk, budget=budget, **kw)
    sch = S.Scheduler(ex, lanes=lanes, max_batch=max_batch)
    summary = S.run_trace(sch, reqs, clock=clk, sleep=clk.sleep)
    return sch, ex, summary


def test_every_request_completes_with_its_own_image():
    reqs = _trace(300, 2000.0, 1)
    sch, ex, summary = _run(reqs)
    assert summary["requests"] == 300 and summary["rejected"] == 0
    for r in reqs:
        assert r.result is not None and r.result[0, 0, 0] == r.rid
        assert r.arrival <= r.admitted <= r.done
    assert summary["p50_ms"] <= summary["p99_ms"]


def test_delivered_images_are_dropped_when_results_are_not_kept():
    """keep_results=False: every request still completes (and is timed), but its image is not held."""
    reqs = _trace(100, 2000.0, 5)
    clk = SimClock()
    ex = FakeExecutor(clk, budget=10_000)
    sch = S.Scheduler(ex, lanes=3, max_batch=4, keep_results=False)
    summary = S.run_trace(sch, reqs, clock=clk, sleep=clk.sleep)
    assert summary["requests"] == 100 and summary["rejected"] == 0
    assert all(r.result is None and r.done is not None and r.arrival <= r.admitted <= r.done for r in reqs)


def test_results_reach_the_delivery_hook_and_per_lane_buffers_need_dropped_results():
    """on_result sees every request with its own image as it completes, also when results are not kept; an
    executor that reuses each lane's host buffer is refused by a scheduler that keeps results."""
    reqs = _trace(120, 2000.0, 9)
    clk = SimClock()
    ex = FakeExecutor(clk, budget=10_000)
    seen = {}
    sch = S.Scheduler(ex, lanes=3, max_batch=4, keep_results=False,
                      on_result=lambda r, img: seen.__setitem__(r.rid, float(img[0, 0, 0])))
    S.run_trace(sch, reqs, clock=clk, sleep=clk.sleep)
    assert seen == {r.rid: float(r.rid) for r in reqs} and all(r.result is None for r in reqs)
    ex.host_buffers = "per_lane"
    with pytest.raises(ValueError):
        S.Scheduler(ex, lanes=3, max_batch=4)
    S.Scheduler(ex, lanes=3, max_batch=4, keep_results=False)


def test_batches_hold_one_key_and_respect_lanes_and_memory():
    reqs = _trace(400, 5000.0, 2)
    sch, ex, summary = _run(reqs, lanes=3, max_batch=4, budget=2500)
    assert all(1 <= len(h["reqs"]) <= 4 for h in ex.launched)
    assert summary["max_in_flight"] <= 3
    assert summary["peak_reserved_bytes"] <= 2500
    # under this load requests queue up, so batches of several views form
    assert summary["mean_batch"] > 1.5


def test_arrivals_while_busy_join_later_batches():
    """Continuous batching: requests admitted while earlier batches are still running."""
    reqs = _trace(200, 3000.0, 3)
    sch, ex, summary = _run(reqs, lanes=2, max_batch=8)
    overlapped = 0
    for h in ex.launched:
        start = min(r.admitted for r in h["reqs"])
        overlapped += any(g is not h and min(q.admitted for q in g["reqs"]) < start < g["end"] for g in ex.launched)
    assert overlapped > 0
    assert summary["max_in_flight"] == 2


def test_fifo_with_one_lane_and_no_batching():
    reqs = _trace(60, 100.0, 4)
    sch, ex, summary = _run(reqs, lanes=1, max_batch=1)
    done = sorted(reqs, key=lambda r: r.done)
    assert [r.rid for r in done] == sorted(r.rid for r in reqs)


def test_oversize_request_rejected_and_others_served():
    reqs = _trace(20, 500.0, 5, res=((100, 50),), p=(1.0,))
    reqs.append(S.Request(99, "a", np.eye(4, dtype=np.float32), 4000, 2000, reqs[-1].arrival + 1e-3))
    sch, ex, summary = _run(reqs, budget=5000)
    assert summary["rejected"] == 1 and reqs[-1].error and reqs[-1].result is None
    assert summary["requests"] == 20


def test_younger_requests_backfill_memory_the_oldest_cannot_use():
    clk = SimClock()
    ex = FakeExecutor(clk, budget=900, base=0.05)
    sch = S.Scheduler(ex, lanes=3, max_batch=1, max_wait=1.0)
    eye = np.eye(4, dtype=np.float32)
    big1 = S.Request(0, "a", eye, 200, 200, 0.0)      # 500 bytes
    big2 = S.Request(1, "a", eye, 200, 200, 0.001)    # does not fit beside big1
    small = S.Request(2, "b", eye, 100, 100, 0.002)   # 200 bytes: fits
    S.run_trace(sch, [big1, big2, small], clock=clk, sleep=clk.sleep)
    assert small.admitted < big2.admitted
    assert big2.admitted >= big1.done


def test_max_wait_stops_backfill():
    clk = SimClock()
    ex = FakeExecutor(clk, budget=900, base=0.05)
    sch = S.Scheduler(ex, lanes=3, max_batch=1, max_wait=0.0)
    eye = np.eye(4, dtype=np.float32)
    big1 = S.Request(0, "a", eye, 200, 200, 0.0)
    big2 = S.Request(1, "a", eye, 200, 200, 0.001)
    small = S.Request(2, "b", eye, 100, 100, 0.002)
    S.run_trace(sch, [big1, big2, small], clock=clk, sleep=clk.sleep)
    assert small.admitted >= big2.admitted


def test_bad_scheduler_arguments():
    with pytest.raises(ValueError):
        S.Scheduler(FakeExecutor(SimClock()), lanes=0)


def test_lane_arena_carves_aligned_disjoint_buffers_and_falls_back_past_its_end():
    """The serving executor's per-lane arena (CPU tensors here): buffers in order, each at a 256-byte boundary,
    disjoint, of the asked shape and type; a request past the arena's end gets an ordinary tensor; reset starts over
    and grows the arena when asked for more."""
    torch = pytest.importorskip("torch")
    ar = S._LaneArena(torch, torch.device("cpu"))
    ar.reset(4096)
    a = ar.alloc((3, 5), torch.float32, "cpu")
    b = ar.alloc((7,), torch.int64, "cpu")
    c = ar.alloc((100,), torch.uint8, "cpu")
    base = ar.buf.data_ptr()
    assert [a.data_ptr() - base, b.data_ptr() - base, c.data_ptr() - base] == [0, 256, 512]
    assert a.shape == (3, 5) and a.dtype == torch.float32 and b.dtype == torch.int64 and c.shape == (100,)
    a.fill_(1.0), b.fill_(2), c.fill_(3)
    assert float(a.sum()) == 15.0 and int(b.sum()) == 14 and int(c.sum()) == 300
    big = ar.alloc((4096,), torch.float32, "cpu")  # does not fit: a tensor of its own
    assert not (base <= big.data_ptr() < base + ar.buf.numel())
    ar.reset(1 << 16)
    assert ar.buf.numel() >= 1 << 16 and ar.off == 0
    assert ar.alloc((2,), torch.float32, "cpu").data_ptr() == ar.buf.data_ptr()
