"""Serving loop: novel-view render requests against resident scenes, with continuous batching.

Requests (scene, pose, resolution) arrive over time. The scheduler keeps every scene's Gaussians resident on the
device and runs batches on a fixed number of lanes (one CUDA stream each), so batches of different scenes or
resolutions overlap on the GPU:
  * a batch is up to `max_batch` waiting requests of the same scene and resolution, rendered as the views of one
    forward pass (one launch per stage for all of them);
  * the oldest waiting request leads the next batch (first come, first served); when its batch does not fit in the
    free device-memory budget, younger requests that do fit are admitted instead, unless the oldest one has waited
    longer than `max_wait` seconds (then nothing passes it);
  * a request is admitted the moment a lane and memory free up, while other batches are still on the GPU, and it
    completes when its image is back in host memory.
A view's image depends only on its pose and the scene (Eqs. 3-8), so a request renders to the same pixels alone or
batched with others.

The scheduler is independent of CUDA: it drives an executor with `bytes_needed`, `launch`, `done` and `collect`
(and, optionally, `wait`, a blocking wait for the next finished batch). `GpuExecutor` is the one that renders with
the CUDA library.
"""
from __future__ import annotations

import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    scene: str
    viewmat: np.ndarray          # [4, 4] world-to-camera pose
    width: int
    height: int
    arrival: float = 0.0         # seconds on the scheduler clock
    admitted: float | None = None
    done: float | None = None
    result: object = None        # [3, H, W] float32 image once complete
    batch: int | None = None
    error: str | None = None

    @property
    def key(self):
        return (self.scene, self.width, self.height)


@dataclass
class Batch:
    bid: int
    lane: int
    requests: list
    nbytes: int
    started: float
    handle: object = None


@dataclass
class Stats:
    completed: int = 0
    rejected: int = 0
    batches: int = 0
    views_in_batches: int = 0
    max_in_flight: int = 0
    peak_reserved: int = 0
    latencies: list = field(default_factory=list)

    def summary(self, makespan: float) -> dict:
        lat = np.asarray(self.latencies) * 1e3
        return {"requests": self.completed, "rejected": self.rejected,
                "views_per_s": self.completed / makespan if makespan > 0 else None,
                "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
                "mean_batch": self.views_in_batches / max(self.batches, 1),
                "max_in_flight": self.max_in_flight, "peak_reserved_bytes": self.peak_reserved}


class Scheduler:
    def __init__(self, executor, lanes: int = 4, max_batch: int = 8, mem_budget: int | None = None,
                 max_wait: float = 0.25, keep_results: bool = True, on_result=None):
        if lanes < 1 or max_batch < 1:
            raise ValueError("lanes and max_batch must be >= 1")
        if keep_results and getattr(executor, "host_buffers", "per_batch") == "per_lane":
            raise ValueError("an executor with per-lane host buffers reuses each image's memory: keep_results=False")
        self.ex = executor
        self.lanes = lanes
        self.max_batch = max_batch
        self.mem_budget = mem_budget if mem_budget is not None else executor.memory_budget()
        self.max_wait = max_wait
        # keep_results=False: a completed request's image is delivered and dropped at once (a server that hands it
        # on), so its host buffer goes back to the allocator instead of being held until the caller lets go
        self.keep_results = keep_results
        self.on_result = on_result  # called with (request, image) as each request completes, before it is dropped
        self.waiting: list[Request] = []
        self.in_flight: dict[int, Batch] = {}
        self.free_lanes = list(range(lanes))
        self.reserved = 0
        self.stats = Stats()
        self._next_bid = 0

    # ------------------------------------------------------------------ admission
    def submit(self, req: Request) -> None:
        self.waiting.append(req)

    def _group(self, head: Request) -> list:
        group = [head]
        for r in self.waiting:
            if len(group) == self.max_batch:
                break
            if r is not head and r.key == head.key:
                group.append(r)
        return group

    def _fit(self, group: list) -> tuple[list, int] | None:
        """Largest prefix of `group` whose batch fits in the free budget, with its size in bytes."""
        free = self.mem_budget - self.reserved
        s, w, h = group[0].key
        while group:
            need = self.ex.bytes_needed(s, w, h, len(group))
            if need <= free:
                return group, need
            group = group[:-1]
        return None

    def pump(self, now: float) -> int:
        """Start as many batches as free lanes and memory allow; returns how many started."""
        started = 0
        while self.free_lanes and self.waiting:
            head = self.waiting[0]
            choice = None
            fit = self._fit(self._group(head))
            if fit is not None:
                choice = fit
            elif not self.in_flight and self.ex.bytes_needed(*head.key, 1) > self.mem_budget:
                # can never fit, even alone on an idle device
                self.waiting.pop(0)
                head.error = "request exceeds the device memory budget"
                head.done = now
                self.stats.rejected += 1
                continue
            elif now - head.arrival < self.max_wait:
                seen = {head.key}
                for r in self.waiting[1:]:
                    if r.key in seen:
                        continue
                    seen.add(r.key)
                    fit = self._fit(self._group(r))
                    if fit is not None:
                        choice = fit
                        break
            if choice is None:
                break
            group, need = choice
            for r in group:
                self.waiting.remove(r)
                r.admitted = now
            lane = self.free_lanes.pop(0)
            b = Batch(self._next_bid, lane, group, need, now)
            self._next_bid += 1
            for r in group:
                r.batch = b.bid
            b.handle = self.ex.launch(lane, group)
            self.in_flight[b.bid] = b
            self.reserved += need
            self.stats.batches += 1
            self.stats.views_in_batches += len(group)
            self.stats.max_in_flight = max(self.stats.max_in_flight, len(self.in_flight))
            self.stats.peak_reserved = max(self.stats.peak_reserved, self.reserved)
            started += 1
        return started

    # ------------------------------------------------------------------ completion
    def poll(self, now: float) -> list:
        """Collect finished batches; returns the requests completed by this call."""
        finished = []
        for bid in list(self.in_flight):
            b = self.in_flight[bid]
            if not self.ex.done(b.handle):
                continue
            images = self.ex.collect(b.handle)
            t = now
            for r, img in zip(b.requests, images):
                if self.on_result is not None:
                    self.on_result(r, img)
                r.result = img if self.keep_results else None
                r.done = t
                self.stats.completed += 1
                self.stats.latencies.append(t - r.arrival)
                finished.append(r)
            del self.in_flight[bid]
            self.reserved -= b.nbytes
            self.free_lanes.append(b.lane)
            self.free_lanes.sort()
        return finished

    def idle(self) -> bool:
        return not self.waiting and not self.in_flight


def run_trace(scheduler: Scheduler, requests: list, clock=time.perf_counter, sleep=time.sleep,
              spin: float = 5e-5) -> dict:
    """Replays `requests` (sorted by arrival, seconds from the start) in real time through the scheduler and
    returns its summary: views/s over the makespan, p50 / p99 latency from arrival to image on the host.

    Between events the loop blocks: on the executor's `wait` (until a batch finishes or the next request is due)
    when the executor has one, else by sleeping `spin` seconds."""
    pending = sorted(requests, key=lambda r: r.arrival)
    wait = getattr(scheduler.ex, "wait", None)
    i = 0
    t0 = clock()
    while i < len(pending) or not scheduler.idle():
        now = clock() - t0
        while i < len(pending) and pending[i].arrival <= now:
            scheduler.submit(pending[i])
            i += 1
        scheduler.poll(now)
        scheduler.pump(now)
        due = pending[i].arrival - (clock() - t0) if i < len(pending) else None
        if scheduler.in_flight and wait is not None:
            wait(None if due is None else max(0.0, due))
        elif scheduler.idle() and due is not None:
            sleep(max(0.0, min(due, 1e-3)))
        elif spin:
            sleep(spin)
    makespan = clock() - t0 - (pending[0].arrival if pending else 0.0)
    return scheduler.stats.summary(makespan)


class _LaneArena:
    """Device memory of one lane, carved into a batch's buffers. A lane runs one batch at a time and its next batch
    is launched only after the previous one was collected, so each launch starts carving from the beginning again.
    The arena grows (one allocation) when a batch needs more than it holds, which the warm-up of every key brings
    about before any timed work; in steady state a batch allocates no device memory, so no allocation of the
    framework's caching allocator can stall the other lanes."""

    def __init__(self, torch, device):
        self.torch, self.device = torch, device
        self.buf = None
        self.off = 0

    def reset(self, nbytes: int) -> None:
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = None
            self.buf = self.torch.empty((nbytes,), dtype=self.torch.uint8, device=self.device)
        self.off = 0

    def alloc(self, shape, dtype, device):
        torch = self.torch
        count = 1
        for d in shape:
            count *= int(d)
        nbytes = count * torch.empty((), dtype=dtype).element_size()
        if self.buf is not None and self.off + nbytes <= self.buf.numel():
            t = self.buf[self.off:self.off + nbytes].view(dtype).view(tuple(shape))
            self.off += (nbytes + 255) // 256 * 256
            return t
        return torch.empty(tuple(shape), dtype=dtype, device=device)  # past the arena (a capacity re-run)


class GpuExecutor:
    """Renders batches with the CUDA library; every scene stays resident on the device.

    scenes: name -> (means, scales, quats, opacity, sh) float32 arrays (host or device), all with one SH degree per
    scene. Instance capacity per batch is sized from the largest per-view count seen for that scene and resolution
    (a probe render on first use) times `headroom`; a batch that still overflows is re-rendered once with growing
    capacity when it is collected, and counted in `overflows`.

    host_buffers: where a batch's images land on the host. "per_batch" (default): a new pinned buffer per batch,
    from the framework's caching host allocator; the images stay valid as long as they are held. "per_lane": one
    pinned buffer per lane, sized by `reserve` and reused by the lane's next batch, so that serving pins no host
    memory (pinning a buffer of hundreds of MB takes far longer than rendering into it); the images a batch returns
    are then valid only until its lane's next batch, and only a Scheduler that does not keep results accepts it.
    """

    def __init__(self, scenes: dict, lanes: int, device="cuda", tile: int = 16, headroom: float = 1.3,
                 bg=(0.0, 0.0, 0.0), host_buffers: str = "per_batch"):
        if host_buffers not in ("per_batch", "per_lane"):
            raise ValueError("host_buffers must be 'per_batch' or 'per_lane'")
        import torch
        import paper_2404_03202_gb300 as og
        self.torch, self.og = torch, og
        self.device = torch.device(device)
        self.tile, self.headroom, self.bg = tile, headroom, bg
        self.scenes = {}
        for name, arrays in scenes.items():
            t = tuple(torch.as_tensor(a, dtype=torch.float32).to(self.device).contiguous() for a in arrays)
            k = int(t[4].shape[1])
            self.scenes[name] = (t, int(t[0].shape[0]), int(round(k ** 0.5)) - 1)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(lanes)]
        self.arenas = [_LaneArena(torch, self.device) for _ in range(lanes)]
        self.host_buffers = host_buffers
        self._lane_host = [None] * lanes  # per_lane: each lane's pinned result buffer (float32, flat)
        self.per_view = {}
        self.overflows = 0
        # one waiter thread per lane blocks on the lane's batches in launch order (its stream runs them in that
        # order) and wakes `wait`; the event wait releases the interpreter lock
        self._cv = threading.Condition()
        self._ready = 0
        self._queues = [queue.Queue() for _ in range(lanes)]
        self._threads = [threading.Thread(target=self._waiter, args=(q,), daemon=True) for q in self._queues]
        for t in self._threads:
            t.start()

    def _waiter(self, q):
        while True:
            h = q.get()
            if h is None:  # close()
                return
            h["ev"].synchronize()
            with self._cv:
                h["finished"] = True
                self._ready += 1
                self._cv.notify_all()

    def reserve(self, keys, max_views: int) -> int:
        """Grow every lane's arena to the largest batch of up to max_views views of the given (scene, (w, h)) keys,
        so that no lane allocates device memory once requests are served. Returns the bytes per lane."""
        nbytes = max(self.bytes_needed(scene, w, h, max_views) for scene, (w, h) in keys)
        for a in self.arenas:
            a.reset(nbytes)
        if self.host_buffers == "per_lane":
            floats = max_views * 3 * max(w * h for _, (w, h) in keys)
            for lane in range(len(self._lane_host)):
                self._lane_host[lane] = self._pinned(lane, floats)
        return nbytes

    def _pinned(self, lane: int, floats: int):
        """The lane's pinned result buffer, grown to hold `floats` values."""
        buf = self._lane_host[lane]
        if buf is None or buf.numel() < floats:
            buf = None
            self._lane_host[lane] = buf = self.torch.empty((floats,), dtype=self.torch.float32, pin_memory=True)
        return buf

    def close(self) -> None:
        """Stop the waiter threads (after the batches already launched) and release the lanes' arenas and the
        resident scenes. The threads hold the executor, so without close() its device memory stays allocated."""
        for q in self._queues:
            q.put(None)
        for t in self._threads:
            t.join()
        self.arenas = []
        self._lane_host = []
        self.scenes = {}

    def wait(self, timeout=None) -> None:
        """Block until some launched batch has finished and not been collected, or `timeout` seconds pass."""
        with self._cv:
            if self._ready == 0:
                self._cv.wait(timeout)

    def _settings(self, scene, w, h, v):
        return self.og.Settings(width=w, height=h, tile=self.tile, num_views=v, sh_degree=self.scenes[scene][2],
                                bg=self.bg)

    def memory_budget(self) -> int:
        free, _ = self.torch.cuda.mem_get_info(self.device)
        return int(free * 0.8)

    def _per_view(self, scene, w, h) -> int:
        key = (scene, w, h)
        if key not in self.per_view:  # probe: identity pose, one view, synchronous
            r = self.og.Rasterizer(self._settings(scene, w, h, 1), device=self.device, capacity=1 << 16)
            vm = self.torch.eye(4, device=self.device).reshape(1, 4, 4)
            r.forward(*self.scenes[scene][0], vm)
            self.per_view[key] = max(int(r.count), 1)
            del r
        return self.per_view[key]

    def _capacity(self, scene, w, h, v) -> int:
        return int(self._per_view(scene, w, h) * v * self.headroom) + 4096

    def bytes_needed(self, scene, w, h, v) -> int:
        from . import _cabi as C
        n = self.scenes[scene][1]
        cap = self._capacity(scene, w, h, v)
        cfg = self._settings(scene, w, h, v).config()
        pixels = v * w * h
        buffers = (pixels * (3 + 1 + 1 + 3) * 4            # rgb, T, n_contrib, dL/dC
                   + v * ((w // self.tile) * (h // self.tile)) * 8  # ranges
                   + cap * 8                                   # instance keys
                   + max(v * n, 1) * (48 + 4 + 48))            # splats, order, 2D gradients
        return int(C.omnigs_workspace_size(cfg, n, cap)) + buffers + pixels * 3 * 4  # + pinned result (host)

    def launch(self, lane: int, requests: list):
        torch = self.torch
        r0 = requests[0]
        s = self.streams[lane]
        v = len(requests)
        params = self.scenes[r0.scene][0]
        vm = np.stack([np.asarray(r.viewmat, np.float32) for r in requests])
        arena = self.arenas[lane]
        arena.reset(self.bytes_needed(r0.scene, r0.width, r0.height, v))
        with torch.cuda.stream(s):
            rast = self.og.Rasterizer(self._settings(r0.scene, r0.width, r0.height, v), device=self.device,
                                      capacity=self._capacity(r0.scene, r0.width, r0.height, v), grow=False,
                                      alloc=arena.alloc, forward_only=True)
            vm_dev = torch.from_numpy(vm).to(self.device, non_blocking=True)
            rast.forward(*params, vm_dev, stream=s)
            shape = tuple(rast.rgb.shape)
            if self.host_buffers == "per_lane":
                # the lane's previous batch was collected before this launch, so its buffer is free
                host = self._pinned(lane, v * 3 * r0.width * r0.height)[:v * 3 * r0.width * r0.height].view(shape)
            else:
                host = torch.empty(shape, dtype=torch.float32, pin_memory=True)
            host.copy_(rast.rgb, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        handle = {"r": rast, "host": host, "ev": ev, "stream": s, "vm": vm_dev, "requests": requests,
                  "finished": False}
        self._queues[lane].put(handle)
        return handle

    def done(self, handle) -> bool:
        return handle["finished"]

    def collect(self, handle) -> list:
        with self._cv:
            self._ready -= 1
        rast, s = handle["r"], handle["stream"]
        try:
            rast.check(stream=s)
        except self.og.OmnigsError:
            # capacity overflow: re-render with a growing capacity (one host synchronisation) and remember the count
            self.overflows += 1
            torch = self.torch
            with torch.cuda.stream(s):
                rast.grow = True
                rast.forward(*self.scenes[handle["requests"][0].scene][0], handle["vm"], stream=s)
                handle["host"].copy_(rast.rgb, non_blocking=True)
            s.synchronize()
            r0 = handle["requests"][0]
            key = (r0.scene, r0.width, r0.height)
            self.per_view[key] = max(self.per_view[key], -(-int(rast.count) // len(handle["requests"])))
        host = handle["host"]
        return [host[i].numpy() for i in range(host.shape[0])]
