"""Serving render requests: continuous batching on one persistent launch, against one plain
launch per request, under an open-loop Poisson arrival process.

The paper's SaaS server (Sec. "Cloud architecture") serves several clients from one
application instance. Here a request names a resident volume, a transfer function, a camera and an
image size. Admission is by an HBM budget for output images (volumes, brick tables and
occupancy stay resident); admitted requests go to

* BatchedServer -- vrc_server_*: requests are appended to a device FIFO while one persistent
  kernel runs; its warps claim 8 x 4 pixel tiles (phase 1 of the split render) and queued rays
  (phase 2) of the oldest unfinished requests, so requests that arrive while others render
  start as soon as warps free up and overlap on the device; each split request holds a ray
  queue of 112 bytes per pixel while it is in flight;
* PlainServer -- one vrc_render launch per request, in arrival order on one stream.

Both render with the split render by default (the per-ray kernel with kernel=1), so images are
bit-identical across them. Admission counts each server's device bytes per pixel in flight.
run_open_loop() replays a request list against a server and reports p50/p99 latency (arrival
to completion observed by the host) and images/s. Only scheduling and bookkeeping happen in
Python; all rendering runs in the library's kernels.
"""
from __future__ import annotations

import collections
import ctypes as C
import dataclasses
import math
import time

import numpy as np

from . import native


@dataclasses.dataclass
class Request:
    arrival: float      # seconds from the start of the run
    vol_id: int
    tf_id: int
    cam: object         # synth.Camera-like record
    step: float = 0.5
    ert: float = 0.999
    brick: int = 8

    @property
    def image_bytes(self) -> int:
        return self.cam.width * self.cam.height * 16


def poisson_requests(seed: int, rate: float, duration: float, vol_ids, tf_ids, sizes,
                     cam_fn, step=0.5, ert=0.999, brick=8) -> list:
    """Arrivals of a Poisson process of `rate` per second over `duration` seconds; each
    request draws a volume, a transfer function and an image size uniformly, and a camera
    from cam_fn(rng, vol_id, width, height)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        v = vol_ids[int(rng.integers(len(vol_ids)))]
        tf = tf_ids[int(rng.integers(len(tf_ids)))]
        w, h = sizes[int(rng.integers(len(sizes)))]
        out.append(Request(t, v, tf, cam_fn(rng, v, w, h), step, ert, brick))


class ImageBudget:
    """Admission by HBM budget: a request is admitted when its device memory -- the output
    image (16 bytes per pixel) plus whatever the server holds per pixel while it renders --
    fits in what the in-flight requests leave of the budget (first come, first served). Image
    buffers are pooled by size and reused."""

    def __init__(self, budget_bytes: int, alloc, extra_bytes_per_pixel: int = 0):
        self.budget = int(budget_bytes)
        self.used = 0
        self.alloc = alloc  # (height, width) -> buffer
        self.per_pixel = 16 + int(extra_bytes_per_pixel)
        self.free = collections.defaultdict(list)

    def try_acquire(self, h: int, w: int):
        need = h * w * self.per_pixel
        if need > self.budget:
            raise ValueError(f"a {w}x{h} request ({need} bytes) exceeds the whole budget")
        if self.used + need > self.budget:
            return None
        self.used += need
        pool = self.free[(h, w)]
        return pool.pop() if pool else self.alloc(h, w)

    def release(self, h: int, w: int, buf):
        self.used -= h * w * self.per_pixel
        self.free[(h, w)].append(buf)


class BatchedServer:
    """Continuous batching on one persistent launch (vrc_server_*). mode 0: the persistent
    kernel's warps render the requests; mode 1 ("launching"): a persistent scheduler starts
    each request's split render on the device as it arrives (split render only)."""

    def __init__(self, renderer, max_slots: int = 1024, budget_ms: float = 250.0,
                 idle_ms: float = 5.0, kernel: int = 0, mode: int = 0):
        self.R = renderer
        self.lib = renderer.lib
        self.kernel = int(kernel)
        self.mode = int(mode)
        self.name = "launching" if self.mode == 1 else "batched"
        # device bytes a request holds per pixel besides its image: its ray queue
        self.extra_bytes_per_pixel = 0 if self.kernel == 1 else 112
        ptr = C.c_void_p()
        native.check(renderer.ctx, self.lib.vrc_server_create_ex(
            renderer.ctx, int(max_slots), self.mode, C.byref(ptr)))
        self.srv = ptr
        self.budget_ns = int(budget_ms * 1e6)
        self.idle_ns = int(idle_ms * 1e6)

    def submit(self, req: Request, out):
        t = C.c_longlong()
        cs = native.camera_struct(req.cam)
        ps = native.params_struct(req.step, req.ert, req.brick, 64, self.kernel)
        native.check(self.R.ctx, self.lib.vrc_server_submit(
            self.srv, int(req.vol_id), int(req.tf_id), C.byref(cs), C.byref(ps),
            C.c_void_p(out.data_ptr()), C.byref(t)))
        return t.value

    def pump(self) -> bool:
        running = C.c_int()
        native.check(self.R.ctx, self.lib.vrc_server_pump(self.srv, self.budget_ns, self.idle_ns,
                                                          C.byref(running)))
        return bool(running.value)

    def done(self, handle) -> bool:
        d = C.c_int()
        native.check(self.R.ctx, self.lib.vrc_server_poll(self.srv, C.c_longlong(handle),
                                                          C.byref(d)))
        return bool(d.value)

    def close(self):
        if self.srv:
            self.lib.vrc_server_destroy(self.srv)
            self.srv = None


class PlainServer:
    """One vrc_render launch per request, FIFO on one stream; completion by CUDA event."""

    name = "plain"
    extra_bytes_per_pixel = 0  # the context's one split queue per stream is not per request

    def __init__(self, renderer, kernel: int = 0):
        import torch
        self.torch = torch
        self.R = renderer
        self.kernel = int(kernel)
        self.stream = torch.cuda.Stream()

    def submit(self, req: Request, out):
        self.R.render(req.vol_id, req.tf_id, req.cam, step=req.step, ert=req.ert,
                      brick=req.brick, out=out, stream=self.stream, kernel=self.kernel)
        ev = self.torch.cuda.Event()
        ev.record(self.stream)
        return ev

    def pump(self) -> bool:
        return True

    def done(self, handle) -> bool:
        return handle.query()

    def close(self):
        self.stream.synchronize()


def percentile(xs, q):
    if not xs:
        return float("nan")
    ys = sorted(xs)
    k = min(len(ys) - 1, max(0, int(math.ceil(q / 100.0 * len(ys))) - 1))
    return ys[k]


def run_open_loop(server, requests, budget: ImageBudget, warmup: float = 0.0,
                  clock=time.perf_counter, sleep=time.sleep, poll_s: float = 1e-4,
                  drain_timeout: float = 60.0):
    """Replays `requests` (sorted by arrival) in real time against `server`. Returns a dict
    with the latencies of the requests that arrived after `warmup`, their p50/p99 (ms),
    images/s over the measured window and the offered rate."""
    waiting = collections.deque()   # arrived, not yet admitted (FIFO)
    inflight = []                   # (request, buffer, handle)
    lat, done_times, records = [], [], []
    i, n = 0, len(requests)
    t0 = clock()
    end_arrivals = requests[-1].arrival if requests else 0.0
    while i < n or waiting or inflight:
        now = clock() - t0
        if now > end_arrivals + drain_timeout:
            raise TimeoutError(f"{len(inflight) + len(waiting)} requests unfinished")
        while i < n and requests[i].arrival <= now:
            waiting.append(requests[i])
            i += 1
        while waiting:
            r = waiting[0]
            buf = budget.try_acquire(r.cam.height, r.cam.width)
            if buf is None:
                break
            waiting.popleft()
            inflight.append((r, buf, server.submit(r, buf)))
        if inflight:
            server.pump()
        still = []
        for r, buf, hnd in inflight:
            if server.done(hnd):
                t = clock() - t0
                budget.release(r.cam.height, r.cam.width, buf)
                if r.arrival >= warmup:
                    lat.append(t - r.arrival)
                    done_times.append(t)
                    records.append((r.arrival, r.cam.width, r.cam.height, t - r.arrival))
            else:
                still.append((r, buf, hnd))
        inflight = still
        if i < n and not inflight and not waiting:
            sleep(max(0.0, min(requests[i].arrival - (clock() - t0), 0.01)))
        elif inflight:
            sleep(poll_s)
    measured = [r for r in requests if r.arrival >= warmup]
    span = (max(done_times) - warmup) if done_times else float("nan")
    window = max(end_arrivals - warmup, 1e-9)
    return {"server": server.name, "requests": len(measured),
            "offered_per_s": len(measured) / window,
            "images_per_s": len(lat) / span if done_times else 0.0,
            "p50_ms": 1e3 * percentile(lat, 50), "p99_ms": 1e3 * percentile(lat, 99),
            "latencies_s": lat, "records": records}
