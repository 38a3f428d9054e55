"""Serving loop: protect / restore requests of mixed sizes, continuously batched.

Requests arrive at any time (``Server.submit`` returns a ``concurrent.futures.Future``).  A
scheduler thread keeps several lanes -- each a CUDA stream with a reusable batch plan --
and, whenever a lane is free, packs the waiting requests of one kind (protect or restore)
that fit into the device-memory budget into one batch: host->device copies, ONE persistent
batched launch for the whole batch, device->host copies, all on the lane's stream.  Requests
that arrive while other batches are on the GPU are admitted into the next free lane as soon
as memory allows, so work of different batches overlaps on the device.  Keys stay resident
on the device (key slots); every request names its slot and its own initial counter block.

Each result is bit-for-bit what the request gives alone: batching changes only which launch
a request's tiles belong to.
"""
from __future__ import annotations

import collections
import queue
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    """One protect request (``pixels`` H x W x 3 uint8) or restore request (``public`` int16
    fragment bytes and ``private`` ciphertext bytes).  Host arrays; pinned memory is copied
    faster."""
    kind: str                      # "protect" or "restore"
    width: int
    height: int
    k: int
    key_slot: int
    iv: bytes
    pixels: object = None          # protect input
    public: object = None          # restore inputs
    private: object = None
    arrival: float = 0.0           # time.perf_counter() at submission
    done: float = 0.0              # time.perf_counter() when the result was ready
    future: Future = field(default_factory=Future)

    def sizes(self):
        from . import api
        pub, priv = api.sizes(self.width, self.height, self.k)
        return self.width * self.height * 3, pub, priv

    def device_bytes(self) -> int:
        px, pub, priv = self.sizes()
        return px + pub + priv


class GpuLane:
    """One CUDA stream and a reusable plan; runs one batch at a time."""

    def __init__(self, device, capacity):
        import torch

        from . import api
        self.torch, self.api = torch, api
        self.device = device
        self.stream = torch.cuda.Stream(device)
        with torch.cuda.device(device):
            self.plan = api.Plan(capacity=capacity)
        self.event = None
        self.batch = None
        self.hold = None

    def busy(self) -> bool:
        return self.batch is not None

    def done(self) -> bool:
        return self.batch is not None and self.event.query()

    def launch(self, batch: list[Request]) -> None:
        torch, api = self.torch, self.api
        kind = batch[0].kind
        descs = [api.ImageDesc(r.width, r.height, r.k, r.key_slot, r.iv) for r in batch]
        npx, npub, npriv = api.layout(descs)
        with torch.cuda.stream(self.stream):
            px = torch.empty(max(npx, 16), dtype=torch.uint8, device=self.device)
            pub = torch.empty(max(npub, 16), dtype=torch.uint8, device=self.device)
            priv = torch.empty(max(npriv, 16), dtype=torch.uint8, device=self.device)
            outs = []
            for r, d in zip(batch, descs):
                n, pb, vb = r.sizes()
                if kind == "protect":
                    px[d.pixel_offset: d.pixel_offset + n].copy_(_as_u8(torch, r.pixels), non_blocking=True)
                else:
                    pub[d.public_offset: d.public_offset + pb].copy_(_as_u8(torch, r.public), non_blocking=True)
                    priv[d.private_offset: d.private_offset + vb].copy_(_as_u8(torch, r.private), non_blocking=True)
            self.plan.update(descs, self.stream)
            if kind == "protect":
                self.plan.protect(px, pub, priv)
            else:
                self.plan.restore(pub, priv, px)
            for r, d in zip(batch, descs):
                n, pb, vb = r.sizes()
                if kind == "protect":
                    hp = torch.empty(pb, dtype=torch.uint8, pin_memory=True)
                    hv = torch.empty(vb, dtype=torch.uint8, pin_memory=True)
                    hp.copy_(pub[d.public_offset: d.public_offset + pb], non_blocking=True)
                    hv.copy_(priv[d.private_offset: d.private_offset + vb], non_blocking=True)
                    outs.append((hp, hv))
                else:
                    hx = torch.empty(n, dtype=torch.uint8, pin_memory=True)
                    hx.copy_(px[d.pixel_offset: d.pixel_offset + n], non_blocking=True)
                    outs.append(hx)
            self.event = torch.cuda.Event()
            self.event.record(self.stream)
        self.batch, self.hold = batch, (px, pub, priv, outs)

    def finish(self) -> list[tuple[Request, object]]:
        """Results of the finished batch: protect -> (public int16 array [H/8, W/8, 3, 63-k],
        private bytes); restore -> H x W x 3 uint8 array."""
        batch, (_, _, _, outs) = self.batch, self.hold
        res = []
        for r, o in zip(batch, outs):
            if r.kind == "protect":
                pub = o[0].numpy().view(np.int16).reshape(r.height // 8, r.width // 8, 3, 63 - r.k)
                res.append((r, (pub, o[1].numpy().tobytes())))
            else:
                res.append((r, o.numpy().reshape(r.height, r.width, 3)))
        self.batch = self.hold = self.event = None
        return res

    def close(self) -> None:
        self.plan.close()


def _as_u8(torch, a):
    if isinstance(a, torch.Tensor):
        return a.reshape(-1).view(torch.uint8)
    if isinstance(a, (bytes, bytearray)):
        return torch.frombuffer(bytearray(a), dtype=torch.uint8)
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1).view(np.uint8))


class Server:
    """Continuous-batching server.

    lanes: batches in flight at once (each on its own stream); max_batch: requests per batch;
    mem_budget: device bytes that admitted requests may hold at once (default: half of the
    device memory free at start).  A request larger than the whole budget is rejected.
    ``lane_factory(i)`` builds a lane (GpuLane by default; tests pass CPU fakes)."""

    def __init__(self, device: int = 0, lanes: int = 3, max_batch: int = 64,
                 mem_budget: int | None = None, lane_factory=None):
        self.max_batch = max_batch
        if lane_factory is None:
            import torch

            from . import api
            api.init(device)
            if mem_budget is None:
                free, _ = torch.cuda.mem_get_info(device)
                mem_budget = free // 2
            lane_factory = lambda i: GpuLane(torch.device("cuda", device), max_batch)  # noqa: E731
        self.mem_budget = int(mem_budget if mem_budget is not None else 1 << 62)
        self.lanes = [lane_factory(i) for i in range(lanes)]
        self.inbox: queue.Queue = queue.Queue()
        self.ready: collections.deque = collections.deque()
        self.in_use = 0                 # device bytes of admitted, unfinished requests
        self.stats = {"batches": 0, "requests": 0, "max_batch": 0, "max_lanes_busy": 0}
        self._stop = False
        self._thread = threading.Thread(target=self._loop, name="fds-serve", daemon=True)
        self._thread.start()

    def submit(self, req: Request) -> Future:
        if req.kind not in ("protect", "restore"):
            raise ValueError("kind must be 'protect' or 'restore'")
        if req.device_bytes() > self.mem_budget:
            raise ValueError("request larger than the server's device-memory budget")
        req.arrival = time.perf_counter()
        self.inbox.put(req)
        return req.future

    def close(self) -> None:
        self._stop = True
        self._thread.join()
        for lane in self.lanes:
            if hasattr(lane, "close"):
                lane.close()

    # scheduler thread
    def _loop(self) -> None:
        try:
            while True:
                progressed = False
                for lane in self.lanes:                       # retire finished batches
                    if lane.busy() and lane.done():
                        now = time.perf_counter()
                        for r, res in lane.finish():
                            self.in_use -= r.device_bytes()
                            r.done = now
                            r.future.set_result(res)
                        progressed = True
                while True:                                   # arrivals join the ready list
                    try:
                        self.ready.append(self.inbox.get_nowait())
                    except queue.Empty:
                        break
                for lane in self.lanes:                       # fill free lanes
                    if lane.busy() or not self.ready:
                        continue
                    batch = self._take_batch()
                    if not batch:
                        break                                 # head request waits for memory
                    lane.launch(batch)
                    self.stats["batches"] += 1
                    self.stats["requests"] += len(batch)
                    self.stats["max_batch"] = max(self.stats["max_batch"], len(batch))
                    progressed = True
                busy = sum(lane.busy() for lane in self.lanes)
                self.stats["max_lanes_busy"] = max(self.stats["max_lanes_busy"], busy)
                if self._stop and not self.ready and busy == 0 and self.inbox.empty():
                    return
                if not progressed:
                    if busy:
                        time.sleep(20e-6)
                    else:
                        try:
                            self.ready.append(self.inbox.get(timeout=0.002))
                        except queue.Empty:
                            pass
        except BaseException as exc:                          # fail every waiting request
            for r in list(self.ready):
                if not r.future.done():
                    r.future.set_exception(exc)
            for lane in self.lanes:
                for r in (lane.batch or []):
                    if not r.future.done():
                        r.future.set_exception(exc)
            raise

    def _take_batch(self) -> list[Request]:
        """Oldest ready request's kind; then every ready request of that kind, in arrival
        order, that fits into the memory budget, up to max_batch (admission by memory)."""
        kind = self.ready[0].kind
        batch, keep = [], collections.deque()
        while self.ready and len(batch) < self.max_batch:
            r = self.ready.popleft()
            need = r.device_bytes()
            if r.kind == kind and self.in_use + need <= self.mem_budget:
                batch.append(r)
                self.in_use += need
            else:
                keep.append(r)
                if r.kind == kind and not batch:
                    break                                     # the oldest does not fit yet
        keep.extend(self.ready)
        self.ready = keep
        return batch


def run_poisson(server: Server, requests: list[Request], arrivals: np.ndarray) -> dict:
    """Submit `requests` at the given arrival times (seconds from now), wait for all, and
    return latency percentiles (ms) and sustained MB/s of pixels."""
    t0 = time.perf_counter()
    for r, at in zip(requests, arrivals):
        delay = t0 + float(at) - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        server.submit(r)
    for r in requests:
        r.future.result()
    t1 = max(r.done for r in requests)
    lat = np.sort(np.array([(r.done - r.arrival) * 1e3 for r in requests]))
    pix = sum(r.width * r.height * 3 for r in requests)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "sustained_MBps": pix / (t1 - t0) / 1e6,
            "seconds": t1 - t0, "requests": len(requests)}
