"""Serving loop: protect / restore requests of mixed sizes, continuously batched.

Requests arrive at any time (``Server.submit`` returns a ``concurrent.futures.Future``).  A
scheduler thread keeps several lanes -- each a CUDA stream with a reusable batch plan --
and, whenever a lane is free, packs the waiting requests of one kind (protect or restore)
that fit into the device-memory budget into one batch: host->device copies, ONE persistent
batched launch for the whole batch, device->host copies, all on the lane's stream.  Requests
that arrive while other batches are on the GPU are admitted into the next free lane as soon
as memory allows, so work of different batches overlaps on the device.  Keys stay resident
on the device (key slots); every request names its slot and its own initial counter block.

Host side: inputs that are not pinned host tensors are copied into pinned memory by a pool of
staging threads when they are submitted (off the scheduler thread); a batch's outputs leave the
device as one copy per fragment buffer into the lane's pinned host buffers, which the same pool
copies out once per batch (the lane takes its next batch once they are out); each request's
result is a view into that copy.  The lane's device and pinned host buffers persist and grow with the largest batch, so
a warm server allocates no pinned memory.

Each result is bit-for-bit what the request gives alone: batching changes only which launch
a request's tiles belong to.
"""
from __future__ import annotations

import collections
import functools
import os
import queue
import threading
import time
from concurrent.futures import Future, ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    """One protect request (``pixels`` H x W x 3 uint8) or restore request (``public`` int16
    fragment bytes and ``private`` ciphertext bytes).  Host arrays or tensors of exactly those
    sizes; pinned memory is copied faster."""
    kind: str                      # "protect" or "restore"
    width: int
    height: int
    k: int
    key_slot: int
    iv: bytes
    pixels: object = None          # protect input
    public: object = None          # restore inputs
    private: object = None
    # optional output buffers the result is copied into straight from the device (contiguous
    # CPU tensors, pinned for speed, each at least the result's bytes): protect (public,
    # private), restore (pixels,); the result is then given as arrays over them
    out: tuple = None
    arrival: float = 0.0           # time.perf_counter() at submission
    done: float = 0.0              # time.perf_counter() when the result was ready
    future: Future = field(default_factory=Future)

    _sizes: tuple = None           # (pixel, public, private) bytes, computed once
    _staged: tuple = None          # pinned host copies of the inputs (the inputs stay as given)

    def inputs(self) -> tuple:
        """The inputs the lane copies to the device: the staged copies once there are some."""
        if self._staged is not None:
            return self._staged
        return (self.pixels,) if self.kind == "protect" else (self.public, self.private)

    def sizes(self):
        if self._sizes is None:
            from . import api
            pub, priv = api.sizes(self.width, self.height, self.k)
            self._sizes = (self.width * self.height * 3, pub, priv)
        return self._sizes

    def device_bytes(self) -> int:
        px, pub, priv = self.sizes()
        return px + pub + priv


class GpuLane:
    """One CUDA stream, a reusable plan, and device and pinned host buffers that grow with the
    largest batch; runs one batch at a time.

    Life of a batch: launch() (copies in, one batched launch, copies out, on the stream);
    done() once the stream has passed it; finish() hands back one result builder per request
    (each copies its result out of the pinned buffers); release() once all have run."""

    def __init__(self, device, capacity):
        import torch

        from . import api
        self.torch, self.api = torch, api
        self.device = device
        self.stream = torch.cuda.Stream(device)
        with torch.cuda.device(device):
            self.plan = api.Plan(capacity=capacity)
        self.bufs = [None, None, None]       # pixels, public, private (device, uint8)
        self.hbufs = [None, None]            # outputs (pinned host, uint8)
        self.event = None
        self.batch = None
        self.hold = None
        self.draining = False

    def busy(self) -> bool:
        return self.batch is not None

    def done(self) -> bool:
        return self.batch is not None and not self.draining and self.event.query()

    def _grow(self, bufs, i: int, n: int, **kw):
        b = bufs[i]
        if b is None or b.numel() < n:
            # this lane's previous batch is over (the lane was free), so the old buffer may go
            b = self.torch.empty(max(n, 16, 2 * (b.numel() if b is not None else 0)), dtype=self.torch.uint8, **kw)
            bufs[i] = b
        return b

    def launch(self, batch: list[Request]) -> None:
        torch, api = self.torch, self.api
        kind = batch[0].kind
        # per-request sizes, offsets and descriptors, as arrays (no per-request objects)
        sz = np.array([r.sizes() for r in batch], dtype=np.int64).reshape(-1, 3)
        offs, (npx, npub, npriv) = api.layout_arrays(sz[:, 0], sz[:, 1], sz[:, 2])
        rec = api.desc_records([r.width for r in batch], [r.height for r in batch], [r.k for r in batch],
                               [r.key_slot for r in batch], [r.iv for r in batch], offs)
        self.nbytes, self.offs = (npx, npub, npriv), offs
        refs = []                                   # host inputs, alive until the batch is over
        with torch.cuda.stream(self.stream):
            dev = dict(device=self.device)
            px, pub, priv = (self._grow(self.bufs, 0, npx, **dev), self._grow(self.bufs, 1, npub, **dev),
                             self._grow(self.bufs, 2, npriv, **dev))
            # every input of the batch by one call, one copy each
            if kind == "protect":
                api.copy_many(px.data_ptr() + offs[0].astype(np.uint64),
                              [_host_ptr(torch, r.inputs()[0], refs) for r in batch], sz[:, 0], self.stream)
            else:
                dsts = np.concatenate([pub.data_ptr() + offs[1].astype(np.uint64),
                                       priv.data_ptr() + offs[2].astype(np.uint64)])
                srcs = [_host_ptr(torch, r.inputs()[0], refs) for r in batch] + \
                       [_host_ptr(torch, r.inputs()[1], refs) for r in batch]
                api.copy_many(dsts, srcs, np.concatenate([sz[:, 1], sz[:, 2]]), self.stream)
            self.plan.update_records(rec, self.stream)
            if kind == "protect":
                self.plan.protect(px, pub, priv)
            else:
                self.plan.restore(pub, priv, px)
            # results: straight into the buffers of the requests that brought them, the rest
            # into the lane's pinned buffers
            direct = np.array([r.out is not None for r in batch], dtype=bool)
            if direct.any():
                idx = np.nonzero(direct)[0]
                if kind == "protect":
                    dsts = [r.out[0].data_ptr() for r in batch if r.out is not None] + \
                           [r.out[1].data_ptr() for r in batch if r.out is not None]
                    srcs = np.concatenate([pub.data_ptr() + offs[1][idx].astype(np.uint64),
                                           priv.data_ptr() + offs[2][idx].astype(np.uint64)])
                    api.copy_many(dsts, srcs, np.concatenate([sz[idx, 1], sz[idx, 2]]), self.stream)
                else:
                    api.copy_many([r.out[0].data_ptr() for r in batch if r.out is not None],
                                  px.data_ptr() + offs[0][idx].astype(np.uint64), sz[idx, 0], self.stream)
            if not direct.all():
                if kind == "protect":
                    h0 = self._grow(self.hbufs, 0, npub, pin_memory=True)
                    h1 = self._grow(self.hbufs, 1, npriv, pin_memory=True)
                    h0[:npub].copy_(pub[:npub], non_blocking=True)
                    h1[:npriv].copy_(priv[:npriv], non_blocking=True)
                else:
                    h0 = self._grow(self.hbufs, 0, npx, pin_memory=True)
                    h0[:npx].copy_(px[:npx], non_blocking=True)
            self.event = torch.cuda.Event()
            self.event.record(self.stream)
        self.batch, self.hold = batch, refs

    def finish(self) -> list[tuple[Request, object]]:
        """One (request, result or builder) per request of the finished batch: protect ->
        (public int16 array [H/8, W/8, 3, 63-k], private bytes); restore -> H x W x 3 uint8
        array.  A request that brought its own output buffers gets its result at once, as
        arrays over those buffers; for the others builder() returns a view into one copy of
        the lane's pinned buffers.  Call release() after every builder has run."""
        self.draining = True
        if self.batch[0].kind == "protect":
            used = [self.nbytes[1], self.nbytes[2]]
        else:
            used = [self.nbytes[0], 0]
        host = _BatchCopy(self.hbufs, used)
        out = []
        for i, r in enumerate(self.batch):
            o = (int(self.offs[0][i]), int(self.offs[1][i]), int(self.offs[2][i]))
            if r.out is not None:
                out.append((r, _result_in(r)))
            else:
                out.append((r, functools.partial(_result_of, r, o, host)))
        return out

    def release(self) -> None:
        self.batch = self.hold = self.event = None
        self.draining = False

    def close(self) -> None:
        self.plan.close()


class _BatchCopy:
    """The used part of a lane's pinned output buffers, copied once per batch into ordinary host
    memory by whichever result builder runs first (a torch clone: it runs without the
    interpreter lock); every request's result is then a view into that copy, which stays alive
    as long as one of them does."""

    def __init__(self, bufs, used):
        self.bufs, self.used = bufs, used
        self.lock = threading.Lock()
        self.copy = None

    def get(self):
        with self.lock:
            if self.copy is None:
                self.copy = [b[:n].clone() if (b is not None and n) else None for b, n in zip(self.bufs, self.used)]
        return self.copy


def _result_of(r: Request, offs, batch_copy: _BatchCopy):
    """Request r's result as a view into its batch's copy of the lane's output buffers; offs =
    its (pixel, public, private) offsets in the batch."""
    host = batch_copy.get()
    n, pb, vb = r.sizes()
    if r.kind == "protect":
        pub = host[0][offs[1]: offs[1] + pb].numpy().view(np.int16).reshape(r.height // 8, r.width // 8, 3, 63 - r.k)
        return pub, host[1][offs[2]: offs[2] + vb].numpy().tobytes()
    return host[0][offs[0]: offs[0] + n].numpy().reshape(r.height, r.width, 3)


def _u8(t):
    """A contiguous CPU tensor's bytes as a numpy uint8 array (no copy)."""
    return t.numpy().reshape(-1).view(np.uint8)


def _result_in(r: Request):
    """The result of a request that brought its own output buffers, over those buffers."""
    n, pb, vb = r.sizes()
    if r.kind == "protect":
        pub = _u8(r.out[0])[:pb].view(np.int16).reshape(r.height // 8, r.width // 8, 3, 63 - r.k)
        return pub, _u8(r.out[1])[:vb].tobytes()
    return _u8(r.out[0])[:n].reshape(r.height, r.width, 3)


def _host_ptr(torch, a, refs: list) -> int:
    """Address of input `a` (a contiguous tensor, a numpy array or bytes); `a`, or the
    contiguous copy whose address this is, is appended to refs."""
    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            a = a.contiguous()
        refs.append(a)
        return a.data_ptr()
    if isinstance(a, (bytes, bytearray, memoryview)):
        arr = np.frombuffer(a, dtype=np.uint8)
    else:
        arr = np.ascontiguousarray(a)
    refs.append(arr)
    return arr.ctypes.data


def _check_buffers(req: Request) -> None:
    """Inputs of exactly the request's sizes; output buffers (if any) large enough."""
    import torch
    n, pb, vb = req.sizes()
    need = (n,) if req.kind == "protect" else (pb, vb)
    for i, (a, b) in enumerate(zip(req.inputs(), need)):
        if a is None or _nbytes(torch, a) != b:
            raise ValueError(f"{req.kind} input {i}: {b} bytes expected")
    if req.out is not None:
        need = (pb, vb) if req.kind == "protect" else (n,)
        if len(req.out) != len(need):
            raise ValueError(f"{req.kind} takes {len(need)} output buffers")
        for o, b in zip(req.out, need):
            if not (isinstance(o, torch.Tensor) and o.device.type == "cpu" and o.is_contiguous()
                    and _nbytes(torch, o) >= b):
                raise ValueError(f"output buffers: contiguous CPU tensors of at least {need} bytes")


def _nbytes(torch, a) -> int:
    if isinstance(a, torch.Tensor):
        return a.numel() * a.element_size()
    if isinstance(a, (bytes, bytearray, memoryview)):
        return len(a)
    return int(np.asarray(a).nbytes)


def _host_u8(torch, a):
    """A request input as a flat uint8 host tensor (pinned once staged)."""
    if isinstance(a, torch.Tensor):
        return a.reshape(-1).view(torch.uint8)
    if isinstance(a, (bytes, bytearray)):
        return torch.frombuffer(bytearray(a), dtype=torch.uint8)
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1).view(np.uint8))


def _stage(torch, a):
    """A pinned host copy of input `a` (itself if it already is a pinned CPU tensor)."""
    if isinstance(a, torch.Tensor) and (a.is_cuda or a.is_pinned()):
        return a
    src = _host_u8(torch, a)
    dst = torch.empty(src.numel(), dtype=torch.uint8, pin_memory=True)
    dst.copy_(src)
    return dst


class Server:
    """Continuous-batching server.

    lanes: batches in flight at once (each on its own stream); max_batch: requests per batch;
    mem_budget: device bytes that admitted requests may hold at once (default: half of the
    device memory free at start).  A request larger than the whole budget is rejected.
    ``lane_factory(i)`` builds a lane (GpuLane by default; tests pass CPU fakes).
    stage_threads: threads that copy inputs which are not pinned host tensors into pinned
    memory before they join the queue (GPU lanes only; 0 = the scheduler copies from pageable
    memory itself)."""

    def __init__(self, device: int = 0, lanes: int = 3, max_batch: int = 64,
                 mem_budget: int | None = None, lane_factory=None, stage_threads: int | None = None):
        self.max_batch = max_batch
        self._stager = None
        if lane_factory is None:
            if stage_threads is None:
                stage_threads = min(8, os.cpu_count() or 1)
            if stage_threads > 0:
                self._stager = ThreadPoolExecutor(max_workers=stage_threads, thread_name_prefix="fds-stage")
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
        self._pending = 0               # requests still being staged
        self._lock = threading.Lock()
        self._stop = False
        self._thread = threading.Thread(target=self._loop, name="fds-serve", daemon=True)
        self._thread.start()

    def submit(self, req: Request) -> Future:
        if req.kind not in ("protect", "restore"):
            raise ValueError("kind must be 'protect' or 'restore'")
        if req.device_bytes() > self.mem_budget:
            raise ValueError("request larger than the server's device-memory budget")
        _check_buffers(req)
        req.arrival = time.perf_counter()
        if self._stager is not None and not self._pinned(req):
            with self._lock:
                self._pending += 1
            self._stager.submit(self._stage_then_queue, req)
        else:
            self.inbox.put(req)
        return req.future

    @staticmethod
    def _pinned(req: Request) -> bool:
        import torch
        return all(isinstance(a, torch.Tensor) and (a.is_cuda or a.is_pinned()) for a in req.inputs())

    def _stage_then_queue(self, req: Request) -> None:
        import torch
        try:
            req._staged = tuple(_stage(torch, a) for a in req.inputs())
        except BaseException as exc:                          # the request fails, not the server
            req.future.set_exception(exc)
            with self._lock:
                self._pending -= 1
            return
        self.inbox.put(req)
        with self._lock:
            self._pending -= 1

    def close(self) -> None:
        self._stop = True
        self._thread.join()
        if self._stager is not None:
            self._stager.shutdown(wait=True)
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
                        self._retire(lane)
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
                if self._stop and not self.ready and busy == 0 and self.inbox.empty() and self._pending == 0:
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

    def _retire(self, lane) -> None:
        """A batch the GPU has finished: its device memory is free; its results are delivered
        (copied out by the staging pool when they come as builders), then the lane is free."""
        parts = lane.finish()
        for r, _ in parts:
            self.in_use -= r.device_bytes()
        deferred = [(r, res) for r, res in parts if callable(res)]
        now = time.perf_counter()
        for r, res in parts:
            if not callable(res):
                r.done = now
                r.future.set_result(res)
        if not deferred:
            if hasattr(lane, "release"):
                lane.release()
            return
        if self._stager is None:
            for r, fn in deferred:
                self._deliver(r, fn)
            lane.release()
            return
        left = [len(deferred)]

        def run(r, fn):
            self._deliver(r, fn)
            with self._lock:
                left[0] -= 1
                last = left[0] == 0
            if last:
                lane.release()

        for r, fn in deferred:
            self._stager.submit(run, r, fn)

    @staticmethod
    def _deliver(r: Request, fn) -> None:
        try:
            res = fn()
        except BaseException as exc:
            r.done = time.perf_counter()
            r.future.set_exception(exc)
            return
        r.done = time.perf_counter()
        r.future.set_result(res)

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
