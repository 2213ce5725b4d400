"""Serving loop for ORP and sort requests (continuous batching; no counterpart in the paper).

Requests arrive at any time (submit). A request is admitted when the device-memory budget
holds its input, output and workspace; admitted work runs on a pool of worker threads, each with
its own CUDA stream, so requests overlap on the device. When a worker frees up it takes the next
admitted request - or, if several small requests are waiting, up to `max_batch` of them as one
batched launch (bos_sort_batched). A request's result never depends on what it ran with: its
seed and Z are its own (Z from the per-size-class table when not given).

The scheduling is independent of the GPU: `executor` does the work; the default executor runs the
library's CUDA path, and tests may pass a fake one.
"""
import collections
import threading
import time

import numpy as np


class Request:
    __slots__ = ("id", "op", "recs", "seed", "Z", "n", "rec_bytes", "t_arrival", "t_start", "t_done",
                 "result", "attempts", "error", "need_bytes", "_event", "batched")

    def __init__(self, rid, op, recs, seed, Z, rec_bytes):
        self.id, self.op, self.recs, self.seed, self.Z = rid, op, recs, seed, Z
        self.rec_bytes = rec_bytes
        self.n = recs.shape[0]
        self.t_arrival = self.t_start = self.t_done = None
        self.result = None
        self.attempts = 0
        self.error = None
        self.need_bytes = 0
        self.batched = False
        self._event = threading.Event()

    def wait(self, timeout=None):
        if not self._event.wait(timeout):
            raise TimeoutError(f"request {self.id} not done")
        if self.error is not None:
            raise self.error
        return self.result

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.t_arrival


def device_bytes(n, rec_bytes, Z, op):
    """Device memory a request holds while it runs: input, output and the library's workspace."""
    from . import bos
    w = bos.workspace_bytes(n, bos.params(rec_bytes, Z, 0)) if n else 0
    return 2 * n * rec_bytes + w


class CudaExecutor:
    """Runs requests with the library's CUDA path; one instance per worker (own stream).

    The worker's device buffers (input, output, workspace) and its pinned host staging buffers
    stay resident: they grow to the largest request the worker has run and are reused, so a
    request costs no device allocation once the worker has seen one as large (the admission
    budget bounds the requests' needs; each worker holds at most its largest request's).

    keep_results=False reads each result back into the pinned buffer and keeps no copy
    (benchmarks of long streams)."""

    def __init__(self, device="cuda:0", keep_results=True):
        import torch
        from . import bos
        self.torch, self.bos = torch, bos
        self.device = torch.device(device)
        self.stream = torch.cuda.Stream(self.device)
        self.keep = keep_results
        self.buf = {}  # name -> resident uint8 tensor

    def _resident(self, name, nbytes, pinned=False):
        t = self.buf.get(name)
        if t is None or t.numel() < nbytes:
            del t
            self.buf.pop(name, None)
            if pinned:
                t = self.torch.empty(max(nbytes, 1), dtype=self.torch.uint8, pin_memory=True)
            elif name == "ws":
                t = self.bos.alloc_workspace(max(nbytes, 256), self.device)
            else:
                t = self.torch.empty(max(nbytes, 1), dtype=self.torch.uint8, device=self.device)
            self.buf[name] = t
        return t

    def _upload(self, flat):
        """Host bytes -> the resident device input, through the pinned staging buffer."""
        nb = flat.size
        hin = self._resident("h_in", nb, pinned=True)
        hin[:nb].numpy()[:] = flat
        x = self._resident("x", nb)
        x[:nb].copy_(hin[:nb], non_blocking=True)
        return x

    def _download(self, out, nb):
        hout = self._resident("h_out", nb, pinned=True)
        hout[:nb].copy_(out[:nb], non_blocking=True)
        return hout

    def run_one(self, r: Request):
        torch, bos = self.torch, self.bos
        nb = r.n * r.rec_bytes
        with torch.cuda.stream(self.stream):
            x = self._upload(np.ascontiguousarray(r.recs).view(np.uint8).reshape(-1))
            out = self._resident("out", nb)
            p = bos.params(r.rec_bytes, r.Z, r.seed)
            ws = self._resident("ws", bos.workspace_bytes(r.n, p))
            fn = bos.sort_raw if r.op == 1 else bos.orp_raw
            info = fn(x.data_ptr(), out.data_ptr(), r.n, p, ws.data_ptr(), ws.numel(),
                      bos._stream_handle(self.stream))
            hout = self._download(out, nb)
        self.stream.synchronize()
        r.result = hout[:nb].numpy().view(r.recs.dtype).copy() if self.keep else None
        r.attempts = int(info.attempts)

    def run_batch(self, rs):
        torch, bos = self.torch, self.bos
        sizes = np.array([r.n for r in rs], dtype=np.int64)
        offs = np.zeros(len(rs) + 1, dtype=np.uint64)
        np.cumsum(sizes, out=offs[1:])
        flat = np.concatenate([np.ascontiguousarray(r.recs).view(np.uint8).reshape(-1) for r in rs])
        nb = flat.size
        with torch.cuda.stream(self.stream):
            x = self._upload(flat)
            out = self._resident("out", nb)
            base = bos.params(rs[0].rec_bytes, 512, 0)
            seeds = np.array([r.seed for r in rs], dtype=np.uint64)
            ops = np.array([r.op for r in rs], dtype=np.uint8)
            Zs = np.array([r.Z for r in rs], dtype=np.uint32)
            need = bos.batched_workspace_bytes(offs, Zs, ops, base)
            batch = bos.Batch(x[:nb], out[:nb], offs, seeds, ops, base, Zs=Zs,
                              workspace=self._resident("ws", need))
            att = batch.run(self.stream)
            hout = self._download(out, nb)
        self.stream.synchronize()
        for j, r in enumerate(rs):
            a, b = int(offs[j]) * r.rec_bytes, int(offs[j + 1]) * r.rec_bytes
            r.result = hout[a:b].numpy().view(r.recs.dtype).copy() if self.keep else None
            r.attempts = int(att[j])


class Server:
    """Admits requests under a device-memory budget and runs them on `workers` streams.

    budget_bytes: device memory the admitted requests may hold at once (input + output +
    workspace each). small_max: requests of at most this many records may be batched together,
    up to max_batch per launch.
    """

    def __init__(self, budget_bytes=64 << 30, workers=4, rec_bytes=16, small_max=1 << 16, max_batch=64,
                 executor_factory=None, need_fn=None, z_fn=None):
        self.budget = budget_bytes
        self.rec_bytes = rec_bytes
        self.small_max = small_max
        self.max_batch = max_batch
        self.need_fn = need_fn or device_bytes
        if z_fn is None:
            from . import autotune
            table = autotune.load_table()
            z_fn = lambda n: autotune.z_for(n, rec_bytes, table)  # noqa: E731
        self.z_fn = z_fn
        self.queue = collections.deque()
        self.cv = threading.Condition()
        self.held = 0
        self.peak_held = 0
        self.closed = False
        self.done = []
        self.next_id = 0
        factory = executor_factory or (lambda: CudaExecutor())
        self.threads = []
        for w in range(workers):
            t = threading.Thread(target=self._worker, args=(factory,), daemon=True, name=f"bos-worker-{w}")
            t.start()
            self.threads.append(t)

    def submit(self, recs, op=1, seed=1, Z=None) -> Request:
        """Queue one request (op 0 = ORP, 1 = sort) of a structured record array."""
        with self.cv:
            if self.closed:
                raise RuntimeError("server closed")
            r = Request(self.next_id, op, recs, seed, Z or self.z_fn(recs.shape[0]), self.rec_bytes)
            self.next_id += 1
            r.need_bytes = self.need_fn(r.n, self.rec_bytes, r.Z, op)
            if r.need_bytes > self.budget:
                r.error = MemoryError(f"request {r.id} needs {r.need_bytes} bytes, budget {self.budget}")
                r.t_arrival = r.t_done = time.perf_counter()
                r._event.set()
                return r
            r.t_arrival = time.perf_counter()
            self.queue.append(r)
            self.cv.notify_all()
        return r

    def _take(self):
        """FIFO admission: the head request when it fits the budget; with it, following small
        requests that also fit (one batched launch)."""
        while True:
            if self.queue:
                head = self.queue[0]
                if self.held + head.need_bytes <= self.budget:
                    self.queue.popleft()
                    taken = [head]
                    self.held += head.need_bytes
                    if head.n <= self.small_max:
                        while (self.queue and len(taken) < self.max_batch and self.queue[0].n <= self.small_max
                               and self.held + self.queue[0].need_bytes <= self.budget):
                            r = self.queue.popleft()
                            self.held += r.need_bytes
                            taken.append(r)
                    self.peak_held = max(self.peak_held, self.held)
                    return taken
            elif self.closed:
                return None
            self.cv.wait()

    def _worker(self, factory):
        ex = None
        while True:
            with self.cv:
                taken = self._take()
            if taken is None:
                return
            try:
                if ex is None:
                    ex = factory()
                t0 = time.perf_counter()
                for r in taken:
                    r.t_start = t0
                    r.batched = len(taken) > 1
                if len(taken) == 1:
                    ex.run_one(taken[0])
                else:
                    ex.run_batch(taken)
            except Exception as e:  # report on every request of the launch
                for r in taken:
                    r.error = e
            t1 = time.perf_counter()
            with self.cv:
                for r in taken:
                    r.t_done = t1
                    self.held -= r.need_bytes
                    self.done.append(r)
                    r._event.set()
                self.cv.notify_all()

    def close(self, wait=True):
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        if wait:
            for t in self.threads:
                t.join()

    def stats(self):
        lat = np.array([r.latency for r in self.done if r.error is None], dtype=np.float64)
        recs = sum(r.n for r in self.done if r.error is None)
        if lat.size == 0:
            return {"requests": 0}
        t0 = min(r.t_arrival for r in self.done)
        t1 = max(r.t_done for r in self.done)
        return {"requests": int(lat.size), "records": int(recs),
                "records_per_s": recs / (t1 - t0) if t1 > t0 else 0.0,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "batched_requests": int(sum(r.batched for r in self.done)), "peak_held_bytes": int(self.peak_held)}
