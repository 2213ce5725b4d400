"""Scheduling logic of the serving loop, with a fake executor (CPU only)."""
import threading
import time

import numpy as np
import pytest

from paper_2008_01765_gb300 import inputs, serve


class FakeExecutor:
    """Records overlap and returns the input reversed (stands in for the GPU work)."""

    live = 0
    peak = 0
    lock = threading.Lock()

    def _enter(self):
        with FakeExecutor.lock:
            FakeExecutor.live += 1
            FakeExecutor.peak = max(FakeExecutor.peak, FakeExecutor.live)

    def _leave(self):
        with FakeExecutor.lock:
            FakeExecutor.live -= 1

    def run_one(self, r):
        self._enter()
        time.sleep(0.002 + r.n * 1e-8)
        r.result = r.recs[::-1].copy()
        r.attempts = 1
        self._leave()

    def run_batch(self, rs):
        self._enter()
        time.sleep(0.002)
        for r in rs:
            r.result = r.recs[::-1].copy()
            r.attempts = 1
        self._leave()


def make_server(budget, workers=4, small_max=1000, max_batch=8):
    return serve.Server(budget_bytes=budget, workers=workers, rec_bytes=8, small_max=small_max,
                        max_batch=max_batch, executor_factory=FakeExecutor,
                        need_fn=lambda n, R, Z, op: 100 * n, z_fn=lambda n: 512)


def test_budget_is_never_exceeded_and_all_requests_finish():
    FakeExecutor.peak = 0
    srv = make_server(budget=100 * 50_000, workers=4)
    rng = np.random.default_rng(1)
    reqs = [srv.submit(inputs.make_records(int(n), 8, seed=i), op=int(i % 2), seed=i)
            for i, n in enumerate(rng.integers(10, 40_000, size=60))]
    for r in reqs:
        out = r.wait(30)
        np.testing.assert_array_equal(out, r.recs[::-1])
    srv.close()
    assert srv.peak_held <= 100 * 50_000
    assert FakeExecutor.peak >= 2  # requests overlapped
    st = srv.stats()
    assert st["requests"] == 60 and st["p99_ms"] >= st["p50_ms"]


def test_small_requests_are_batched_and_large_are_not():
    srv = make_server(budget=1 << 40, workers=1, small_max=1000, max_batch=8)
    gate = srv.submit(inputs.make_records(5000, 8, seed=0))  # occupies the only worker
    smalls = [srv.submit(inputs.make_records(100, 8, seed=i), seed=i) for i in range(1, 20)]
    big = srv.submit(inputs.make_records(4000, 8, seed=99))
    for r in [gate, big] + smalls:
        r.wait(30)
    srv.close()
    assert not gate.batched and not big.batched
    assert sum(r.batched for r in smalls) >= 8


def test_fifo_start_order_and_oversize_rejection():
    srv = make_server(budget=100 * 10_000, workers=1)
    too_big = srv.submit(inputs.make_records(20_000, 8))
    with pytest.raises(MemoryError):
        too_big.wait(5)
    reqs = [srv.submit(inputs.make_records(5000, 8, seed=i), seed=i) for i in range(6)]
    for r in reqs:
        r.wait(30)
    srv.close()
    starts = [r.t_start for r in reqs]
    assert starts == sorted(starts)
    with pytest.raises(RuntimeError):
        srv.submit(inputs.make_records(10, 8))
