"""Serving loop on the GPU: requests that run together (overlapping on several streams, small
ones merged into batched launches) give exactly the result they give alone."""
import numpy as np
import pytest

import oracle
from paper_2008_01765_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bos():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_01765_gb300 import _build
    _build.build()
    from paper_2008_01765_gb300 import bos as b
    return b


def test_results_same_alone_and_in_the_mix(bos):
    from paper_2008_01765_gb300 import serve
    rng = np.random.default_rng(4)
    sizes = np.floor(np.exp2(rng.uniform(8, 19, size=48))).astype(int)
    jobs = [(inputs.make_records(int(n), 16, "uniform" if j % 3 else "dup1024", seed=j, payload="random"),
             int(j % 2), 1000 + j) for j, n in enumerate(sizes)]
    srv = serve.Server(budget_bytes=2 << 30, workers=4, rec_bytes=16, small_max=1 << 13, max_batch=16)
    reqs = [srv.submit(recs, op=op, seed=seed) for recs, op, seed in jobs]
    got = [r.wait(300) for r in reqs]
    srv.close()
    assert sum(r.batched for r in reqs) > 0  # some requests shared a batched launch
    for (recs, op, seed), r, out in zip(jobs, reqs, got):
        x = bos.to_device(recs)
        alone, info = (bos.sort if op else bos.orp)(x, 16, Z=r.Z, seed=seed)
        np.testing.assert_array_equal(out, bos.to_host(alone, recs.dtype))
        ref, rinfo = (oracle.sort if op else oracle.orp)(recs, r.Z, seed, method=oracle.CLOSED)
        np.testing.assert_array_equal(out, ref)
        assert r.attempts == rinfo.attempts
    st = srv.stats()
    assert st["requests"] == len(jobs)
