"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

n = 2^30 16-byte records (Z = 1024, B = 2^21): sampled final buckets of the ORP are compared bit
for bit with the oracle's bucket-by-bucket computation; the sort is checked over the whole
output (non-decreasing keys, a permutation of the input; with all keys equal it must equal the
ORP output, ties keeping ORP order). The 4096-array batch is checked array by array on a sample.
"""
import numpy as np
import pytest

import oracle
from paper_2008_01765_gb300 import inputs

pytestmark = pytest.mark.gpu

N30 = 1 << 30
Z30 = 1024


@pytest.fixture(scope="module")
def bos():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_01765_gb300 import _build
    _build.build()
    from paper_2008_01765_gb300 import bos as b
    return b


@pytest.fixture(scope="module")
def big(bos):
    import torch
    free, _ = torch.cuda.mem_get_info()
    p = bos.params(16, Z30, 7)
    need = 2 * N30 * 16 + bos.workspace_bytes(N30, p)
    if free < need + (4 << 30):
        pytest.skip(f"needs {need / 2**30:.0f} GiB of device memory")
    ws = bos.alloc_workspace(bos.workspace_bytes(N30, p))
    x = torch.empty(N30 * 16, dtype=torch.uint8, device="cuda")
    out = torch.empty_like(x)
    rng = np.random.default_rng(2)
    B = N30 * 2 // Z30
    buckets = np.unique(np.concatenate([[0, 1, B // 2, B - 1], rng.integers(0, B, size=8)]))
    off, load, src = oracle.orp_sample(N30, Z30, 7, buckets)  # labels do not depend on the data
    yield dict(ws=ws, x=x, out=out, buckets=buckets, off=off, load=load, src=src)
    del ws, x, out
    torch.cuda.empty_cache()


def _slice(t, a, b):
    return t[a * 16:b * 16].cpu().numpy().view(inputs.REC16)


@pytest.mark.parametrize("dist", ["uniform", "equal", "reverse"])
def test_orp_2p30_sampled_buckets(bos, big, dist):
    import torch
    recs = inputs.make_records(N30, 16, dist, seed=1)
    big["x"].copy_(torch.from_numpy(recs.view(np.uint8)))
    _, info = bos.orp(big["x"], 16, Z=Z30, seed=7, out=big["out"], workspace=big["ws"])
    torch.cuda.synchronize()
    assert info.attempts == 1 and info.B == N30 * 2 // Z30 and info.L == 21
    for o, m, src in zip(big["off"], big["load"], big["src"]):
        seg = _slice(big["out"], int(o), int(o) + int(m))
        np.testing.assert_array_equal(seg["payload"], src)          # payload = input index
        np.testing.assert_array_equal(seg["key"], recs["key"][src])


@pytest.mark.parametrize("dist", ["uniform", "equal", "reverse"])
def test_sort_2p30_whole_output(bos, big, dist):
    import torch
    recs = inputs.make_records(N30, 16, dist, seed=1)
    big["x"].copy_(torch.from_numpy(recs.view(np.uint8)))
    _, info = bos.sort(big["x"], 16, Z=Z30, seed=7, out=big["out"], workspace=big["ws"])
    torch.cuda.synchronize()
    assert info.attempts == 1
    got = big["out"].cpu().numpy().view(inputs.REC16)
    keys = got["key"]
    assert np.all(keys[1:] >= keys[:-1])
    seen = np.zeros(N30, dtype=bool)
    seen[got["payload"]] = True
    assert seen.all()  # every input record exactly once (payload = index, n entries)
    np.testing.assert_array_equal(keys, recs["key"][got["payload"]])
    if dist == "equal":  # every tie keeps the ORP order: the sort output is the ORP output
        for o, m, src in zip(big["off"], big["load"], big["src"]):
            np.testing.assert_array_equal(got["payload"][int(o):int(o) + int(m)], src)
    if dist == "reverse":
        np.testing.assert_array_equal(keys, np.arange(N30, dtype=np.uint64))


def _trace_digest(bos, recs, Z, seed):
    import torch
    buf = torch.zeros(1 << 28, dtype=torch.uint8, device="cuda")
    bos.trace_attach(buf)
    try:
        bos.orp(bos.to_device(recs), 16, Z=Z, seed=seed)
        torch.cuda.synchronize()
    finally:
        bos.trace_attach(None)
    w = buf.view(torch.int64).cpu().numpy().view(np.uint64)
    cnt = int(w[0])
    assert 0 < cnt <= buf.numel() // 16 - 1
    ent = w[2:2 + 2 * cnt].reshape(cnt, 2)
    return ent[np.lexsort((ent[:, 1], ent[:, 0]))]


def test_address_trace_2p20_identical_across_inputs(bos):
    # Same n, Z and seed; uniform, all-equal and reverse-sorted keys: the multiset of global
    # accesses (kind, buffer, bytes, offset) of the whole ORP is identical (Section 3.1).
    n, Z = 1 << 20, 1024
    base = _trace_digest(bos, inputs.make_records(n, 16, "uniform", seed=3), Z, 9)
    for dist in ("equal", "reverse"):
        np.testing.assert_array_equal(_trace_digest(bos, inputs.make_records(n, 16, dist, seed=3), Z, 9), base)


@pytest.mark.parametrize("dist", ["equal", "reverse"])
def test_trace_digest_2p30_identical_across_inputs(bos, big, dist):
    # The full n = 2^30 benchmark ORP, in bench.py's plan, through the order-independent trace
    # digest (count and sum of a 64-bit mix of every global access, Section 3.1): uniform,
    # all-equal and reverse-sorted keys give the same digest for one seed.
    import torch

    def digest(d):
        recs = inputs.make_records(N30, 16, d, seed=1)
        big["x"].copy_(torch.from_numpy(recs.view(np.uint8)))
        buf = torch.zeros(256 * 16, dtype=torch.uint8, device="cuda")
        bos.trace_attach_digest(buf)
        try:
            bos.orp(big["x"], 16, Z=Z30, seed=7, out=big["out"], workspace=big["ws"])
            torch.cuda.synchronize()
        finally:
            bos.trace_attach_digest(None)
        w = buf.view(torch.int64).cpu().numpy().view(np.uint64).reshape(256, 2)
        return int(w[:, 0].sum()), int(w[:, 1].sum(dtype=np.uint64))

    if "digest_uniform" not in big:
        big["digest_uniform"] = digest("uniform")
    cnt, h = big["digest_uniform"]
    assert cnt > 2 * N30  # every slot of the first pass's output and the LAST pass's input, at least
    assert digest(dist) == (cnt, h)


def test_batched_4096_arrays_sampled(bos):
    # The benchmark's batch (4096 arrays, sizes log-uniform in [2^10, 2^20], Z per size class),
    # run as one launch sequence; 24 arrays are checked against the oracle run alone.
    import torch
    from paper_2008_01765_gb300 import autotune
    sizes = inputs.batched_sizes(4096, 10.0, 20.0, seed=1)
    recs, offs = inputs.make_batch(sizes, 8, seed=1)
    Zs = autotune.z_array(sizes, 8)
    seeds = np.arange(1, sizes.size + 1, dtype=np.uint64)
    ops = np.ones(sizes.size, dtype=np.uint8)
    ops[::2] = 0
    x = bos.to_device(recs)
    out = torch.empty_like(x)
    att = bos.sort_batched(x, out, offs, seeds, ops, bos.params(8, 512, 0), Zs=Zs)
    got = out.cpu().numpy().view(inputs.REC8)
    rng = np.random.default_rng(3)
    for j in np.unique(np.concatenate([[0, sizes.size - 1], rng.integers(0, sizes.size, size=22)])):
        a, b = int(offs[j]), int(offs[j + 1])
        f = oracle.sort if ops[j] else oracle.orp
        ref, rinfo = f(recs[a:b], int(Zs[j]), int(seeds[j]), method=oracle.CLOSED)
        assert att[j] == rinfo.attempts
        np.testing.assert_array_equal(got[a:b], ref, err_msg=f"array {j}")
