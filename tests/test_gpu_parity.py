"""CUDA path against the oracle, element by element, through the C ABI (libbos.so).

Integer and byte work: every comparison is bit-exact. The oracle's closed form is used for
speed; it is pinned to the literal Algorithm 3.1 by the CPU tests.
"""
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
    b.lib()
    return b


def gpu_orp(bos, recs, Z, seed, **kw):
    out, info = bos.orp(bos.to_device(recs), recs.dtype.itemsize, Z=Z, seed=seed, **kw)
    return bos.to_host(out, recs.dtype), info


def gpu_sort(bos, recs, Z, seed, **kw):
    out, info = bos.sort(bos.to_device(recs), recs.dtype.itemsize, Z=Z, seed=seed, **kw)
    return bos.to_host(out, recs.dtype), info


def test_philox_matches_curand_and_oracle(bos):
    import torch
    rng = np.random.default_rng(5)
    n = 1 << 20
    ctr = rng.integers(0, 1 << 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 1 << 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:1000] = 0  # include the all-zero corner and small counters
    ctr[:1000, 2] = np.arange(1000)
    mine, ref = bos.selftest_philox(torch.from_numpy(ctr.view(np.int32)).cuda(),
                                    torch.from_numpy(key.view(np.int32)).cuda())
    mine = mine.cpu().numpy().view(np.uint32)
    ref = ref.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(mine, ref)
    np.testing.assert_array_equal(mine, oracle.philox_many(ctr, key))


ORP_CASES = [
    # (n, Z, rec_bytes, k)
    (1, 512, 8, 0), (2, 4, 8, 0), (3, 4, 16, 0), (5, 2, 8, 0), (7, 3, 16, 0),
    (100, 8, 8, 0), (1000, 32, 16, 0), (4097, 64, 8, 0), (4097, 64, 8, 1),
    (12345, 12, 16, 0), (30000, 5, 8, 0),
    (1 << 16, 512, 8, 1), (1 << 16, 512, 8, 0), (1 << 16, 512, 16, 0),
    ((1 << 20) + 3, 512, 16, 0), (300000, 1024, 16, 0), (300000, 1024, 16, 2),
    ((1 << 18) - 1, 96, 8, 0), (1 << 19, 4096, 8, 0), (1 << 17, 2, 8, 0),
]


@pytest.mark.parametrize("n,Z,rec_bytes,k", ORP_CASES)
def test_orp_matches_oracle(bos, n, Z, rec_bytes, k):
    recs = inputs.make_records(n, rec_bytes, "uniform", seed=n + Z)
    for seed in (1, 0xDEADBEEFCAFEF00D):
        try:
            ref, rinfo = oracle.orp(recs, Z, seed, max_attempts=64, method=oracle.CLOSED)
        except oracle.OracleError as e:
            # tiny Z: every attempt overflows (Lemma 3.2); the library must say so too
            assert e.status == oracle.ERR_OVERFLOW
            with pytest.raises(bos.BosError) as ge:
                gpu_orp(bos, recs, Z, seed, k=k, max_attempts=64)
            assert ge.value.status == bos.ERR_OVERFLOW
            continue
        got, info = gpu_orp(bos, recs, Z, seed, k=k, max_attempts=64)
        assert info.attempts == rinfo.attempts
        assert info.B == rinfo.B and info.L == rinfo.L
        np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("rec_bytes", [8, 16])
@pytest.mark.parametrize("dist", inputs.DISTRIBUTIONS)
def test_sort_matches_oracle(bos, rec_bytes, dist):
    for n, Z in [(5000, 64), (1 << 16, 512), (200003, 256)]:
        recs = inputs.make_records(n, rec_bytes, dist, seed=3)
        ref, rinfo = oracle.sort(recs, Z, 7, method=oracle.CLOSED)
        got, info = gpu_sort(bos, recs, Z, 7)
        assert info.attempts == rinfo.attempts
        np.testing.assert_array_equal(got, ref)
        if dist == "equal":
            assert info.radix_passes == 0


def test_result_independent_of_k(bos):
    recs = inputs.make_records(1 << 18, 16, "dup1024", seed=9)
    outs = []
    for k in (1, 2, 3, 4, 0):
        got, info = gpu_sort(bos, recs, 256, 11, k=k)
        outs.append(got)
        if k == 1:
            assert info.passes == info.L
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])


def test_forced_overflow_retry(bos):
    recs = inputs.make_records(50000, 16, "uniform", seed=2)
    got, info = gpu_orp(bos, recs, 128, 5, flags=bos.FLAG_FORCE_OVERFLOW(2))
    assert info.attempts == 3
    ref, _ = oracle.orp(recs, 128, 5, method=oracle.CLOSED, first_attempt=2)
    np.testing.assert_array_equal(got, ref)
    with pytest.raises(bos.BosError) as e:
        gpu_orp(bos, recs, 128, 5, flags=bos.FLAG_FORCE_OVERFLOW(3), max_attempts=3)
    assert e.value.status == bos.ERR_OVERFLOW


def test_real_overflow_retries_match_oracle(bos):
    # n = 4096, Z = 32 (B = 256) overflows in about 14% of attempts (Lemma 3.2); the attempt
    # that first succeeds must agree with the oracle's.
    recs = inputs.make_records(4096, 8, "uniform", seed=4)
    seen_retry = False
    for seed in range(60):
        try:
            ref, rinfo = oracle.orp(recs, 32, seed, max_attempts=16, method=oracle.CLOSED)
        except oracle.OracleError:
            with pytest.raises(bos.BosError):
                gpu_orp(bos, recs, 32, seed, max_attempts=16)
            continue
        got, info = gpu_orp(bos, recs, 32, seed, max_attempts=16)
        assert info.attempts == rinfo.attempts
        seen_retry |= info.attempts > 1
        np.testing.assert_array_equal(got, ref)
    assert seen_retry


def test_lookback_timeout_reports_status_and_context_survives(bos):
    recs = inputs.make_records(20000, 8, "uniform", seed=6)
    with pytest.raises(bos.BosError) as e:
        gpu_orp(bos, recs, 64, 3, flags=bos.FLAG_SKIP_PUBLISH)
    assert e.value.status == bos.ERR_TIMEOUT
    got, _ = gpu_orp(bos, recs, 64, 3)
    ref, _ = oracle.orp(recs, 64, 3, method=oracle.CLOSED)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("rec_bytes", [8, 16])
@pytest.mark.parametrize("n", [1, 2, 64, 4096, 1 << 16, 1 << 20])
def test_bitonic_matches_sort_by_key_payload(bos, rec_bytes, n):
    recs = inputs.make_records(n, rec_bytes, "dup1024", seed=n, payload="random")
    out = bos.bitonic_sort(bos.to_device(recs), rec_bytes)
    got = bos.to_host(out, recs.dtype)
    np.testing.assert_array_equal(got, np.sort(recs, order=["key", "payload"]))


def test_batched_equals_alone(bos):
    sizes = inputs.batched_sizes(24, 4, 16, seed=3)
    sizes[0] = 0
    sizes[1] = 1
    recs, offs = inputs.make_batch(sizes, 8, seed=2)
    seeds = np.arange(100, 100 + sizes.size, dtype=np.uint64)
    ops = (np.arange(sizes.size) % 2).astype(np.uint8)
    Zs = np.where(np.arange(sizes.size) % 3 == 0, 64, 512).astype(np.uint32)
    x = bos.to_device(recs)
    import torch
    out = torch.empty_like(x)
    att = bos.sort_batched(x, out, offs, seeds, ops, bos.params(8, 512, 0), Zs=Zs)
    got = bos.to_host(out, recs.dtype)
    for j in range(sizes.size):
        a, b = int(offs[j]), int(offs[j + 1])
        f = oracle.sort if ops[j] else oracle.orp
        ref, rinfo = f(recs[a:b], int(Zs[j]), int(seeds[j]), method=oracle.CLOSED)
        assert att[j] == (rinfo.attempts if b > a else 0)
        np.testing.assert_array_equal(got[a:b], ref)


def _trace(bos, recs, Z, seed, k=0, flags=0):
    import torch
    buf = torch.zeros(1 << 27, dtype=torch.uint8, device="cuda")
    bos.trace_attach(buf)
    try:
        gpu_orp(bos, recs, Z, seed, k=k, flags=flags)
        torch.cuda.synchronize()
    finally:
        bos.trace_attach(None)
    w = buf.view(torch.int64).cpu().numpy().view(np.uint64)
    cnt = int(w[0])
    assert 0 < cnt <= (buf.numel() // 16 - 1)
    ent = w[2:2 + 2 * cnt].reshape(cnt, 2)
    order = np.lexsort((ent[:, 1], ent[:, 0]))
    return ent[order]


@pytest.mark.parametrize("k", [1, 0])
def test_address_trace_is_input_independent(bos, k):
    n, Z = 1 << 14, 256
    base = None
    for dist in ("uniform", "equal", "sorted", "reverse"):
        recs = inputs.make_records(n, 16, dist, seed=12)
        t = _trace(bos, recs, Z, seed=4, k=k)
        if base is None:
            base = t
        else:
            np.testing.assert_array_equal(t, base)
    # Across seeds the butterfly passes (everything but the compacted output writes, whose
    # addresses follow the final loads, Lemma 3.3) are identical too.
    t2 = _trace(bos, inputs.make_records(n, 16, "uniform", seed=12), Z, seed=99, k=k)
    kind_buf = lambda t: ((t[:, 0] >> np.uint64(48)) & np.uint64(0xFF))
    keep = lambda t: t[kind_buf(t) != 5]
    np.testing.assert_array_equal(keep(t2), keep(base))
    # every slot of every bucket is read and written by each butterfly pass: counts check
    assert len(keep(base)) > 0


OBLIVIOUS_CASES = [
    (1, 2, 8), (3, 4, 16), (1000, 64, 8), (5000, 96, 16), (1 << 16, 512, 8), (300001, 256, 16),
    ((1 << 18) + 5, 1024, 16), (20000, 4096, 8), (700, 8, 8),
]


@pytest.mark.parametrize("n,Z,rec_bytes", OBLIVIOUS_CASES)
def test_oblivious_split_matches_oracle(bos, n, Z, rec_bytes):
    # Section 4.1's form (bitonic MergeSplits, bitonic in-bin permutations) gives the oracle's ORP:
    # L = 0, 1 and many levels, Z not a power of two, Z = 4096, and a small Z that overflows and
    # retries (same attempts as the oracle, or overflow on every attempt on both sides).
    recs = inputs.make_records(n, rec_bytes, "uniform", seed=n % 997 + 5)
    seed = 0xABC + n
    try:
        ref, rinfo = oracle.orp(recs, Z, seed, max_attempts=16, method=oracle.CLOSED)
    except oracle.OracleError as e:
        assert e.status == oracle.ERR_OVERFLOW
        with pytest.raises(bos.BosError) as ge:
            gpu_orp(bos, recs, Z, seed, flags=bos.FLAG_OBLIVIOUS_SPLIT, max_attempts=16)
        assert ge.value.status == bos.ERR_OVERFLOW
        return
    got, info = gpu_orp(bos, recs, Z, seed, flags=bos.FLAG_OBLIVIOUS_SPLIT, max_attempts=16)
    assert info.attempts == rinfo.attempts
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("n,Z,rec_bytes,dist", [(1, 2, 16, "uniform"), (5000, 96, 16, "dup1024"),
                                                 (1 << 16, 512, 8, "uniform"), (700, 8, 8, "sorted"),
                                                 ((1 << 18) + 5, 1024, 16, "reverse")])
def test_oblivious_split_sort_matches_oracle(bos, n, Z, rec_bytes, dist):
    # The whole oblivious sort with Section 4.1's ORP, followed by the radix sort or by the merge
    # sort, equals the oracle's stable sort of its ORP (ties in ORP order).
    recs = inputs.make_records(n, rec_bytes, dist, seed=n % 991 + 7)
    seed = 0xDEF + n
    ref, rinfo = oracle.sort(recs, Z, seed, max_attempts=16, method=oracle.CLOSED)
    for flags in (bos.FLAG_OBLIVIOUS_SPLIT, bos.FLAG_OBLIVIOUS_SPLIT | bos.FLAG_MERGE_SORT):
        got, info = gpu_sort(bos, recs, Z, seed, flags=flags, max_attempts=16)
        assert info.attempts == rinfo.attempts, flags
        np.testing.assert_array_equal(got, ref, err_msg=str(flags))


def test_oblivious_split_trace_is_input_independent(bos):
    # Every global access of the Section 4.1 form (placement, each level's bucket pairs, the final
    # buckets, the strip) is the same multiset for different inputs of one size and seed.
    n, Z = 1 << 12, 64
    base = None
    for dist in ("uniform", "equal", "sorted", "reverse"):
        t = _trace(bos, inputs.make_records(n, 16, dist, seed=12), Z, seed=4, flags=bos.FLAG_OBLIVIOUS_SPLIT)
        if base is None:
            base = t
        else:
            np.testing.assert_array_equal(t, base)


def test_cfg1_plain_form_full_size(bos):
    # n = 2^16 8-byte records, uniform u32 keys, payload = index, Z = 512 (B = 256), seed 1,
    # one level per launch.
    recs = inputs.make_records(1 << 16, 8, "uniform", seed=1)
    ref, rinfo = oracle.sort(recs, 512, 1, method=oracle.CLOSED)
    got, info = gpu_sort(bos, recs, 512, 1, k=1)
    assert (info.B, info.L, info.passes) == (256, 8, 8)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("dist", ["uniform", "dup1024", "sorted"])
def test_cfg2_full_size(bos, dist):
    # n = 2^24 16-byte records, Z = 512 (B = 2^16), fused k-level passes.
    recs = inputs.make_records(1 << 24, 16, dist, seed=2)
    ref, rinfo = oracle.sort(recs, 512, 2, method=oracle.CLOSED)
    got, info = gpu_sort(bos, recs, 512, 2)
    assert (info.B, info.L) == (1 << 16, 16)
    assert info.passes < info.L
    np.testing.assert_array_equal(got, ref)


KERNEL_CASES = [
    # (n, Z, rec_bytes, k): Z a multiple of 32 selects the persistent cluster kernel
    (1 << 12, 64, 8, 0), ((1 << 16) + 77, 512, 8, 0), (1 << 16, 512, 8, 1), ((1 << 20) - 5, 512, 16, 0),
    (1 << 22, 1024, 16, 0), (300001, 96, 16, 0), (1 << 18, 32, 16, 0), (1 << 19, 4096, 8, 0),
    (999, 32, 8, 0), (1 << 21, 256, 8, 3), (1 << 12, 32, 16, 0),
]


@pytest.mark.parametrize("n,Z,rec_bytes,k", KERNEL_CASES)
def test_cluster_kernel_matches_generic_and_oracle(bos, n, Z, rec_bytes, k):
    recs = inputs.make_records(n, rec_bytes, "uniform", seed=n ^ Z)
    seed = 0x1234 + n
    try:
        ref, rinfo = oracle.orp(recs, Z, seed, max_attempts=16, method=oracle.CLOSED)
    except oracle.OracleError as e:  # every attempt overflows (small Z): all kernels must say so
        assert e.status == oracle.ERR_OVERFLOW
        for flags in (0, bos.FLAG_FEWEST_PASSES, bos.FLAG_NO_CLUSTER, bos.FLAG_GENERIC):
            with pytest.raises(bos.BosError) as ge:
                gpu_orp(bos, recs, Z, seed, k=k, flags=flags, max_attempts=16)
            assert ge.value.status == bos.ERR_OVERFLOW
        return
    outs = {}
    for name, flags in (("auto", 0), ("no_stream", bos.FLAG_NO_STREAM), ("fewest", bos.FLAG_FEWEST_PASSES),
                        ("no_cluster", bos.FLAG_NO_CLUSTER),
                        ("no_cluster_no_stream", bos.FLAG_NO_CLUSTER | bos.FLAG_NO_STREAM),
                        ("generic", bos.FLAG_GENERIC)):
        got, info = gpu_orp(bos, recs, Z, seed, k=k, flags=flags, max_attempts=16)
        assert info.attempts == rinfo.attempts, name
        np.testing.assert_array_equal(got, ref, err_msg=name)
        outs[name] = info
    if Z % 32 == 0 and k == 0 and outs["auto"].L >= 8:
        assert outs["fewest"].max_cluster > 1
        assert outs["fewest"].passes <= outs["no_stream"].passes <= outs["no_cluster_no_stream"].passes
        assert outs["auto"].passes <= outs["no_stream"].passes
    assert outs["no_cluster"].max_cluster == 1


MERGE_CASES = [
    (1, 512, 16, "uniform"), (2047, 512, 8, "uniform"), (2048, 512, 16, "dup1024"), (2049, 512, 16, "uniform"),
    (3 * 4096 + 5, 256, 16, "equal"), (1 << 16, 512, 8, "uniform"), (300001, 96, 16, "dup1024"),
    (1 << 20, 1024, 16, "reverse"), (1 << 22, 1024, 16, "uniform"), ((1 << 21) + 777, 512, 8, "sorted"),
]


@pytest.mark.parametrize("n,Z,rec_bytes,dist", MERGE_CASES)
def test_merge_sort_matches_oracle(bos, n, Z, rec_bytes, dist):
    # The comparison-based sort after the ORP (stable merge sort) gives the oracle's stable sort of
    # the ORP output: sizes around the 2048-record runs and merge chunks, odd and even numbers of
    # merge passes, duplicate and equal keys (ties keep the ORP order), Z of the generic kernel.
    recs = inputs.make_records(n, rec_bytes, dist, seed=n % 1000 + 3)
    ref, rinfo = oracle.sort(recs, Z, 21, method=oracle.CLOSED, max_attempts=16)
    got, info = gpu_sort(bos, recs, Z, 21, flags=bos.FLAG_MERGE_SORT, max_attempts=16)
    assert info.attempts == rinfo.attempts and info.radix_passes == 0
    np.testing.assert_array_equal(got, ref)


def test_cfg3_geometry_plans(bos):
    # n = 2^30 and Z = 1024 give L = 21. The fewest-passes plan uses 16-CTA clusters (7 levels a
    # pass); the measured-cost plan uses fewer levels per pass. Both give the oracle's result.
    # Checked on n = 2^22 (L = 13) with the same Z and record width.
    recs = inputs.make_records(1 << 22, 16, "uniform", seed=3)
    ref, _ = oracle.sort(recs, 1024, 5, method=oracle.CLOSED)
    got, info = gpu_sort(bos, recs, 1024, 5, flags=bos.FLAG_FEWEST_PASSES)
    np.testing.assert_array_equal(got, ref)
    assert info.max_k == 7 and info.max_cluster == 16 and info.passes == 2
    got, info = gpu_sort(bos, recs, 1024, 5)
    np.testing.assert_array_equal(got, ref)
    assert 2 <= info.passes <= 5


def _check_batch_against_oracle(recs, offs, seeds, ops, Zs, got, att):
    for j in range(len(offs) - 1):
        a, b = int(offs[j]), int(offs[j + 1])
        f = oracle.sort if ops[j] else oracle.orp
        ref, rinfo = f(recs[a:b], int(Zs[j]), int(seeds[j]), method=oracle.CLOSED)
        assert att[j] == (rinfo.attempts if b > a else 0), j
        np.testing.assert_array_equal(got[a:b], ref, err_msg=f"array {j}")


def test_batched_graph_replay_equals_alone(bos):
    # The launch sequence of a batch is captured once into a CUDA graph and replayed; every
    # array's result equals that array run alone (oracle), for mixed sizes, ops and Z.
    import torch
    sizes = inputs.batched_sizes(64, 6, 17, seed=11)
    sizes[3] = 0
    recs, offs = inputs.make_batch(sizes, 8, seed=5)
    seeds = np.arange(7, 7 + sizes.size, dtype=np.uint64) * 1000003
    ops = (np.arange(sizes.size) % 3 != 0).astype(np.uint8)
    Zs = np.array([[512, 1024, 256, 2048][j % 4] for j in range(sizes.size)], dtype=np.uint32)
    x = bos.to_device(recs)
    out = torch.empty_like(x)
    batch = bos.Batch(x, out, offs, seeds, ops, bos.params(8, 512, 0), Zs=Zs)
    batch.prepare()
    stream = torch.cuda.Stream()
    batch.enqueue(stream)  # warm-up outside the capture
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
        batch.enqueue(stream)
    out.zero_()
    graph.replay()
    att = batch.collect(stream)
    _check_batch_against_oracle(recs, offs, seeds, ops, Zs, bos.to_host(out, recs.dtype), att)
    out.zero_()
    graph.replay()  # a second replay gives the same result
    att2 = batch.collect(stream)
    np.testing.assert_array_equal(att2, att)
    _check_batch_against_oracle(recs, offs, seeds, ops, Zs, bos.to_host(out, recs.dtype), att2)


def test_batched_retries_only_overflowing_arrays(bos):
    # Z = 32 with 4096 records overflows in about 14% of attempts: such arrays rerun with the next
    # attempt counter and still match the oracle; the others keep attempt 1.
    import torch
    sizes = np.full(24, 4096, dtype=np.int64)
    recs, offs = inputs.make_batch(sizes, 16, seed=8)
    seeds = np.arange(24, dtype=np.uint64)
    ops = np.ones(24, dtype=np.uint8)
    Zs = np.full(24, 32, dtype=np.uint32)
    x = bos.to_device(recs)
    out = torch.empty_like(x)
    try:
        att = bos.sort_batched(x, out, offs, seeds, ops, bos.params(16, 32, 0, max_attempts=16), Zs=Zs)
    except bos.BosError as e:
        pytest.skip(f"an array exhausted its attempts: {e}")
    assert (att >= 1).all() and (att > 1).any()
    _check_batch_against_oracle(recs, offs, seeds, ops, Zs, bos.to_host(out, recs.dtype), att)


STREAM_CASES = [
    # (n, Z, rec_bytes, k): automatic plans whose first and middle passes run the streaming kernel
    # (orp_stream.cu). Ragged n (groups of unequal size), the Z values it takes, both widths.
    ((1 << 20) + 3, 512, 16, 0), (1 << 20, 256, 8, 0), (300001, 96, 8, 0), (4097, 64, 8, 0),
    (1 << 21, 2048, 8, 0), ((1 << 22) + 12345, 1024, 16, 0), (1 << 24, 512, 16, 0), (1 << 21, 64, 8, 0),
    (1 << 25, 1024, 16, 0),
    # k = 5 with Z = 2048: a batch brings 32-64 reals to each of the 32 output buckets, more than a
    # ring holds, so every batch is redone in rounds of 16 slots (the kernel's slow path)
    (1 << 20, 2048, 8, 5), ((1 << 20) + 1, 2048, 16, 5), (1 << 20, 1024, 16, 6),
]


@pytest.mark.parametrize("n,Z,rec_bytes,k", STREAM_CASES)
def test_stream_pass_matches_oracle(bos, n, Z, rec_bytes, k):
    recs = inputs.make_records(n, rec_bytes, "uniform", seed=(n * 7 + Z) % 100003)
    seed = 0x5EED + n
    plan = bos.plan(n, rec_bytes, Z, k=k, sort=False)
    assert plan.stream_passes >= 1
    try:
        ref, rinfo = oracle.orp(recs, Z, seed, max_attempts=16, method=oracle.CLOSED)
    except oracle.OracleError as e:
        assert e.status == oracle.ERR_OVERFLOW
        with pytest.raises(bos.BosError) as ge:
            gpu_orp(bos, recs, Z, seed, k=k, max_attempts=16)
        assert ge.value.status == bos.ERR_OVERFLOW
        return
    got, info = gpu_orp(bos, recs, Z, seed, k=k, max_attempts=16)
    assert info.attempts == rinfo.attempts and info.stream_passes == plan.stream_passes
    np.testing.assert_array_equal(got, ref)
    got2, info2 = gpu_orp(bos, recs, Z, seed, k=k, max_attempts=16, flags=bos.FLAG_NO_STREAM)
    assert info2.stream_passes == 0
    np.testing.assert_array_equal(got2, ref)


def test_stream_pass_overflow_and_retry(bos):
    # Z = 32 at n = 2^14 (B = 2^10) overflows in most attempts (Lemma 3.2); the streaming first
    # pass must flag exactly the attempts the oracle flags, intermediate levels included.
    recs = inputs.make_records(1 << 14, 16, "uniform", seed=8)
    seen = 0
    for seed in range(40):
        try:
            ref, rinfo = oracle.orp(recs, 32, seed, max_attempts=8, method=oracle.CLOSED)
        except oracle.OracleError:
            with pytest.raises(bos.BosError):
                gpu_orp(bos, recs, 32, seed, max_attempts=8, k=5)
            continue
        got, info = gpu_orp(bos, recs, 32, seed, max_attempts=8, k=5)
        assert info.stream_passes >= 1
        assert info.attempts == rinfo.attempts
        seen += info.attempts > 1
        np.testing.assert_array_equal(got, ref)
    assert seen > 0


@pytest.mark.parametrize("n", [100003, 1 << 20])
def test_stream_first_pass_8_byte_aligned_input(bos, n):
    # d_in need only be aligned to the record size: the first pass's bulk copies must start on a
    # 16-byte address, so 8-byte records at either end of a batch are loaded separately.
    import torch
    recs = inputs.make_records(n, 8, "uniform", seed=31)
    buf = torch.empty(n * 8 + 16, dtype=torch.uint8, device="cuda")
    x = buf[8:8 + n * 8]
    x.copy_(bos.to_device(recs))
    assert x.data_ptr() % 16 == 8
    ref, rinfo = oracle.orp(recs, 256, 3, method=oracle.CLOSED)
    out, info = bos.orp(x, 8, Z=256, seed=3)
    assert info.stream_passes >= 1 and info.attempts == rinfo.attempts
    np.testing.assert_array_equal(bos.to_host(out, recs.dtype), ref)
    sref, _ = oracle.sort(recs, 256, 3, method=oracle.CLOSED)
    sout, _ = bos.sort(x, 8, Z=256, seed=3)
    np.testing.assert_array_equal(bos.to_host(sout, recs.dtype), sref)


def test_stream_trace_is_input_and_seed_independent(bos):
    # The streaming pass reads whole input ranges and buckets and writes every 8-slot chunk of every
    # output bucket once: its address multiset depends on neither the input nor the seed.
    n, Z = 1 << 18, 256
    assert bos.plan(n, 16, Z, sort=False).stream_passes >= 1
    base = None
    for dist in ("uniform", "equal", "sorted", "reverse"):
        t = _trace(bos, inputs.make_records(n, 16, dist, seed=12), Z, seed=4)
        if base is None:
            base = t
        else:
            np.testing.assert_array_equal(t, base)
    t2 = _trace(bos, inputs.make_records(n, 16, "uniform", seed=12), Z, seed=99)
    kind_buf = lambda t: ((t[:, 0] >> np.uint64(48)) & np.uint64(0xFF))
    keep = lambda t: t[kind_buf(t) != 5]
    np.testing.assert_array_equal(keep(t2), keep(base))
    # the first pass wrote every chunk of the B*Z slot array exactly once
    B = 1 << 11
    wr_tag = base[(kind_buf(base) == 2) & ((base[:, 0] >> np.uint64(56)) == 2)]
    assert len(wr_tag) >= B * Z // 8


def _kind_buf(t):
    return (t[:, 0] >> np.uint64(48)) & np.uint64(0xFF)


def test_address_trace_cfg1_plain_form(bos):
    # Config 1's shape: n = 2^16 8-byte records, Z = 512 (B = 256), the plain form (one level per
    # launch). The multiset of global accesses is the same for every input (Section 3.1), and for
    # every seed but the compacted output writes (their addresses follow the final loads, Lemma 3.3).
    n, Z = 1 << 16, 512
    base = None
    for dist in ("uniform", "equal", "sorted", "reverse"):
        t = _trace(bos, inputs.make_records(n, 8, dist, seed=12), Z, seed=1, k=1)
        if base is None:
            base = t
        else:
            np.testing.assert_array_equal(t, base)
    t2 = _trace(bos, inputs.make_records(n, 8, "uniform", seed=12), Z, seed=77, k=1)
    np.testing.assert_array_equal(t2[_kind_buf(t2) != 5], base[_kind_buf(base) != 5])
    # eight passes, each reading and writing every slot of both slot arrays in turn
    assert int((_kind_buf(base) != 5).sum()) > 0


def _batch_trace(bos, sizes, rec_bytes, dist, seeds, Zs, ops):
    import torch
    recs, offs = inputs.make_batch(sizes, rec_bytes, seed=5)
    if dist == "equal":
        recs["key"] = 0x55
    elif dist == "reverse":
        recs["key"] = np.arange(recs.size, 0, -1, dtype=recs["key"].dtype)
    x = bos.to_device(recs)
    out = torch.empty_like(x)
    buf = torch.zeros(1 << 26, dtype=torch.uint8, device="cuda")
    bos.trace_attach(buf)
    try:
        bos.sort_batched(x, out, offs, seeds, ops, bos.params(rec_bytes, 512, 0), Zs=Zs)
        torch.cuda.synchronize()
    finally:
        bos.trace_attach(None)
    w = buf.view(torch.int64).cpu().numpy().view(np.uint64)
    cnt = int(w[0])
    assert 0 < cnt <= buf.numel() // 16 - 1
    ent = w[2:2 + 2 * cnt].reshape(cnt, 2)
    return ent[np.lexsort((ent[:, 1], ent[:, 0]))]


def test_batched_kernel_trace_is_input_independent(bos):
    # The batched (one-CTA-per-subproblem) kernel that the batched and serving workloads run, on a
    # mixed batch: uneven sizes, two bucket sizes, ORP and sort arrays. Its ORP accesses are the
    # same multiset for every input content, and for other seeds except the compacted writes.
    sizes = np.array([1024, 3000, 4096, 777, 12000, 20000, 1, 0, 65536, 5000], dtype=np.int64)
    Zs = np.where(np.arange(sizes.size) % 2 == 0, 512, 64).astype(np.uint32)
    ops = (np.arange(sizes.size) % 3 == 0).astype(np.uint8)
    seeds = np.arange(7, 7 + sizes.size, dtype=np.uint64)
    base = _batch_trace(bos, sizes, 8, "uniform", seeds, Zs, ops)
    for dist in ("equal", "reverse"):
        np.testing.assert_array_equal(_batch_trace(bos, sizes, 8, dist, seeds, Zs, ops), base)
    t2 = _batch_trace(bos, sizes, 8, "uniform", seeds + np.uint64(1000), Zs, ops)
    np.testing.assert_array_equal(t2[_kind_buf(t2) != 5], base[_kind_buf(base) != 5])


SHARD_CASES = [
    # (G, n, Z, rec_bytes, k): the shard plan on one device, against bos_orp and the oracle
    (2, 1 << 16, 512, 8, 0), (4, (1 << 20) + 3, 512, 16, 0), (2, 300001, 96, 16, 0), (8, 1 << 22, 1024, 16, 0),
    (4, 100003, 64, 8, 1), (2, 50000, 40, 8, 0), (4, 20000, 32, 8, 0),  # the last two overflow and retry
]


@pytest.mark.parametrize("G,n,Z,rec_bytes,k", SHARD_CASES)
def test_shard_plan_on_gpu_equals_single_device(bos, G, n, Z, rec_bytes, k):
    # Local levels on every rank's buckets, one all-to-all of whole buckets (device copies here),
    # the fused last levels with the in-bin permutation: the ranks' parts in rank order equal
    # bos_orp of the whole array and the oracle, with the same attempts (Algorithm 3.1).
    recs = inputs.make_records(n, rec_bytes, "uniform", seed=n % 997 + G)
    seed = 77 + G
    x = bos.to_device(recs)
    try:
        ref, rinfo = oracle.orp(recs, Z, seed, max_attempts=16, method=oracle.CLOSED)
    except oracle.OracleError:
        with pytest.raises(bos.BosError):
            bos.sharded_orp(x, rec_bytes, G, Z=Z, seed=seed, k=k, max_attempts=16)
        return
    out, attempts, counts = bos.sharded_orp(x, rec_bytes, G, Z=Z, seed=seed, k=k, max_attempts=16)
    got = bos.to_host(out, recs.dtype)
    assert attempts == rinfo.attempts and sum(counts) == n
    np.testing.assert_array_equal(got, ref)
    alone, ainfo = gpu_orp(bos, recs, Z, seed, k=k, max_attempts=16)
    np.testing.assert_array_equal(got, alone)


OOC_CASES = [
    # (G, n, Z, rec_bytes): the out-of-core ORP (host memory, one rank's share on the device)
    (4, 1 << 22, 1024, 16), (16, (1 << 22) + 77, 512, 16), (4, 100003, 64, 8), (8, 1 << 20, 96, 8),
    (2, 8192, 32, 8),  # overflows and retries
]


@pytest.mark.parametrize("G,n,Z,rec_bytes", OOC_CASES)
def test_out_of_core_orp_equals_in_memory(bos, G, n, Z, rec_bytes):
    # Section 4.3's setting: the data stay in host memory and move in runs of whole buckets; the
    # result equals bos_orp in device memory and the oracle, with the same attempts.
    recs = inputs.make_records(n, rec_bytes, "uniform", seed=n % 991 + 3)
    seed = 2 if n == 8192 else 5 + G
    if n == 8192:
        recs = inputs.make_records(n, rec_bytes, "uniform", seed=2)
    ref, rinfo = oracle.orp(recs, Z, seed, max_attempts=16, method=oracle.CLOSED)
    got, info = bos.orp_out_of_core(recs, G, Z=Z, seed=seed, max_attempts=16)
    assert info.attempts == rinfo.attempts
    np.testing.assert_array_equal(got, ref)
    alone, _ = gpu_orp(bos, recs, Z, seed, max_attempts=16)
    np.testing.assert_array_equal(got, alone)


def _hybrid_keys(n, rec_bytes, recipe, seed):
    """Records whose keys steer the hybrid sort's plan (shaped from the seeded generators)."""
    if recipe in inputs.DISTRIBUTIONS:
        return inputs.make_records(n, rec_bytes, recipe, seed=seed)
    recs = inputs.make_records(n, rec_bytes, "uniform", seed=seed)
    kt = recs.dtype["key"].type
    bits = recs.dtype["key"].itemsize * 8
    k = recs["key"].copy()
    if recipe == "low16_zero":  # digits 0 and 1 constant: the on-chip sort starts at digit 2
        k &= kt(~np.uint64(0xFFFF) & np.uint64((1 << bits) - 1))
    elif recipe == "top_two_values":  # top digit: 2 values over n/2 records each, next digit constant
        top = np.where(np.arange(n) % 2 == 0, 1, 2).astype(np.uint64) << np.uint64(bits - 8)
        k = ((k.astype(np.uint64) & np.uint64((1 << (bits - 24)) - 1)) | top).astype(kt)
    elif recipe == "half_equal":  # half the keys one value: a group larger than any range
        k[::2] = kt(12345)
    elif recipe == "d6_few":  # digit 6 takes 16 values: on-chip sub-buckets too large for a warp
        sh = np.uint64(bits - 16)
        k64 = k.astype(np.uint64)
        k = ((k64 & ~(np.uint64(0xFF) << sh)) | (((k64 >> sh) & np.uint64(0x0F)) << sh)).astype(kt)
    elif recipe == "few_values":  # 64 distinct keys: whole ranges of equal keys
        table = inputs.make_records(64, rec_bytes, "uniform", seed=seed + 1)["key"]
        k = table[np.arange(n) % 64]
    recs["key"] = k
    return recs


HYBRID_CAP = {16: 19456, 8: 28672}  # records one CTA sorts on chip (sort_hybrid.cu)


def _hybrid_mode(keys, rec_bytes):
    """The plan's rule stated on the keys: 1 if all fit one CTA, 2 if every bucket of the top
    varying digit does, 3 if the top two digits both vary and every pair of them does, else 0."""
    n, cap, D = keys.size, HYBRID_CAP[rec_bytes], rec_bytes // 2
    k = keys.astype(np.uint64)
    digit = [(k >> np.uint64(8 * d)) & np.uint64(255) for d in range(D)]
    live = [d for d in range(D) if np.bincount(digit[d].astype(np.int64), minlength=256).max() < n]
    if n < 2 or not live:
        return 0
    if n <= cap:
        return 1
    dA = live[-1]
    if np.bincount(digit[dA].astype(np.int64), minlength=256).max() <= cap:
        return 2
    if len(live) >= 2 and dA == D - 1 and live[-2] == D - 2:
        pair = (digit[D - 1] << np.uint64(8)) | digit[D - 2]
        if np.bincount(pair.astype(np.int64), minlength=65536).max() <= cap:
            return 3
    return 0


HYBRID_CASES = [
    # (n, rec_bytes, keys, sort_mode the plan must pick)
    (1, 16, "uniform", 0), (2, 16, "uniform", 1), (33, 8, "uniform", 1), (10000, 16, "dup1024", 1),
    (19456, 16, "uniform", 1), (19457, 16, "uniform", 2), (28672, 8, "uniform", 1), (28673, 8, "reverse", 2),
    (1 << 20, 16, "uniform", 2), (1 << 20, 8, "uniform", 2), ((1 << 22) + 5, 16, "uniform", 2),
    (1 << 23, 16, "uniform", 3), ((1 << 23) - 7, 8, "uniform", 3), (1 << 20, 16, "dup1024", 2),
    (1 << 20, 16, "sorted", 2), (1 << 20, 16, "reverse", 0), (200003, 16, "equal", 0),
    (1 << 20, 16, "low16_zero", 2), (1 << 20, 16, "top_two_values", 0), (1 << 20, 8, "half_equal", 0),
    (1 << 20, 16, "few_values", None), (1 << 22, 16, "d6_few", 2), (1 << 24, 8, "uniform", 3),
    # ranges of at most 1024 records go to the warp-per-range kernels: one whole array, or many
    # single-group ranges of about 256 / 512 / 1024 records
    (500, 16, "uniform", 1), (512, 8, "dup1024", 1), (1 << 24, 16, "uniform", 3), (1 << 25, 16, "uniform", 3),
    (1000, 16, "uniform", 1), (1 << 26, 16, "uniform", 3),
]


@pytest.mark.parametrize("n,rec_bytes,keys,mode", HYBRID_CASES)
def test_hybrid_sort_matches_oracle_and_lsd(bos, n, rec_bytes, keys, mode):
    # The hybrid radix sort (the default) and the LSD radix sort both give the oracle's stable
    # sort of the ORP output; the plan's mode is the one the key distribution calls for.
    recs = _hybrid_keys(n, rec_bytes, keys, seed=n % 1000 + rec_bytes)
    Z = 512
    ref, rinfo = oracle.sort(recs, Z, 21, method=oracle.CLOSED)
    got, info = gpu_sort(bos, recs, Z, 21)
    assert info.sort_mode == _hybrid_mode(recs["key"], rec_bytes)
    if mode is not None:
        assert info.sort_mode == mode
    assert info.attempts == rinfo.attempts
    np.testing.assert_array_equal(got, ref)
    lsd, linfo = gpu_sort(bos, recs, Z, 21, flags=bos.FLAG_LSD_SORT)
    assert linfo.sort_mode == 0
    np.testing.assert_array_equal(lsd, ref)
