"""Pins of the oracle against facts that do not come from the oracle itself.

Each test names the passage of the paper (Asharov et al., SOSA 2020) or the library routine it
pins against. CPU only.
"""
import ctypes
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2008_01765_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_claims.json")


# --------------------------------------------------------------------------------------------
# Philox4x32-10 against cuRAND's host generator (an independent library implementation). The
# host generator seeded with S emits, for output block j, Philox4x32-10(counter = (0, 0, j, 0),
# key = (lo S, hi S)); the multiply words, the xor words and the key schedule all take part.
# --------------------------------------------------------------------------------------------
def _curand_host_blocks(seed, nblocks):
    path = "/usr/local/cuda/lib64/libcurand.so"
    if not os.path.exists(path):
        pytest.skip("libcurand not present")
    lib = ctypes.CDLL(path)
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:  # PHILOX4_32_10
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(4 * nblocks, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(out.size)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out.reshape(nblocks, 4)


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(seed):
    nblocks = 4096
    ref = _curand_host_blocks(seed, nblocks)
    ctrs = np.zeros((nblocks, 4), dtype=np.uint32)
    ctrs[:, 2] = np.arange(nblocks, dtype=np.uint32)
    keys = np.tile(np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32), (nblocks, 1))
    np.testing.assert_array_equal(oracle.philox_many(ctrs, keys), ref)


def test_philox_counter_words_all_matter():
    # Changing any one counter word or key word changes every output word (avalanche); a
    # dropped word in the round function would leave outputs unchanged.
    base_c = np.array([5, 7, 11, 13], dtype=np.uint32)
    base_k = np.array([17, 19], dtype=np.uint32)
    ref = oracle.philox(base_c, base_k)
    for w in range(4):
        c = base_c.copy()
        c[w] ^= 1
        assert np.all(oracle.philox(c, base_k) != ref)
    for w in range(2):
        k = base_k.copy()
        k[w] ^= 1
        assert np.all(oracle.philox(base_c, k) != ref)


# --------------------------------------------------------------------------------------------
# Geometry (Algorithm 3.1: B = smallest power of two >= 2n/Z)
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n,Z,B,L", [(1 << 16, 512, 256, 8), (1 << 24, 512, 1 << 16, 16),
                                     (1 << 30, 1024, 1 << 21, 21), (0, 512, 1, 0),
                                     (1, 2, 1, 0), (3, 4, 2, 1), (5, 4, 4, 2), (1000, 32, 64, 6)])
def test_geometry(n, Z, B, L):
    assert oracle.geometry(n, Z) == (B, L)


def test_geometry_is_smallest_power_of_two():
    rng = np.random.default_rng(3)
    for _ in range(500):
        n = int(rng.integers(0, 1 << 20))
        Z = int(rng.integers(2, 2048))
        B, L = oracle.geometry(n, Z)
        assert B == 1 << L
        assert B * Z >= 2 * n
        assert B == 1 or (B // 2) * Z < 2 * n


# --------------------------------------------------------------------------------------------
# Labels: uniform over [0, B) (Algorithm 3.1) - chi-square, and the top-L-bits rule.
# --------------------------------------------------------------------------------------------
def test_labels_uniform_and_in_range():
    from scipy import stats
    n, L = 1 << 18, 8
    lab = oracle.labels(n, seed=99, attempt=0, L=L)
    assert lab.max() < (1 << L)
    counts = np.bincount(lab, minlength=1 << L)
    chi2 = ((counts - n / 256) ** 2 / (n / 256)).sum()
    assert chi2 < stats.chi2.ppf(0.9999, 255)
    # The label is a prefix of the same Philox word for every L: label_L = label_{L+1} >> 1.
    lab9 = oracle.labels(n, seed=99, attempt=0, L=L + 1)
    np.testing.assert_array_equal(lab9 >> 1, lab)
    # Attempts draw fresh labels.
    lab_a1 = oracle.labels(n, seed=99, attempt=1, L=L)
    assert (lab_a1 != lab).mean() > 0.99


# --------------------------------------------------------------------------------------------
# Literal Algorithm 3.1 against its closed form (Figure 1 caption: after level i every 2^i
# consecutive buckets are semi-sorted by the top i label bits), over random sizes including
# B not dividing n, B = 1 and n in {0, 1, 2, 3}.
# --------------------------------------------------------------------------------------------
def _cases():
    rng = np.random.default_rng(11)
    cases = [(0, 4), (1, 4), (2, 4), (3, 4), (3, 2), (7, 2), (1, 2), (5, 64), (100, 8)]
    for _ in range(40):
        Z = int(rng.choice([2, 3, 4, 8, 12, 16, 32, 64]))
        n = int(rng.integers(0, 3000))
        cases.append((n, Z))
    return cases


@pytest.mark.parametrize("n,Z", _cases())
def test_literal_equals_closed_form(n, Z):
    for rec_bytes in (8, 16):
        recs = inputs.make_records(n, rec_bytes, "uniform", seed=n * 31 + Z)
        for seed in (1, 2, 77):
            try:
                lit, li, loads = oracle.orp(recs, Z, seed, max_attempts=64, want_loads=True)
            except oracle.OracleError as e:
                assert e.status == oracle.ERR_OVERFLOW
                with pytest.raises(oracle.OracleError):
                    oracle.orp(recs, Z, seed, max_attempts=64, method=oracle.CLOSED)
                continue
            clo, ci, cloads = oracle.orp(recs, Z, seed, max_attempts=64, method=oracle.CLOSED,
                                         want_loads=True)
            assert li.attempts == ci.attempts
            np.testing.assert_array_equal(lit, clo)
            np.testing.assert_array_equal(loads, cloads)
            # Output is a permutation of the input (payload = index).
            np.testing.assert_array_equal(np.sort(lit["payload"]), np.arange(n))
            assert loads.sum() == n


@pytest.mark.parametrize("n,Z", [(5, 2), (37, 3), (1000, 8), (4097, 64), (12345, 12), (300001, 96),
                                 (99991, 512), (64, 4), (1 << 12, 32), (3, 4)])
def test_groups_divide_the_input_evenly(n, Z):
    # Algorithm 3.1 "evenly divides X into B groups": every group has floor(n/B) or ceil(n/B)
    # elements, the groups tile [0, n) in order, exactly n mod B of them are the larger size, and
    # none is larger than Z/2 rounded up (so a padded bucket always holds its group).
    B, L = oracle.geometry(n, Z)
    b = oracle.group_bounds(n, Z).astype(np.int64)
    assert b.size == B + 1 and b[0] == 0 and b[-1] == n
    sizes = np.diff(b)
    assert (sizes >= 0).all()
    assert set(np.unique(sizes)) <= {n // B, -(-n // B)}
    assert int((sizes == -(-n // B)).sum()) == (n % B if n % B else B)
    assert sizes.max() <= -(-Z // 2)


def test_literal_overflow_follows_the_groups():
    # The literal butterfly overflows exactly when some level-i bucket gathers more than Z reals,
    # where level-i bucket (G, t) holds the elements of groups [G 2^i, (G+1) 2^i) whose top i label
    # bits are t. Counted here by brute force from the exported group bounds and labels, for sizes
    # B does not divide, so an uneven split would change the outcome on some seed.
    for n, Z in [(5, 2), (37, 3), (97, 6), (200, 8), (1000, 12)]:
        B, L = oracle.geometry(n, Z)
        assert n % B != 0
        grp = np.repeat(np.arange(B), np.diff(oracle.group_bounds(n, Z).astype(np.int64)))
        seen = set()
        for seed in range(200):
            lab = oracle.labels(n, seed, 0, L).astype(np.int64)
            over = False
            for i in range(1, L + 1):
                cell = ((grp >> i) << i) | (lab >> (L - i))
                over |= np.bincount(cell, minlength=B).max() > Z
            assert oracle.overflow(n, Z, seed, 0, oracle.LITERAL) == over, (n, Z, seed)
            seen.add(over)
        assert seen == {False, True}, (n, Z)


def test_overflow_literal_equals_closed_form():
    # Small Z makes overflow frequent at every level; both forms must agree seed by seed.
    for n, Z in [(64, 4), (200, 8), (37, 3), (512, 16), (96, 6)]:
        for seed in range(300):
            assert (oracle.overflow(n, Z, seed, 0, oracle.LITERAL)
                    == oracle.overflow(n, Z, seed, 0, oracle.CLOSED)), (n, Z, seed)


def test_final_bucket_is_label_class_in_input_order():
    # Closed form restated as a check: the element order before the in-bin permutation is the
    # stable counting sort by label; the in-bin permutation only reorders within a label class.
    n, Z, seed = 3000, 64, 5
    recs = inputs.make_records(n, 8, "uniform", seed=1)
    out, info, loads = oracle.orp(recs, Z, seed, want_loads=True)
    lab = oracle.labels(n, seed, info.attempts - 1, info.L)
    np.testing.assert_array_equal(loads, np.bincount(lab, minlength=info.B))
    offs = np.concatenate([[0], np.cumsum(loads)]).astype(np.int64)
    for b in range(info.B):
        seg = out["payload"][offs[b]:offs[b + 1]]
        np.testing.assert_array_equal(np.sort(seg), np.flatnonzero(lab == b))


def test_in_bin_order_is_the_sorted_slot_list_without_empty_slots():
    # Section 3.2 orders a final bucket's m reals (slots 0..m-1) by (r(b, s), s), r the key from
    # Philox(b*Z + s, attempt, stream 1). Dropping entries from a sorted list keeps the order of
    # the rest, so the same order is the list of ALL Z slots sorted by (r, s) with the entries
    # >= m removed (what the GPU's permutation table relies on). Both are checked against the
    # oracle's output, bucket by bucket.
    n, Z, seed = 5000, 64, 9
    recs = inputs.make_records(n, 8, "uniform", seed=2)
    out, info, loads = oracle.orp(recs, Z, seed, want_loads=True)
    attempt = info.attempts - 1
    lab = oracle.labels(n, seed, attempt, info.L)
    offs = np.concatenate([[0], np.cumsum(loads)]).astype(np.int64)
    for b in range(info.B):
        idx = np.uint64(b * Z) + np.arange(Z, dtype=np.uint64)
        ctr = np.zeros((Z, 4), dtype=np.uint32)
        ctr[:, 0] = (idx & np.uint64(0xFFFFFFFF)).astype(np.uint32)
        ctr[:, 1] = (idx >> np.uint64(32)).astype(np.uint32)
        ctr[:, 2] = attempt
        ctr[:, 3] = 1
        key = np.tile(np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32), (Z, 1))
        w = oracle.philox_many(ctr, key)
        r = (w[:, 0].astype(np.uint64) << np.uint64(32)) | w[:, 1].astype(np.uint64)
        m = int(loads[b])
        reals_only = sorted(range(m), key=lambda s: (int(r[s]), s))
        filtered = [s for s in sorted(range(Z), key=lambda s: (int(r[s]), s)) if s < m]
        assert filtered == reals_only
        members = np.flatnonzero(lab == b)  # slot s holds the s-th element of the class
        np.testing.assert_array_equal(out["payload"][offs[b]:offs[b + 1]], members[reals_only])


# --------------------------------------------------------------------------------------------
# Lemma 3.3: the ORP output is a uniformly random permutation. n = 4 with Z = 4 (B = 2, no
# overflow possible) and Z = 2 (B = 4; only the last level can overflow and that event is a
# symmetric function of the final loads), chi-square over the 24 permutations; n = 8, Z = 4 over
# all 40320 permutations.
# --------------------------------------------------------------------------------------------
def _perm_histogram(n, Z, nseeds, seed0):
    recs = inputs.make_records(n, 8, "uniform", seed=1)
    outs, _ = oracle.orp_many(recs, Z, seed0, nseeds, max_attempts=64)
    perms = outs["payload"].astype(np.int64)
    # Lehmer code -> permutation rank in [0, n!)
    rank = np.zeros(nseeds, dtype=np.int64)
    for i in range(n):
        smaller_after = (perms[:, i + 1:] < perms[:, i:i + 1]).sum(axis=1)
        rank = rank * (n - i) + smaller_after
    return np.bincount(rank, minlength=math.factorial(n))


@pytest.mark.parametrize("Z", [4, 2])
def test_orp_uniform_n4(Z):
    from scipy import stats
    nseeds = 240_000
    h = _perm_histogram(4, Z, nseeds, seed0=1000 * Z)
    exp = nseeds / 24
    chi2 = ((h - exp) ** 2 / exp).sum()
    assert chi2 < stats.chi2.ppf(0.999, 23), (chi2, h)


@pytest.mark.slow
def test_orp_uniform_n8():
    from scipy import stats
    nseeds = 4_000_000
    h = _perm_histogram(8, 4, nseeds, seed0=7)
    exp = nseeds / 40320
    chi2 = ((h - exp) ** 2 / exp).sum()
    assert chi2 < stats.chi2.ppf(0.999, 40319), chi2


def test_orp_without_in_bin_permutation_would_fail_uniformity():
    # The stable butterfly alone keeps input order inside each bin: only the in-bin
    # permutation of Section 3.2 makes all 24 orders reachable. With Z = 4, n = 4 (B = 2)
    # every permutation must occur.
    h = _perm_histogram(4, 4, 24_000, seed0=5)
    assert (h > 0).all()


# --------------------------------------------------------------------------------------------
# Lemma 3.2: overflow probability. B = 64, n = 32 Z. The measured attempt-failure frequency
# falls with Z and lies between the largest single-bucket binomial tail and the union bound
# over all (level, bucket) exact binomial tails; every such tail is at most e^{-Z/6}.
# --------------------------------------------------------------------------------------------
def test_overflow_decay_lemma_3_2():
    from scipy import stats
    nseeds = 100_000
    B = 64
    freqs = []
    for Z in (8, 16, 32):
        n = 32 * Z
        assert oracle.geometry(n, Z) == (B, 6)
        fails = oracle.overflow_count(n, Z, seed0=123456, nseeds=nseeds)
        f = fails / nseeds
        # level-i bucket load ~ Bin(2^i * n/B, 2^-i)
        tails = [stats.binom.sf(Z, (1 << i) * (n // B), 2.0 ** -i) for i in range(1, 7)]
        lower = max(tails)
        upper = min(1.0, B * sum(tails))
        for t in tails:
            assert t <= math.exp(-Z / 6.0)
        sigma = math.sqrt(max(f * (1 - f), 1e-12) / nseeds) + 1.0 / nseeds
        assert lower - 5 * sigma <= f <= upper + 5 * sigma, (Z, f, lower, upper)
        freqs.append(f)
    assert freqs[0] > freqs[1] > freqs[2]


def test_paper_error_bound_formula():
    claims = json.load(open(GOLDEN))
    # Section 3.4: Z = 512 gives failure <= 2^-80 for reasonable n (we take n up to 2^40).
    Z = claims["z_for_2_pow_minus_80"]
    for logn in range(10, 41):
        n = 2 ** logn
        eps = (2 * n / Z) * math.log2(2 * n / Z) * math.exp(-Z / claims["chernoff_exponent_divisor"])
        assert eps <= 2.0 ** -claims["failure_bits_for_z512"]


# --------------------------------------------------------------------------------------------
# Section 3.4: access count. Each level reads and writes B*Z slots; with B*Z = 2n that is
# 4 n log2(2n/Z) accesses (< 4 n log n).
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n,Z", [(4096, 64), (1 << 14, 512), (1000, 32), (3, 4)])
def test_access_count(n, Z):
    claims = json.load(open(GOLDEN))
    recs = inputs.make_records(n, 8, "uniform", seed=2)
    _, info = oracle.orp(recs, Z, seed=9)
    B, L = info.B, info.L
    assert info.slot_reads == B * Z * L
    assert info.slot_writes == B * Z * L
    if B * Z == 2 * n and n > 1:
        assert info.slot_reads + info.slot_writes == 4 * n * math.log2(2 * n / Z)
        assert info.slot_reads + info.slot_writes < claims["orp_accesses_per_n_log_n"] * n * math.log2(n)


def test_table1_ratios():
    claims = json.load(open(GOLDEN))
    n_log2 = claims["bucket_sort_vs_bitonic_speedup_at_n"]["n_log2"]
    bitonic = claims["bitonic_comparisons_per_n_log2_n"] * claims["accesses_per_comparison"] * n_log2 ** 2
    bucket = claims["sort_accesses_per_n_log_n"] * n_log2
    assert bitonic / bucket == claims["bucket_sort_vs_bitonic_speedup_at_n"]["speedup"]
    assert (claims["sort_accesses_per_n_log_n"] / claims["merge_sort_accesses_per_n_log_n"]
            == claims["bucket_sort_vs_merge_sort_slowdown"])


# --------------------------------------------------------------------------------------------
# Obliviousness (Section 3.1: the order of bucket reads and writes is fixed and independent of
# the input). The literal trace is identical across inputs and across seeds, and has the
# butterfly shape of Algorithm 3.1.
# --------------------------------------------------------------------------------------------
def test_literal_trace_is_input_and_seed_independent():
    n, Z = 1024, 64
    traces = []
    for dist in ("uniform", "sorted", "equal", "reverse"):
        recs = inputs.make_records(n, 16, dist, seed=4)
        for seed in (1, 2):
            _, info, tr = oracle.orp(recs, Z, seed, trace_cap=1 << 20)
            assert info.attempts == 1
            traces.append(tr)
    for t in traces[1:]:
        np.testing.assert_array_equal(t, traces[0])
    w, lvl, bkt, slot = oracle.trace_fields(traces[0])
    B, L = oracle.geometry(n, Z)
    per_pair = 4 * Z
    pos = 0
    for i in range(L):
        for j in range(B // 2):
            jp = (j >> i) << i
            seg = slice(pos, pos + per_pair)
            exp_b = np.concatenate([np.full(Z, jp + j), np.full(Z, jp + j + (1 << i)),
                                    np.full(Z, 2 * j), np.full(Z, 2 * j + 1)])
            np.testing.assert_array_equal(bkt[seg], exp_b)
            np.testing.assert_array_equal(w[seg], np.repeat([0, 1], 2 * Z))
            np.testing.assert_array_equal(lvl[seg], np.repeat([i, i + 1], 2 * Z))
            np.testing.assert_array_equal(slot[seg], np.tile(np.arange(Z), 4))
            pos += per_pair
    assert pos == len(traces[0])


# --------------------------------------------------------------------------------------------
# Sort (Section 3.3): sorted, a permutation of the input, equal to the ORP output stably sorted
# (std::stable_sort and an LSD radix sort agree), and to numpy's stable argsort.
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("rec_bytes", [8, 16])
@pytest.mark.parametrize("dist", ["uniform", "dup1024", "sorted", "equal", "reverse"])
def test_sort(rec_bytes, dist):
    n, Z, seed = 5000, 64, 3
    recs = inputs.make_records(n, rec_bytes, dist, seed=8)
    out, info = oracle.sort(recs, Z, seed)
    out_r, _ = oracle.sort(recs, Z, seed, sorter=1)
    np.testing.assert_array_equal(out, out_r)
    orp_out, _ = oracle.orp(recs, Z, seed)
    np.testing.assert_array_equal(out, orp_out[np.argsort(orp_out["key"], kind="stable")])
    assert np.all(out["key"][1:] >= out["key"][:-1])
    np.testing.assert_array_equal(np.sort(out["payload"]), np.arange(n))


def test_radix_equals_stable_sort_with_many_ties():
    rng = np.random.default_rng(1)
    for rec_bytes in (8, 16):
        r = np.zeros(20000, dtype=inputs.rec_dtype(rec_bytes))
        r["key"] = rng.integers(0, 7, size=r.size) << (8 * (rec_bytes // 2) - 3)
        r["payload"] = np.arange(r.size)
        np.testing.assert_array_equal(oracle.radix_sort(r), oracle.stable_sort(r))
        np.testing.assert_array_equal(oracle.stable_sort(r), r[np.argsort(r["key"], kind="stable")])


@pytest.mark.parametrize("n", [1, 2, 16, 1024])
def test_bitonic_network(n):
    for rec_bytes in (8, 16):
        r = inputs.make_records(n, rec_bytes, "dup1024", seed=n, payload="random")
        got = oracle.bitonic_sort(r)
        np.testing.assert_array_equal(got, np.sort(r, order=["key", "payload"]))
    with pytest.raises(oracle.OracleError):
        oracle.bitonic_sort(inputs.make_records(12, 8))


def test_orp_sample_equals_full_orp():
    # The sampled form (bucket by bucket, any n) agrees with the full literal ORP on every bucket.
    n, Z, seed = 20000, 64, 13
    recs = inputs.make_records(n, 8, "uniform", seed=2)
    out, info, loads = oracle.orp(recs, Z, seed, want_loads=True)
    assert info.attempts == 1
    buckets = np.arange(info.B)
    off, load, src = oracle.orp_sample(n, Z, seed, buckets)
    np.testing.assert_array_equal(load, loads)
    for b in buckets:
        seg = out["payload"][int(off[b]):int(off[b]) + int(load[b])]
        np.testing.assert_array_equal(seg, src[b])


@pytest.mark.parametrize("n,Z,rec_bytes,dist", [(0, 4, 8, "uniform"), (5, 2, 16, "uniform"), (3001, 16, 8, "dup1024"), (3001, 8, 8, "uniform"),
                                                (20000, 64, 16, "uniform"), (65536, 512, 8, "reverse")])
def test_threaded_baseline_equals_one_thread(n, Z, rec_bytes, dist):
    # The threaded CPU baseline is the same literal algorithm (Algorithm 3.1, Section 3.2, an LSD
    # radix sort as Section 3.3's sort) with each step's independent work split across threads:
    # its output and attempt count equal the one-thread oracle's for every thread count.
    recs = inputs.make_records(n, rec_bytes, dist, seed=n + 1)
    for seed in (1, 9):
        try:
            ref, ri = oracle.sort(recs, Z, seed, max_attempts=32, method=oracle.LITERAL, sorter=1)
        except oracle.OracleError as e:  # every attempt overflows: so must the threaded run
            assert e.status == oracle.ERR_OVERFLOW
            with pytest.raises(oracle.OracleError):
                oracle.sort_threads(recs, Z, seed, 4, max_attempts=32)
            continue
        for threads in (1, 3, 8):
            got, gi = oracle.sort_threads(recs, Z, seed, threads, max_attempts=32)
            assert gi.attempts == ri.attempts
            np.testing.assert_array_equal(got, ref)
