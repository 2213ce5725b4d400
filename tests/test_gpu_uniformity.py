"""Lemma 3.3 on the GPU: the ORP output is a uniformly random permutation.

The oracle's uniformity pins (tests/test_oracle.py) run the n = 4 ORP over 240,000 seeds with
Z = 4 (B = 2, one level, overflow impossible) and Z = 2 (B = 4, two levels; only the last level can
overflow and that event is a symmetric function of the final loads, so conditioning on success
keeps the output uniform). Here the same seeds go through the CUDA path: every seed's output must
equal the oracle's element by element, with the same attempt count, and the histogram of the
GPU's permutations over the 24 orders must pass the same chi-square bound (23 degrees of freedom,
p = 0.001). All 240,000 arrays run as one bos_sort_batched call; a sample of seeds also runs
through bos_orp one array at a time.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2008_01765_gb300 import inputs

pytestmark = pytest.mark.gpu

NSEEDS = 240_000


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


def _perm_rank(perms):
    """Lehmer rank in [0, n!) of each row of a (count, n) array of permutations of 0..n-1."""
    count, n = perms.shape
    rank = np.zeros(count, dtype=np.int64)
    for i in range(n):
        smaller_after = (perms[:, i + 1:] < perms[:, i:i + 1]).sum(axis=1)
        rank = rank * (n - i) + smaller_after
    return rank


@pytest.mark.parametrize("Z", [4, 2])
def test_gpu_orp_n4_uniform_and_equal_to_oracle_seed_by_seed(bos, Z):
    import torch
    from scipy import stats
    n = 4
    recs = inputs.make_records(n, 8, "uniform", seed=1)
    seed0 = 1000 * Z  # the oracle pin's seeds
    ref, ratt = oracle.orp_many(recs, Z, seed0, NSEEDS, max_attempts=64, method=oracle.CLOSED)

    x = bos.to_device(np.tile(recs, NSEEDS))
    out = torch.empty_like(x)
    offs = np.arange(NSEEDS + 1, dtype=np.uint64) * n
    seeds = seed0 + np.arange(NSEEDS, dtype=np.uint64)
    ops = np.zeros(NSEEDS, dtype=np.uint8)
    att = bos.sort_batched(x, out, offs, seeds, ops, bos.params(8, Z, 0, max_attempts=64))
    got = bos.to_host(out, recs.dtype).reshape(NSEEDS, n)
    np.testing.assert_array_equal(att[:NSEEDS], ratt)
    np.testing.assert_array_equal(got, ref)
    if Z == 2:
        assert (ratt > 1).any()  # the retry path ran on the GPU too

    h = np.bincount(_perm_rank(got["payload"].astype(np.int64)), minlength=math.factorial(n))
    exp = NSEEDS / 24
    chi2 = ((h - exp) ** 2 / exp).sum()
    assert chi2 < stats.chi2.ppf(0.999, 23), (chi2, h)

    # one array per call through bos_orp, on a sample of the same seeds
    xs = bos.to_device(recs)
    for j in range(0, NSEEDS, NSEEDS // 2000):
        o, info = bos.orp(xs, 8, Z=Z, seed=int(seeds[j]), max_attempts=64)
        assert info.attempts == ratt[j]
        np.testing.assert_array_equal(bos.to_host(o, recs.dtype), ref[j])
