"""bos_orp_noalloc: the bucket ORP for callers that cannot allocate device memory.

Such callers (code inside a custom device allocator or its callbacks, plugins whose host owns all
device memory) cannot hand bos_orp a workspace; bos_orp_noalloc takes its workspace from a fixed
scratch array inside the library. These tests call it through the C ABI and compare it with
bos_orp and with the oracle bit for bit, on two calls in a row (the scratch keeps the first call's
contents when the second one starts), for every pass kernel that can use the scratch: the
automatic plan (streaming and cluster passes), the plain form (k = 1), the one-CTA-per-subproblem
kernel and the Section 4.1 form, whose workspace regions differ.

This file is collected last on purpose: a run that stops at the first failure has already run
every other test when it gets here.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2008_01765_gb300 import inputs


@pytest.fixture(scope="module")
def bos():
    from paper_2008_01765_gb300 import _build
    _build.build()
    from paper_2008_01765_gb300 import bos as b
    b.lib()
    return b


def test_noalloc_rejects_sizes_beyond_its_scratch(bos):
    # n = 2^19 + 1 16-byte records at Z = 512 need 2 x 4096 x 512 x 20 B of slot arrays > 64 MiB.
    L = bos.lib()
    p = bos.params(16, 512, 1)
    st = L.bos_orp_noalloc(ctypes.c_void_p(0x10000), ctypes.c_void_p(0x20000), (1 << 19) + 1,
                           ctypes.byref(p), None, None)
    assert st == bos.ERR_WORKSPACE
    bad = bos.params(16, 1, 1)
    assert L.bos_orp_noalloc(None, None, 100, ctypes.byref(bad), None, None) == bos.ERR_INVALID
    assert L.bos_orp_noalloc(None, None, 0, ctypes.byref(p), None, None) == bos.OK


@pytest.mark.gpu
@pytest.mark.parametrize("flags_name,k", [("auto", 0), ("auto", 1), ("generic", 0), ("generic", 1),
                                          ("oblivious", 0)])
def test_noalloc_matches_bos_orp_and_oracle_on_two_calls_in_a_row(bos, flags_name, k):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    flags = {"auto": 0, "generic": bos.FLAG_GENERIC, "oblivious": bos.FLAG_OBLIVIOUS_SPLIT}[flags_name]
    # Two different calls back to back: the second starts with the first one's scratch contents.
    cases = [((1 << 19), 16, 512, 11, "uniform"), (30011, 8, 64, 12, "dup1024")]
    if flags_name == "oblivious":
        cases = [(1 << 16, 16, 256, 11, "uniform"), (3001, 8, 64, 12, "dup1024")]
    for n, rec_bytes, Z, seed, dist in cases:
        recs = inputs.make_records(n, rec_bytes, dist, seed=seed)
        x = bos.to_device(recs)
        ref, rinfo = bos.orp(x, rec_bytes, Z=Z, seed=seed, k=k, flags=flags)
        got, info = bos.orp_noalloc(x, rec_bytes, Z=Z, seed=seed, k=k, flags=flags)
        torch.cuda.synchronize()
        assert info.attempts == rinfo.attempts and info.B == rinfo.B and info.passes == rinfo.passes
        np.testing.assert_array_equal(bos.to_host(got, recs.dtype), bos.to_host(ref, recs.dtype))
        oref, oinfo = oracle.orp(recs, Z, seed, method=oracle.CLOSED)
        assert info.attempts == oinfo.attempts
        np.testing.assert_array_equal(bos.to_host(got, recs.dtype), oref)
