"""The C ABI library loads, exports every entry point declared in include/*.h, and rejects bad
arguments with the documented status codes before touching a GPU. CPU only."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bos():
    from paper_2008_01765_gb300 import _build
    _build.build()
    from paper_2008_01765_gb300 import bos as b
    return b


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(bos_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(bos):
    names = _declared()
    assert {"bos_orp", "bos_sort", "bos_sort_batched", "bos_workspace_bytes",
            "bos_bitonic_sort", "bos_trace_attach", "bos_status_str"} <= names
    lib = bos.lib()
    for n in names:
        assert hasattr(lib, n), n


def test_workspace_bytes(bos):
    p = bos.params(16, 1024, 1)
    assert bos.workspace_bytes(0, p) == 0
    w = bos.workspace_bytes(1 << 20, p)
    # two slot arrays of 2n slots of (16 + 4) bytes, plus the sort's scratch of n records
    assert w >= 2 * (2 << 20) * 20 + (1 << 20) * 16
    bad = bos.params(16, 1, 1)
    assert bos.workspace_bytes(100, bad) == 0


def test_invalid_arguments_are_rejected(bos):
    L = bos.lib()
    info = bos.Info()
    for p in (bos.Params(12, 4, 512, 0, 0, 0, 1), bos.Params(16, 4, 512, 0, 0, 0, 1),
              bos.Params(16, 8, 1, 0, 0, 0, 1), bos.Params(16, 8, 8192, 0, 0, 0, 1)):
        st = L.bos_orp(None, None, 1000, ctypes.byref(p), None, 0, None, ctypes.byref(info))
        assert st == bos.ERR_INVALID
    p = bos.params(16, 512, 1)
    # null pointers with n > 0
    assert L.bos_sort(None, None, 10, ctypes.byref(p), None, 0, None, None) == bos.ERR_INVALID
    # n = 0 is a no-op
    assert L.bos_orp(None, None, 0, ctypes.byref(p), None, 0, None, ctypes.byref(info)) == bos.OK
    assert info.B == 1 and info.L == 0
    # workspace too small (aligned fake pointers; rejected before any device access)
    assert L.bos_orp(ctypes.c_void_p(0x10000), ctypes.c_void_p(0x20000), 16, ctypes.byref(p),
                     ctypes.c_void_p(0x100000), 16, None, None) == bos.ERR_WORKSPACE
    # output overlapping the input
    ws = bos.workspace_bytes(16, p)
    assert L.bos_orp(ctypes.c_void_p(0x10000), ctypes.c_void_p(0x10010), 16, ctypes.byref(p),
                     ctypes.c_void_p(0x1000000), ws, None, None) == bos.ERR_INVALID
    # misaligned input
    assert L.bos_orp(ctypes.c_void_p(0x10008), ctypes.c_void_p(0x20000), 16, ctypes.byref(p),
                     ctypes.c_void_p(0x1000000), ws, None, None) == bos.ERR_INVALID
    # the Section 4.1 form needs two slot arrays even for L < 2
    po = bos.params(16, 512, 1, flags=bos.FLAG_OBLIVIOUS_SPLIT)
    assert bos.workspace_bytes(16, po) >= 2 * bos.plan(16, 16, 512).B * 512 * 20
    # bitonic needs a power of two
    assert L.bos_bitonic_sort(ctypes.c_void_p(0x10000), ctypes.c_void_p(0x20000), 12, 16, 8,
                              None) == bos.ERR_INVALID
    assert bos.status_str(bos.ERR_OVERFLOW).startswith("bucket overflow")


def test_plan_geometry_matches_paper(bos):
    # Algorithm 3.1: B is the smallest power of two >= 2n/Z (reported through info at n=0 only on
    # CPU; the GPU tests check info.B for n > 0).
    import oracle
    for n, Z in [(1 << 16, 512), (1 << 24, 512), (1 << 30, 1024)]:
        assert oracle.geometry(n, Z)[0] * Z >= 2 * n


def test_plans_cover_every_level(bos):
    # The planner (no device work with FLAG_PLAN_ONLY): for record widths, bucket sizes, sizes and
    # cluster caps, a plan exists, its passes apply L levels (passes x max_k >= L), B matches
    # Algorithm 3.1's smallest power of two with B*Z >= 2n, the cluster sizes respect the cap, and
    # the fewest-passes plan never has more passes than the default without the streaming kernel,
    # which never has more than the cluster-free one.
    import oracle
    for R in (8, 16):
        for Z in (32, 64, 96, 256, 512, 1024, 2048, 4096):
            for n in (1, 2, 100, 4097, 1 << 16, 300001, 1 << 22, (1 << 26) + 3, 1 << 30):
                B, L = oracle.geometry(n, Z)
                if B * Z >= 1 << 32:
                    continue
                plans = {}
                for name, flags in (("auto", 0), ("nostream", bos.FLAG_NO_STREAM), ("fewest", bos.FLAG_FEWEST_PASSES),
                                    ("nocl", bos.FLAG_NO_CLUSTER), ("cap2", bos.FLAG_MAX_CLUSTER(2)),
                                    ("nocl_nostream", bos.FLAG_NO_CLUSTER | bos.FLAG_NO_STREAM),
                                    ("generic", bos.FLAG_GENERIC)):
                    try:
                        info = bos.plan(n, R, Z, flags=flags)
                    except bos.BosError as e:  # beyond the documented Z range for 16-byte records
                        assert name == "generic" and Z * R > 48 << 10 and e.status == bos.ERR_INVALID
                        continue
                    assert (info.B, info.L) == (B, L), (R, Z, n, name)
                    assert info.passes >= 1 and info.passes * max(info.max_k, 1) >= L, (R, Z, n, name)
                    plans[name] = info
                assert plans["nocl"].max_cluster == 1
                assert "generic" not in plans or plans["generic"].max_cluster == 1
                assert plans["cap2"].max_cluster <= 2
                assert plans["fewest"].passes <= plans["nostream"].passes <= plans["nocl_nostream"].passes, (R, Z, n)
                # the streaming kernel (no clusters) is chosen only where it needs no more passes
                assert plans["auto"].passes <= plans["nostream"].passes, (R, Z, n)
                assert plans["nocl"].passes <= plans["nocl_nostream"].passes, (R, Z, n)
                assert plans["nostream"].stream_passes == 0
                assert "generic" not in plans or plans["generic"].stream_passes == 0


def test_shard_layout_and_input_ranges(bos):
    # The shard plan's geometry (no device work): B_local = B / G, g = log2 G, the local step runs
    # L - g levels, the send and receive regions lie inside the workspace and hold G chunks of
    # B_local / G whole buckets each, and the ranks' input ranges tile [0, n) in rank order.
    import oracle
    for R, Z, n, G in [(8, 64, 5000, 2), (16, 512, 1 << 20, 4), (16, 1024, (1 << 22) + 5, 8), (8, 96, 300001, 4)]:
        p = bos.params(R, Z, 1)
        lay = bos.shard_layout(n, G, p)
        B, L = oracle.geometry(n, Z)
        assert (lay.B, lay.L, lay.B_local, 1 << lay.g) == (B, L, B // G, G)
        assert lay.chunk_rec_bytes == (B // G // G) * Z * R and lay.chunk_tag_bytes == (B // G // G) * Z * 4
        for off, cb in ((lay.send_rec_offset, lay.chunk_rec_bytes), (lay.recv_rec_offset, lay.chunk_rec_bytes),
                        (lay.send_tag_offset, lay.chunk_tag_bytes), (lay.recv_tag_offset, lay.chunk_tag_bytes)):
            assert off % 256 == 0 and off + G * cb <= lay.ws_bytes
        assert lay.send_rec_offset != lay.recv_rec_offset
        end = 0
        for r in range(G):
            lo, hi = bos.shard_input_range(n, G, r, p)
            assert lo == end and hi >= lo
            end = hi
        assert end == n
    with pytest.raises(bos.BosError):
        bos.shard_layout(5000, 3, bos.params(8, 64, 1))  # not a power of two
    with pytest.raises(bos.BosError):
        bos.shard_layout(100, 8, bos.params(8, 64, 1))  # G^2 > B
