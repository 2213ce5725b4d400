"""Python face of the oracle (oracle.cpp): bucket ORP and bucket oblivious sort on the CPU.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the CUDA library and its binding never do. Records are
numpy structured arrays with a ``key`` field at offset 0 (uint32 for 8-byte records, uint64 for
16-byte records) and a ``payload`` field after it.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_vp = ctypes.c_void_p


class OrpInfo(ctypes.Structure):
    _fields_ = [("attempts", _u32), ("L", _u32), ("B", _u64), ("slot_reads", _u64),
                ("slot_writes", _u64)]


OK, ERR_INVALID, ERR_OVERFLOW = 0, 1, 2
LITERAL, CLOSED = 0, 1

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.or_philox4x32_10.argtypes = [_vp, _vp, _vp]
        L.or_philox_many.argtypes = [_u64, _vp, _vp, _vp]
        L.or_geometry.argtypes = [_u64, _u32, ctypes.POINTER(_u64), ctypes.POINTER(_u32)]
        L.or_labels.argtypes = [_u64, _u64, _u32, _u32, _vp]
        L.or_group_bounds.argtypes = [_u64, _u32, _vp]
        L.or_overflow.argtypes = [_u64, _u32, _u64, _u32, ctypes.c_int]
        L.or_overflow.restype = ctypes.c_int
        L.or_overflow_count.argtypes = [_u64, _u32, _u64, _u64, _u32, ctypes.c_int]
        L.or_overflow_count.restype = _u64
        L.or_orp.argtypes = [_vp, _vp, _u64, _u32, _u32, _u64, _u32, ctypes.c_int,
                             ctypes.POINTER(OrpInfo), _vp, _vp, _u64, ctypes.POINTER(_u64)]
        L.or_orp.restype = ctypes.c_int
        L.or_orp_from.argtypes = [_vp, _vp, _u64, _u32, _u32, _u64, _u32, _u32, ctypes.c_int,
                                  ctypes.POINTER(OrpInfo), _vp, _vp, _u64, ctypes.POINTER(_u64)]
        L.or_orp_from.restype = ctypes.c_int
        L.or_orp_many.argtypes = [_vp, _vp, _u64, _u32, _u32, _u64, _u64, _u32, ctypes.c_int, _vp]
        L.or_orp_many.restype = ctypes.c_int
        L.or_stable_sort.argtypes = [_vp, _u64, _u32, _u32]
        L.or_radix_sort.argtypes = [_vp, _u64, _u32, _u32]
        L.or_sort.argtypes = [_vp, _vp, _u64, _u32, _u32, _u32, _u64, _u32, ctypes.c_int,
                              ctypes.c_int, ctypes.POINTER(OrpInfo)]
        L.or_sort.restype = ctypes.c_int
        L.or_sort_threads.argtypes = [_vp, _vp, _u64, _u32, _u32, _u32, _u64, _u32, _u32,
                                      ctypes.POINTER(OrpInfo)]
        L.or_sort_threads.restype = ctypes.c_int
        L.or_orp_sample.argtypes = [_u64, _u32, _u64, _u32, _vp, _u32, _vp, _vp, _vp, _u64]
        L.or_orp_sample.restype = ctypes.c_int
        L.or_bitonic_sort.argtypes = [_vp, _u64, _u32, _u32]
        L.or_bitonic_sort.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_vp)


def _rec_bytes(recs):
    return recs.dtype.itemsize


def _key_bytes(recs):
    return recs.dtype["key"].itemsize


class OracleError(RuntimeError):
    def __init__(self, status):
        super().__init__(f"oracle status {status}")
        self.status = status


def philox(ctr, key):
    """Philox4x32-10 of one 4-word counter and 2-word key -> 4 uint32 words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox_many(ctrs, keys):
    c = np.ascontiguousarray(ctrs, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(keys, dtype=np.uint32).reshape(-1, 2)
    assert c.shape[0] == k.shape[0]
    out = np.zeros_like(c)
    lib().or_philox_many(c.shape[0], _ptr(c), _ptr(k), _ptr(out))
    return out


def geometry(n, Z):
    B, L = _u64(), _u32()
    lib().or_geometry(n, Z, ctypes.byref(B), ctypes.byref(L))
    return B.value, L.value


def group_bounds(n, Z):
    """Boundaries of the B groups of Algorithm 3.1's placement: group j = [b[j], b[j+1])."""
    B, _ = geometry(n, Z)
    out = np.zeros(B + 1, dtype=np.uint64)
    lib().or_group_bounds(n, Z, _ptr(out))
    return out


def labels(n, seed, attempt, L):
    out = np.zeros(n, dtype=np.uint32)
    lib().or_labels(n, seed, attempt, L, _ptr(out))
    return out


def overflow(n, Z, seed, attempt=0, method=LITERAL):
    return bool(lib().or_overflow(n, Z, seed, attempt, method))


def overflow_count(n, Z, seed0, nseeds, attempt=0, method=CLOSED):
    return int(lib().or_overflow_count(n, Z, seed0, nseeds, attempt, method))


def orp(recs, Z, seed, max_attempts=8, method=LITERAL, want_loads=False, trace_cap=0,
        first_attempt=0):
    """Bucket ORP of a structured record array. Returns (out, info[, loads][, trace])."""
    recs = np.ascontiguousarray(recs)
    n = recs.shape[0]
    out = np.zeros_like(recs)
    info = OrpInfo()
    B, _ = geometry(n, Z)
    loads = np.zeros(B, dtype=np.uint32) if want_loads else None
    trace = np.zeros(trace_cap, dtype=np.uint64) if trace_cap else None
    tlen = _u64(0)
    st = lib().or_orp_from(_ptr(recs), _ptr(out), n, _rec_bytes(recs), Z, seed, first_attempt,
                           max_attempts, method, ctypes.byref(info),
                           _ptr(loads) if loads is not None else None,
                           _ptr(trace) if trace is not None else None, trace_cap,
                           ctypes.byref(tlen))
    if st != OK:
        raise OracleError(st)
    res = [out, info]
    if want_loads:
        res.append(loads)
    if trace_cap:
        assert tlen.value <= trace_cap, "trace buffer too small"
        res.append(trace[: tlen.value])
    return tuple(res)


def orp_many(recs, Z, seed0, count, max_attempts=8, method=LITERAL):
    """ORP of one small array under seeds seed0 .. seed0+count-1 -> (count, n) records."""
    recs = np.ascontiguousarray(recs)
    n = recs.shape[0]
    out = np.zeros((count, n), dtype=recs.dtype)
    att = np.zeros(count, dtype=np.uint32)
    st = lib().or_orp_many(_ptr(recs), _ptr(out), n, _rec_bytes(recs), Z, seed0, count,
                           max_attempts, method, _ptr(att))
    if st != OK:
        raise OracleError(st)
    return out, att


def orp_sample(n, Z, seed, buckets, attempt=0):
    """Output offset, load and input indices (in output order) of the given final buckets of the
    ORP of n records (no overflow check; for runs that reported none)."""
    b = np.ascontiguousarray(buckets, dtype=np.uint64)
    off = np.zeros(b.size, dtype=np.uint64)
    load = np.zeros(b.size, dtype=np.uint32)
    B, _ = geometry(n, Z)
    cap = int(min(n, b.size * max(4 * n // max(B, 1), 16) + 64))
    src = np.zeros(cap, dtype=np.uint64)
    st = lib().or_orp_sample(n, Z, seed, attempt, _ptr(b), b.size, _ptr(off), _ptr(load), _ptr(src), cap)
    if st != OK:
        raise OracleError(st)
    out, pos = [], 0
    for x in range(b.size):
        out.append(src[pos:pos + int(load[x])].copy())
        pos += int(load[x])
    return off, load, out


def stable_sort(recs):
    r = np.array(recs, copy=True)
    lib().or_stable_sort(_ptr(r), r.shape[0], _rec_bytes(r), _key_bytes(r))
    return r


def radix_sort(recs):
    r = np.array(recs, copy=True)
    lib().or_radix_sort(_ptr(r), r.shape[0], _rec_bytes(r), _key_bytes(r))
    return r


def sort(recs, Z, seed, max_attempts=8, method=LITERAL, sorter=0, first_attempt=0):
    """Bucket oblivious sort: ORP, then a stable sort by key. Returns (out, info)."""
    recs = np.ascontiguousarray(recs)
    if first_attempt:
        out, info = orp(recs, Z, seed, max_attempts, method, first_attempt=first_attempt)
        return (radix_sort(out) if sorter == 1 else stable_sort(out)), info
    out = np.zeros_like(recs)
    info = OrpInfo()
    st = lib().or_sort(_ptr(recs), _ptr(out), recs.shape[0], _rec_bytes(recs), _key_bytes(recs),
                       Z, seed, max_attempts, method, sorter, ctypes.byref(info))
    if st != OK:
        raise OracleError(st)
    return out, info


def sort_threads(recs, Z, seed, threads, max_attempts=8):
    """or_sort (literal ORP + LSD radix) with each step split across `threads` host threads:
    the threaded CPU baseline. Returns (out, info)."""
    recs = np.ascontiguousarray(recs)
    out = np.zeros_like(recs)
    info = OrpInfo()
    st = lib().or_sort_threads(_ptr(recs), _ptr(out), recs.shape[0], _rec_bytes(recs), _key_bytes(recs),
                               Z, seed, max_attempts, threads, ctypes.byref(info))
    if st != OK:
        raise OracleError(st)
    return out, info


def bitonic_sort(recs):
    r = np.array(recs, copy=True)
    st = lib().or_bitonic_sort(_ptr(r), r.shape[0], _rec_bytes(r), _key_bytes(r))
    if st != OK:
        raise OracleError(st)
    return r


def trace_fields(trace):
    """Split packed trace words into (write, level, bucket, slot) arrays."""
    t = np.asarray(trace, dtype=np.uint64)
    return ((t >> np.uint64(63)) & np.uint64(1), (t >> np.uint64(56)) & np.uint64(0x7F),
            (t >> np.uint64(24)) & np.uint64(0xFFFFFFFF), t & np.uint64(0xFFFFFF))
