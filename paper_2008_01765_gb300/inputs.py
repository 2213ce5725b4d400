"""Seeded synthetic inputs for the ORP and the sort (numpy only).

This module holds no step of the method: it only draws records, sizes and arrival times from
numpy's PCG64 generator. Both the CUDA path's tests/benchmark and the oracle take their inputs
from here.

Record layouts (little-endian, key first):
  * 8-byte records  ``REC8``  = {uint32 key, uint32 payload}
  * 16-byte records ``REC16`` = {uint64 key, uint64 payload}
"""
import numpy as np

REC8 = np.dtype([("key", "<u4"), ("payload", "<u4")])
REC16 = np.dtype([("key", "<u8"), ("payload", "<u8")])

DISTRIBUTIONS = ("uniform", "dup1024", "sorted", "equal", "reverse")


def rec_dtype(rec_bytes: int) -> np.dtype:
    if rec_bytes == 8:
        return REC8
    if rec_bytes == 16:
        return REC16
    raise ValueError(f"rec_bytes must be 8 or 16, got {rec_bytes}")


def make_records(n: int, rec_bytes: int = 16, dist: str = "uniform", seed: int = 1,
                 payload: str = "index") -> np.ndarray:
    """n records whose keys follow ``dist``; payload = index (or uniform random).

    uniform : keys uniform over the full key width
    dup1024 : a table of 1024 distinct uniform keys; each record picks a uniform table entry
    sorted  : uniform keys sorted ascending
    equal   : every key 0x5555...
    reverse : key = n - 1 - i
    """
    dt = rec_dtype(rec_bytes)
    kt = dt["key"]
    kbits = kt.itemsize * 8
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty(n, dtype=dt)
    if dist in ("uniform", "sorted"):
        keys = rng.integers(0, np.iinfo(kt).max, size=n, dtype=kt, endpoint=True)
        if dist == "sorted":
            keys.sort()
        out["key"] = keys
    elif dist == "dup1024":
        table = np.unique(rng.integers(0, np.iinfo(kt).max, size=4096, dtype=kt, endpoint=True))
        while table.size < 1024:  # pragma: no cover - 4096 draws give >= 1024 distinct values
            table = np.unique(np.concatenate(
                [table, rng.integers(0, np.iinfo(kt).max, size=4096, dtype=kt, endpoint=True)]))
        table = rng.permutation(table)[:1024]
        out["key"] = table[rng.integers(0, 1024, size=n)]
    elif dist == "equal":
        out["key"] = np.array(0x5555555555555555 if kbits == 64 else 0x55555555, dtype=kt)
    elif dist == "reverse":
        out["key"] = (n - 1 - np.arange(n, dtype=np.uint64)).astype(kt)
    else:
        raise ValueError(f"unknown key distribution {dist!r}")
    if payload == "index":
        out["payload"] = np.arange(n, dtype=np.uint64).astype(dt["payload"])
    else:
        out["payload"] = rng.integers(0, np.iinfo(dt["payload"]).max, size=n,
                                      dtype=dt["payload"], endpoint=True)
    return out


def batched_sizes(count: int = 4096, lo_log2: float = 10.0, hi_log2: float = 20.0,
                  seed: int = 1) -> np.ndarray:
    """Array sizes n_j = floor(2^U_j), U_j ~ Uniform[lo_log2, hi_log2]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.uniform(lo_log2, hi_log2, size=count)
    return np.floor(np.exp2(u)).astype(np.int64)


def make_batch(sizes, rec_bytes: int = 8, seed: int = 1):
    """Concatenated records of all arrays (uniform keys, payload = index within its array) and
    the offsets table (len(sizes) + 1 entries)."""
    sizes = np.asarray(sizes, dtype=np.int64)
    offsets = np.zeros(sizes.size + 1, dtype=np.uint64)
    np.cumsum(sizes, out=offsets[1:])
    total = int(offsets[-1])
    dt = rec_dtype(rec_bytes)
    rng = np.random.Generator(np.random.PCG64(seed))
    recs = np.empty(total, dtype=dt)
    kt = dt["key"]
    recs["key"] = rng.integers(0, np.iinfo(kt).max, size=total, dtype=kt, endpoint=True)
    idx = np.arange(total, dtype=np.int64) - np.repeat(offsets[:-1].astype(np.int64), sizes)
    recs["payload"] = idx.astype(dt["payload"])
    return recs, offsets


def poisson_stream(count: int, rate_per_s: float, lo_log2: float = 12.0, hi_log2: float = 26.0,
                   seed: int = 1):
    """Serving workload: arrival times (s) of a Poisson process, log-uniform sizes, and an op per
    request (0 = ORP, 1 = sort, 50/50)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    arrivals = np.cumsum(gaps) - gaps[0]
    sizes = np.floor(np.exp2(rng.uniform(lo_log2, hi_log2, size=count))).astype(np.int64)
    ops = rng.integers(0, 2, size=count).astype(np.uint8)
    seeds = rng.integers(1, 1 << 62, size=count, dtype=np.uint64)
    return arrivals, sizes, ops, seeds
