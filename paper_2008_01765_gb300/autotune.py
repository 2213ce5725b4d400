"""Per-size-class bucket size Z for batched ORP/sort, picked by measurement.

Z changes the result (it sets the buckets and the labels' width), so for the same input a batch
must always use the same Z for an array of a given size: the table maps a size class (round of
log2 n) to Z and is part of the result contract. Candidates are restricted by Lemma 3.2's bound:
eps(n, Z) = (2n/Z) log2(2n/Z) e^(-Z/6) <= 2^-security_bits for every n of the class (Section 3.4
takes 2^-80). Among them the tuner keeps the fastest measured one.

    python -m paper_2008_01765_gb300.autotune --write     # on a GPU: measure and save the table
"""
import json
import math
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "autotune_table.json")
DEFAULT_Z = 512
CANDIDATES = (256, 512, 1024, 2048, 4096)


def size_class(n: int) -> int:
    return int(round(math.log2(n))) if n > 0 else 0


def eps_bound(n: int, Z: int) -> float:
    """Lemma 3.2: overflow probability <= (2n/Z) log2(2n/Z) e^(-Z/6) (0 when 2n <= Z)."""
    r = 2.0 * n / Z
    if r <= 1.0:
        return 0.0
    return r * math.log2(r) * math.exp(-Z / 6.0)


def secure(n_max: int, Z: int, bits: int = 80) -> bool:
    return eps_bound(n_max, Z) <= 2.0 ** -bits


def load_table(path: str = TABLE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def z_for(n: int, rec_bytes: int = 8, table: dict = None) -> int:
    """Z of the size class of n (DEFAULT_Z when the class is not in the table)."""
    table = load_table() if table is None else table
    return int(table.get("Z", {}).get(str(rec_bytes), {}).get(str(size_class(n)), DEFAULT_Z))


def z_array(sizes, rec_bytes: int = 8, table: dict = None) -> np.ndarray:
    table = load_table() if table is None else table
    return np.array([z_for(int(n), rec_bytes, table) for n in sizes], dtype=np.uint32)


def tune(rec_bytes=8, classes=range(10, 21), records_per_class=1 << 24, reps=3, bits=80, verbose=True):
    """Measures batched sort throughput per (size class, candidate Z) on the current GPU."""
    import torch

    from . import bos, inputs
    result, measured = {}, {}
    for c in classes:
        n = 1 << c
        count = max(1, records_per_class // n)
        sizes = np.full(count, n, dtype=np.int64)
        recs, offs = inputs.make_batch(sizes, rec_bytes, seed=c)
        x = bos.to_device(recs)
        out = torch.empty_like(x)
        seeds = np.arange(count, dtype=np.uint64) + 1
        ops = np.ones(count, dtype=np.uint8)
        best = None
        for Z in CANDIDATES:
            hi = int(round(2 ** (c + 0.5)))  # largest n of the class
            if not secure(hi, Z, bits):
                continue
            try:
                batch = bos.Batch(x, out, offs, seeds, ops, bos.params(rec_bytes, Z, 0),
                                  Zs=np.full(count, Z, dtype=np.uint32))
                batch.run()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(reps):
                    batch.run()
                torch.cuda.synchronize()
                dt = (time.perf_counter() - t0) / reps
            except bos.BosError:
                continue
            rate = count * n / dt
            measured.setdefault(str(c), {})[str(Z)] = rate
            if verbose:
                print(f"class 2^{c}: Z={Z} {rate / 1e9:.3f} G records/s", flush=True)
            if best is None or rate > best[1]:
                best = (Z, rate)
            del batch
        if best:
            result[str(c)] = best[0]
        del x, out
        torch.cuda.empty_cache()
    return result, measured


if __name__ == "__main__":
    import argparse
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--write", action="store_true")
    ap.add_argument("--rec-bytes", type=int, default=8)
    ap.add_argument("--out", default=TABLE, help="where --write saves the table")
    args = ap.parse_args()
    table, measured = tune(args.rec_bytes)
    doc = load_table()
    doc.setdefault("Z", {})[str(args.rec_bytes)] = table
    doc.setdefault("measured_records_per_s", {})[str(args.rec_bytes)] = measured
    doc["device"] = torch.cuda.get_device_name(0)
    doc["security_bits"] = 80
    print(json.dumps(doc["Z"], indent=1))
    if args.write:
        with open(args.out, "w") as f:
            json.dump(doc, f, indent=1, sort_keys=True)
