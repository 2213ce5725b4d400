"""The ORP's multi-GPU shard plan, run on CPU ranks (oracle side).

TEST INFRASTRUCTURE ONLY: like the rest of ``oracle/``, only the tests may import this module.

Algorithm 3.1 shards over G = 2^g ranks with one fixed exchange. Rank r holds the initial buckets
[r B/G, (r+1) B/G). Level i of the butterfly pairs buckets inside aligned blocks of 2^(i+1) (it
merges buckets a and a + 2^i and writes buckets 2j and 2j+1, j = a without bit i), so levels
0 .. L-g-1 stay inside a rank's block and run locally. The last g levels form one fused subproblem
for every t < B/G, whose inputs are bucket s B/G + t of every rank s: rank d takes the subproblems
t in [d B/G^2, (d+1) B/G^2), so every rank sends every other rank one contiguous run of B/G^2
whole buckets. This is an all-to-all whose volume and addresses do not depend on the data, so the
plan stays oblivious. Rank d then runs levels L-g .. L-1 on what it received, which leaves it
exactly the final buckets [d B/G, (d+1) B/G). It applies the in-bin permutation of Section 3.2
to them and strips the dummies. An exclusive scan of the ranks' real counts places each rank's
part of the output. An overflow on any rank fails the attempt everywhere (a max-reduction), and
the ranks retry with the next attempt counter, as the single-device path does.
"""
import numpy as np

from . import geometry, labels, philox_many

DUMMY = 0xFFFFFFFF


def _group_lo(j, n, B):
    return (j * n) // B


def _level(held, i, L, Z):
    """One butterfly level on the buckets a rank holds: {bucket: [(label, src), ...]} (reals in
    slot order). Returns the new buckets and whether a MergeSplit output exceeded Z reals."""
    bit = L - 1 - i
    out, over = {}, False
    for a in sorted(held):
        if (a >> i) & 1:
            continue
        b = a | (1 << i)
        assert b in held, "the plan must hold both buckets of every pair"
        j = ((a >> (i + 1)) << i) | (a & ((1 << i) - 1))
        sides = ([], [])
        for lab, src in held[a] + held[b]:  # A_0's reals in slot order, then A_1's
            sides[(lab >> bit) & 1].append((lab, src))
        over |= len(sides[0]) > Z or len(sides[1]) > Z
        out[2 * j], out[2 * j + 1] = sides
    return out, over


def _permute(bucket, reals, Z, seed, attempt):
    """Section 3.2: slot s of final bucket b gets the key (w0 << 32 | w1) of Philox counter
    (lo32(b Z + s), hi32(b Z + s), attempt, 1), key (lo32 seed, hi32 seed); ascending (key, s)."""
    m = len(reals)
    if m == 0:
        return []
    idx = np.uint64(bucket * Z) + np.arange(m, dtype=np.uint64)
    ctr = np.zeros((m, 4), dtype=np.uint32)
    ctr[:, 0] = (idx & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    ctr[:, 1] = (idx >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = attempt
    ctr[:, 3] = 1
    key = np.tile(np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32), (m, 1))
    w = philox_many(ctr, key)
    r = (w[:, 0].astype(np.uint64) << np.uint64(32)) | w[:, 1].astype(np.uint64)
    order = sorted(range(m), key=lambda s: (int(r[s]), s))
    return [reals[s][1] for s in order]


def _pack(buckets, keys, Z):
    """Fixed-size wire form of whole buckets: Z (label, src) slots each, dummies as DUMMY."""
    a = np.full((len(keys), Z, 2), DUMMY, dtype=np.int64)
    for x, k in enumerate(keys):  # an overflowing bucket (the attempt fails) sends its first Z
        for s, (lab, src) in enumerate(buckets[k][:Z]):
            a[x, s] = (lab, src)
    return a


def sharded_orp(recs, Z, seed, rank, world, max_attempts=8):
    """This rank's part of ORP(recs) under the shard plan on `world` gloo ranks (a power of two
    with world^2 <= B). Returns (offset of the part in the output, the part, attempts)."""
    import torch
    import torch.distributed as dist
    n = recs.shape[0]
    B, L = geometry(n, Z)
    g = world.bit_length() - 1
    assert 1 << g == world and world * world <= B, "need a power-of-two world with world^2 <= B"
    per, sub = B // world, B // (world * world)  # buckets per rank; subproblems per rank
    for attempt in range(max_attempts):
        lab = labels(n, seed, attempt, L)
        held = {}
        for j in range(rank * per, (rank + 1) * per):  # placement: group j into bucket j
            lo, hi = _group_lo(j, n, B), _group_lo(j + 1, n, B)
            held[j] = [(int(lab[x]), x) for x in range(lo, hi)]
        over = any(len(v) > Z for v in held.values())
        for i in range(L - g):  # local levels
            held, o = _level(held, i, L, Z)
            over |= o
        assert set(held) == set(range(rank * per, (rank + 1) * per))
        # the exchange: to rank d, local buckets t in [d sub, (d+1) sub), Z slots each
        send = _pack(held, [rank * per + t for t in range(per)], Z)  # rows in destination order
        recv = np.empty_like(send)
        st, rt = torch.from_numpy(send.reshape(-1)), torch.from_numpy(recv.reshape(-1))
        dist.all_to_all_single(rt, st)
        recv = rt.numpy().reshape(world, sub, Z, 2)
        held = {}
        for s in range(world):
            for x in range(sub):
                t = rank * sub + x
                row = recv[s, x]
                held[s * per + t] = [(int(a), int(b)) for a, b in row if a != DUMMY]
        for i in range(L - g, L):  # the fused last levels of this rank's subproblems
            held, o = _level(held, i, L, Z)
            over |= o
        assert set(held) == set(range(rank * per, (rank + 1) * per))
        flag = torch.tensor([int(over)], dtype=torch.int64)
        dist.all_reduce(flag, op=dist.ReduceOp.MAX)
        if flag.item():
            continue
        src = []
        for b in range(rank * per, (rank + 1) * per):
            src += _permute(b, held[b], Z, seed, attempt)
        counts = torch.zeros(world, dtype=torch.int64)
        counts[rank] = len(src)
        dist.all_reduce(counts)
        offset = int(counts[:rank].sum())
        return offset, recs[np.array(src, dtype=np.int64)], attempt + 1
    raise RuntimeError("every attempt overflowed")
