"""The ORP's multi-GPU shard plan on gloo CPU ranks (oracle side): local butterfly levels, one
fixed all-to-all of whole buckets, the fused last levels, then the in-bin permutation. The ranks'
parts, put at their scanned offsets, equal the single-device ORP of the same input, seed and Z,
and take the same attempts. CPU only."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, n, Z, seed, q):
    import datetime

    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    from oracle import shard
    from paper_2008_01765_gb300 import inputs
    recs = inputs.make_records(n, 8, "uniform", seed=seed)
    off, part, attempts = shard.sharded_orp(recs, Z, seed, rank, world, max_attempts=16)
    q.put((rank, off, part.tobytes(), attempts))
    dist.destroy_process_group()


CASES = [(2, 5000, 64, 3), (4, 5000, 64, 3), (2, (1 << 13) + 3, 32, 11), (4, 20000, 96, 5), (2, 3, 2, 1),
         (2, 200, 8, 1), (4, 500, 8, 15), (4, 500, 16, 2)]  # the last three overflow and retry


@pytest.mark.parametrize("world,n,Z,seed", CASES)
def test_shard_plan_equals_single_device_orp(world, n, Z, seed):
    import torch.multiprocessing as mp

    import oracle
    from paper_2008_01765_gb300 import inputs
    B, L = oracle.geometry(n, Z)
    if world * world > B:
        pytest.skip("the plan needs world^2 <= B")
    recs = inputs.make_records(n, 8, "uniform", seed=seed)
    ref, info = oracle.orp(recs, Z, seed, max_attempts=16, method=oracle.CLOSED)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n, Z, seed, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=120) for _ in range(world))
    finally:
        for p in procs:
            p.join(60)
            if p.is_alive():
                p.terminate()
    assert all(p.exitcode == 0 for p in procs)
    out = np.zeros_like(recs)
    end = 0
    for rank, off, part, attempts in res:
        part = np.frombuffer(part, dtype=recs.dtype)
        assert off == end  # the parts tile the output in rank order
        out[off:off + part.shape[0]] = part
        end = off + part.shape[0]
        assert attempts == info.attempts
    assert end == n
    np.testing.assert_array_equal(out, ref)
