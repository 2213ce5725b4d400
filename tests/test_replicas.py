"""bench.py's multi-GPU mode runs independent replicas (one array per rank, no data exchange):
the only collectives are the timing barrier and the max over ranks. Checked here with two gloo
ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(dist)
    # each rank "measured" a different step time; everyone must see the slowest
    ms = 10.0 + 5.0 * rank
    worst = bench.max_over_ranks(dist, ms)
    n_per_rank = 1 << 20
    value = world * n_per_rank / (worst / 1e3)  # whole-job records/s, as bench.py reports it
    q.put((rank, worst, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_step():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] == res[1][2] == pytest.approx(2 * (1 << 20) / 0.015)
