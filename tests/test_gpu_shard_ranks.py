"""The shard plan as separate ranks: two processes, one gloo process group, both on the one GPU.

Each rank runs its own steps through the C ABI (bos_shard_local, bos_shard_final) on its own
workspace. The exchange is one all_to_all of whole buckets staged through host memory, the
overflow decision a max all-reduce, and the output offsets an all-reduce of the counts, as a
multi-GPU deployment would do them over NCCL. No kernel of one rank waits on the other's: the
ranks meet only in host collectives between launches. The ranks' parts, put together, equal
bos_orp of the whole array and the oracle, with the same attempts.
"""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, n, Z, rec_bytes, seed, q):
    import ctypes
    import datetime

    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
    from paper_2008_01765_gb300 import bos, inputs
    torch.cuda.set_device(0)
    L = bos.lib()
    recs = inputs.make_records(n, rec_bytes, "uniform", seed=seed)
    p = bos.params(rec_bytes, Z, seed)
    lay = bos.shard_layout(n, world, p)
    lo, hi = bos.shard_input_range(n, world, rank, p)
    x = bos.to_device(recs[lo:hi])  # this rank's input records only
    ws = bos.alloc_workspace(lay.ws_bytes, "cuda:0")
    part = torch.empty(lay.out_capacity * rec_bytes, dtype=torch.uint8, device="cuda:0")
    sh = bos._stream_handle(torch.cuda.current_stream())
    for attempt in range(16):
        st = L.bos_shard_local(ctypes.c_void_p(x.data_ptr()), n, world, rank, ctypes.byref(p), attempt,
                               ctypes.c_void_p(ws.data_ptr()), ws.numel(), sh)
        assert st == bos.OK, st
        # the exchange: chunk d of the send regions to rank d (records and tags), staged in host memory
        send = torch.cat([torch.cat([ws[off + d * cb:off + (d + 1) * cb] for off, cb in
                                     ((lay.send_rec_offset, lay.chunk_rec_bytes),
                                      (lay.send_tag_offset, lay.chunk_tag_bytes))]) for d in range(world)]).cpu()
        recv = torch.empty_like(send)
        dist.all_to_all_single(recv, send)
        per = lay.chunk_rec_bytes + lay.chunk_tag_bytes
        for s in range(world):
            blk = recv[s * per:(s + 1) * per].cuda()
            ws[lay.recv_rec_offset + s * lay.chunk_rec_bytes:lay.recv_rec_offset + (s + 1) * lay.chunk_rec_bytes].copy_(
                blk[:lay.chunk_rec_bytes])
            ws[lay.recv_tag_offset + s * lay.chunk_tag_bytes:lay.recv_tag_offset + (s + 1) * lay.chunk_tag_bytes].copy_(
                blk[lay.chunk_rec_bytes:])
        c, o = ctypes.c_uint64(), ctypes.c_uint32()
        st = L.bos_shard_final(n, world, rank, ctypes.byref(p), attempt, ctypes.c_void_p(part.data_ptr()),
                               lay.out_capacity, ctypes.c_void_p(ws.data_ptr()), ws.numel(), sh,
                               ctypes.byref(c), ctypes.byref(o))
        assert st == bos.OK, st
        flag = torch.tensor([int(o.value)], dtype=torch.int64)
        dist.all_reduce(flag, op=dist.ReduceOp.MAX)
        if flag.item():
            continue
        counts = torch.zeros(world, dtype=torch.int64)
        counts[rank] = int(c.value)
        dist.all_reduce(counts)
        off = int(counts[:rank].sum())
        q.put((rank, off, part[:int(c.value) * rec_bytes].cpu().numpy().tobytes(), attempt + 1))
        break
    else:
        q.put((rank, -1, b"", 16))
    dist.destroy_process_group()


@pytest.mark.parametrize("n,Z,rec_bytes,seed", [(1 << 18, 512, 16, 5), (100003, 64, 8, 9), (8192, 32, 8, 2)])
def test_two_rank_processes_on_one_gpu(n, Z, rec_bytes, seed):
    import torch
    import torch.multiprocessing as mp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2008_01765_gb300 import _build, bos, inputs
    _build.build()
    world = 2
    recs = inputs.make_records(n, rec_bytes, "uniform", seed=seed)
    ref, info = oracle.orp(recs, Z, seed, max_attempts=16, method=oracle.CLOSED)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n, Z, rec_bytes, seed, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=300) for _ in range(world))
    finally:
        for p in procs:
            p.join(120)
            if p.is_alive():
                p.terminate()
    assert all(p.exitcode == 0 for p in procs)
    out = np.zeros_like(recs)
    end = 0
    for rank, off, part, attempts in res:
        assert off == end and attempts == info.attempts
        part = np.frombuffer(part, dtype=recs.dtype)
        out[off:off + part.shape[0]] = part
        end = off + part.shape[0]
    assert end == n
    np.testing.assert_array_equal(out, ref)
    got, _ = bos.orp(bos.to_device(recs), rec_bytes, Z=Z, seed=seed, max_attempts=16)
    np.testing.assert_array_equal(out, bos.to_host(got, recs.dtype))
