"""Benchmark: bucket oblivious sort (bucket ORP + stable LSD radix sort) of n = 2^30 16-byte
records {uint64 key uniform, uint64 payload = index}, Z = 1024 (B = 2^21), on GB300.

One step = one bos_sort call over the whole array (all butterfly passes, the in-bin permutation,
the radix histogram and every radix pass), inputs resident in HBM. Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--n-log2 30]

--impl reference times the oracle (plain C++, single thread) on a bounded sample of the same
workload on the host cores. Under torchrun (N > 1) every rank sorts its own independent array
(replicas: the method has no exchange step on one array), rank 0 prints the line.
"""
import argparse
import hashlib
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

Z_DEFAULT = 1024
REC = 16
METRIC = "records/sec & HBM GB/s (% roofline), oblivious sort n=2^30 16-B records vs plain"
UNIT = "records/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n-log2", type=int, default=30)
    ap.add_argument("--Z", type=int, default=Z_DEFAULT)
    ap.add_argument("--dist", default="uniform")
    ap.add_argument("--no-compare", action="store_true", help="skip the plain-form and bitonic comparators")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample-log2", type=int, default=26,
                    help="log2 records of the CPU baseline sample (threaded; one thread: 4x fewer)")
    ap.add_argument("--flags", type=lambda x: int(x, 0), default=0, help="bos_params.flags (comparisons)")
    ap.add_argument("--k", type=int, default=0, help="levels per ORP pass (0 = automatic)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the ORP-by-distribution timings and the batched and serving summaries")
    ap.add_argument("--workload", default="sort", choices=["sort", "batched", "serving"],
                    help="sort: n=2^30 16-B records (the headline); batched: 4096 arrays of 2^10..2^20 "
                         "8-B records in one CUDA graph; serving: a Poisson request stream")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x, device=None):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"bos_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def source_hash(files=None):
    """Hash of the kernel sources (all of csrc/, or the named files of it)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2008_01765_gb300", "csrc")
    names = files if files else [f for f in sorted(os.listdir(csrc)) if f.endswith((".cu", ".cuh", ".h"))]
    for f in names:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if the sources that define the kernel
    (its entry's "sources", else all of csrc/) are the ones it was taken on."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        e = t.get(workload, {}).get(kernel)
        if e and e.get("source_hash") == source_hash(e.get("sources")):
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(n_log2, Z, dist):
    """The oracle (literal Algorithm 3.1 + in-bin permutation + LSD radix sort) on a bounded
    sample of the workload: on all the host's cores (its threaded build: each step's independent
    work split across std::threads) and on one thread."""
    import oracle
    from paper_2008_01765_gb300 import inputs
    n = 1 << n_log2
    recs = inputs.make_records(n, REC, dist, seed=1)
    oracle.lib()
    cores = host_cores()
    t0 = time.perf_counter()
    oracle.sort_threads(recs, Z, 1, cores)
    dt = time.perf_counter() - t0
    n1 = n >> 2 if n_log2 >= 12 else n  # the one-thread sample: a quarter of the records
    t0 = time.perf_counter()
    oracle.sort(recs[:n1], Z, 1, method=oracle.LITERAL, sorter=1)
    dt1 = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"n=2^{n_log2} 16-B records ({dist} u64 keys), Z={Z}, literal Algorithm 3.1 + in-bin "
                      f"permutation + LSD radix sort, {cores} host threads (nproc = {cores}), {dt:.2f} s",
            "one_thread": {"value": n1 / dt1, "unit": UNIT, "seconds": dt1, "n": n1}}


def run_reference(args):
    world, rank, _, pg = dist_setup(args)
    if rank != 0:
        return
    import oracle
    from paper_2008_01765_gb300 import inputs
    n = 1 << args.cpu_sample_log2
    recs = inputs.make_records(n, REC, args.dist, seed=1)
    oracle.lib()
    cores = host_cores()
    for _ in range(args.warmup):
        oracle.sort_threads(recs, args.Z, 1, cores)
    t0 = time.perf_counter()
    for s in range(args.steps):
        oracle.sort_threads(recs, args.Z, 1 + s, cores)
    dt = (time.perf_counter() - t0) / args.steps
    v = n / dt
    sample = (f"each step: n=2^{args.cpu_sample_log2} 16-B records ({args.dist} u64 keys), Z={args.Z}, "
              f"oracle (literal Algorithm 3.1 + in-bin permutation + LSD radix sort), {cores} host threads")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"sort n=2^{args.n_log2} rec16 Z={args.Z}", "n": 1 << args.n_log2,
                       "rec_bytes": REC, "Z": args.Z, "keys": f"{args.dist} u64, payload = index",
                       "sample_n": n, "parallelism": f"{cores} host threads"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_step_bytes(offs, Zs, R=8):
    """Algorithmic HBM bytes of one batched sort: per array, its ORP passes as the batched
    (one-CTA-per-subproblem) kernel plans them - input and output records once, the B*Z slot
    array written and read between passes - plus the radix histogram and its live digit passes
    (4 for uniform 32-bit keys)."""
    from paper_2008_01765_gb300 import bos
    total, cache = 0.0, {}
    for j in range(len(offs) - 1):
        n = int(offs[j + 1] - offs[j])
        if n == 0:
            continue
        key = (n, int(Zs[j]))
        if key not in cache:
            info = bos.plan(n, R, int(Zs[j]), flags=bos.FLAG_GENERIC)
            slot = info.B * int(Zs[j]) * (R + 4)
            cache[key] = 2 * n * R + 2 * (info.passes - 1) * slot + n * 4 + 4 * 2 * n * R
        total += cache[key]
    return total


def run_batched(args):
    import torch
    from paper_2008_01765_gb300 import _build
    _build.build()
    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    line = batched_measure(args, torch.device("cuda", local), world, rank, pg)
    if rank == 0:
        print(json.dumps(line), flush=True)


def batched_measure(args, dev, world=1, rank=0, pg=None):
    """The batched workload: 4096 arrays of 2^10..2^20 8-byte records in one CUDA graph."""
    import torch
    from paper_2008_01765_gb300 import autotune, bos, inputs
    local = dev.index
    sizes = inputs.batched_sizes(4096, 10.0, 20.0, seed=1 + rank)
    recs, offs = inputs.make_batch(sizes, 8, seed=1 + rank)
    Zs = autotune.z_array(sizes, 8)
    seeds = np.arange(1, sizes.size + 1, dtype=np.uint64)
    ops = np.ones(sizes.size, dtype=np.uint8)
    host_in = torch.from_numpy(recs.view(np.uint8).reshape(-1))
    x = host_in.to(dev)
    out = torch.empty_like(x)
    batch = bos.Batch(x, out, offs, seeds, ops, bos.params(8, 512, 0), Zs=Zs)
    stream = torch.cuda.Stream(dev)
    batch.prepare(stream)
    batch.enqueue(stream)
    batch.collect(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
        batch.enqueue(stream)
    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            graph.replay()
        batch.collect(stream)
    torch.cuda.synchronize()
    barrier(pg)
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            graph.replay()  # the graph's work is on `stream`, between the events
        att = batch.collect(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(pg, e0.elapsed_time(e1) / args.steps, dev)
    n_total = int(offs[-1])
    hbm, _ = peaks()
    step_bytes = batched_step_bytes(offs, Zs)
    line = {"metric": "records/sec, batched bucket oblivious sort (4096 arrays, CUDA graph)",
            "value": world * n_total / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "batched sort, 4096 arrays, n_j = floor(2^U), U ~ U[10, 20], 8-B records "
                                   "{u32 key uniform, u32 payload}, Z per size class from the autotune table",
                       "records": n_total, "arrays": int(sizes.size), "Z_values": sorted(set(int(z) for z in Zs)),
                       "attempts_max": int(att.max()), "l2": "batch (%.1f GiB) larger than L2" % (n_total * 8 / 2**30)},
            "hbm_gbs": step_bytes / (ms / 1e3) / 1e9, "hbm_frac": step_bytes / (ms / 1e3) / 1e9 / hbm,
            "clocks": clk}
    if not args.no_e2e:
        pin_in = host_in.pin_memory()
        pin_out = torch.empty_like(pin_in).pin_memory()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(max(1, min(args.steps, 3))):
            with torch.cuda.stream(stream):
                x.copy_(pin_in, non_blocking=True)
                graph.replay()
            batch.collect(stream)
            with torch.cuda.stream(stream):
                pin_out.copy_(out, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        k = max(1, min(args.steps, 3))
        ems = e0.elapsed_time(e1) / k
        line["e2e"] = {"value": world * n_total / (ems / 1e3), "unit": UNIT, "h2d_bytes_per_step": n_total * 8,
                       "d2h_bytes_per_step": n_total * 8, "ms_per_step": ems}
    return line


def run_serving(args):
    """Poisson stream of ORP and sort requests (50/50), n log-uniform in [2^12, 2^26], 16-B
    records {u64 key uniform, u64 payload}, 64 GiB admission budget. The arrival rate is 70% of
    the capacity measured by a burst of the same requests first."""
    import torch
    from paper_2008_01765_gb300 import _build
    _build.build()
    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    line = serving_measure(args, local, world, rank, max(40, args.steps * 40))
    if rank == 0:
        print(json.dumps(line), flush=True)


def serving_measure(args, local, world=1, rank=0, count=40):
    from paper_2008_01765_gb300 import inputs, serve
    pool = inputs.make_records(1 << 26, 16, "uniform", seed=7 + rank, payload="random")
    arrivals, sizes, ops, seeds = inputs.poisson_stream(count, 1.0, 12.0, 26.0, seed=3 + rank)
    rng = np.random.default_rng(5 + rank)
    offs = [int(rng.integers(0, pool.size - n + 1)) for n in sizes]
    jobs = [(pool[o:o + int(n)], int(op), int(sd)) for o, n, op, sd in zip(offs, sizes, ops, seeds)]

    def make_server():
        return serve.Server(budget_bytes=64 << 30, workers=4, rec_bytes=16,
                            executor_factory=lambda: serve.CudaExecutor(f"cuda:{local}", keep_results=False))

    # capacity: the whole stream submitted at once
    srv = make_server()
    for recs, op, sd in jobs[: min(len(jobs), 16)]:  # warm-up (allocator, kernels)
        srv.submit(recs, op=op, seed=sd)
    srv.close()
    srv = make_server()
    t0 = time.perf_counter()
    reqs = [srv.submit(recs, op=op, seed=sd) for recs, op, sd in jobs]
    try:
        for r in reqs:
            r.wait(600)
    finally:
        srv.close()
    t1 = time.perf_counter()
    capacity_jobs = len(jobs) / (t1 - t0)
    rate = 0.7 * capacity_jobs
    # the Poisson stream at 70% of that capacity
    srv = make_server()
    clocks = ClockSampler(local)
    clocks.start()
    reqs = []
    start = time.perf_counter()
    for (recs, op, sd), ta in zip(jobs, arrivals / rate):
        delay = start + ta - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        reqs.append(srv.submit(recs, op=op, seed=sd))
    try:
        for r in reqs:
            r.wait(600)
    finally:
        srv.close()
    clk = clocks.stop()
    st = srv.stats()
    line = {"metric": "records/sec and p50/p99 latency, serving a Poisson stream of ORP/sort requests",
            "value": st["records_per_s"] * world, "unit": UNIT, "n_gpus": world, "steps": 1, "warmup": 1,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic",
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "config": {"workload": "serving: Poisson arrivals, 50/50 ORP/sort, n log-uniform in [2^12, 2^26], "
                                   "16-B records, 64 GiB admission budget, 4 worker streams",
                       "requests": st["requests"], "records": st["records"],
                       "arrival_rate_per_s": rate, "capacity_requests_per_s": capacity_jobs,
                       "capacity_records_per_s": sum(int(n) for n in sizes) / (t1 - t0),
                       "batched_requests": st["batched_requests"], "peak_held_bytes": st["peak_held_bytes"]},
            "clocks": clk}
    return line


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    import torch
    from paper_2008_01765_gb300 import _build
    _build.build()
    from paper_2008_01765_gb300 import bos, inputs

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    n = 1 << args.n_log2
    Z = args.Z
    recs = inputs.make_records(n, REC, args.dist, seed=1 + rank)
    host_in = torch.from_numpy(recs.view(np.uint8).reshape(-1))
    x = host_in.to(dev)
    del recs
    out = torch.empty_like(x)
    p = bos.params(REC, Z, seed=1, flags=args.flags)
    ws = bos.alloc_workspace(bos.workspace_bytes(n, p), dev)
    sh = bos._stream_handle(stream)

    def step(seed, k=None):
        p.seed = seed
        p.k = args.k if k is None else k
        return bos.sort_raw(x.data_ptr(), out.data_ptr(), n, p, ws.data_ptr(), ws.numel(), sh)

    for w in range(args.warmup):
        info = step(1000 + w)
    torch.cuda.synchronize()
    bos.profile_enable(True)
    clocks = ClockSampler(local)
    barrier(pg)
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(args.steps):
        info = step(1 + s)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(pg, ms, dev)
    stats, launches = bos.profile_read()
    bos.profile_enable(False)

    value = world * n / (ms_max / 1e3)
    hbm, peak_src = peaks()
    # whole-step algorithmic bytes / step time
    step_bytes = sum(v["bytes"] for v in stats.values()) / args.steps
    top_name, top = max(((k, v) for k, v in stats.items()), key=lambda kv: kv[1]["ms"])
    top_gbs = top["bytes"] / (top["ms"] / 1e3) / 1e9
    workload = f"sort n=2^{args.n_log2} rec16 Z={Z}"
    roof = {"bound": "hbm", "achieved": top_gbs, "peak": hbm, "unit": "GB/s", "frac": top_gbs / hbm,
            "traffic": traffic_for(top_name, workload), "kernel": top_name,
            "bytes_per_launch": top["bytes"] / top["launches"], "ms_per_launch": top["ms"] / top["launches"],
            "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback 6.8 TB/s"}
    kernels = {k: {"launches_per_step": v["launches"] / args.steps, "ms_per_step": v["ms"] / args.steps,
                   "GBps": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] > 0 else 0.0}
               for k, v in stats.items()}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": workload, "n": n, "rec_bytes": REC, "Z": Z, "B": int(info.B),
                       "L": int(info.L), "orp_passes": int(info.passes), "radix_passes": int(info.radix_passes),
                       "max_cluster": int(info.max_cluster), "max_k": int(info.max_k), "flags": args.flags,
                       "keys": f"{args.dist} u64, payload = index", "l2": "inputs (16 GiB) larger than L2",
                       "parallelism": f"replicas x{world}"},
            "hbm_gbs": step_bytes / (ms / 1e3) / 1e9, "hbm_frac": step_bytes / (ms / 1e3) / 1e9 / hbm,
            "roofline": roof, "kernels": kernels, "gpu_launches": launches,
            "clocks": clk}

    # ---- the ORP alone (Algorithm 3.1 + Section 3.2) on uniform, all-equal and reverse-sorted
    # keys: its time does not depend on the data. Inputs are made on the device (x is refilled from
    # the host by the end-to-end leg below). ----
    if not args.no_extras:
        ws_orp = ws
        by_dist = {}
        xv = x.view(torch.int64).view(n, 2)
        for dist in ("uniform", "equal", "reverse"):
            if dist == "equal":
                xv[:, 0] = 0x5555555555555555
            elif dist == "reverse":
                xv[:, 0] = torch.arange(n - 1, -1, -1, dtype=torch.int64, device=dev)
            if dist != "uniform":
                xv[:, 1] = torch.arange(n, dtype=torch.int64, device=dev)
            p.seed, p.k = 4000, args.k
            bos.orp_raw(x.data_ptr(), out.data_ptr(), n, p, ws_orp.data_ptr(), ws_orp.numel(), sh)
            torch.cuda.synchronize()
            e0.record(stream)
            for s2 in range(2):
                p.seed = 1 + s2
                oinfo = bos.orp_raw(x.data_ptr(), out.data_ptr(), n, p, ws_orp.data_ptr(), ws_orp.numel(), sh)
            e1.record(stream)
            torch.cuda.synchronize()
            by_dist[dist] = {"ms": e0.elapsed_time(e1) / 2, "attempts": int(oinfo.attempts)}
        t = [v["ms"] for v in by_dist.values()]
        line["orp_by_dist"] = dict(by_dist, spread=(max(t) - min(t)) / min(t),
                                   note="bos_orp alone at the benchmark size, seeds 1-2 each")
        del ws_orp
        if args.no_e2e:  # the end-to-end leg would refill x from the host
            x.copy_(host_in)

    # ---- end to end through the public API with host buffers (H2D + sort + D2H every step) ----
    # A stream of sorts from pinned host memory: every step copies its input in and reads its
    # result back inside the timed region. Buffers are doubled so that the copy of step s+1's
    # input and the read-back of step s-1's result run on copy streams while step s sorts.
    if not args.no_e2e:
        pin_in = host_in.pin_memory()
        pin_out = torch.empty_like(pin_in).pin_memory()
        xin, xo = [x, torch.empty_like(x)], [out, torch.empty_like(out)]
        h2d, d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

        def tev():
            return torch.cuda.Event(enable_timing=True)

        spans = {"h2d": [], "sort": [], "d2h": []}

        def e2e_run(ke, seed0, start=None):
            spans["h2d"].clear(), spans["sort"].clear(), spans["d2h"].clear()
            if start is not None:
                h2d.wait_event(start)
            ev_in = [None] * ke
            ev_out = [None, None]

            def copy_in(s):
                b0, b1 = tev(), tev()
                with torch.cuda.stream(h2d):
                    if s >= 2 and ev_out[s % 2] is not None:
                        # after the read-back of step s - 2 (the previous D2H): the two copies
                        # would share the host link, and the next sort starts only when that
                        # read-back ends, so it should end as early as it can
                        h2d.wait_event(ev_out[s % 2])
                    b0.record(h2d)
                    xin[s % 2].copy_(pin_in, non_blocking=True)
                    b1.record(h2d)
                spans["h2d"].append((b0, b1))
                ev_in[s] = b1

            copy_in(0)
            for s in range(ke):
                b = s % 2
                if s + 1 < ke:  # xin[1 - b] was last read by sort s - 1, which has returned
                    copy_in(s + 1)
                stream.wait_event(ev_in[s])
                if ev_out[b] is not None:
                    stream.wait_event(ev_out[b])
                p.seed, p.k = seed0 + s, args.k
                s0, s1 = tev(), tev()
                s0.record(stream)
                bos.sort_raw(xin[b].data_ptr(), xo[b].data_ptr(), n, p, ws.data_ptr(), ws.numel(), sh)
                s1.record(stream)
                spans["sort"].append((s0, s1))
                with torch.cuda.stream(d2h):
                    d2h.wait_event(s1)
                    d0, d1 = tev(), tev()
                    d0.record(d2h)
                    pin_out.copy_(xo[b], non_blocking=True)
                    d1.record(d2h)
                    ev_out[b] = d1
                spans["d2h"].append((d0, d1))
            stream.wait_stream(h2d)
            stream.wait_stream(d2h)

        e2e_run(2, 2000)
        torch.cuda.synchronize()
        barrier(pg)
        ke = max(3, min(args.steps, 5))
        e0.record(stream)
        e2e_run(ke, 1, start=e0)
        e1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(pg, e0.elapsed_time(e1) / ke, dev)
        avg = {k: float(np.mean([a.elapsed_time(b) for a, b in v])) for k, v in spans.items()}
        # start and end of every copy and sort of the first three steps, ms after the timed start
        timeline = {k: [[round(e0.elapsed_time(a), 1), round(e0.elapsed_time(b), 1)] for a, b in v[:3]]
                    for k, v in spans.items()}
        line["e2e"] = {"value": world * n / (ems / 1e3), "unit": UNIT, "h2d_bytes_per_step": n * REC,
                       "d2h_bytes_per_step": n * REC, "ms_per_step": ems, "steps": ke,
                       "h2d_ms": avg["h2d"], "d2h_ms": avg["d2h"], "sort_ms": avg["sort"],
                       "h2d_GBps": n * REC / (avg["h2d"] / 1e3) / 1e9, "d2h_GBps": n * REC / (avg["d2h"] / 1e3) / 1e9,
                       "timeline_ms": timeline,
                       "pipeline": "double buffers on copy streams: H2D of step s+1 during sort s, after the D2H of "
                                   "step s-1; per-stream times are CUDA events around each copy and each bos_sort"}
        del pin_in, pin_out, xin, xo

    # ---- comparators: plain one-level-per-launch form, GPU bitonic sort (rank-local) ----
    if not args.no_compare:
        comp = {}
        step(3000, k=1)
        torch.cuda.synchronize()
        e0.record(stream)
        for s in range(2):
            pinfo = step(1 + s, k=1)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / 2
        comp["plain_k1"] = {"value": n / (pms / 1e3), "unit": UNIT, "ms_per_step": pms,
                            "orp_passes": int(pinfo.passes)}
        # the comparison-based sort after the ORP (stable merge sort) in place of the radix sort
        p.flags = args.flags | bos.FLAG_MERGE_SORT
        step(3500)
        torch.cuda.synchronize()
        e0.record(stream)
        for s in range(2):
            step(1 + s)
        e1.record(stream)
        torch.cuda.synchronize()
        p.flags = args.flags
        mms = e0.elapsed_time(e1) / 2
        comp["orp_merge_sort"] = {"value": n / (mms / 1e3), "unit": UNIT, "ms_per_step": mms}
        del ws
        torch.cuda.empty_cache()
        bos.bitonic_sort(x, REC, out=out)
        torch.cuda.synchronize()
        e0.record(stream)
        for s in range(2):
            bos.bitonic_sort(x, REC, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        bms = e0.elapsed_time(e1) / 2
        comp["bitonic"] = {"value": n / (bms / 1e3), "unit": UNIT, "ms_per_step": bms}
        line["comparators"] = comp
        line["speedup_vs_plain"] = pms / ms
        line["speedup_vs_bitonic"] = bms / ms

    # ---- the batched and serving workloads, summarised beside the headline ----
    if not args.no_extras and world == 1:
        del x, out  # the headline's buffers (its workspace went before the bitonic comparator)
        torch.cuda.empty_cache()
        try:
            bl = batched_measure(args, dev)
            line["batched"] = {"records_per_s": bl["value"], "ms_per_step": bl["ms_per_step"],
                               "hbm_gbs": bl["hbm_gbs"], "hbm_frac": bl["hbm_frac"],
                               "arrays": bl["config"]["arrays"], "records": bl["config"]["records"],
                               "e2e_records_per_s": bl.get("e2e", {}).get("value")}
        except Exception as ex:  # pragma: no cover
            line["batched"] = {"error": str(ex)}
        torch.cuda.empty_cache()
        try:
            sl = serving_measure(args, local, count=40)
            line["serving"] = {"records_per_s": sl["value"], "p50_ms": sl["p50_ms"], "p99_ms": sl["p99_ms"],
                               "requests": sl["config"]["requests"],
                               "arrival_rate_per_s": sl["config"]["arrival_rate_per_s"]}
        except Exception as ex:  # pragma: no cover
            line["serving"] = {"error": str(ex)}

    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            line["cpu_baseline"] = cpu_baseline(args.cpu_sample_log2, Z, args.dist)
        except Exception as e:  # pragma: no cover
            line["cpu_baseline"] = {"value": None, "error": str(e)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
