"""ctypes binding of libbos.so (the C ABI declared in include/bos.h).

Argument marshalling only: every step of the ORP and the sort runs in the library's CUDA
kernels. PyTorch provides device memory and streams. There is no CPU fallback: if libbos.so
cannot be loaded the calls raise.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbos.so")

OK, ERR_INVALID, ERR_OVERFLOW, ERR_WORKSPACE, ERR_CUDA, ERR_TIMEOUT = range(6)
FLAG_SKIP_PUBLISH = 0x1
FLAG_GENERIC = 0x2
FLAG_NO_CLUSTER = 0x4
FLAG_FEWEST_PASSES = 0x8
FLAG_PLAN_ONLY = 0x10
FLAG_MERGE_SORT = 0x20
FLAG_OBLIVIOUS_SPLIT = 0x40
FLAG_NO_STREAM = 0x80
FLAG_LSD_SORT = 0x200000


def FLAG_FORCE_OVERFLOW(n):
    return (n & 0xFF) << 8


def FLAG_MAX_CLUSTER(c):
    return (c & 0x1F) << 16


class Params(ctypes.Structure):
    _fields_ = [("rec_bytes", ctypes.c_uint32), ("key_bytes", ctypes.c_uint32),
                ("Z", ctypes.c_uint32), ("k", ctypes.c_uint32), ("max_attempts", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("seed", ctypes.c_uint64)]


class Info(ctypes.Structure):
    _fields_ = [("attempts", ctypes.c_uint32), ("L", ctypes.c_uint32), ("passes", ctypes.c_uint32),
                ("radix_passes", ctypes.c_uint32), ("B", ctypes.c_uint64),
                ("max_cluster", ctypes.c_uint32), ("max_k", ctypes.c_uint32),
                ("stream_passes", ctypes.c_uint32), ("sort_mode", ctypes.c_uint32)]


class ShardLayout(ctypes.Structure):
    _fields_ = [("B", ctypes.c_uint64), ("B_local", ctypes.c_uint64), ("L", ctypes.c_uint32),
                ("g", ctypes.c_uint32), ("local_passes", ctypes.c_uint32), ("ws_bytes", ctypes.c_size_t),
                ("send_rec_offset", ctypes.c_size_t), ("send_tag_offset", ctypes.c_size_t),
                ("recv_rec_offset", ctypes.c_size_t), ("recv_tag_offset", ctypes.c_size_t),
                ("chunk_rec_bytes", ctypes.c_size_t), ("chunk_tag_bytes", ctypes.c_size_t),
                ("out_capacity", ctypes.c_uint64)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint32),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


class BosError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {status_str(status)} ({status})")


_lib = None
_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32


def lib():
    """Load libbos.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libbos.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.bos_workspace_bytes.argtypes = [_u64, ctypes.POINTER(Params)]
        L.bos_workspace_bytes.restype = ctypes.c_size_t
        for name in ("bos_orp", "bos_sort"):
            f = getattr(L, name)
            f.argtypes = [_vp, _vp, _u64, ctypes.POINTER(Params), _vp, ctypes.c_size_t, _vp,
                          ctypes.POINTER(Info)]
            f.restype = ctypes.c_int
        L.bos_batched_workspace_bytes.argtypes = [_vp, _u32, _vp, _vp, ctypes.POINTER(Params)]
        L.bos_batched_workspace_bytes.restype = ctypes.c_size_t
        for name in ("bos_sort_batched", "bos_batched_collect"):
            f = getattr(L, name)
            f.argtypes = [_vp, _vp, _vp, _u32, _vp, _vp, _vp, ctypes.POINTER(Params), _vp,
                          ctypes.c_size_t, _vp, _vp]
            f.restype = ctypes.c_int
        for name in ("bos_batched_prepare", "bos_batched_enqueue"):
            f = getattr(L, name)
            f.argtypes = [_vp, _vp, _vp, _u32, _vp, _vp, _vp, ctypes.POINTER(Params), _vp,
                          ctypes.c_size_t, _vp]
            f.restype = ctypes.c_int
        L.bos_bitonic_sort.argtypes = [_vp, _vp, _u64, _u32, _u32, _vp]
        L.bos_bitonic_sort.restype = ctypes.c_int
        L.bos_trace_attach.argtypes = [_vp, ctypes.c_size_t]
        L.bos_trace_attach.restype = ctypes.c_int
        L.bos_shard_layout.argtypes = [_u64, _u32, ctypes.POINTER(Params), ctypes.POINTER(ShardLayout)]
        L.bos_shard_layout.restype = ctypes.c_int
        L.bos_shard_input_range.argtypes = [_u64, _u32, _u32, ctypes.POINTER(Params), ctypes.POINTER(_u64),
                                            ctypes.POINTER(_u64)]
        L.bos_shard_input_range.restype = ctypes.c_int
        L.bos_shard_local.argtypes = [_vp, _u64, _u32, _u32, ctypes.POINTER(Params), _u32, _vp, ctypes.c_size_t, _vp]
        L.bos_shard_local.restype = ctypes.c_int
        L.bos_shard_final.argtypes = [_u64, _u32, _u32, ctypes.POINTER(Params), _u32, _vp, _u64, _vp,
                                      ctypes.c_size_t, _vp, ctypes.POINTER(_u64), ctypes.POINTER(_u32)]
        L.bos_shard_final.restype = ctypes.c_int
        L.bos_orp_out_of_core_bytes.argtypes = [_u64, _u32, ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_size_t),
                                                ctypes.POINTER(ctypes.c_size_t)]
        L.bos_orp_out_of_core_bytes.restype = ctypes.c_int
        L.bos_orp_out_of_core.argtypes = [_vp, _vp, _u64, ctypes.POINTER(Params), _u32, _vp, ctypes.c_size_t, _vp,
                                          ctypes.c_size_t, _vp, ctypes.POINTER(Info)]
        L.bos_orp_out_of_core.restype = ctypes.c_int
        L.bos_trace_attach_digest.argtypes = [_vp, ctypes.c_size_t]
        L.bos_trace_attach_digest.restype = ctypes.c_int
        L.bos_status_str.argtypes = [ctypes.c_int]
        L.bos_status_str.restype = ctypes.c_char_p
        L.bos_version.restype = _u32
        L.bos_selftest_philox.argtypes = [_vp, _vp, _vp, _vp, _u64, _vp]
        L.bos_selftest_philox.restype = ctypes.c_int
        L.bos_orp_noalloc.argtypes = [_vp, _vp, _u64, ctypes.POINTER(Params), _vp,
                                      ctypes.POINTER(Info)]
        L.bos_orp_noalloc.restype = ctypes.c_int
        L.bos_profile_enable.argtypes = [ctypes.c_int]
        L.bos_profile_enable.restype = ctypes.c_int
        L.bos_profile_read.argtypes = [ctypes.POINTER(KernelStat), _u32, ctypes.POINTER(_u64)]
        L.bos_profile_read.restype = _u32
        _lib = L
    return _lib


def status_str(s):
    return lib().bos_status_str(int(s)).decode()


def params(rec_bytes=16, Z=512, seed=1, k=0, max_attempts=0, flags=0):
    return Params(rec_bytes, 4 if rec_bytes == 8 else 8, Z, k, max_attempts, flags, seed)


def plan(n, rec_bytes=16, Z=512, k=0, flags=0, sort=True) -> Info:
    """The library's pass plan for n records (no device work)."""
    p = params(rec_bytes, Z, 0, k, 0, flags | FLAG_PLAN_ONLY)
    info = Info()
    fn = lib().bos_sort if sort else lib().bos_orp
    _check(fn(None, None, n, ctypes.byref(p), None, 0, None, ctypes.byref(info)), "plan")
    return info


def workspace_bytes(n, p: Params) -> int:
    return int(lib().bos_workspace_bytes(n, ctypes.byref(p)))


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(st, what):
    if st != OK:
        raise BosError(st, what)


def alloc_workspace(nbytes, device="cuda"):
    import torch
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def orp_raw(d_in, d_out, n, p: Params, ws, ws_bytes, stream_handle) -> Info:
    """bos_orp on raw device pointers (ints); returns Info, raises BosError."""
    info = Info()
    st = lib().bos_orp(_vp(d_in), _vp(d_out), n, ctypes.byref(p), _vp(ws), ws_bytes,
                       stream_handle, ctypes.byref(info))
    _check(st, "bos_orp")
    return info


def sort_raw(d_in, d_out, n, p: Params, ws, ws_bytes, stream_handle) -> Info:
    info = Info()
    st = lib().bos_sort(_vp(d_in), _vp(d_out), n, ctypes.byref(p), _vp(ws), ws_bytes,
                        stream_handle, ctypes.byref(info))
    _check(st, "bos_sort")
    return info


def _run(fn, x, out, n, rec_bytes, Z, seed, k, max_attempts, flags, workspace, stream):
    import torch
    p = params(rec_bytes, Z, seed, k, max_attempts, flags)
    if out is None:
        out = torch.empty_like(x)
    need = workspace_bytes(n, p)
    if workspace is None or workspace.numel() < need:
        workspace = alloc_workspace(need, x.device)
    info = fn(x.data_ptr(), out.data_ptr(), n, p, workspace.data_ptr(), workspace.numel(),
              _stream_handle(stream))
    return out, info


def orp(x, rec_bytes, Z=512, seed=1, k=0, max_attempts=0, flags=0, out=None, workspace=None,
        stream=None):
    """Bucket ORP of a contiguous CUDA tensor holding n records of rec_bytes bytes each."""
    n = x.numel() * x.element_size() // rec_bytes
    return _run(orp_raw, x, out, n, rec_bytes, Z, seed, k, max_attempts, flags, workspace, stream)


NOALLOC_SCRATCH_BYTES = 64 << 20


def orp_noalloc(x, rec_bytes, Z=512, seed=1, k=0, max_attempts=0, flags=0, out=None, stream=None):
    """bos_orp_noalloc: the bucket ORP without a caller workspace (the library's fixed scratch
    is used; calls on one device must not overlap). Returns (out, Info)."""
    import torch
    n = x.numel() * x.element_size() // rec_bytes
    if out is None:
        out = torch.empty_like(x)
    p = params(rec_bytes, Z, seed, k, max_attempts, flags)
    info = Info()
    st = lib().bos_orp_noalloc(_vp(x.data_ptr()), _vp(out.data_ptr()), n, ctypes.byref(p),
                               _stream_handle(stream), ctypes.byref(info))
    _check(st, "bos_orp_noalloc")
    return out, info


def sort(x, rec_bytes, Z=512, seed=1, k=0, max_attempts=0, flags=0, out=None, workspace=None,
         stream=None):
    """Bucket oblivious sort of a contiguous CUDA tensor of records."""
    n = x.numel() * x.element_size() // rec_bytes
    return _run(sort_raw, x, out, n, rec_bytes, Z, seed, k, max_attempts, flags, workspace, stream)


def bitonic_sort(x, rec_bytes, out=None, stream=None):
    import torch
    n = x.numel() * x.element_size() // rec_bytes
    if out is None:
        out = torch.empty_like(x)
    st = lib().bos_bitonic_sort(_vp(x.data_ptr()), _vp(out.data_ptr()), n, rec_bytes,
                                4 if rec_bytes == 8 else 8, _stream_handle(stream))
    _check(st, "bos_bitonic_sort")
    return out


def batched_workspace_bytes(offsets, Zs, ops, base: Params) -> int:
    """bos_batched_workspace_bytes for host arrays (offsets num + 1, Zs or None, ops)."""
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    ops = np.ascontiguousarray(ops, dtype=np.uint8)
    Zs = None if Zs is None else np.ascontiguousarray(Zs, dtype=np.uint32)
    return int(lib().bos_batched_workspace_bytes(off.ctypes.data_as(_vp), off.size - 1,
                                                 None if Zs is None else Zs.ctypes.data_as(_vp),
                                                 ops.ctypes.data_as(_vp), ctypes.byref(base)))


class Batch:
    """A batch of back-to-back arrays (bos_sort_batched and its prepare/enqueue/collect steps).

    x, out: CUDA uint8 tensors holding all records; offsets: num + 1 record offsets; seeds, ops
    (0 = ORP, 1 = sort) and Zs (optional) per array. The host tables are kept alive here, as the
    enqueue step may be captured into a CUDA graph.
    """

    def __init__(self, x, out, offsets, seeds, ops, base: Params, Zs=None, workspace=None):
        self.x, self.out, self.base = x, out, base
        self.off = np.ascontiguousarray(offsets, dtype=np.uint64)
        self.seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
        self.ops = np.ascontiguousarray(ops, dtype=np.uint8)
        self.Zs = None if Zs is None else np.ascontiguousarray(Zs, dtype=np.uint32)
        self.num = self.off.size - 1
        need = int(lib().bos_batched_workspace_bytes(
            self.off.ctypes.data_as(_vp), self.num,
            None if self.Zs is None else self.Zs.ctypes.data_as(_vp), self.ops.ctypes.data_as(_vp),
            ctypes.byref(base)))
        if need == 0 and self.num:
            raise BosError(ERR_INVALID, "bos_batched_workspace_bytes")
        if workspace is None or workspace.numel() < need:
            workspace = alloc_workspace(need, x.device)
        self.ws = workspace
        self.attempts = np.zeros(max(self.num, 1), dtype=np.uint32)

    def _args(self):
        return (_vp(self.x.data_ptr()), _vp(self.out.data_ptr()), self.off.ctypes.data_as(_vp),
                self.num, self.seeds.ctypes.data_as(_vp),
                None if self.Zs is None else self.Zs.ctypes.data_as(_vp),
                self.ops.ctypes.data_as(_vp), ctypes.byref(self.base), _vp(self.ws.data_ptr()),
                self.ws.numel())

    def run(self, stream=None):
        st = lib().bos_sort_batched(*self._args(), _stream_handle(stream),
                                    self.attempts.ctypes.data_as(_vp))
        _check(st, "bos_sort_batched")
        return self.attempts[:self.num]

    def prepare(self, stream=None):
        _check(lib().bos_batched_prepare(*self._args(), _stream_handle(stream)), "bos_batched_prepare")

    def enqueue(self, stream=None):
        _check(lib().bos_batched_enqueue(*self._args(), _stream_handle(stream)), "bos_batched_enqueue")

    def collect(self, stream=None):
        st = lib().bos_batched_collect(*self._args(), _stream_handle(stream),
                                       self.attempts.ctypes.data_as(_vp))
        _check(st, "bos_batched_collect")
        return self.attempts[:self.num]


def sort_batched(x, out, offsets, seeds, ops, base: Params, Zs=None, workspace=None, stream=None):
    """Batched ORP/sort of back-to-back arrays; returns the attempts per array."""
    return Batch(x, out, offsets, seeds, ops, base, Zs, workspace).run(stream)


def trace_attach(buf):
    """Attach a uint8/uint64 CUDA tensor as the address-trace buffer (None detaches)."""
    if buf is None:
        _check(lib().bos_trace_attach(None, 0), "bos_trace_attach")
    else:
        _check(lib().bos_trace_attach(_vp(buf.data_ptr()), buf.numel() * buf.element_size()),
               "bos_trace_attach")


def shard_layout(n, G, p: Params) -> ShardLayout:
    """bos_shard_layout: geometry and workspace layout of the G-rank shard plan."""
    lay = ShardLayout()
    _check(lib().bos_shard_layout(n, G, ctypes.byref(p), ctypes.byref(lay)), "bos_shard_layout")
    return lay


def shard_input_range(n, G, r, p: Params):
    lo, hi = _u64(), _u64()
    _check(lib().bos_shard_input_range(n, G, r, ctypes.byref(p), ctypes.byref(lo), ctypes.byref(hi)),
           "bos_shard_input_range")
    return lo.value, hi.value


def sharded_orp(x, rec_bytes, G, Z=512, seed=1, k=0, max_attempts=8, flags=0, stream=None):
    """The G-rank shard plan run on one device (each rank its own workspace; the exchange is a
    device copy of every rank-to-rank chunk). Returns (out, attempts, counts per rank)."""
    import torch
    n = x.numel() * x.element_size() // rec_bytes
    p = params(rec_bytes, Z, seed, k, 0, flags)
    lay = shard_layout(n, G, p)
    sh = _stream_handle(stream)
    ws = [alloc_workspace(lay.ws_bytes, x.device) for _ in range(G)]
    parts = [torch.empty(lay.out_capacity * rec_bytes, dtype=torch.uint8, device=x.device) for _ in range(G)]
    ranges = [shard_input_range(n, G, r, p) for r in range(G)]
    for attempt in range(max_attempts):
        for r in range(G):
            lo, hi = ranges[r]
            _check(lib().bos_shard_local(_vp(x.data_ptr() + lo * rec_bytes), n, G, r, ctypes.byref(p), attempt,
                                         _vp(ws[r].data_ptr()), ws[r].numel(), sh), "bos_shard_local")
        with torch.cuda.stream(stream) if stream is not None else _nullctx():
            for s in range(G):
                for d in range(G):
                    for src_off, dst_off, cb in ((lay.send_rec_offset, lay.recv_rec_offset, lay.chunk_rec_bytes),
                                                 (lay.send_tag_offset, lay.recv_tag_offset, lay.chunk_tag_bytes)):
                        ws[d][dst_off + s * cb:dst_off + (s + 1) * cb].copy_(
                            ws[s][src_off + d * cb:src_off + (d + 1) * cb])
        counts, over = [], False
        for r in range(G):
            c, o = _u64(), _u32()
            _check(lib().bos_shard_final(n, G, r, ctypes.byref(p), attempt, _vp(parts[r].data_ptr()),
                                         lay.out_capacity, _vp(ws[r].data_ptr()), ws[r].numel(), sh,
                                         ctypes.byref(c), ctypes.byref(o)), "bos_shard_final")
            counts.append(int(c.value))
            over |= bool(o.value)
        if over:
            continue
        out = torch.cat([parts[r][:counts[r] * rec_bytes] for r in range(G)])
        return out, attempt + 1, counts
    raise BosError(ERR_OVERFLOW, "sharded_orp")


def orp_out_of_core(recs: np.ndarray, G, Z=512, seed=1, k=0, max_attempts=0, flags=0, device="cuda",
                    stream=None):
    """bos_orp_out_of_core of a host record array (copied to pinned host memory); returns
    (host result array, Info). The device holds one rank's share of the shard plan at a time."""
    import torch
    rec_bytes = recs.dtype.itemsize
    n = recs.shape[0]
    p = params(rec_bytes, Z, seed, k, max_attempts, flags)
    dev_b, host_b = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().bos_orp_out_of_core_bytes(n, G, ctypes.byref(p), ctypes.byref(dev_b), ctypes.byref(host_b)),
           "bos_orp_out_of_core_bytes")
    h_in = torch.from_numpy(np.ascontiguousarray(recs).view(np.uint8).reshape(-1)).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    h_stage = torch.empty(max(host_b.value, 1), dtype=torch.uint8).pin_memory()
    d_buf = alloc_workspace(dev_b.value, device)
    info = Info()
    _check(lib().bos_orp_out_of_core(_vp(h_in.data_ptr()), _vp(h_out.data_ptr()), n, ctypes.byref(p), G,
                                     _vp(d_buf.data_ptr()), d_buf.numel(), _vp(h_stage.data_ptr()), h_stage.numel(),
                                     _stream_handle(stream), ctypes.byref(info)), "bos_orp_out_of_core")
    return h_out.numpy().view(recs.dtype).copy(), info


class _nullctx:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def trace_attach_digest(buf):
    """Attach a zeroed CUDA tensor (>= 4096 bytes) as the address-trace digest (None detaches)."""
    if buf is None:
        _check(lib().bos_trace_attach_digest(None, 0), "bos_trace_attach_digest")
    else:
        _check(lib().bos_trace_attach_digest(_vp(buf.data_ptr()), buf.numel() * buf.element_size()),
               "bos_trace_attach_digest")


def selftest_philox(ctr, key, with_curand=True, stream=None):
    """Library Philox (and cuRAND's) of CUDA uint32 tensors ctr (n,4) and key (n,2)."""
    import torch
    n = ctr.shape[0]
    out = torch.empty((n, 4), dtype=torch.int32, device=ctr.device)
    ref = torch.empty_like(out) if with_curand else None
    st = lib().bos_selftest_philox(_vp(ctr.data_ptr()), _vp(key.data_ptr()), _vp(out.data_ptr()),
                                   _vp(ref.data_ptr()) if ref is not None else None, n,
                                   _stream_handle(stream))
    _check(st, "bos_selftest_philox")
    return out, ref


def profile_enable(on=True):
    _check(lib().bos_profile_enable(1 if on else 0), "bos_profile_enable")


def profile_read():
    """{kernel class: {launches, ms, bytes}} and the total launch count since enable."""
    arr = (KernelStat * 16)()
    tot = _u64(0)
    m = lib().bos_profile_read(arr, 16, ctypes.byref(tot))
    stats = {arr[i].name.decode(): {"launches": int(arr[i].launches), "ms": float(arr[i].ms),
                                    "bytes": float(arr[i].bytes)} for i in range(m)}
    return stats, int(tot.value)


# ---- numpy <-> torch helpers for structured record arrays ----
def to_device(recs: np.ndarray, device="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(recs).view(np.uint8).reshape(-1)).to(device)


def to_host(t, dtype) -> np.ndarray:
    return t.cpu().numpy().view(dtype)
