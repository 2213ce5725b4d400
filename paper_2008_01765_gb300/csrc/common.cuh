// Shared device helpers of the CUDA path: Philox4x32-10, record types, bounded look-back
// waits and the debug address trace. sm_103a only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bos {

constexpr uint32_t kDummy = 0xFFFFFFFFu;  // tag of a dummy slot; real tags are labels < 2^31

// Dynamic shared memory limit of every kernel that may use more than 48 KB: the device's opt-in
// maximum minus the kernel's static shared memory - one value per kernel, never the launch's own
// size. The attribute is per-function process state, and host threads launching the same kernel
// with different sizes must not lower it under one another.
template <typename Kernel>
inline cudaError_t set_smem_optin(Kernel kern) {
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  int dev = 0, optin = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

// ---------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC 2011). Ten rounds; each multiplies counter words 0 and 2 by
// the two round multipliers, xors the high halves into words 1 and 3 with the round key, and
// bumps the key by the Weyl constants between rounds.
// ---------------------------------------------------------------------------------------------
struct PhiloxOut {
  uint32_t w0, w1, w2, w3;
};

__host__ __device__ __forceinline__ PhiloxOut philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                            uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
#ifdef __CUDA_ARCH__
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
#else
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return {c0, c1, c2, c3};
}

// Philox block at position `index` of stream `stream` for attempt `attempt`:
// counter = (lo index, hi index, attempt, stream), key = (lo seed, hi seed).
__host__ __device__ __forceinline__ PhiloxOut philox_at(uint64_t index, uint32_t attempt,
                                                        uint32_t stream, uint64_t seed) {
  return philox4x32_10((uint32_t)index, (uint32_t)(index >> 32), attempt, stream, (uint32_t)seed,
                       (uint32_t)(seed >> 32));
}

// Label of element i: top L bits of word 0 of stream 0 (Algorithm 3.1, random key in [0, B)).
__device__ __forceinline__ uint32_t label_of(uint64_t i, uint64_t seed, uint32_t attempt, uint32_t L) {
  if (L == 0) return 0;
  return philox_at(i, attempt, 0, seed).w0 >> (32 - L);
}

// ---------------------------------------------------------------------------------------------
// Records: 8-byte {u32 key, u32 payload} as uint2, 16-byte {u64 key, u64 payload} as uint4.
// ---------------------------------------------------------------------------------------------
template <int R> struct RecT;
template <> struct RecT<8> {
  using T = uint2;
  using Key = uint32_t;
  static constexpr int kDigits = 4;
  __device__ __forceinline__ static Key key(const T& r) { return r.x; }
  __device__ __forceinline__ static T zero() { return make_uint2(0, 0); }
};
template <> struct RecT<16> {
  using T = uint4;
  using Key = unsigned long long;
  static constexpr int kDigits = 8;
  __device__ __forceinline__ static Key key(const T& r) {
    return (unsigned long long)r.x | ((unsigned long long)r.y << 32);
  }
  __device__ __forceinline__ static T zero() { return make_uint4(0, 0, 0, 0); }
};

// Lanes of the warp whose value equals this lane's in the low nbits bits: one ballot per bit.
// Measured on this part: cheaper than the match instruction when a warp holds many distinct
// values (8-bit radix digits), dearer when it holds few (the butterfly's 2^k routing digits).
__device__ __forceinline__ uint32_t ballot_peers(uint32_t v, uint32_t nbits) {
  uint32_t peers = 0xFFFFFFFFu;
#pragma unroll 4
  for (uint32_t b = 0; b < nbits; ++b) {
    const uint32_t bit = (v >> b) & 1u;
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, bit);
    peers &= bit ? bal : ~bal;
  }
  return peers;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ---------------------------------------------------------------------------------------------
// Control block at the start of the workspace (zeroed at the start of every attempt).
// ---------------------------------------------------------------------------------------------
struct Ctrl {
  uint32_t overflow;         // any MergeSplit output received more than Z reals
  uint32_t timeout;          // a bounded wait gave up
  uint32_t forced;           // debug: attempts still to be reported as overflowed
  uint32_t radix_live;       // bit d set: digit d of the keys is not constant (a radix pass runs)
  uint32_t sort_mode;        // sort after the ORP: 0 = LSD radix passes, m = 1..3: the hybrid sort's m passes
  uint32_t bad;              // a device-side consistency check failed (the work it guards was skipped)
  uint32_t tickets[58];      // dynamic work counters, one per launch that orders its CTAs
};
static_assert(sizeof(Ctrl) == 256, "control block size");

// The LAST ORP pass writes the sort's scratch buffer (instead of the output) when an odd number of
// sort passes follows it, so that the last sort pass writes the output.
__device__ __forceinline__ bool sort_passes_odd(const Ctrl* c) {
  const uint32_t p = c->sort_mode ? c->sort_mode : (uint32_t)__popc(c->radix_live);
  return (p & 1u) != 0;
}

// Bounded spin: number of polls before a wait gives up (~0.5 s with the back-off below).
constexpr uint32_t kSpinLimit = 1u << 22;

// Look-back status words carry their own value (state, tag and count in one 64-bit word) and
// no other data depends on them, so relaxed device-scope accesses suffice (no fences).
__device__ __forceinline__ unsigned long long ld_status(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_status(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Look-back status word: bits 62..63 = state (1 aggregate, 2 inclusive prefix), bits 56..61 =
// tag of the launch that wrote it (so one zeroed array serves several passes), bits 0..55 value.
constexpr unsigned long long kStAgg = 1ull << 62;
constexpr unsigned long long kStIncl = 2ull << 62;
constexpr unsigned long long kStValue = (1ull << 56) - 1;

__device__ __forceinline__ unsigned long long st_word(unsigned long long state, uint32_t tag,
                                                      unsigned long long value) {
  return state | ((unsigned long long)(tag & 63u) << 56) | (value & kStValue);
}

// Exclusive prefix of tile `tile` over its predecessors (decoupled look-back, one thread). The
// word of tile j is status[j * stride]. Spins with a limit; on timeout raises ctrl->timeout and
// returns the prefix gathered so far.
__device__ __forceinline__ unsigned long long lookback(const unsigned long long* status, uint64_t tile,
                                                       uint64_t stride, uint32_t tag, Ctrl* ctrl) {
  unsigned long long prefix = 0;
  int64_t j = (int64_t)tile - 1;
  while (j >= 0) {
    unsigned long long w = 0;
    uint32_t spins = 0;
    while (true) {
      w = ld_status(status + (uint64_t)j * stride);
      if ((w >> 62) != 0 && ((w >> 56) & 63u) == tag) break;
      if (++spins > kSpinLimit) {
        atomicExch(&ctrl->timeout, 1u);
        return prefix;
      }
      if (spins > 32) __nanosleep(64);
    }
    prefix += w & kStValue;
    if (w & kStIncl) break;
    --j;
  }
  return prefix;
}

// Windowed variant: each step issues the loads of W predecessors at once (independent loads, one
// round-trip per W tiles), then folds them in order, waiting (bounded) on any not yet published.
template <int W>
__device__ __forceinline__ unsigned long long lookback_window(const unsigned long long* status, uint64_t tile,
                                                              uint64_t stride, uint32_t tag, Ctrl* ctrl) {
  unsigned long long prefix = 0;
  int64_t j = (int64_t)tile - 1;
  while (j >= 0) {
    unsigned long long w[W];
#pragma unroll
    for (int x = 0; x < W; ++x) w[x] = (j - x >= 0) ? ld_status(status + (uint64_t)(j - x) * stride) : 0ull;
#pragma unroll
    for (int x = 0; x < W; ++x) {
      if (j - x < 0) return prefix;
      unsigned long long v = w[x];
      uint32_t spins = 0;
      while (!((v >> 62) != 0 && ((v >> 56) & 63u) == tag)) {
        if (++spins > kSpinLimit) {
          atomicExch(&ctrl->timeout, 1u);
          return prefix;
        }
        if (spins > 16) __nanosleep(32);
        v = ld_status(status + (uint64_t)(j - x) * stride);
      }
      prefix += v & kStValue;
      if (v & kStIncl) return prefix;
    }
    j -= W;
  }
  return prefix;
}

// ---------------------------------------------------------------------------------------------
// Shared-memory addresses, mbarriers and TMA bulk copies (cp.async.bulk)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// ---- mbarrier + TMA bulk copies ----
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bounded wait on an mbarrier phase; false (and ctrl->timeout) if it never completed.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, Ctrl* ctrl) {
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  atomicExch(&ctrl->timeout, 1u);
  return false;
}
__device__ __forceinline__ void tma_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_store(void* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_store_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void tma_store_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void tma_store_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------------------------------------
// Debug address trace: {(kind << 56) | (buffer << 48) | bytes, byte offset}.
// ---------------------------------------------------------------------------------------------
enum TraceBuf : uint32_t {
  kBufIn = 0, kBufRecA = 1, kBufTagA = 2, kBufRecB = 3, kBufTagB = 4, kBufOut = 5, kBufTmp = 6,
  kBufPerm = 7
};
enum TraceKind : uint32_t { kRead = 1, kWrite = 2 };

struct Trace {
  unsigned long long* buf;  // word 0 = entry counter; entries start at word 2 (digest: 256 slots)
  unsigned long long cap;   // entries that fit
  uint32_t digest;          // 1: order-independent digest instead of the entries
};

// SplitMix64's output function (Steele, Lea, Flood 2014): a 64-bit mix for the trace digest.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Entry {(kind << 56) | (buffer << 48) | bytes, offset}. Digest mode: slot (SM id mod 256) of the
// buffer counts the entries and sums mix64(word0 ^ mix64(offset)) modulo 2^64, so the sum over the
// slots depends only on the multiset of entries, not on their order or on which SM logged them.
template <bool TRACE>
__device__ __forceinline__ void trace_log(const Trace& tr, uint32_t kind, uint32_t buffer,
                                          uint32_t bytes, uint64_t offset) {
  if constexpr (TRACE) {
    if (tr.buf == nullptr) return;
    const unsigned long long w0 = ((unsigned long long)kind << 56) | ((unsigned long long)buffer << 48) | bytes;
    if (tr.digest) {
      uint32_t smid;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
      unsigned long long* slot = tr.buf + 2 * (smid & 255u);
      atomicAdd(slot, 1ull);
      atomicAdd(slot + 1, mix64(w0 ^ mix64(offset)));
      return;
    }
    const unsigned long long e = atomicAdd(tr.buf, 1ull);
    if (e < tr.cap) {
      tr.buf[2 + 2 * e] = w0;
      tr.buf[3 + 2 * e] = offset;
    }
  }
}

}  // namespace bos
